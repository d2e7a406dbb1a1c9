// Checkpoint of the solver precompute (Section 5: the smoother precompute is
// expensive and normally read back from disk) and the C_l update of a plan.
//
// File layout (little-endian, fixed-size fields):
//   magic "CRPRECMP", u32 version, u32 reserved
//   identity: i32 nside, lmax, H, ld, smoother kind; per pixel level i32 nside_h, lmax_h,
//             ntile, i64 nblocks; u64 hashes of C_l, b_l and the N^-1 map
//   per pixel level: f64 alpha, amax, lambda_max; f32 factor blocks
//                    [nblocks][64][64] (Schwarz: the first ntile blocks hold
//                    the tiles' inverse blocks)
//   top level:       f64 top_lambda, top_scale; f64 inv_diag_hp [n_lm(lmax)]
//   bottom level:    i32 nd; f64 A_bottom [nd][nd], A_bottom^-1 [nd][nd];
//                    dof map [nd] (i32 l, m, part)
//   u64 hash of everything above (trailer)
// The identity fields must match the plan a checkpoint is loaded into.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

namespace {

constexpr char kMagic[8] = {'C', 'R', 'P', 'R', 'E', 'C', 'M', 'P'};
constexpr uint32_t kVersion = 2;
constexpr int kBlock = 64 * 64;  // floats per factor block

// 64-bit FNV-1a over bytes
struct Hash {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
};

// Writer and Reader own their FILE: close() ends it, the destructor closes it
// on any other way out (an error return or a host allocation failure)
struct Writer {
  FILE* f = nullptr;
  Hash hash;
  bool ok = true;
  ~Writer() {
    if (f) std::fclose(f);
  }
  bool close() {
    const bool c = std::fclose(f) == 0;
    f = nullptr;
    return c;
  }
  void put(const void* p, size_t n) {
    if (!ok || n == 0) return;
    hash.add(p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  }
  template <typename X> void val(const X& x) { put(&x, sizeof(X)); }
};

struct Reader {
  FILE* f = nullptr;
  Hash hash;
  bool ok = true;
  ~Reader() {
    if (f) std::fclose(f);
  }
  void close() {
    std::fclose(f);
    f = nullptr;
  }
  void get(void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) hash.add(p, n);
  }
  template <typename X> X val() {
    X x{};
    get(&x, sizeof(X));
    return x;
  }
};

// hashes of the inputs that the precompute depends on
int input_hashes(cr_plan* P, uint64_t out[3]) {
  Hash hc, hb, hn;
  hc.add(P->h_cl.data(), P->h_cl.size() * sizeof(double));
  hb.add(P->h_bl.data(), P->h_bl.size() * sizeof(double));
  std::vector<double> ninv(P->obs.npix);
  CR_CUDA(cudaStreamSynchronize(P->stream));
  CR_CUDA(cudaMemcpy(ninv.data(), P->d_ninv, ninv.size() * sizeof(double), cudaMemcpyDeviceToHost));
  hn.add(ninv.data(), ninv.size() * sizeof(double));
  out[0] = hc.h;
  out[1] = hb.h;
  out[2] = hn.h;
  return CR_OK;
}

struct Identity {
  int32_t nside = 0, lmax = 0, H = 0, ld = 0, smoother = 0;
  std::vector<int32_t> nside_h, lmax_h, ntile;
  std::vector<int64_t> nblocks;
  uint64_t hash[3] = {0, 0, 0};
};

int plan_identity(cr_plan* P, Identity& id) {
  const Hierarchy& H = *P->hier;
  id.nside = P->obs.nside;
  id.lmax = P->lmax;
  id.H = H.H;
  id.ld = H.ld;
  id.smoother = H.smoother_kind;
  for (const PixLevel& lev : H.pix) {
    id.nside_h.push_back(lev.nside_h);
    id.lmax_h.push_back(lev.lmax_h);
    id.ntile.push_back(lev.pat.ntile);
    id.nblocks.push_back(lev.pat.nblocks);
  }
  return input_hashes(P, id.hash);
}

}  // namespace

}  // namespace cr

using namespace cr;

static int save_impl(cr_plan* plan, const char* path) {
  if (!plan || !path) return fail(CR_EINVAL, "cr_save: null argument");
  if (!plan->hier) return fail(CR_EINVAL, "cr_save: plan was created without levels");
  Hierarchy& H = *plan->hier;
  if (!H.numeric_ready) return fail(CR_ESTATE, "cr_save: the precompute has not been run");
  Identity id;
  int rc = plan_identity(plan, id);
  if (rc) return rc;
  Writer w;
  w.f = std::fopen(path, "wb");
  if (!w.f) return fail(CR_EIO, std::string("cr_save: cannot open ") + path);
  w.put(kMagic, sizeof(kMagic));
  w.val(kVersion);
  w.val<uint32_t>(0);
  w.val(id.nside);
  w.val(id.lmax);
  w.val(id.H);
  w.val(id.ld);
  w.val(id.smoother);
  for (int i = 0; i < id.H; ++i) {
    w.val(id.nside_h[i]);
    w.val(id.lmax_h[i]);
    w.val(id.ntile[i]);
    w.val(id.nblocks[i]);
  }
  for (uint64_t h : id.hash) w.val(h);
  std::vector<float> fbuf;
  for (const PixLevel& lev : H.pix) {
    w.val(lev.alpha);
    w.val(lev.amax);
    w.val(lev.lambda_max);
    const int64_t nel = lev.pat.nblocks * kBlock;
    // in slices, to bound the host buffer
    const int64_t slice = (int64_t)1 << 26;
    for (int64_t o = 0; o < nel && w.ok; o += slice) {
      const int64_t n = std::min(slice, nel - o);
      fbuf.resize(n);
      cudaError_t e = cudaMemcpy(fbuf.data(), lev.d_L + o, n * sizeof(float), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "cr_save: factor copy");
      w.put(fbuf.data(), n * sizeof(float));
    }
  }
  w.val(H.top_lambda);
  w.val(H.top_scale);
  {
    std::vector<double> hv(n_lm(plan->lmax));
    cudaError_t e = cudaMemcpy(hv.data(), H.inv_diag_hp.d, hv.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cr_save: top smoother copy");
    w.put(hv.data(), hv.size() * sizeof(double));
  }
  w.val<int32_t>(H.nd);
  if (H.nd > 0) {
    const size_t nn = (size_t)H.nd * H.nd;
    std::vector<double> a(nn), ai(nn);
    std::vector<int32_t> dofs(3 * (size_t)H.nd);
    cudaError_t e = cudaMemcpy(a.data(), H.d_Abottom, nn * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ai.data(), H.d_Ainv, nn * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dofs.data(), H.d_dof_lm, dofs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cr_save: bottom copy");
    w.put(a.data(), nn * sizeof(double));
    w.put(ai.data(), nn * sizeof(double));
    w.put(dofs.data(), dofs.size() * sizeof(int32_t));
  }
  const uint64_t trailer = w.hash.h;
  if (w.ok) w.ok = std::fwrite(&trailer, 1, sizeof(trailer), w.f) == sizeof(trailer);
  const bool closed = w.close();
  if (!w.ok || !closed) return fail(CR_EIO, std::string("cr_save: write failed: ") + path);
  return CR_OK;
}

static int load_impl(cr_plan* plan, const char* path) {
  if (!plan || !path) return fail(CR_EINVAL, "cr_load: null argument");
  if (!plan->hier) return fail(CR_EINVAL, "cr_load: plan was created without levels");
  Hierarchy& H = *plan->hier;
  Identity id;
  int rc = plan_identity(plan, id);
  if (rc) return rc;
  Reader r;
  r.f = std::fopen(path, "rb");
  if (!r.f) return fail(CR_EIO, std::string("cr_load: cannot open ") + path);
  auto bad = [&](int code, const std::string& why) { return fail(code, "cr_load: " + why); };
  char magic[8];
  r.get(magic, sizeof(magic));
  const uint32_t ver = r.val<uint32_t>();
  r.val<uint32_t>();
  if (!r.ok || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) return bad(CR_EIO, "not a precompute checkpoint");
  if (ver != kVersion) return bad(CR_EIO, "unsupported checkpoint version");
  Identity fid;
  fid.nside = r.val<int32_t>();
  fid.lmax = r.val<int32_t>();
  fid.H = r.val<int32_t>();
  fid.ld = r.val<int32_t>();
  fid.smoother = r.val<int32_t>();
  if (!r.ok) return bad(CR_EIO, "truncated header");
  if (fid.nside != id.nside || fid.lmax != id.lmax || fid.H != id.H || fid.ld != id.ld ||
      fid.smoother != id.smoother)
    return bad(CR_EINVAL, "checkpoint was made for another grid, band limit, level table or smoother");
  for (int i = 0; i < fid.H; ++i) {
    const int32_t ns = r.val<int32_t>(), lm = r.val<int32_t>(), nt = r.val<int32_t>();
    const int64_t nb = r.val<int64_t>();
    if (!r.ok) return bad(CR_EIO, "truncated header");
    if (ns != id.nside_h[i] || lm != id.lmax_h[i] || nt != id.ntile[i] || nb != id.nblocks[i])
      return bad(CR_EINVAL, "checkpoint was made for another level table");
  }
  for (int k = 0; k < 3; ++k) {
    const uint64_t h = r.val<uint64_t>();
    if (!r.ok) return bad(CR_EIO, "truncated header");
    if (h != id.hash[k]) {
      static const char* what[3] = {"C_l", "b_l", "the N^-1 map"};
      return bad(CR_EINVAL, std::string("checkpoint was made for different ") + what[k]);
    }
  }
  // read everything into host memory first, so that a bad file changes nothing
  struct LevelData {
    double alpha, amax, lambda_max;
    std::vector<float> L;
  };
  std::vector<LevelData> lv(H.H);
  for (int i = 0; i < H.H; ++i) {
    lv[i].alpha = r.val<double>();
    lv[i].amax = r.val<double>();
    lv[i].lambda_max = r.val<double>();
    lv[i].L.resize(H.pix[i].pat.nblocks * kBlock);
    r.get(lv[i].L.data(), lv[i].L.size() * sizeof(float));
  }
  const double top_lambda = r.val<double>(), top_scale = r.val<double>();
  std::vector<double> hv(n_lm(plan->lmax));
  r.get(hv.data(), hv.size() * sizeof(double));
  const int32_t nd = r.val<int32_t>();
  if (!r.ok || nd < 0) return bad(CR_EIO, "truncated or corrupt body");
  // the bottom dof map indexes device vectors in the dense solve: it must be
  // exactly the map the plan builds from its own C_l and band limit, not
  // merely one of the same length (checked before the bottom arrays, whose
  // size nd^2 comes from the file, are allocated)
  const std::vector<int32_t> dofs_plan = bottom_dof_map(plan, H.ld);
  if ((size_t)nd * 3 != dofs_plan.size()) return bad(CR_EINVAL, "bottom level does not match the plan's C_l");
  std::vector<double> a((size_t)nd * nd), ai((size_t)nd * nd);
  std::vector<int32_t> dofs(3 * (size_t)nd);
  r.get(a.data(), a.size() * sizeof(double));
  r.get(ai.data(), ai.size() * sizeof(double));
  r.get(dofs.data(), dofs.size() * sizeof(int32_t));
  const uint64_t want = r.hash.h;
  uint64_t trailer = 0;
  const bool got = std::fread(&trailer, 1, sizeof(trailer), r.f) == sizeof(trailer);
  if (!r.ok || !got) return bad(CR_EIO, "truncated body");
  if (trailer != want) return bad(CR_EIO, "checksum mismatch");
  r.close();
  if (dofs != dofs_plan) return fail(CR_EINVAL, "cr_load: bottom level does not match the plan's C_l");
  // upload
  CR_CUDA(cudaStreamSynchronize(plan->stream));
  H.numeric_ready = false;
  for (int i = 0; i < H.H; ++i) {
    PixLevel& lev = H.pix[i];
    CR_CUDA(cudaMemcpy(lev.d_L, lv[i].L.data(), lv[i].L.size() * sizeof(float), cudaMemcpyHostToDevice));
    lev.alpha = lv[i].alpha;
    lev.amax = lv[i].amax;
    lev.lambda_max = lv[i].lambda_max;
    lev.lt_valid = false;
  }
  H.top_lambda = top_lambda;
  H.top_scale = top_scale;
  if ((rc = H.inv_diag_hp.assign(hv))) return rc;
  if (nd > 0) {
    if ((rc = bottom_upload(plan, H, nd, a.data(), ai.data(), dofs.data()))) return rc;
  }
  H.nd = nd;
  H.numeric_ready = true;
  return CR_OK;
}

// The file is staged through host memory (the fine levels' factors are
// gigabytes at Nside 2048): a failed host allocation is reported, not thrown
// across the C ABI.
extern "C" int cr_save(cr_plan* plan, const char* path) {
  try {
    return save_impl(plan, path);
  } catch (const std::bad_alloc&) {
    return fail(CR_ENOMEM, "cr_save: host allocation");
  }
}

extern "C" int cr_load(cr_plan* plan, const char* path) {
  try {
    return load_impl(plan, path);
  } catch (const std::bad_alloc&) {
    return fail(CR_ENOMEM, "cr_load: host allocation");
  }
}
