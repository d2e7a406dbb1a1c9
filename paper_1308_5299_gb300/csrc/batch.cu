// Batched realizations: the fixed-count CR-Solves (Fig. code:mg) of many
// right-hand sides, over one or several plans (mixed resolutions), captured
// once into a CUDA graph and replayed with a single graph launch.  Replays
// run the same kernels with the same arguments as the uncaptured solves, so
// their results are identical; the host issues one launch per batch instead
// of one per kernel.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {
int solve(cr_plan* P, void* x, const void* b, double eps, int max_cycles, int mode, int* cycles_out,
          double* relres_out, double* history);
int solve_tc(cr_plan* P, void* x, const void* b, int nrhs, double eps, int max_cycles, bool fixed, int* cycles_out,
             double* relres_out, double* history);
}  // namespace cr

struct cr_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  size_t nodes = 0;
  int64_t kernels = 0;  // kernel nodes
};

using namespace cr;

extern "C" {

int cr_batch_create(cr_batch** out, int nplans, cr_plan* const* plans, void* const* x, const void* const* b,
                    const int* nrhs, int cycles, int mode) {
  if (!out || nplans < 1 || !plans || !x || !b || !nrhs || cycles < 1)
    return fail(CR_EINVAL, "cr_batch_create: bad arguments");
  const bool tc = (mode & CR_TC_CYCLES) != 0;
  if ((mode & ~(3 | CR_TC_CYCLES | CR_TC_TOP_F32 | CR_TC_SPLIT)) != 0 ||
      ((mode & 3) != CR_F64 && (mode & 3) != CR_MIXED) || (tc && (mode & 3) != CR_MIXED) ||
      ((mode & (CR_TC_TOP_F32 | CR_TC_SPLIT)) && !tc))
    return fail(CR_EINVAL, "cr_batch_create: mode must be CR_F64 or CR_MIXED (stationary, fixed count), "
                           "CR_TC_CYCLES only with CR_MIXED");
  cudaStream_t st = plans[0] ? plans[0]->stream : nullptr;
  if (!st) return fail(CR_EINVAL, "cr_batch_create: graph capture needs a created stream, not the default stream");
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || !plans[i]->hier) return fail(CR_EINVAL, "cr_batch_create: every plan needs levels");
    if (!plans[i]->hier->numeric_ready)
      return fail(CR_ESTATE, "cr_batch_create: a plan's C_l-dependent precompute was deferred");
    if (plans[i]->stream != st) return fail(CR_EINVAL, "cr_batch_create: plans must share one stream");
    if (nrhs[i] < 0) return fail(CR_EINVAL, "cr_batch_create: nrhs < 0");
  }
  const int fmode = (mode & 3) | CR_FIXED;
  // one uncaptured solve per plan first: it builds the tables created lazily
  // on first use, which must not be allocated inside the capture
  for (int i = 0; i < nplans; ++i) {
    plans[i]->tc_top_f32 = (mode & CR_TC_TOP_F32) != 0;
    plans[i]->tc_split = (mode & CR_TC_SPLIT) ? 1 : plans[i]->tc_split_param;
  }
  for (int i = 0; i < nplans; ++i) {
    if (nrhs[i] == 0) continue;
    int rc = tc ? solve_tc(plans[i], x[i], b[i], nrhs[i], 0.0, 1, true, nullptr, nullptr, nullptr)
                : solve(plans[i], x[i], b[i], 0.0, 1, fmode, nullptr, nullptr, nullptr);
    if (rc) {
      for (int k = 0; k < nplans; ++k) plans[k]->tc_split = plans[k]->tc_split_param;
      return rc;
    }
  }
  CR_CUDA(cudaStreamSynchronize(st));
  cr_batch* bt = new cr_batch();
  bt->stream = st;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    delete bt;
    for (int k = 0; k < nplans; ++k) plans[k]->tc_split = plans[k]->tc_split_param;
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  int rc = CR_OK;
  for (int i = 0; i < nplans && !rc; ++i) {
    const int64_t nlm = n_lm(plans[i]->lmax);
    plans[i]->capturing = true;
    if (tc && nrhs[i] > 0)
      rc = solve_tc(plans[i], x[i], b[i], nrhs[i], 0.0, cycles, true, nullptr, nullptr, nullptr);
    for (int j = 0; !tc && j < nrhs[i] && !rc; ++j)
      rc = solve(plans[i], (char*)x[i] + j * nlm * sizeof(double2), (const char*)b[i] + j * nlm * sizeof(double2), 0.0,
                 cycles, fmode, nullptr, nullptr, nullptr);
    plans[i]->capturing = false;
  }
  e = cudaStreamEndCapture(st, &bt->graph);
  for (int i = 0; i < nplans; ++i) plans[i]->tc_split = plans[i]->tc_split_param;
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
  if (!rc) {
    e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
  }
  if (!rc) {
    e = cudaGraphGetNodes(bt->graph, nullptr, &bt->nodes);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphGetNodes");
  }
  if (!rc && bt->nodes) {
    std::vector<cudaGraphNode_t> nodes(bt->nodes);
    size_t n = bt->nodes;
    e = cudaGraphGetNodes(bt->graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++bt->kernels;
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "graph node types");
  }
  if (rc) {
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    delete bt;
    return rc;
  }
  *out = bt;
  return CR_OK;
}

int cr_batch_run(cr_batch* bt) {
  if (!bt || !bt->exec) return fail(CR_EINVAL, "cr_batch_run: no batch");
  CR_CUDA(cudaGraphLaunch(bt->exec, bt->stream));
  return CR_OK;
}

int cr_batch_nodes(const cr_batch* bt, int64_t* nodes, int64_t* kernels) {
  if (!bt) return fail(CR_EINVAL, "cr_batch_nodes: null argument");
  if (nodes) *nodes = (int64_t)bt->nodes;
  if (kernels) *kernels = bt->kernels;
  return CR_OK;
}

int cr_batch_destroy(cr_batch* bt) {
  if (!bt) return CR_OK;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  delete bt;
  return CR_OK;
}

}  // extern "C"
