/*
 * cr.h -- C ABI of the GB300-native multi-level constrained-realization (CR)
 * solver for CMB skies (Seljebotn, Mardal, Jewell, Eriksen & Bull 2013,
 * "A multi-level solver for Gaussian constrained CMB realizations").
 *
 * The system solved is (Section 2.3, Eqs. system-explicit and cr-system)
 *     A x = b,   A = S^-1 + B Y^T N^-1 Y B,
 * with S = diag(C_l) the prior, B = diag(b_l p_l) the beam and pixel window,
 * N^-1 the per-pixel inverse noise (zero under the mask), Y spherical-harmonic
 * synthesis to the HEALPix observation grid and Y^T its transpose (adjoint
 * synthesis, Section 2.1 -- not analysis).
 *
 * Conventions shared by every entry point
 *  - Spherical-harmonic vectors ("alm") are complex, m >= 0 only, stored
 *    m-major with l = m..L contiguous: element (l, m) sits at
 *    off_m + (l - m), off_m = m (L + 1) - m (m - 1) / 2, N_lm = (L+1)(L+2)/2.
 *    Real and imaginary parts are interleaved (double2 / float2).  Im(a_l0)
 *    is not a degree of freedom: outputs write it as 0 and inputs ignore it.
 *    The inner product that makes Y^T the transpose of Y is
 *    <a,b> = sum_l a_l0 b_l0 + 2 sum_{m>0} Re(a_lm conj b_lm).
 *  - Coefficients whose C_l is 0 are not unknowns (the C_l -> 0 limit):
 *    operators write 0 there.
 *  - Maps are real, HEALPix RING order (or Gauss-Legendre ring order), north
 *    to south.
 *  - Units: uK for maps and alm, uK^2 for C_l, uK^-2 for N^-1.
 *  - All data pointers are DEVICE pointers owned by the caller unless a
 *    parameter says "host".  The plan owns only its own tables and
 *    workspace.  Calls are asynchronous on the plan's stream unless stated.
 *  - Every entry point returns an int status: CR_OK (0) or a negative error
 *    code; cr_last_error() gives a one-line message for the calling thread.
 *    An error leaves outputs undefined but the plan usable, except where
 *    noted.
 *  - dtype selects the arithmetic of a call: CR_F64 (double/double2 buffers)
 *    or CR_F32 (float/float2 buffers).
 */
#ifndef CR_H_
#define CR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CR_OK 0
#define CR_EINVAL (-1)     /* bad argument or size */
#define CR_ENOMEM (-2)     /* device or host allocation failed */
#define CR_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define CR_EICC (-4)       /* incomplete Cholesky failed even with the largest ridge */
#define CR_EDIVERGED (-5)  /* residual grew over two consecutive cycles */
#define CR_EMAXITER (-6)   /* iteration cap reached before the tolerance */
#define CR_ENONFINITE (-7) /* a NaN or Inf appeared in a vector */
#define CR_ESTATE (-8)     /* call not valid in the plan's current state */
#define CR_EIO (-9)        /* checkpoint file could not be read or written */

/* arithmetic of a call */
#define CR_F64 0
#define CR_F32 1
/* dtype of cr_sht_synth, cr_sht_adjoint and cr_apply_A (level 0): FP32 data
 * (complex64 alm, float32 maps), many right-hand sides, the Legendre
 * contractions on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation; 16 right-hand sides per launch): about BF16 accuracy (1e-2
 * relative) for batched throughput.  The call synchronises the plan's
 * stream to read the kernels' completion status (CR_ECUDA if a wait gave up). */
#define CR_TC 3
/* solve mode: FP32 W-cycles inside an FP64 iterative-refinement loop */
#define CR_MIXED 2
/* solve flag (or-ed with CR_F64 / CR_MIXED): flexible preconditioned CG with
 * one CR-Cycle as the preconditioner instead of repeated cycles */
#define CR_PCG 4
/* solve flag: run exactly max_cycles cycles with no stop test; in the
 * stationary form the residual after the last cycle (needed only by the
 * stop test) is not formed, so relres_out reports the residual before the
 * last cycle and the last history entry is NaN.  For timing a cycle count
 * found beforehand. */
#define CR_FIXED 8
/* solve flag: diagonal-preconditioned conjugate gradients on A instead of the
 * multi-level cycle (the comparison method of Sections 1 and 2.4), FP64 only,
 * needs no levels; max_cycles caps the CG iterations and cycles_out counts
 * them (one FP64 A per iteration). */
#define CR_CG 16
/* solve flag (with CR_MIXED, stationary): the FP32 cycles of up to 16
 * right-hand sides run together, every Legendre stage of the hierarchy (the
 * level operators and the pixel levels' transforms around the smoothers) as
 * one tensor-core contraction over the right-hand sides (BF16 operands, FP32
 * accumulation); the outer residual b - A x stays FP64 per right-hand side.
 * Also accepted by cr_batch_create. */
#define CR_TC_CYCLES 32
/* solve flag (with CR_TC_CYCLES): the top level's residuals (full band
 * limit, the most accuracy-sensitive step of the cycle) run per right-hand
 * side on the FP32 CUDA-core kernels; the pixel levels stay batched on the
 * tensor cores.  A replayed batch graph keeps the choice it was captured
 * with. */
#define CR_TC_TOP_F32 64
/* solve flag (with CR_TC_CYCLES): the cycles' tensor-core contractions with
 * hi + lo BF16 operands (three MMAs per step, about 2^-17 relative instead
 * of the 2^-9 of plain BF16), as the plan option tc_split does for every
 * tensor-core call.  Also accepted by cr_batch_create (a replayed graph
 * keeps the choice it was captured with). */
#define CR_TC_SPLIT 128

/* grid kinds */
#define CR_GRID_HEALPIX 0
#define CR_GRID_GL 1

/* grid selector of the transform entry points */
#define CR_OBS 0 /* the observation grid at the plan's lmax; level grids are CR_OBS + h, h >= 1 */

typedef struct cr_plan cr_plan;

/*
 * One spherical-harmonic level with its sibling pixel grid (Section 3.2):
 * HEALPix Nside_h (power of two, >= 8, <= the observation Nside), band limit
 * lmax_h (non-increasing from level to level), n_rec recursions into the
 * next coarser level, and the cumulative filter f^h_l (HOST [lmax + 1];
 * entries above lmax_h are ignored).
 */
typedef struct cr_level_spec {
  int nside_h;
  int lmax_h;
  int n_rec;
  const double* fl;
} cr_level_spec;

/*
 * Plan parameters.  struct_size must be sizeof(cr_params).
 *   grid_kind   CR_GRID_HEALPIX (nside, a power of two >= 1) or CR_GRID_GL
 *               (gl_ntheta rings at Gauss-Legendre nodes, gl_nphi pixels per
 *               ring, gl_nphi even).
 *   lmax        band limit L of the unknowns (>= 0).
 *   cl, bl      HOST arrays [lmax+1]: prior C_l (>= 0) and b_l p_l.  NULL cl
 *               means "transforms only" (no operator).  NULL bl means 1.
 *   ninv        DEVICE array [npix] of doubles, N^-1 per pixel (0 = masked),
 *               finite and >= 0 (else CR_EINVAL naming the first bad pixel).
 *               Copied into the plan at creation.  NULL means no noise term.
 *   stream      cudaStream_t for every call on this plan (NULL = default).
 */
typedef struct cr_params {
  int struct_size;
  int grid_kind;
  int nside;
  int gl_ntheta;
  int gl_nphi;
  int lmax;
  const double* cl;
  const double* bl;
  const double* ninv;
  void* stream;
  /* multi-level solver (needs cl).  nlevels: -1 = the default level table
   * (the paper's Planck table for Nside 2048 / lmax 3000, otherwise levels
   * from the power of two nearest lmax / 2.93 down to 8, with fourth-power
   * and Gaussian filters),
   * 0 = no levels (transforms and A only), > 0 = the `levels` array (fine to
   * coarse).  lmax_dense: band limit of the bottom dense level (-1: default
   * min(40, lmax_H / 2)).  ridge_factor (0: 1.5) and ridge_bisections
   * (0: 30) set the incomplete-Cholesky ridge search (Section 3.5);
   * ridge_alpha (HOST [nlevels], or NULL) fixes the ridges instead.
   * ridge_lambda_target (0: 1.5; < 0: off): after the ridge search the
   * ridge is raised further until a power-iteration estimate of the largest
   * eigenvalue of S_h A_h (smoother times level operator) is at most this
   * value, so that no error-smoothing step over-corrects (not applied when
   * ridge_alpha is given); the top-level diagonal smoother is scaled down to
   * the same bound when its estimate exceeds it. */
  int nlevels;
  const cr_level_spec* levels;
  int lmax_dense;
  double ridge_factor;
  int ridge_bisections;
  const double* ridge_alpha;
  double ridge_lambda_target;
  /* gl_downgrade (Section 3.4, Eqs. Ni-rewrite and Xi): a pixel level's
   * Y_obs^T N^-1 Y_obs at band limit lmax_h only sees the inverse-noise map
   * up to multipole 2 lmax_h, so it is applied on a Gauss-Legendre grid of
   * 2 lmax_h + 1 rings and a power-of-two nphi >= 4 lmax_h + 1 with the
   * quadrature-weighted map w_j (sum_{L<=2 lmax_h} xi_LM Y_LM)(n_j),
   * xi = Y_obs^T n: the same operator (exact by the Gaunt expansion, up to
   * rounding) at O(lmax_h^3) cost.  0 = on for levels whose GL grid has at
   * most 3/5 of the observation grid's rings, 1 = on for every pixel level,
   * -1 = off. */
  int gl_downgrade;
  /* fp64_df: 1 = evaluate the FP64 Legendre stages (FP64 transforms, FP64
   * A, the outer residual of CR_MIXED) in double-float arithmetic on the
   * FP32 pipes -- pairs of floats with error-free sums and products, about
   * 2^-44 relative per operation -- which GB300 runs several times faster
   * than native FP64; 0 = native FP64. */
  int fp64_df;
  /* defer_precompute: 1 = build the level structure (grids, tile patterns,
   * the observation-dependent inverse-noise terms) but not the
   * C_l-dependent numerical precompute (smoother factorisations with the
   * ridge search, top-level diagonal smoother, bottom dense inverse); fill
   * it in later with cr_load or cr_plan_update_cl.  Until then the solver
   * entry points return CR_ESTATE.  0 = run everything at creation. */
  int defer_precompute;
  /* autotune: 1 = run cr_plan_autotune at the end of creation. */
  int autotune;
  /* smoother of the pixel levels: 0 = multicolour block ICC(0) (Section
   * 3.5); 1 = additive Schwarz without overlap (block Jacobi): every tile is
   * a subdomain solved exactly, M = blockdiag(A_hat_pp + alpha I)^-1, applied
   * in one fully parallel pass -- the domain-decomposition smoother Section
   * 3.5 names as the parallel alternative.  The ridge alpha is found as for
   * ICC(0) (smallest alpha for which every block factorises, times
   * ridge_factor) and raised under ridge_lambda_target. */
  int smoother;
  /* triangular sweeps of the ICC(0) smoother: 0 = automatic (levels of at
   * most 1024 tiles, Nside_h <= 64, run both sweeps of one application in
   * one cooperative persistent launch, larger levels one launch per
   * colour); 1 = one launch
   * per colour on every level; 2 = the cooperative launch wherever the
   * device supports it.  The same operator either way. */
  int smoother_sweep;
  /* tensor-core contractions of batched right-hand sides (CR_TC, and the
   * cycles of CR_TC_CYCLES): 0 = BF16 operands (about 2^-9 relative per
   * product, FP32 accumulation); 1 = each operand carried as a BF16 pair
   * hi + lo and the product as A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs
   * per step, about 2^-17 relative). */
  int tc_split;
} cr_params;

/* One-line message describing the last error on the calling thread. */
const char* cr_last_error(void);

/*
 * Create a plan: ring geometry (Section 2.1; HEALPix pixel centres of
 * Gorski et al. 2005, or Gauss-Legendre nodes), Legendre recurrence tables,
 * per-ring FFT tables, and the operator diagonals.  Synchronous.  *out is set
 * only on success.  Errors: CR_EINVAL, CR_ENOMEM, CR_ECUDA.
 */
int cr_plan_create(cr_plan** out, const cr_params* p);

/*
 * Autotuner of the Legendre kernels (Section 2.1 transforms): times the
 * FP32 and FP64 synthesis and adjoint Legendre stages with 2, 4 and 8 ring
 * pairs per thread (the ring block of one CTA; 16 too for the FP32 adjoint),
 * each with the m tile 1 and 2 (one m per CTA, or m paired with L - m), on
 * every grid and band limit the plan transforms on, and keeps the fastest
 * shape.  Choices are cached for the process per (grid shape, band limit,
 * precision, stage) and used by every plan with those shapes; shapes already
 * in the cache are not re-timed.  Untuned shapes use 4 and 1.  *nentries (may be
 * NULL) receives the size of the cache.  Synchronous; a few seconds at
 * Nside 2048.  The batched tensor-core synthesis (16 right-hand sides) is
 * tuned too: its stage shape (variant 0: K 32 per parity, 2 pipeline
 * stages; 1: K 32, 3 stages; 2: K 16, 3 stages), cached with precision 2
 * and stage 2.  cr_tune_entry reads cache entry i (0 <= i < size): grid
 * ring and pixel counts, band limit, precision in bytes (4 or 8; 2 for the
 * tensor-core entries), stage (0 synthesis, 1 adjoint, 2 tensor-core
 * synthesis), the chosen pairs per thread (or variant), the chosen m tile
 * (1: one m per CTA; 2: each CTA takes m and L - m, so that every CTA has
 * about the same l range; 1 for the tensor-core entries) and the measured
 * ms (HOST [8]; -1 where there is no such choice): choices 2, 4, 8, 16 pairs
 * per thread with m tile 1, then the same with m tile 2 (tensor-core
 * entries: variants 0, 1, 2 in the first three); any output may be NULL.
 * Errors: CR_EINVAL, CR_ECUDA.
 */
int cr_plan_autotune(cr_plan* plan, int* nentries);
int cr_tune_entry(int i, int* nring, int64_t* npix, int* lmax, int* precision_bytes, int* stage, int* rp,
                  int* m_tile, double* ms);
/* Pin the choice for one (grid shape, band limit, precision, stage): rp 2,
 * 4 or 8, or 16 for the FP32 adjoint, with m tile 1 or 2; precision 2 with
 * stage 2: the tensor-core synthesis variant 0, 1 or 2 (m tile 1).  Errors:
 * CR_EINVAL. */
int cr_tune_set(int nring, int64_t npix, int lmax, int precision_bytes, int stage, int rp, int m_tile);

/*
 * Replace the prior C_l of a plan (HOST [lmax + 1], finite, >= 0) and redo
 * only the precompute that depends on it (Section 5): the diagonals S^-1 and
 * B, the level operators' D_h, each pixel level's prior term of the
 * assembled block matrix (its inverse-noise term is kept unless the set of
 * l with C_l > 0 changes), the ridge search and incomplete-Cholesky
 * factorisation, the top-level diagonal smoother and the bottom dense
 * inverse.  Device arrays are rewritten in place, so CUDA graphs of
 * cr_batch_create stay valid unless the set of l with C_l > 0 changes.
 * Synchronous.  Errors: CR_EINVAL (null, bad C_l; the plan is unchanged),
 * CR_ESTATE (plan created without C_l), CR_EICC, CR_ECUDA (after which the
 * solver entry points return CR_ESTATE until a successful update or load).
 */
int cr_plan_update_cl(cr_plan* plan, const double* cl);

/*
 * Checkpoint of the C_l-dependent numerical precompute (Section 5: the
 * precomputed smoothers are normally read from disk).  cr_save writes, to
 * the file `path`, each pixel level's ridge and block incomplete-Cholesky
 * factor, the top-level diagonal smoother, and the bottom dense matrix and
 * its inverse, after a header identifying the plan (grid, band limits,
 * level table, tile-pattern sizes) and 64-bit FNV-1a hashes of C_l, b_l and
 * the N^-1 map, and followed by a hash of the whole file.  cr_load reads
 * such a file into a plan built from the same inputs, normally created with
 * defer_precompute = 1, and makes it ready to solve; solutions then equal
 * those of the plan that was saved.  Both synchronous.  Errors: CR_EINVAL
 * (null argument, plan without levels, a checkpoint made for other inputs),
 * CR_ESTATE (cr_save before the precompute), CR_EIO (cannot open, read or
 * write; not a checkpoint; truncated; checksum mismatch -- the plan is then
 * unchanged), CR_ECUDA.
 */
int cr_save(cr_plan* plan, const char* path);
int cr_load(cr_plan* plan, const char* path);

/* Grid on which pixel level h (1..nlevels) applies its inverse-noise term:
 * *kind = CR_GRID_HEALPIX (the observation grid) or CR_GRID_GL (the
 * downgraded grid of gl_downgrade), with its ring and pixel counts.  Any
 * output pointer may be NULL.  Errors: CR_EINVAL (no levels, h out of
 * range). */
int cr_plan_level_grid(const cr_plan* plan, int h, int* kind, int* nring, int64_t* npix);

/*
 * Right-hand side of the CR system (Section 2.3, Eq. system-explicit and the
 * constrained-realization construction it cites):
 *   b = B Y^T N^-1 d + S^-1/2 omega_1 + B Y^T N^-1/2 omega_2
 * with omega_1 ~ N(0, I) in the real orthonormal coefficient basis and
 * omega_2 ~ N(0, I) per pixel (N^-1/2 = 0 under the mask); without
 * CR_DRAW_FLUCT only the Wiener-filter term is formed.  d: device FP64
 * [nrhs][npix] RING map, or NULL for d = 0.  b: device FP64 complex
 * [nrhs][N_lm(lmax)], overwritten (0 at C_l = 0, Im a_l0 = 0).  Normals come
 * from Philox4x32-10 (Salmon et al. 2011) keyed by `seed`: element k of
 * stream s (3 = omega_1 at k = 2 i + part of coefficient i, 4 = omega_2 at
 * pixel k) for right-hand side j uses counter (k >> 2, k >> 34, s, j) and
 * Box-Muller slot k & 3.  Allocates one FP64 map for the call; synchronous.
 * Errors: CR_EINVAL (no C_l in the plan, bad flag), CR_ECUDA.
 */
#define CR_DRAW_FLUCT 1
/* CR_DRAW_PLAIN: the data term is B Y^T d (no N^-1), e.g. for trace probes */
#define CR_DRAW_PLAIN 2
int cr_draw(cr_plan* plan, uint64_t seed, const void* d, void* b, int nrhs, int flags);

/*
 * Gradient contractions for differentiating the solve of Section 2.3 (A is
 * symmetric, so the adjoint lambda = A^-1 g is another CR-Solve).
 * cr_grad_cl: out[l] = alpha C_l^-2 <u, v>_l + beta C_l^-3/2 <u, w1>_l
 *   + kappa (2l+1) / C_l for l = 0..lmax (0 where C_l = 0), <.,.>_l the real
 *   inner product restricted to multipole l and w1 the constrained-realization
 *   normals of cr_draw (seed, right-hand side rhs) in complex storage.  u, v:
 *   device FP64 complex [N_lm] (v may be NULL: its term is 0); out: device
 *   FP64 [lmax+1], overwritten, or added to when accumulate != 0.
 *   A realization x = A^-1 b with loss gradient g uses (u, v) = (A^-1 g, x),
 *   alpha = 1, beta = -1/2; the Wiener-filter data term uses u = v = A^-1 b,
 *   alpha = 1/2, beta = 0.
 * cr_grad_ninv: out_i = alpha p_i q_i + p_i (gamma d_i + delta w2_i / sqrt n_i)
 *   + eps d_i^2 + kappa / n_i with p = Y B u, q = Y B v synthesised in FP64
 *   (v may be NULL: q = 0), w2 the pixel normals of cr_draw, n the plan's
 *   N^-1 (the w2 and 1/n terms only where n_i > 0); d: device FP64 [npix] or
 *   NULL; out: device FP64 [npix], overwritten or accumulated.  Realization:
 *   alpha = -1, gamma = 1, delta = 1/2, eps = 0; Wiener-filter data term:
 *   u = v = A^-1 b, alpha = -1/2, gamma = 1, delta = 0, eps = -1/2.
 *   Allocates two FP64 maps for the call.
 * Log-determinant part of the Wiener-filter log-likelihood,
 *   -1/2 ln det M = -1/2 (ln det N + ln det S + ln det A) (determinant lemma):
 *   d/dC_l = -1/2 ((2l+1)/C_l - C_l^-2 tr_l A^-1), d/dn_i = -1/2 (-1/n_i +
 *   (Y B A^-1 B Y^T)_ii), the traces by Hutchinson estimates over Rademacher
 *   probes z (cr_probe CR_PROBE_ALM: <z, A^-1 z>_l) and w (CR_PROBE_MAP:
 *   (Y B A^-1 B Y^T w)_i w_i, with B Y^T w from cr_draw CR_DRAW_PLAIN).
 * cr_probe: Rademacher probe j: CR_PROBE_ALM a complex [N_lm] vector in the
 *   real orthonormal basis (0 at C_l = 0), CR_PROBE_MAP an FP64 [npix] map
 *   (0 where n_i = 0); element k of stream 5 (coefficients, k = 2 i + part)
 *   or 6 (pixels) takes word k & 3 of Philox4x32-10 at counter
 *   (k >> 2, k >> 34, stream, j), sign + for an even word.
 * cr_map_wdot: *out = sum_i n_i a_i b_i (host result; a, b device FP64 maps).
 * cr_alm_dot: *out = <u, v> (real inner product, S^-1-weighted if weighted).
 * All synchronous.  Errors: CR_EINVAL (null pointers, plan without C_l),
 * CR_ECUDA.
 */
int cr_grad_cl(cr_plan* plan, const void* u, const void* v, double alpha, double beta, double kappa, uint64_t seed,
               int rhs, int accumulate, double* out);
int cr_grad_ninv(cr_plan* plan, const void* u, const void* v, const double* d, double alpha, double gamma,
                 double delta, double eps, double kappa, uint64_t seed, int rhs, int accumulate, double* out);
#define CR_PROBE_ALM 0
#define CR_PROBE_MAP 1
int cr_probe(cr_plan* plan, uint64_t seed, int kind, int j, void* out);
int cr_map_wdot(cr_plan* plan, const double* a, const double* b, double* out);
int cr_alm_dot(cr_plan* plan, const void* u, const void* v, int weighted, double* out);

/*
 * Batched realizations in one CUDA graph.  cr_batch_create captures, on the
 * plans' common stream, the fixed-count CR-Solve (max_cycles = cycles, no
 * stop test) of nrhs[i] right-hand sides for every plan i -- plans may have
 * different resolutions -- after one uncaptured solve per plan (which builds
 * tables created on first use), and instantiates the graph.  x[i], b[i]:
 * device FP64 complex [nrhs[i]][N_lm(lmax_i)]; the buffers are bound into
 * the graph, so later runs read b and write x at the same addresses.  mode:
 * CR_F64 or CR_MIXED (stationary), or CR_MIXED | CR_TC_CYCLES (the cycles of
 * each plan's right-hand sides batched 16 at a time on the tensor cores; a
 * completion wait that gives up inside a replay is reported by the plan's
 * next uncaptured tensor-core call).  cr_batch_run launches the graph on that
 * stream (asynchronous); replays give results identical to the uncaptured
 * solves.  cr_batch_nodes: number of graph nodes (kernels and copies) and of
 * kernel nodes (either pointer may be NULL).
 * Errors: CR_EINVAL (plans without levels, on different streams or on the
 * legacy default stream, which cannot be captured; bad mode), CR_ECUDA.  The
 * plans must outlive the batch.
 */
typedef struct cr_batch cr_batch;
int cr_batch_create(cr_batch** out, int nplans, cr_plan* const* plans, void* const* x, const void* const* b,
                    const int* nrhs, int cycles, int mode);
int cr_batch_run(cr_batch* batch);
int cr_batch_nodes(const cr_batch* batch, int64_t* nodes, int64_t* kernels);
int cr_batch_destroy(cr_batch* batch);

/*
 * Tensor-core self-test: one 128 x 32 x K tile (K in {16, 32, 48, 64}) of
 * BF16 products accumulated in FP32 tensor memory by tcgen05.mma, against the
 * same product on the CUDA cores; *max_abs_err receives the largest
 * difference (0 for a correct tile: the inputs are small integers).  Errors:
 * CR_EINVAL (bad K), CR_ECUDA (including a completion wait that gave up).
 */
int cr_tc_selftest(int K, float* max_abs_err);
/* The same tile with both operands in the MN-major (transposed) layout
 * without swizzle, the layout the batched adjoint writes: core matrices of
 * 8 K rows x 8 MN elements, 128 bytes apart along MN and (MN / 8) * 128
 * bytes apart along K.  swap = 0 passes the MN stride as the descriptor's
 * leading byte offset and the K stride as its stride byte offset, swap = 1
 * the other way round (the operand buffers are large enough for either);
 * swap = 1 is the reading the hardware uses for this layout (exact on
 * GB300), and the batched adjoint's descriptors follow it.
 * Errors: CR_EINVAL, CR_ECUDA. */
int cr_tc_selftest_mn(int K, int swap, float* max_abs_err);

/*
 * Arithmetic peak probe (measurement tooling, no counterpart in the paper):
 * the sustained FMA rate of one pipe on the current device, in TFLOP/s
 * (2 flop per FMA), timed with CUDA events on the default stream as the best
 * of five launches of independent FMA chains that fill every SM.
 *   kind 0: FP32 scalar FMA; 1: FP32 packed pairs (fma.rn.f32x2);
 *   2: FP64 FMA.
 * These are the denominators of the Legendre stages' rooflines (they are
 * bound by the FMA pipes, not by HBM or a dense contraction).  Allocates and
 * frees a small output buffer.  Errors: CR_EINVAL, CR_ECUDA.
 */
int cr_probe_fma_peak(int kind, double* tflops);

/* Release every resource of the plan (NULL is accepted). */
int cr_plan_destroy(cr_plan* plan);

/* Sizes: pixels of grid `grid` (CR_OBS or level), rings, and N_lm at that
 * grid's band limit.  Any output pointer may be NULL. */
int cr_plan_sizes(const cr_plan* plan, int grid, int64_t* npix, int* nring, int* lmax, int64_t* nlm);

/*
 * Spherical-harmonic synthesis, map = Y alm (Section 2.1, Eq. sh-synthesis):
 *   map(n_i) = sum_{l<=L, |m|<=l} a_lm Y_lm(n_i),  real field.
 * alm: [nrhs][N_lm] complex; map: [nrhs][npix] real; dtype CR_F64, CR_F32
 * or CR_TC.
 * Band limits above what a ring resolves alias by folding m mod n_ring, so
 * Y^T below stays its exact transpose.
 */
int cr_sht_synth(cr_plan* plan, int grid, const void* alm, void* map, int nrhs, int dtype);

/*
 * Adjoint synthesis, alm = Y^T map (Section 2.1: the transpose of Y, with no
 * quadrature weights):  a_lm = sum_i conj(Y_lm(n_i)) map_i.
 * map: [nrhs][npix]; alm: [nrhs][N_lm] (overwritten); dtype CR_F64, CR_F32
 * or CR_TC.
 */
int cr_sht_adjoint(cr_plan* plan, int grid, const void* map, void* alm, int nrhs, int dtype);

/*
 * y = A x with A = S^-1 + B Y^T N^-1 Y B (Section 2.3, Eq. system-explicit):
 * one synthesis, the pixel-diagonal N^-1, one adjoint synthesis and the
 * diagonals.  level 0 is the full system; level h >= 1 applies the level
 * operator A_h = D_h + B_h Y^T N^-1 Y B_h (Section 3.2, Eq. A_h) at that
 * level's band limit.  x, y: [nrhs][N_lm]; x and y must not overlap.
 * dtype CR_F64, CR_F32, or at level 0 CR_TC (batched, tensor cores).  With
 * CR_F64 at level 0 and several right-hand sides the two Legendre stages run
 * 8 right-hand sides at a time (one evaluation of the recurrence for all of
 * them; the same FP64 operator, summed in another order).
 * Requires a plan created with cl.  Errors: CR_EINVAL, CR_ESTATE, CR_ECUDA.
 */
int cr_apply_A(cr_plan* plan, int level, const void* x, void* y, int nrhs, int dtype);

/*
 * Multi-level solver (Section 3.2, Fig. code:mg).  Levels are numbered
 * h = 0 (top, lmax, diagonal smoother), 1..H (pixel levels), H + 1 (bottom
 * dense level).  Vectors of level h use that level's band limit lmax_h.
 * All entry points below need a plan created with levels; a dtype argument
 * is CR_F64 or CR_F32 (anything else: CR_EINVAL).
 */
/* Number of pixel levels H. */
int cr_plan_nlevels(cr_plan* plan, int* H);
/* Level h: pixel grid Nside_h (0 for the top and bottom), lmax_h, n_rec,
 * the cumulative filter (HOST out [lmax + 1]), the ridge alpha used by its
 * incomplete Cholesky (for h = 0: the damping factor applied to the
 * diagonal smoother) and the estimate of lambda_max(S_h A_h) (for h >= 1
 * after the ridge adjustment; for h = 0 before damping; 0 when not
 * estimated).  Any output pointer may be NULL. */
int cr_plan_level(cr_plan* plan, int h, int* nside_h, int* lmax_h, int* n_rec, double* fl, double* ridge,
                  double* lambda_max);
/* y = A_h x, A_h = D_h + B_h Y^T N^-1 Y B_h (Eq. A_h); h = 0 is A. */
int cr_level_apply(cr_plan* plan, int h, const void* x, void* y, int dtype);
/* r_H = I_h^H r_h: diagonal f^{h+1}/f^h, truncated at lmax_{h+1} (Eq. f_l). */
int cr_restrict(cr_plan* plan, int h, const void* r_h, void* r_H, int dtype);
/* x_h += (I_h^H)^T c_H (interpolation = transposed restriction). */
int cr_prolong_add(cr_plan* plan, int h, const void* c_H, void* x_h, int dtype);
/* c = S_h(r), the error-smoothing correction of level h for residual r:
 * h = 0: (1 - f^1) diag(A)^-1 r (Section 3.2);  h >= 1: Y_h^T M_h Y_h r with
 * M_h the block incomplete-Cholesky smoother (Section 3.5, Eqs.
 * pixel-correction-1..3), or the additive Schwarz smoother of the plan
 * option `smoother`.  c is overwritten. */
int cr_smooth(cr_plan* plan, int h, const void* r, void* c, int dtype);
/* map_out = M_h map_in for nrhs maps (1 <= nrhs <= 16) of pixel level h >= 1:
 * the pixel-space smoother of Section 3.5 (Eqs. pixel-correction-2, the
 * block incomplete-Cholesky solve L^-T L^-1 in the tiles' elimination
 * order, or the additive Schwarz form).  map_in, map_out: DEVICE
 * [nrhs][12 nside_h^2], RING order of the level's grid, FP32 or FP64 (the
 * factor is FP32).  With several maps every factor block is read once for
 * all of them (the form the batched cycles use).  Errors: CR_EINVAL,
 * CR_ESTATE, CR_ECUDA. */
int cr_pixel_smoother(cr_plan* plan, int h, const void* map_in, void* map_out, int nrhs, int dtype);
/* x = A_bottom^-1 b on the bottom level (l <= lmax_dense), dense (FP64). */
int cr_bottom_solve(cr_plan* plan, const void* b, void* x, int dtype);
/* The assembled real-basis matrix of the bottom level (before factorising):
 * A_bottom = D + B (Y^T N^-1 Y) B over the active real dofs with l <= lmax_dense,
 * from the ring formula (Section 3.3, Eq. Ni-dense).  Dof order: a_l0 for
 * l = 0..lmax_dense, then (sqrt2 Re a_lm, sqrt2 Im a_lm) for m >= 1 in storage
 * order, inactive (C_l = 0) dofs removed.  *nd receives the dimension; host
 * (may be NULL) receives nd x nd doubles, row-major. */
int cr_bottom_matrix(cr_plan* plan, double* host, int* nd);
/* One CR-Cycle from the top level, improving x in place for right-hand
 * side b (Fig. code:mg).  x, b: [nrhs][N_lm(lmax)]. */
int cr_wcycle(cr_plan* plan, void* x, const void* b, int nrhs, int dtype);
/*
 * CR-Solve (Fig. code:mg): x = 0, repeat CR-Cycle and r = b - A x until
 * r^T S^-1 r < eps b^T S^-1 b (eps = 1e-12 is a 1e-6 relative residual).
 * x, b: FP64 [nrhs][N_lm(lmax)].  mode CR_F64: every cycle in FP64;
 * CR_MIXED: each cycle in FP32 applied to the FP64 residual (iterative
 * refinement; the residual r = b - A x is always FP64).  Or-ed with CR_PCG:
 * flexible preconditioned CG (Polak-Ribiere beta) whose preconditioner is
 * one CR-Cycle from zero, in the chosen precision, with A and the residual in
 * FP64; one cycle and one FP64 A per iteration.  Outputs (may be
 * NULL): cycles_out[nrhs], relres_out[nrhs] (final sqrt of the ratio),
 * history[nrhs][max_cycles] (relative residual after each cycle).
 * Further flags: CR_FIXED (exactly max_cycles cycles, no stop test),
 * CR_CG (diagonal-preconditioned CG instead of the cycles; needs no levels),
 * CR_TC_CYCLES with CR_MIXED (the FP32 cycles of up to 16 right-hand sides
 * batched on the tensor cores; CR_TC_TOP_F32 keeps the top level's
 * residuals on the CUDA cores).
 * Errors: CR_EDIVERGED (residual grew over two consecutive cycles),
 * CR_EMAXITER, CR_ENONFINITE; x holds the last iterate in each case.
 * CR_ESTATE: the plan was created with defer_precompute and has not been
 * loaded or updated since.
 */
int cr_solve(cr_plan* plan, void* x, const void* b, int nrhs, double eps, int max_cycles, int mode, int* cycles_out,
             double* relres_out, double* history);

/*
 * Per-stage timing (the per-level, per-action cost breakdown of the paper's
 * Table "cycle-cost"): while enabled, every kernel stage launched by the plan
 * is bracketed by CUDA events on the plan's stream and accumulated by stage
 * name.  cr_plan_set_timing(plan, 1) clears and enables, 0 disables.
 * cr_plan_timing synchronises the recorded events and reports stage i
 * (0 <= i < *count) in name order: its name (NUL-terminated, truncated to
 * name_cap; transform stages carry a _f64 / _f32 suffix), total
 * milliseconds, number of recorded scopes, and the algorithmic work of those
 * scopes (flops for the Legendre stages: 8 per ring pair and (l, m); bytes
 * for the pixel smoother: the factor blocks read twice; 0 where not
 * defined); i < 0 only sets *count.  Any output pointer may be NULL.
 */
int cr_plan_set_timing(cr_plan* plan, int enable);
/* Number of kernels the library has launched in this process on the
 * transform, operator, smoother and solver paths (plan-time table builders
 * excluded); the difference across a region counts its launches. */
long cr_launch_count(void);
int cr_plan_timing(cr_plan* plan, int i, char* name, int name_cap, double* ms, long* launches, double* work,
                   int* count);
/* The executed work of stage i (same order as cr_plan_timing): for the
 * Legendre stages, 8 flops per (ring pair, l, m) term the kernels evaluate,
 * i.e. only the terms at or past each (m, ring pair)'s start in the 2^-60
 * start table (the dense count of cr_plan_timing credits the skipped region
 * below the turning point too); 0 for stages without a flop count.
 * Errors: CR_EINVAL. */
int cr_plan_timing_exec(cr_plan* plan, int i, double* work_exec);

/*
 * Allocation-free synthesis (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc at all -- code running while a CUDA
 * graph is captured, allocator callbacks, real-time loops, or code working
 * inside a device-memory budget owned by another framework -- and therefore
 * cannot create a plan: map = Y alm in FP64 on the HEALPix grid of `nside`
 * (RING order) at band limit `lmax`, the same operation and layouts as
 * cr_sht_synth with dtype CR_F64, but with no plan and no allocation.
 *   alm   DEVICE [N_lm(lmax)] double2 (16-byte aligned), input.
 *   map   DEVICE [12 nside^2] double, output.
 *   stream  cudaStream_t (NULL = default stream).
 * The library's only scratch for this call is a fixed 16 MiB device array in
 * the library itself, so (4 nside - 1)(lmax + 1) * 16 bytes must not exceed
 * 16 MiB (e.g. nside 256 with lmax <= 1023); larger sizes return CR_EINVAL.
 * The array exists on every GPU that loads the library until the process
 * exits.  The first call on a device looks up the array's device address
 * (with that device current); make that first call before any stream
 * capture.  The address is looked up again when the device's context has
 * been rebuilt (after cudaDeviceReset), so the call after a reset is again
 * a "first call".  lmax is at most 16384, as for a plan.  All calls share the one array: calls that overlap on the GPU
 * (different streams, or different host threads on the same device) race, so
 * serialise them.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.  Errors: CR_EINVAL, CR_ECUDA.
 */
int cr_sht_synth_noalloc(int nside, int lmax, const void* alm, void* map, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CR_H_ */
