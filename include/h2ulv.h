/*
 * h2ulv.h -- C ABI of the GB300 H^2-ULV dense solver.
 *
 * The library solves A x = b for a dense kernel matrix A_ab = G(p_a, p_b)
 * over 3-D points, following Ma & Yokota, "An inherently parallel H^2-ULV
 * factorization for solving dense linear systems on GPUs" (arXiv 2502.02395):
 *
 *   h2_build   compresses A into an H^2 matrix whose shared bases also span
 *              the factorization's fill-ins (Algorithm 1, Section 3.4-3.5).
 *   h2_factor  the level-by-level ULV factorization (Algorithm 2 / 4,
 *              Section 3.6), every level one wide batch on the GPU.
 *   h2_solve   forward/backward substitution in the parallel product form of
 *              Eq. 24-31 (Section 3.7), wrapped in iterative refinement whose
 *              residual is the H^2 matrix-vector product to FP64 accuracy.
 *   h2_matvec  y = A_H2 x in FP64.
 *
 * Conventions (all entry points):
 *   - Vectors are in the caller's original point order; the tree permutation
 *     stays inside the library.
 *   - A pointer argument may be host or device memory unless stated;
 *     the library tells them apart with cudaPointerGetAttributes.
 *   - The context owns all device memory it allocates; the caller owns every
 *     buffer it passes.  The library copies what it keeps.
 *   - Work is issued on the context's stream (h2_set_stream; default: the
 *     legacy default stream).  Calls that return results to host memory
 *     synchronise that stream.
 *   - Every call returns an h2_status.  On failure h2_last_error(ctx) gives a
 *     one-line reason (for H2_ERR_SINGULAR: the level and box).
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef H2ULV_H
#define H2ULV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_ctx h2_ctx;

typedef enum {
  H2_OK = 0,
  H2_ERR_INVALID_ARG = -1,   /* a size, pointer or parameter is out of range */
  H2_ERR_OOM = -2,           /* device or host allocation failed            */
  H2_ERR_SINGULAR = -3,      /* a zero pivot in an LU (level and box in the message) */
  H2_ERR_NOT_CONVERGED = -4, /* refinement stopped at max_iters above target */
  H2_ERR_CUDA = -5,          /* a CUDA runtime call failed                  */
  H2_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up          */
  H2_ERR_STATE = -7          /* call out of order (e.g. solve before factor) */
} h2_status;

/* Kernel functions G(x, y).  The diagonal entry (a == b, the same point)
 * is listed after each formula.  eps, ell and diag_shift come from h2_params.
 *   H2_K_LAPLACE_EPS   1/(r + eps);           diagonal 1/eps + diag_shift
 *   H2_K_YUKAWA_EPS    exp(-r)/(r + eps);     diagonal 1/eps + diag_shift
 *   H2_K_GAUSSIAN      exp(-r^2/ell^2);       diagonal 1 + diag_shift
 *   H2_K_LAPLACE_PAPER 1/r (Eq. 35);          diagonal 1e3 + diag_shift
 *   H2_K_YUKAWA_PAPER  exp(-r)/r (Eq. 36);    diagonal 1e3 + diag_shift
 *   H2_K_POLY2_TEST    (1 + x.y)^2;           diagonal (1+|x|^2)^2 + diag_shift (1+|x|^2)
 *                      (every off-diagonal block has rank <= 10: a test kernel) */
typedef enum {
  H2_K_LAPLACE_EPS = 0,
  H2_K_YUKAWA_EPS = 1,
  H2_K_GAUSSIAN = 2,
  H2_K_LAPLACE_PAPER = 3,
  H2_K_YUKAWA_PAPER = 4,
  H2_K_POLY2_TEST = 5
} h2_kernel;

/* The problem statement of Section 3 and Section 6: kernel function, leaf
 * size, admissibility eta (Section 6.2: boxes i != j are well separated when
 * |c_i - c_j| > eta (R_i + R_j), c the centre and R the half-diagonal of the
 * tight bounding box; eta = 0 gives HSS, Section 6.3), truncation tolerance
 * (relative to the largest pivot of each box's composite matrix, Section 3.4),
 * a rank cap (0: half the level's box dimension; Section 4.1 pads every box
 * of a level to one rank) and the far/near sample sizes of Algorithm 1
 * (<= 0: no sampling). */
typedef struct {
  int32_t kernel;      /* h2_kernel */
  double eps;          /* softening of the *_EPS kernels (e.g. 1e-3) */
  double ell;          /* Gaussian length scale */
  double diag_shift;   /* added to the diagonal as described above */
  int32_t leaf_size;   /* 1..1024: maximum points per leaf box */
  double eta;          /* >= 0 */
  double tol;          /* > 0 */
  int32_t max_rank;    /* >= 0 */
  int32_t far_samples; /* far-field sample size per box */
  int32_t near_samples;/* sample size per close box */
} h2_params;

/* Arithmetic of the factorization (Algorithm 4), of the substitution
 * (Eq. 24-31) and of the refinement around it.
 *   H2_PREC_FP64   FP64 everywhere (the plain H^2-ULV): complement bases,
 *                  projection, LU and inverse of Ahat_ii^RR, Schur update,
 *                  couplings, merge and substitution; the refinement's
 *                  residual and update in FP64.
 *   H2_PREC_FP16   the projection U_i^T A_ij U_j and the couplings
 *                  T_i S_ij T_j^T on the tensor cores with FP16 operands
 *                  (scaled by powers of two) and FP32 accumulation; the
 *                  complement bases (Householder QR), the Schur update and
 *                  the merge in FP32; the inverse of Ahat_ii^RR by FP32
 *                  Gauss-Jordan elimination with partial pivoting (default)
 *                  or by FP64 partial-pivot elimination rounded once to FP32
 *                  (h2_set_option H2_OPT_RR_LU_FP64 = 1).  The substitution
 *                  reads 16-bit RR/RS/SR quadrants and FP32 bases and
 *                  inverses.  Refinement (scheme 2 of h2_solve): the
 *                  residual b - A_H2 x with each FP64 matrix entry held as
 *                  two FP32 numbers and FP32-pair sums (about 2^-46
 *                  relative per product sum; default) or with FP64
 *                  instructions (H2_OPT_RESIDUAL_FP64 = 1); the update
 *                  x += d in FP64; the inner FGMRES in FP32.
 *   H2_PREC_BF16   as FP16 with BF16 operands. */
typedef enum { H2_PREC_FP64 = 0, H2_PREC_FP16 = 1, H2_PREC_BF16 = 2 } h2_prec;

/* An H^2 instance given as plain host arrays (for h2_import).  Layouts:
 *   points        N x 3 row-major, original order
 *   perm          N: original index of tree position t
 *   leaf_offsets  2^L + 1: leaf box i holds tree positions
 *                 [leaf_offsets[i], leaf_offsets[i+1])
 *   D, K          L + 1 each: box dimension and rank of every level
 *                 (D[L] >= every leaf size, D[l] = 2 K[l+1] for l < L,
 *                 K[0] = 0)
 *   n_near[l], near[l]  ordered near pairs (i, j) of level l, 2 int32 each,
 *                 sorted by (i, j); level 0 is {(0, 0)}
 *   n_far[l], far[l]    ordered far (admissible) pairs of level l
 *   X[l]          l >= 1: 2^l x D[l] x K[l] row-major ID basis of each box
 *                 (rows beyond a leaf box's point count are zero)
 *   SK[l]         l >= 1: 2^l x K[l] original point index of each skeleton
 * X[0] and SK[0] are ignored. */
typedef struct {
  int64_t N;
  int32_t L;
  const double* points;
  const int64_t* perm;
  const int64_t* leaf_offsets;
  const int32_t* D;
  const int32_t* K;
  const int64_t* n_near;
  const int32_t* const* near;
  const int64_t* n_far;
  const int32_t* const* far;
  const double* const* X;
  const int64_t* const* SK;
} h2_instance;

/* Build the H^2 matrix of the N points (host, N x 3 row-major) with the
 * construction of Algorithm 1 including the pre-factorization basis
 * (Section 3.4-3.5): cluster tree, near/far lists, interpolative
 * decomposition of [G(B_i, S_F) | G(B_i, S_C) G(S_C, S_C)^-1] per box, dense
 * near blocks at the leaves and couplings G(SK_i, SK_j).  The tree, lists and
 * IDs are computed on the host; kernel blocks are evaluated on the GPU.
 * On success *out owns the instance.  Errors: H2_ERR_INVALID_ARG (N < 1,
 * leaf_size < 1, eta < 0, tol <= 0, a non-finite coordinate, unknown
 * kernel), H2_ERR_OOM, H2_ERR_CUDA.  Every box dimension (leaf size, or twice
 * the children's rank above the leaves) must stay <= 1024. */
h2_status h2_build(h2_ctx** out, const h2_params* p, const double* points, int64_t N);

/* Depth L of the cluster tree h2_build makes for N points and the given
 * leaf size: the smallest L with leaf_size * 2^L >= N.  -1 for N < 1 or
 * leaf_size < 1. */
int32_t h2_tree_depth(int64_t N, int32_t leaf_size);

/* Several independent systems as one instance (a forest; no counterpart in
 * the paper): each system's H^2 matrix is built as by h2_build with the
 * same parameters p (points[k]: N[k] x 3 row-major, host), and the trees,
 * which must all have the same depth L >= 1 (h2_tree_depth), are laid side
 * by side: system k holds boxes [k 2^l, (k + 1) 2^l) of level l, so every
 * level's batched kernels cover all systems in one launch and the root
 * level has one block per system (count roots factored by one batched
 * launch).  The systems share p (a Gaussian batch with per-system length
 * scales passes points divided by l_k and ell = 1: the matrix depends on
 * |x - y| / l only).  Every level has one rank for all systems, the
 * largest of the systems' tolerance ranks: the systems below it are
 * compressed again at that rank (the pivoted QR's leading pivots), and
 * every leaf is padded to the largest leaf with padding points (1 on the
 * diagonal), as a single instance pads its own leaves.
 * A_H2 is then block diagonal with the systems' own H^2 matrices as its
 * blocks; vectors are the systems' vectors concatenated in input order.
 * Errors: as h2_build; H2_ERR_INVALID_ARG also for count < 1 or depths that
 * differ or are 0 (h2_last_error(NULL) names the system). */
h2_status h2_build_forest(h2_ctx** out, const h2_params* p, const double* const* points, const int64_t* N,
                          int32_t count);

/* Plan without a GPU: run the host part of h2_build (cluster tree, near/far
 * lists and the interpolative decompositions of Algorithm 1) and write a
 * JSON summary to json (cap bytes including the terminating zero): N, L and
 * per level the box count, dimension D, rank K, near and far pair counts, the
 * largest per-box tolerance rank, and the device bytes h2_build and one
 * factorization would allocate.  Errors: as h2_build (H2_ERR_INVALID_ARG
 * also when cap is too small). */
h2_status h2_plan(const h2_params* p, const double* points, int64_t N, char* json, size_t cap);

/* Create a context from an H^2 instance built elsewhere (the same layout
 * h2_build produces internally).  The library evaluates the dense leaf
 * blocks and the couplings G(SK_i, SK_j) itself from the points and p.
 * Errors: as h2_build, plus H2_ERR_INVALID_ARG for inconsistent sizes. */
h2_status h2_import(h2_ctx** out, const h2_params* p, const h2_instance* inst);

/* The ULV factorization, Algorithm 4 with partial-pivot LU of the redundant
 * blocks, level by level from the leaves (Section 3.6):
 *   complement bases U_i = [U_i^R U_i^S] from the QR of the skeleton basis
 *   (Eq. 6-7); two-sided projection U_i^T A_ij U_j of every near block;
 *   LU of Ahat_ii^RR; the self Schur update Ahat_ii^SS -= Ahat_ii^SR
 *   (Ahat_ii^RR)^-1 Ahat_ii^RS (the only trailing update, Eq. 21); couplings
 *   T_i S_ij T_j^T; merge of the children's skeleton blocks into the parent
 *   level (Algorithm 2); LU of the root.
 * prec is an h2_prec.  A later call replaces the previous factorization.
 * Errors: H2_ERR_INVALID_ARG (prec), H2_ERR_SINGULAR (zero pivot),
 * H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_factor(h2_ctx* c, int32_t prec);

/* Free the device arrays of the context's factorizations (FP64 and
 * FP16/BF16) and their CUDA graphs; the instance stays.  Solves need a new
 * h2_factor, which allocates them again.  Errors: H2_ERR_INVALID_ARG. */
h2_status h2_release_factorization(h2_ctx* c);

/* Solve A_H2 x = b by refinement with the factorization as preconditioner.
 * Every refinement residual r = b - A_H2 x is FP64-accurate: FP64
 * instructions (the h2_matvec operator) in schemes 0 and 1, FP32-pair
 * arithmetic by default in scheme 2 (H2_OPT_RESIDUAL_FP64 selects FP64
 * instructions there too).  Every update x += d is FP64; each
 * preconditioner application is the parallel substitution of Eq. 24-31 and
 * its mirror, in the factorization's storage precision.  Schemes
 * (h2_set_refinement):
 *   0 plain iterative refinement: x += M^-1 (b - A_H2 x);
 *   1 FGMRES-based refinement: restarted right-preconditioned flexible
 *     GMRES in FP64, true residual recomputed after every cycle;
 *   2 mixed-precision refinement (FP16/BF16 factorizations): each
 *     correction d of A d = r comes from FGMRES in FP32 with an FP32 copy of
 *     A_H2 and the ULV preconditioner, to 1e-6 relative accuracy (or the
 *     accuracy the target needs, if coarser); residual and update in FP64;
 *   3 automatic (default): 1 for FP64 factorizations, 2 otherwise.
 * Stops when ||r|| / ||b|| <= target or after max_iters preconditioner
 * applications.  b and x hold one vector of N doubles (host or device).
 * relres_out and iters_out (host, may be NULL) receive the final relative
 * residual and the number of preconditioner applications.  target <= 0 runs
 * exactly max_iters applications. */
h2_status h2_solve(h2_ctx* c, const double* b, double* x, double target,
                   int32_t max_iters, double* relres_out, int32_t* iters_out);

/* Several right-hand sides (the paper's solve is per vector; the columns
 * are independent): B and X hold nrhs vectors of N doubles each, one after
 * another (column-major N x nrhs), host or device.  Each column is solved
 * as h2_solve solves one vector, with the same target and max_iters;
 * relres_out and iters_out (host, may be NULL) receive nrhs values.
 * Errors: H2_ERR_INVALID_ARG (nrhs < 0), else as h2_solve; the first
 * failing column ends the call (its index is in h2_last_error). */
h2_status h2_solve_many(h2_ctx* c, const double* B, double* X, int32_t nrhs, double target,
                        int32_t max_iters, double* relres_out, int32_t* iters_out);

/* One application of the factorization, x = ULV^-1 b, without refinement
 * (the parallel substitution of Eq. 24-31 and its mirror).  N doubles each,
 * host or device.  Errors: H2_ERR_STATE, H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_ulv_apply(h2_ctx* c, const double* b, double* x);

/* y = A_H2 x in FP64: upward pass through the nested bases, couplings on
 * every level, downward pass and the dense near blocks of the leaves.
 * N doubles each, host or device.  Errors: H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_matvec(h2_ctx* c, const double* x, double* y);

/* Y = A_H2 X for nrhs vectors laid out as in h2_solve_many (host or
 * device).  Errors: H2_ERR_INVALID_ARG (nrhs < 0), else as h2_matvec. */
h2_status h2_matvec_many(h2_ctx* c, const double* X, double* Y, int32_t nrhs);

/* Choose the refinement scheme of h2_solve (0..3, see h2_solve; default 3)
 * and the FGMRES restart length (1..1000, default 30).
 * Errors: H2_ERR_INVALID_ARG. */
h2_status h2_set_refinement(h2_ctx* c, int32_t method, int32_t restart);

/* y = A_H2 x like h2_matvec, for callers that must not allocate device
 * memory once their context exists (a host framework that owns all device
 * memory and forbids library allocations, or a loop on a latency budget
 * where cudaMalloc / cudaFree may block or synchronize).  No counterpart in
 * the paper: this is a service of the library, not a step of the method.
 *   - x and y: device pointers, N doubles, original point order; the call
 *     allocates nothing and only enqueues work on the context's stream
 *     (y is ready when that stream reaches this point).
 *   - Scratch comes from one fixed 16 MiB device array inside the library
 *     (2^21 doubles); problems needing more (2 padded vectors plus the
 *     skeleton coefficients of every level) are rejected with
 *     H2_ERR_INVALID_ARG.  A GPU holds the array from the first call on that
 *     device until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.  The context's device must be current.
 *   - All calls share the array: calls whose work overlaps on the GPU race.
 * Errors: H2_ERR_INVALID_ARG (NULL or host pointers, wrong device, too
 * large), H2_ERR_CUDA. */
h2_status h2_matvec_noalloc(h2_ctx* c, const double* x, double* y);

/* Options of a context (h2_set_option).  They apply to the next
 * h2_factor / h2_solve.
 *   H2_OPT_RR_LU_FP64     FP16/BF16 factorizations: 0 (default) inverts
 *                         Ahat_ii^RR (and the root block) by Gauss-Jordan
 *                         elimination with partial pivoting in FP32; 1 does
 *                         the partial-pivot elimination in FP64 and rounds
 *                         the inverse once to FP32 (same pivot rule; LAPACK's
 *                         pivots).  FP64 factorizations always use FP64.
 *   H2_OPT_RESIDUAL_FP64  refinement scheme 2: 0 (default) forms
 *                         b - A_H2 x in FP32-pair arithmetic, 1 with FP64
 *                         instructions (the h2_matvec operator).
 *   H2_OPT_GRAPHS         1 (default): the FP32 substitution of FP16/BF16
 *                         factorizations is captured once per factorization
 *                         as a CUDA graph (on a private stream) and replayed
 *                         for every preconditioner application; 0: plain
 *                         launches.  A capture that fails falls back to
 *                         plain launches.
 *   H2_OPT_TC_KERNEL      the kernel form of the factorization's main-chain
 *                         tensor-core GEMMs (projection, Schur update;
 *                         process-wide, all contexts): 0 one CTA per batch
 *                         entry; 1 a persistent grid of two CTAs per SM
 *                         looping over the entries; 2 (default) a
 *                         persistent warp-specialized kernel, one CTA per
 *                         SM, whose epilogue of one tile overlaps the MMAs
 *                         of the next (two TMEM accumulators).  The coupling
 *                         products, on their own stream, always use form 0.
 *   H2_OPT_FP64_LEAF      1 (default): keep the FP64 leaf near blocks; 0
 *                         releases them (the largest array of an instance,
 *                         8 bytes per entry), keeping the FP32 pair and FP16
 *                         copies the FP16 path reads.  Afterwards FP64 and
 *                         BF16 factorizations, the FP64 matvec (h2_matvec,
 *                         arith 0, h2_matvec_noalloc), the FP64 residual
 *                         option and the leaf "A" export return
 *                         H2_ERR_STATE; 1 cannot undo a release (H2_ERR_STATE).
 *                         0 also returns H2_ERR_STATE when the instance has
 *                         no FP16 copy of its leaf blocks.
 *   H2_OPT_BOX_STREAM     the per-box steps of the FP32 substitution on
 *                         levels with at least one box per SM (D = 256,
 *                         R = 128 or D = 128, R = 64; process-wide):
 *                         1 a persistent kernel per step whose factor rows
 *                         stream through a shared-memory ring of bulk
 *                         copies; 2 the same on every level of those
 *                         shapes, whatever its box count; 0 (default)
 *                         row-split kernels (measured faster at N = 2^18:
 *                         22.6 against 24.9 ms of substitution per step).
 *   H2_OPT_PAIR_CTAS      CTAs per SM of the TMA-fed pair kernels of the
 *                         FP16/BF16 substitution, 1..3 (default 3;
 *                         process-wide).
 *   H2_OPT_BOX_CTAS       CTAs per SM the substitution's per-box row splits
 *                         aim at, 1..8 (default 1, the autotuner's choice at
 *                         N = 2^15 and 2^18; process-wide). */
typedef enum {
  H2_OPT_RR_LU_FP64 = 0,
  H2_OPT_RESIDUAL_FP64 = 1,
  H2_OPT_GRAPHS = 2,
  H2_OPT_TC_KERNEL = 3,
  H2_OPT_FP64_LEAF = 4,
  H2_OPT_BOX_STREAM = 5,
  H2_OPT_PAIR_CTAS = 6,
  H2_OPT_BOX_CTAS = 7
} h2_option;

/* Autotuner of the kernel forms and launch shapes (no counterpart in the
 * paper), process-wide settings measured on this context's instance:
 * (1) the form of the factorization's main-chain tensor-core GEMMs
 * (H2_OPT_TC_KERNEL 0, 1, 2: each factors twice, the second timed);
 * (2) the substitution's launch shapes: TMA pair-kernel CTAs per SM (2 or
 * 3), per-box row-split CTAs per SM (1, 2 or 4), the streamed per-box form
 * (H2_OPT_BOX_STREAM 0 or 1) and CUDA-graph replay (H2_OPT_GRAPHS 0 or 1),
 * each of the 24 combinations timed over six ULV applications after two.
 * The fastest of each is kept (set for every context) and the context is
 * left factored in prec (H2_PREC_FP16 or H2_PREC_BF16).  json (may be NULL)
 * receives the choices and the times: {"tc_kernel", "factor_s": [3],
 * "pair_ctas_per_sm", "box_ctas_per_sm", "box_stream", "graphs",
 * "subst_ms", "tried": [[pair, box, stream, graphs, ms], ...]}.
 * Errors: H2_ERR_INVALID_ARG (prec, cap too small), those of h2_factor,
 * H2_ERR_OOM, H2_ERR_TIMEOUT. */
h2_status h2_autotune(h2_ctx* c, int32_t prec, char* json, size_t cap);

/* Set an h2_option to value (0 or 1; 0 .. 2 for H2_OPT_TC_KERNEL and H2_OPT_BOX_STREAM).
 * Errors: H2_ERR_INVALID_ARG. */
h2_status h2_set_option(h2_ctx* c, int32_t option, int64_t value);

/* y = A_H2 x in one of the library's three matvec arithmetics (the same
 * kernels the solver runs), for inspection and tests:
 *   0  FP64 (h2_matvec; the refinement residual of FP64 factorizations);
 *   1  FP32: the FP32 copy of A_H2 that the inner solver of refinement
 *      scheme 2 multiplies by, applied to x rounded to FP32; y is that FP32
 *      result widened to FP64;
 *   2  FP32 pairs: every FP64 matrix entry held as hi = fl32(a) plus
 *      lo = fl32(a - hi), x split the same way, and products summed as
 *      FP32 pairs through the bases, couplings and near blocks; each y_i
 *      converted to FP64 once (about 2^-46 of sum_j |a_ij x_j|; the
 *      default residual of scheme 2).
 * N doubles each, host or device.  Errors: H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_matvec_arith(h2_ctx* c, const double* x, double* y, int32_t arith);

/* Self-test of the library's bounded device-side waits (no counterpart in
 * the paper).  Launches one CTA whose thread 0 waits, with the same
 * bounded mbarrier wait the TMA-fed kernels use, on a barrier that nothing
 * ever completes; after timeout_ns (1 .. 10^10) of GPU global time the wait
 * gives up and the kernel records it in the context's status word, exactly
 * as a kernel whose copies never landed would.  Returns H2_ERR_TIMEOUT with
 * the reason in h2_last_error when the wait gave up as designed (the
 * context stays usable), H2_OK if it did not, H2_ERR_INVALID_ARG or
 * H2_ERR_CUDA. */
h2_status h2_wait_selftest(h2_ctx* c, int64_t timeout_ns);

/* Process-wide cap on the device memory one context may allocate (bytes;
 * 0: no cap beyond the device's free memory).  h2_build and h2_import check
 * the instance's device bytes, and h2_factor the factorization's, against
 * the cap and against cudaMemGetInfo's free memory before allocating or
 * launching anything, and return H2_ERR_OOM with both figures in
 * h2_last_error when it does not fit.  The check against the cap comes
 * before any CUDA call.  The byte counts are estimates of the largest
 * arrays (blocks, bases, couplings), not of every small buffer. */
h2_status h2_set_memory_limit(uint64_t bytes);

/* ---------------------------------------------------------------------------
 * Learned rank predictor (an extension of Algorithm 1; the paper has no
 * counterpart).  A 16 -> 64 -> 64 -> 1 multilayer perceptron with ReLU
 * activations maps a cluster's geometry features to the fraction k / n of
 * its dimension n that the rank-revealing compression keeps, so that every
 * level's rank (the batch layout) is known before any compression runs.
 * The network is trained and evaluated on the GPU by the library's own
 * kernels: BF16 weights, inputs and hidden activations with FP32
 * accumulation, FP32 master weights, full-batch Adam.
 * Parameters, flat, 5313 floats: W1 (64 x 16 row-major), b1 (64),
 * W2 (64 x 64 row-major), b2 (64), w3 (64), b3 (1).
 * Features of box i at level l (16 floats, in this order): log10 of the
 * three extents of the box's bounding box, largest first; log2 of its point
 * count; log2 of its dimension n (points at the leaves, twice the
 * children's rank above); log2 of its near-box count; log2(1 + far-box
 * count); log10 of the smallest centre distance to a far box over the box
 * radius (0 without far boxes); eta; l / L; log10(tol); three indicators of
 * the kernel family (1/r-type, exp(-r)/r-type, Gaussian); log10 of the
 * kernel's length parameter (eps, or ell; 0 for the paper's kernels);
 * log10 of the diagonal entry.
 * ------------------------------------------------------------------------- */
typedef struct h2_rank_model h2_rank_model;

/* Training data from the plain compression: runs the host part of h2_build
 * (no GPU) and writes, for every box of levels L .. 1 (leaves first, boxes
 * in order), its 16 features (feats, nbox x 16 row-major), the fraction
 * k_i / n_i its tolerance rank keeps (targets; k_i before the level's rank
 * cap) and its level (levels).  cap is the room of the arrays in boxes;
 * *nbox receives the box count (with cap too small: H2_ERR_INVALID_ARG and
 * *nbox the count needed).  feats, targets and levels may be NULL when cap
 * is 0.  Errors: as h2_plan. */
h2_status h2_rank_data(const h2_params* p, const double* points, int64_t N, float* feats, float* targets,
                       int32_t* levels, int64_t cap, int64_t* nbox);

/* Create a model on the current device with He-uniform weights drawn from
 * splitmix64(seed) and zero biases.  Errors: H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_rank_model_create(h2_rank_model** out, uint64_t seed);

/* Set the 5313 parameters (host floats; rounded to BF16 for the kernels,
 * kept in FP32 as the master copy) and reset the optimizer state. */
h2_status h2_rank_model_set_weights(h2_rank_model* m, const float* theta);

/* Copy the FP32 master parameters to theta (host, 5313 floats) and, when
 * not NULL, the feature normalization (mean and 1 / standard deviation,
 * 16 floats each) the last training set gave. */
h2_status h2_rank_model_get_weights(h2_rank_model* m, float* theta, float* mean, float* istd);

/* Loss mean((o - y)^2) and its gradient (host, 5313 floats) at the current
 * weights for n samples whose network inputs are given directly (inputs:
 * n x 16, rounded to BF16; no feature normalization), targets y (n).
 * Inputs and targets host or device.  For checking the training kernels. */
h2_status h2_rank_model_grad(h2_rank_model* m, const float* inputs, const float* targets, int64_t n, float* loss,
                             float* grad);

/* Train on n samples (features n x 16 and targets, host or device): the
 * features are normalized by their mean and standard deviation over this
 * set (kept with the model), then steps full-batch Adam steps (learning
 * rate lr, beta 0.9 / 0.999) run on the GPU, 64 steps per CUDA graph.
 * *loss_out (may be NULL) receives the last step's loss. */
h2_status h2_rank_model_train(h2_rank_model* m, const float* feats, const float* targets, int64_t n, int32_t steps,
                              float lr, float* loss_out);

/* Network outputs (predicted k / n) for n feature rows (host or device in
 * and out), with the model's normalization. */
h2_status h2_rank_model_predict(h2_rank_model* m, const float* feats, int64_t n, float* out);

/* One-line description of the model's last error ("" if none). */
const char* h2_rank_model_last_error(const h2_rank_model* m);

/* Free the model.  NULL is ignored. */
void h2_rank_model_destroy(h2_rank_model* m);

/* The batch layout from the predictor alone: cluster tree, near/far lists,
 * features and one inference per level (leaves first; each level's
 * dimension is twice the predicted rank below), no compression.  The JSON
 * (as h2_plan's) gives per level nb, D, predicted K, NP, FP and the
 * device bytes.  Needs the model's device.  Errors: as h2_plan. */
h2_status h2_plan_predicted(const h2_params* p, const double* points, int64_t N, h2_rank_model* model, char* json,
                            size_t cap);

/* h2_build with the ranks laid out by the predictor: each level's rank is
 * K_l = max_i ceil(1.05 prediction_i n_i) + 2, raised to the level's cap
 * once it is within 10 % of it and never above it, and each box's
 * interpolative decomposition comes from a randomized sketch M_i Omega of
 * K_l + 26 columns (Rademacher Omega from splitmix64) followed by a pivoted
 * QR truncated at K_l, in place of the full rank-revealing pass over M_i.
 * The plain pivoted-QR compression stays the fallback and the error check: a box
 * whose sketch shows more than tol of its leading pivot beyond K_l (below
 * the cap), or whose error on 6 further random probes of M_i exceeds
 * 10 max(tol, that estimate), is compressed the plain way; if that needs a
 * larger rank the level is redone the plain way.  h2_stats reports the
 * predicted and final ranks, the fallback count and the host compression
 * time.  Errors: as h2_build. */
h2_status h2_build_predicted(h2_ctx** out, const h2_params* p, const double* points, int64_t N,
                             h2_rank_model* model);

/* h2_build with Algorithm 1's compression on the GPU, each level at a rank
 * laid out beforehand: the predictor's (model; as in h2_build_predicted) or,
 * with model NULL, the level's cap (fixed-rank truncation).  For every box
 * of a level at once, in FP64: W_j = G(S_C(j), S_C(j))^-1 Omega(S_C(j)) per
 * close-sample set (Gauss-Jordan with partial pivoting, or gs_sweeps
 * Gauss-Seidel sweeps from 0 when gs_sweeps > 0: the shortcut of Section
 * 3.5), the sketch Y_i = G(B_i, S_F) Omega(S_F) + sum_j G(B_i, S_C(j)) W_j
 * with K + 32 columns, 6 of them probes (Omega(p, t) = +-1 from splitmix64 of the sample point
 * p and column t), and a column-pivoted QR of the sketch truncated at K + 1
 * steps giving the skeleton and X_i.  The acceptance test and the plain
 * host fallback are those of h2_build_predicted.  Levels the kernels do not
 * cover (box dimension above 256, K above 128, near_samples outside 1..64)
 * run on the host.  h2_stats "construction" reports the GPU levels and the
 * flops of the close-field (pre-factorization) and far-field parts.
 * Errors: as h2_build; H2_ERR_INVALID_ARG also for gs_sweeps outside 0..16. */
h2_status h2_build_gpu(h2_ctx** out, const h2_params* p, const double* points, int64_t N, h2_rank_model* model,
                       int32_t gs_sweeps);

/* ---------------------------------------------------------------------------
 * Batches of independent systems (uneven N and per-cluster ranks; no
 * counterpart in the paper).  Every system keeps its own context; a pool
 * of host workers, each with its own CUDA stream, factors and solves them
 * concurrently, largest system first, so that systems too small to fill
 * the GPU alone share it.  Each context's FP32 substitution replays as a
 * CUDA graph (H2_OPT_GRAPHS).  The worker count is picked by measurement
 * (h2_batch_tune).  A context in a batch must not be used elsewhere while
 * a batch call runs; the batch sets each context's stream.
 * ------------------------------------------------------------------------- */
typedef struct h2_batch h2_batch;

/* A batch over count contexts (not owned) with their sizes n[i].
 * Errors: H2_ERR_INVALID_ARG. */
h2_status h2_batch_create(h2_batch** out, h2_ctx* const* ctxs, const int64_t* n, int32_t count);

/* A batch in forest form over count systems that share the parameters p
 * but the leaf size (points[k]: N[k] x 3, host; leaf[k] the leaf size of
 * system k, or NULL for p->leaf_size): the systems are grouped by (leaf
 * size, tree depth) and each group is built as one h2_build_forest
 * instance, owned by the batch, whose FP64 leaf blocks are then released
 * (H2_OPT_FP64_LEAF; the batch factors in FP16 or BF16 from the FP16 copy,
 * so prec must be H2_PREC_FP16).  h2_batch_run then factors each group
 * (one launch per kernel and level for all its systems) and solves its
 * systems together: each right-hand side is scaled to unit norm, the group
 * is refined to target / sqrt(m) for its m systems (then |r_k| <= |r| <=
 * target for every system), and each system's relative residual, written
 * to relres, is recomputed from one FP32-pair matvec of the group
 * (h2_matvec_arith arith 2); iters receives the group's count.  The vectors
 * B[k], X[k] of a forest batch are host memory (the scaling and splitting
 * run on the host; device vectors give H2_ERR_INVALID_ARG).  The worker pool
 * runs the groups; a group's factorization is released after its solve
 * (h2_release_factorization), so prec = -1 is not available, and a worker
 * whose factorization does not fit (H2_ERR_OOM) waits for another group to
 * release its arrays and tries again (the error stands when no other group
 * holds any).  Errors: as h2_build_forest (the group's message is in
 * h2_last_error(NULL)). */
h2_status h2_batch_create_forest(h2_batch** out, const h2_params* p, const double* const* points,
                                 const int64_t* N, const int32_t* leaf, int32_t count);

/* Factor every system in precision prec (prec = -1: keep the current
 * factorizations) and, with B non-NULL, solve system i for B[i] into X[i]
 * as h2_solve does (target, max_iters).  relres and iters (host, may be
 * NULL) receive count values; *seconds (may be NULL) the wall time.
 * Errors: those of h2_factor / h2_solve, with the system in the message
 * (h2_batch_last_error). */
h2_status h2_batch_run(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                       int32_t max_iters, double* relres, int32_t* iters, double* seconds);

/* Autotune the batch: first h2_autotune on the largest context (kernel
 * forms and launch shapes, process-wide), then the worker count: run the
 * whole batch (factor and solve) with
 * 1, 2, 4, 8 and 16 workers (up to twice the system count) and keep the
 * fastest; *workers_out (may be NULL) receives it.  A system that stops
 * above the target does not end the tuning (H2_ERR_NOT_CONVERGED is
 * returned at the end).  Errors: as h2_batch_run. */
h2_status h2_batch_tune(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                        int32_t max_iters, int32_t* workers_out);

/* JSON: system count, mode ("pool" or "forest"), group count (forest: the
 * systems per group), worker count, the last run's seconds, the tuning
 * times by worker count and h2_autotune's choices ("kernels").  Errors:
 * H2_ERR_INVALID_ARG (cap too small). */
h2_status h2_batch_stats(const h2_batch* b, char* json, size_t cap);

/* One-line description of the batch's last error ("" if none). */
const char* h2_batch_last_error(const h2_batch* b);

/* Free the batch: a pool batch's contexts are not freed (they go back to
 * the legacy default stream); a forest batch's group contexts are.  NULL
 * is ignored. */
void h2_batch_destroy(h2_batch* b);

/* Issue all later work on the given cudaStream_t (NULL: legacy default). */
h2_status h2_set_stream(h2_ctx* c, void* stream);

/* Sizes, ranks, per-phase device times of the last factorization and solve,
 * algorithmic flop and byte counts, as one JSON object written to json
 * (at most cap bytes including the terminating zero).  Returns
 * H2_ERR_INVALID_ARG if cap is too small. */
h2_status h2_stats(const h2_ctx* c, char* json, size_t cap);

/* Copy an internal array to host memory for inspection (tests).  name is
 * one of "X", "U", "T", "Ahat", "lu", "piv", "root", "root_piv", "A" (the
 * level's input near blocks) or "perm"; level selects the level.
 * Arrays are copied in the library's storage type (8-byte doubles for FP64
 * factorizations and for "X"/"A"-FP64, 4-byte floats otherwise); *elem_size
 * receives that size.  With dst == NULL only *count (elements) and
 * *elem_size are set.  Errors: H2_ERR_INVALID_ARG (unknown name or level,
 * cap too small; "lu" and "root" after a mixed-precision factorization,
 * which inverts the blocks by Gauss-Jordan elimination and keeps no LU
 * factors), H2_ERR_STATE (not computed yet). */
h2_status h2_export(const h2_ctx* c, const char* name, int32_t level, void* dst,
                    size_t cap_bytes, size_t* count, int32_t* elem_size);

/* One-line description of the last error on this context ("" if none).
 * With c == NULL, the last error of a failed h2_build / h2_import. */
const char* h2_last_error(const h2_ctx* c);

/* Free the context and all its device memory.  NULL is ignored. */
void h2_destroy(h2_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* H2ULV_H */
