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
 *              residual uses the FP64 H^2 matrix-vector product.
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

/* Arithmetic of the projection and Schur-update contractions (Algorithm 4
 * line 3, line 6 and line 10).  The LU of the redundant diagonal blocks, the
 * refinement residual and update always run in FP64.
 *   H2_PREC_FP64   FP64 everywhere (the plain H^2-ULV).
 *   H2_PREC_FP16   FP16 inputs, FP32 accumulation on the tensor cores;
 *                  FP32 bases, factors and substitution.
 *   H2_PREC_BF16   as FP16 with BF16 inputs. */
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
 *   level (Algorithm 2 line 18-20); LU of the root.
 * prec is an h2_prec.  A later call replaces the previous factorization.
 * Errors: H2_ERR_INVALID_ARG (prec), H2_ERR_SINGULAR (zero pivot),
 * H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_factor(h2_ctx* c, int32_t prec);

/* Solve A_H2 x = b by refinement with the factorization as preconditioner.
 * Every refinement residual r = b - A_H2 x is computed in FP64 (the
 * h2_matvec operator) and every update x += d is FP64; each preconditioner
 * application is the parallel substitution of Eq. 24-31 and its mirror, in
 * the factorization's storage precision.  Schemes (h2_set_refinement):
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
