// Internal declarations of the H^2-ULV library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/h2ulv.h"

#if defined(__CUDACC__)
#define H2_HD __host__ __device__ __forceinline__
#else
#define H2_HD inline
#endif

namespace h2 {

// ---------------------------------------------------------------------------
// Kernel function G(x, y) (the formulas listed in h2ulv.h).  Shared by the
// host-side construction and the device-side block evaluation.
// ---------------------------------------------------------------------------
struct KernelFn {
  int kind;
  double eps, ell, diag_shift;

  H2_HD double off(const double* a, const double* b) const {
    if (kind == H2_K_POLY2_TEST) {
      double d = 1.0 + a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
      return d * d;
    }
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    switch (kind) {
      case H2_K_LAPLACE_EPS: return 1.0 / (r + eps);
      case H2_K_YUKAWA_EPS: return exp(-r) / (r + eps);
      case H2_K_GAUSSIAN: return exp(-r2 / (ell * ell));
      case H2_K_LAPLACE_PAPER: return 1.0 / r;
      default: return exp(-r) / r;  // H2_K_YUKAWA_PAPER
    }
  }
  H2_HD double diag(const double* a) const {
    switch (kind) {
      case H2_K_LAPLACE_EPS:
      case H2_K_YUKAWA_EPS: return 1.0 / eps + diag_shift;
      case H2_K_GAUSSIAN: return 1.0 + diag_shift;
      case H2_K_LAPLACE_PAPER:
      case H2_K_YUKAWA_PAPER: return 1e3 + diag_shift;
      default: {
        double q = 1.0 + a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        return q * q + diag_shift * q;
      }
    }
  }
  // Entry for point indices ia, ib (-1 = padding: 1 on the diagonal, else 0).
  H2_HD double entry(const double* pts, int64_t ia, int64_t ib, bool same_slot) const {
    if (ia < 0 || ib < 0) return (ia < 0 && ib < 0 && same_slot) ? 1.0 : 0.0;
    if (ia == ib) return diag(pts + 3 * ia);
    return off(pts + 3 * ia, pts + 3 * ib);
  }
};

// ---------------------------------------------------------------------------
// Host-side H^2 structure (tree, lists, ID bases) produced by the
// construction or by h2_import.
// ---------------------------------------------------------------------------
struct HostLevel {
  int nb = 0, D = 0, K = 0;
  std::vector<int32_t> near;  // 2 * NP, sorted (i, j)
  std::vector<int32_t> far;   // 2 * FP, sorted (i, j)
  std::vector<double> X;      // nb * D * K
  std::vector<int64_t> SK;    // nb * K
};

// Features of the learned rank predictor per box (the list in h2ulv.h).
constexpr int kRankFeatures = 16;

// What the construction records about its ranks.
struct RankRecord {
  std::vector<std::vector<float>> feats;  // per level: nb * kRankFeatures
  std::vector<std::vector<int>> ranks;    // per level: tolerance rank of each box (plain boxes; -1 sketched)
  std::vector<std::vector<int>> dims;     // per level: box dimension n_i
  std::vector<int> K_pred;                // per level: the predictor's rank (-1: not used)
  int fallback_boxes = 0;                 // boxes compressed the plain way after a failed sketch check
  int fallback_levels = 0;                // levels redone the plain way (rank too small)
  double compress_s = 0;                  // wall time of the per-box compression passes
  int gpu_levels = 0;                     // levels whose sketches ran on the GPU
  double flops_prefactor = 0;             // GPU construction: the close-field (pre-factorization) part
  double flops_far = 0;                   //                   the far-field part
};

// One level of the GPU construction (construct_gpu.cu): nb boxes of at most
// D points (nbox[i]; bpts: nb * D original indices, -1 pad), far samples
// (fptr / fidx), close boxes (nptr / nidx: the near list, j == i skipped),
// close samples of each box (cptr / cidx), rank K, m sketch + probe columns
// (ms of them sketch), q = m - ms probes, Gauss-Seidel sweeps gs (0: exact
// solve).  Outputs: X (nb * D * K row-major), SK (nb * K), piv (nb * D),
// the pivot ratio rho and probe error err per box.
struct GpuLevelJob {
  int nb = 0, D = 0, K = 0, m = 0, ms = 0, q = 0, gs = 0;
  uint64_t seed = 0;
  std::vector<int> nbox;
  std::vector<int64_t> bpts, fptr, fidx, nptr, cptr, cidx;
  std::vector<int32_t> nidx;
  std::vector<double> X, rho, err;
  std::vector<int64_t> SK;
  std::vector<int32_t> piv;
  double flops_prefactor = 0, flops_far = 0;
};
struct GpuCompressor {
  virtual bool supported(int D, int K) const = 0;
  virtual std::string run(GpuLevelJob& job) = 0;  // "" on success
  virtual ~GpuCompressor() = default;
};

struct HostH2 {
  int64_t N = 0;
  int L = 0;
  std::vector<double> points;        // N * 3
  std::vector<int64_t> perm;         // N
  std::vector<int64_t> leaf_offsets; // 2^L + 1
  std::vector<HostLevel> lv;         // L + 1
  std::vector<int> ranks_leaf;       // tol-rank per leaf box (diagnostic)
  RankRecord rec;
};

// The rank predictor as the construction calls it: predictions k / n for
// nb rows of features (nb * kRankFeatures floats).  False on failure.
struct RankPredictor {
  virtual bool predict(const std::vector<float>& feats, int nb, std::vector<float>& out) = 0;
  virtual ~RankPredictor() = default;
};

// Host construction (host_build.cpp).  Returns an empty string on success.
// With pred, every level's rank comes from the predictor and the boxes are
// compressed by randomized sketches (plain pivoted QR as the fallback);
// with layout_only, the levels are laid out from predictions alone (no
// compression; X and SK stay empty).
// With force_K, level l's rank is force_K[l] (where > 0, at most the level's
// smallest box) in place of the largest tolerance rank (plain path only).
std::string build_host(const h2_params& p, const double* pts, int64_t N, HostH2& out,
                       RankPredictor* pred = nullptr, bool layout_only = false, GpuCompressor* gpu = nullptr,
                       const std::vector<int>* force_K = nullptr);
// Depth of the binary tree over n points with leaves of at most `leaf`.
int depth_of(int64_t n, int leaf);
// Independent systems of one tree depth L >= 1 and one rank per level as
// one instance (a forest): system s holds boxes [s 2^l, (s + 1) 2^l) of
// level l, so box i's children stay 2i and 2i + 1 and the root level has one
// box per system.  Leaves are padded to the largest leaf (padding points).
// Empty string on success.
std::string combine_forest(const std::vector<HostH2>& parts, HostH2& out);
// The GPU compressor of construct_gpu.cu over the N points (kernel G);
// nullptr if the device upload fails.
GpuCompressor* make_gpu_compressor(const KernelFn& G, const double* pts, int64_t N, int gs_sweeps);

// ---------------------------------------------------------------------------
// Device-side state.
// ---------------------------------------------------------------------------
struct DevLevel {
  int nb = 0, D = 0, K = 0, R = 0;
  int64_t NP = 0, FP = 0;
  int max_near = 0, max_far = 0;  // largest near / far count of one box
  // pair lists (device)
  int32_t *near_i = nullptr, *near_j = nullptr;  // NP
  int64_t* near_ptr = nullptr;                   // nb + 1 (CSR over i)
  int32_t* diag_pair = nullptr;                  // nb
  int32_t *far_i = nullptr, *far_j = nullptr;    // FP
  int64_t* far_ptr = nullptr;                    // nb + 1
  int32_t *near_dst = nullptr, *far_dst = nullptr;  // parent near-pair index of each pair
  // sub-lists of the near pairs for the substitution: j < i (lo) and j > i
  // (hi), in pair order, with their count per box
  int32_t *lo_pairs = nullptr, *hi_pairs = nullptr;
  int32_t *lo_cnt = nullptr, *hi_cnt = nullptr;
  int64_t n_lo = 0, n_hi = 0;
  // host copies
  std::vector<int32_t> h_near_i, h_near_j, h_far_i, h_far_j, h_diag_pair, h_near_dst, h_far_dst;
  std::vector<int64_t> h_near_ptr, h_far_ptr;
  // construction data (FP64)
  double* X = nullptr;    // nb * D * K
  int64_t* SK = nullptr;  // nb * K
  double* S = nullptr;    // FP * K * K couplings G(SK_i, SK_j)
  float* X32 = nullptr;   // FP32 copies for the inner solver of the mixed refinement
  float* S32 = nullptr;
  // symmetric coupling storage for the FP32 matvec (S_ji = S_ij^T): the far
  // pairs i < j ("stored"), their FP32 couplings, and per box the list of
  // partial products (2k: S_k xh_j for i = box, 2k + 1: S_k^T xh_i for
  // j = box), CSR over boxes
  bool far_sym = false;
  int64_t fpu = 0;
  int64_t fs_goff = 0;  // first index of this level's stored pairs in the all-level batch
  int32_t *fs_i = nullptr, *fs_j = nullptr, *fs_ent = nullptr;
  int64_t* fs_ptr = nullptr;
  float* S32u = nullptr;
  void* S16[2] = {nullptr, nullptr};        // couplings scaled into FP16 [0] / BF16 [1]
  float* S16_scale[2] = {nullptr, nullptr};  // their scale and inverse scale (device)
  // symmetric near list (pair (j, i) present for every (i, j)): the pairs
  // i <= j ("upper", su_*: their index, i, j) and the others (lw_q) with the
  // index of their mirror (lw_m); h_mirror[q] on the host (-1: no mirror)
  bool near_sym = false;
  int64_t n_up = 0, n_lw = 0;
  int32_t *su_q = nullptr, *su_i = nullptr, *su_j = nullptr;
  int32_t *lw_q = nullptr, *lw_m = nullptr, *mirror = nullptr;
  std::vector<int32_t> h_mirror;
};

// Factorization storage of one level in storage type T (double or float).
template <typename T>
struct FacLevel {
  T* U = nullptr;      // nb * D * D   [U^R U^S], column-major
  T* Ur = nullptr;     // nb * D * D   the same, row-major (for x = U z in the substitution)
  T* Tm = nullptr;     // nb * K * K   row-major, upper triangular
  T* Xo = nullptr;     // nb * D * K   X^orth (row-major)
  T* Vq = nullptr;     // nb * D * K   Householder reflectors (column-major, unit diagonal)
  T* tau = nullptr;    // nb * K
  T* Tw = nullptr;     // nb * K * K   compact-WY triangular factor
  T* Qs = nullptr;     // nb * D * K   panel scratch when it does not fit in shared memory
  T* Ain = nullptr;    // NP * D * D   input near blocks of this level (row-major)
  T* Ahat = nullptr;   // NP * D * D   projected blocks (row-major)
  T* Shat = nullptr;   // FP * K * K   couplings in orthogonal coordinates
  T* Z = nullptr;      // nb * R * K   (Ahat_ii^RR)^-1 Ahat_ii^RS
  double* lu = nullptr;    // nb * R * R  LU of Ahat_ii^RR, column-major (FP64 factorization only)
  T* luT = nullptr;        // nb * R * R  the same factors in T (aliases lu when T is double)
  T* Ainv = nullptr;       // nb * R * R  (Ahat_ii^RR)^-1, row-major
  T* M1 = nullptr;         // nb * R * D  Ainv (U^R)^T, row-major (the substitution's first product)
  int32_t* piv = nullptr;  // nb * R (LAPACK-style row interchanges)
  // substitution vectors
  T *vin = nullptr, *c = nullptr, *u = nullptr, *v = nullptr, *om = nullptr, *xs = nullptr;
  // per-pair partial products of the substitution (Factor::part, shared by
  // all levels)
  T* part = nullptr;
  // tensor-core path (mixed precision): 16-bit scaled input blocks and bases
  bool tc = false;
  void* Ain16 = nullptr;  // NP * D * D (scale in Factor::scales[2l], inverse at [2l+1])
  void* U16 = nullptr;    // nb * D * D, column-major like U
  bool tc_coup = false;   // couplings on the tensor cores
  void* T16 = nullptr;    // nb * K * K scaled 16-bit T (scale in Factor::tscale[2l])
  // projection of the upper pairs only (Ahat_ji = Ahat_ij^T): the FP32 SS of
  // a lower off-diagonal pair is then its mirror's, transposed
  bool proj_sym = false;
  // s * Ahat in 16 bits (same layout as Ahat), read by the substitution in
  // place of the FP32 Ahat; ahat_isc -> 1 / s on the device.  NULL where the
  // level keeps the substitution on the FP32 Ahat.
  void* Ahat16 = nullptr;
  const float* ahat_isc = nullptr;
  bool ahat_ss_only = false;  // FP32 Ahat of off-diagonal pairs holds only the SS quadrant
  // tensor maps over Ahat16 (rows NP * D, cols D) with the RR, SR and RS
  // quadrants as tiles, for the TMA-fed pair kernels; tma is false where
  // the shapes do not allow them
  bool tma = false;
  CUtensorMap tm_rr, tm_sr, tm_rs;
  int32_t* err = nullptr;  // device word set by a substitution kernel whose wait timed out
};

template <typename T>
struct Factor {
  bool ready = false;
  std::vector<FacLevel<T>> lv;
  double* root_lu = nullptr;  // D0 * D0 column-major (FP64 factorization only)
  T* root_luT = nullptr;      // the same in T
  T* root_inv = nullptr;      // D0 * D0 row-major
  int32_t* root_piv = nullptr;
  T* root_vec = nullptr;      // D0
  T* root_x = nullptr;        // D0
  T* Wk = nullptr;            // workspace: max NP * D * D
  void* W16 = nullptr;        // 16-bit workspace: max NP * D * D (tensor-core path)
  // workspaces of the basis stream (complement bases and couplings run
  // there, beside the projection / LU / merge chain)
  T* Wq = nullptr;            // max nb * (K * K + D * K): Gram matrix and V Tw
  T* Wc = nullptr;            // max FP * K * K: SIMT coupling products
  void* W16c = nullptr;       // max FP * K * K: 16-bit coupling products
  T* part = nullptr;          // max NP * max(R, K): partial products of the substitution
  double* rr_lu = nullptr;    // FP64 LU / inverse scratch of Ahat_ii^RR for the FP16/BF16
  double* rr_inv = nullptr;   // factorizations' FP64 a3: max(nb R^2, D0^2) doubles each
  float* scales = nullptr;    // 2 (L + 1): per-level operand scale and its inverse
  float* tscale = nullptr;    // 2 (L + 1): scale of T16 and its inverse
  float* cscale = nullptr;    // L + 1: 1 / (scale(S16) scale(T16)^2) for the couplings
  unsigned int* amax = nullptr;  // 2 (L + 1) max-abs accumulators: [l] merge, [L + 1 + l] couplings
  // tensor-core Schur update (FP16/BF16 factorizations): scales of the 16-bit
  // (Ahat_ii^RR)^-1 [0, 1] and Z^T [2, 3], the two GEMMs' output scales
  // [4, 5]; max-abs accumulators [0, 1]
  float* sch = nullptr;
  unsigned int* sch_amax = nullptr;
  bool schur_tc = false;  // the last factorization ran a4/a5 on the tensor cores at some level
  int bf16 = -1;              // operand type the 16-bit buffers hold
  std::vector<void*> allocs;  // this factorization's device arrays (h2_release_factorization)
};

struct PhaseTimes {
  double a1_qr = 0, a2_proj = 0, a3_lu = 0, a5_schur = 0, a2c_coupling = 0, a6_merge = 0,
         a7_root = 0, total_factor = 0;
  double wait_basis = 0;  // the main factorization stream waiting for the basis stream
  double solve_total = 0, subst = 0, matvec = 0;
  double matvec32 = 0, leaf32 = 0;
  int iters = 0, n_subst = 0, n_matvec = 0, n_matvec32 = 0, n_leaf32 = 0, method = 0;
  double relres = 0;
  std::vector<double> history;  // relative residual after every correction (IR) or cycle (GMRES)
};

}  // namespace h2

struct h2_ctx {
  h2_params params{};
  h2::KernelFn kfn{};
  h2::HostH2 host;
  std::vector<h2::DevLevel> lv;
  int L = 0;
  int64_t N = 0;
  int dev = 0;
  cudaStream_t stream = nullptr;
  // the factorization's basis, coupling and substitution-product streams
  // (created on first use)
  cudaStream_t basis_stream = nullptr, coupling_stream = nullptr, product_stream = nullptr;
  // device geometry and vectors
  double* pts = nullptr;         // N * 3
  int64_t* slot_pt = nullptr;    // nbL * DL: original index of each padded leaf slot, -1 pad
  double* A64 = nullptr;         // NP_L * DL * DL leaf near blocks (FP64, for the matvec)
  void* A16[2] = {nullptr, nullptr};     // the leaf blocks scaled into FP16 [0] / BF16 [1]
  float* A16_scale[2] = {nullptr, nullptr};  // their scale and inverse scale (device)
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *y64 = nullptr, *t64 = nullptr;  // padded tree vectors
  double *io_a = nullptr, *io_b = nullptr;  // original-order staging vectors (N)
  double* xhat = nullptr;  // matvec upward/downward scratch (sum over levels nb*K)
  double* yhat = nullptr;
  float* A32 = nullptr;    // FP32 copy of the leaf near blocks (inner solver)
  // fl32(A64 - A32), and the same for the couplings and the leaf basis: with
  // the FP32 copies, the FP64 matrix as FP32 pairs (the mixed refinement's
  // residual)
  float* Alo = nullptr;
  std::vector<float*> Xlo;   // per level (index l; [0] unused)
  std::vector<float*> Slo;   // per level (index l; [0] unused)
  // Symmetric leaf storage of A32 / Alo: only the near pairs i <= j
  // ("stored pairs", sym_q: their index among the near pairs), and per box
  // the list of partial products (2k: A_k x_j of stored pair k with i = box,
  // 2k + 1: A_k^T x_i with j = box), CSR over boxes.
  bool sym = false;
  int64_t npu = 0;
  int32_t *sym_q = nullptr, *sym_i = nullptr, *sym_j = nullptr, *sym_ent = nullptr;
  int64_t* sym_ptr = nullptr;
  float* part32 = nullptr;   // npu * 2 D partial products (FP32 matvec)
  float* part32c = nullptr;  // cb_n * 2 cb_K coupling partial products (beside the leaf's)
  // the FP32 matvec's leaf near field runs on leaf_stream beside the passes
  // through the bases (created on first use), forked and joined by events
  cudaStream_t leaf_stream = nullptr;
  cudaEvent_t mv_fork = nullptr, mv_join = nullptr;
  double* part64 = nullptr;  // the same for the FP32-pair matvec
  // the FP32-pair matvec's input vector (split once per matvec) and its
  // basis coefficients xhat, yhat of all levels, as FP32 pairs
  float *xdf_h = nullptr, *xdf_l = nullptr, *hdf_h = nullptr, *hdf_l = nullptr, *ydf_h = nullptr, *ydf_l = nullptr;
  float *xhat32 = nullptr, *yhat32 = nullptr;
  // the stored coupling pairs of every level as one batch (levels with the
  // same rank cb_K): the FP32 matvec forms all levels' coupling products in
  // one launch; cb_i / cb_j index K-slots of xhat32
  bool cb_ok = false;
  int cb_K = 0;
  int64_t cb_n = 0;
  int32_t *cb_i = nullptr, *cb_j = nullptr;
  float* S32u_all = nullptr;
  std::vector<double*> X64p, S64p;  // per-level pointers (index l; [0] unused)
  std::vector<float*> X32p, S32p;
  std::vector<int64_t> hat_off;  // per-level offsets into xhat / yhat
  double* red = nullptr;         // reduction scratch
  int32_t* status = nullptr;     // device error word(s)
  int prec = -1;                 // precision of the current factorization
  bool used_tc = false;          // the last factorization ran contractions on the tensor cores
  int refine_method = 3;         // 0: plain IR, 1: FGMRES-IR in FP64, 2: FP64 outer / FP32 FGMRES inner,
                                 // 3: automatic (1 for FP64 factorizations, 2 otherwise)
  bool rr_lu64 = false;          // FP16/BF16 factorizations: Ahat_ii^RR inverted in FP64 (else FP32)
  bool resid64 = false;          // refinement scheme 2: residual with FP64 instructions (else FP32 pairs)
  float *mv32_x = nullptr, *mv32_y = nullptr;  // h2_matvec_arith's FP32 tree vectors (created on first use)
  // the FP32 substitution sweep of the current FP16/BF16 factorization as a
  // CUDA graph (captured on first use after each h2_factor; H2_OPT_GRAPHS)
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g_ulv = nullptr;
  long long g_ulv_kernels = 0;  // kernels in that graph (added to the launch count per replay)
  double inner_tol = 1e-6;       // relative accuracy of the FP32 inner solves
  int restart = 30;              // FGMRES restart length
  double* gm_V = nullptr;        // (restart + 1) * nslot Krylov basis
  double* gm_Z = nullptr;        // restart * nslot preconditioned directions
  double* gm_h = nullptr;        // h1, h2 (restart + 2 each), the norm slot (257), y (restart + 2)
  double* gm_host = nullptr;     // pinned copy of h1, h2 and the norm (one read per FGMRES step)
  double* gm_part = nullptr;     // (restart + 1) * 128 dot-product partials
  float* gm_V32 = nullptr;       // FP32 Krylov basis / directions of the inner solver
  float* gm_Z32 = nullptr;
  float* gm_r32 = nullptr;
  int gm_cap = 0;                // restart the buffers were sized for
  h2::Factor<double> f64;
  h2::Factor<float> f32;
  h2::PhaseTimes times;
  std::vector<void*> allocs;
  std::vector<void*>* alloc_sink = nullptr;  // where dalloc records (NULL: allocs)
  std::string err;
};

namespace h2 {

// records allocations made while it lives in the given list (a
// factorization's own arrays)
struct AllocSink {
  h2_ctx* c;
  std::vector<void*>* prev;
  AllocSink(h2_ctx* ctx, std::vector<void*>* to) : c(ctx), prev(ctx->alloc_sink) { c->alloc_sink = to; }
  ~AllocSink() { c->alloc_sink = prev; }
};

// device allocation helper: records the pointer in ctx->allocs (or the
// active AllocSink's list)
template <typename T>
inline cudaError_t dalloc(h2_ctx* c, T** p, size_t n) {
  if (n == 0) n = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e == cudaSuccess) {
    (c->alloc_sink ? *c->alloc_sink : c->allocs).push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

}  // namespace h2
