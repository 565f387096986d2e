// Launchers of the device kernels (internal).
#pragma once

#include <atomic>

#include "h2_internal.h"

namespace h2 {

// Number of kernels this library has launched (reported by h2_stats).
extern std::atomic<long long> g_launches;
// Tensor-core GEMM kernel form of the factorization's main chain
// (projection, Schur update), process-wide (H2_OPT_TC_KERNEL): 0 one CTA per
// batch entry, 1 a persistent grid of two CTAs per SM, 2 (default) the
// persistent warp-specialized kernel with two TMEM accumulators.  The coupling
// products on their own stream always use form 0, so that they keep sharing
// the SMs with the main chain.
extern std::atomic<int> g_tc_kernel;
// The substitution's per-box steps: 1 the streamed persistent form
// (bulk-copy ring) on levels with at least one box per SM, 2 on every level
// of a supported shape, 0 (default) never (row-split kernels); process-wide
// (H2_OPT_BOX_STREAM).
extern std::atomic<int> g_box_stream;
// Launch shapes of the substitution (h2_autotune): CTAs per SM targeted by
// the per-box row splits (default 1) and of the TMA-fed pair kernels
// (default 3; at most 3 fit their shared-memory rings).
extern std::atomic<int> g_box_ctas_per_sm;
extern std::atomic<int> g_pair_ctas_per_sm;

// kernels_factor.cu
void launch_eval_blocks(const KernelFn& G, const double* pts, int64_t npairs, const int32_t* pi,
                        const int32_t* pj, const int64_t* idx, int idx_stride, int rows, int cols,
                        double* out, cudaStream_t st);
template <typename S, typename T>
void launch_convert(const S* in, T* out, int64_t n, cudaStream_t st);
template <typename T, typename TB>
void gemm_simt(int M, int N, int K, const T* A, int64_t sA, const int32_t* ia, int lda, bool tA, const TB* B,
               int64_t sB, const int32_t* ib, int ldb, bool tB, T* C, int64_t sC, const int32_t* ic, int ldc,
               T alpha, T beta, int64_t batch, cudaStream_t st);
template <typename T>
// true when the compact-WY factor Tw was formed too (Tw non-NULL, FP32 register form)
bool launch_qr_panel(int nb, int D, int K, const T* Xin, T* Vout, T* tau, T* Tm, T* gscr, cudaStream_t st,
                     T* Tw = nullptr);
template <typename T>
void launch_wy_tfactor(int nb, int K, const T* S, const T* tau, T* Tw, cudaStream_t st);
template <typename T>
void launch_perm_identity(int nb, int D, int K, T* U, cudaStream_t st);
// U = [Q[:, K:] Q[:, :K]], Q = I - W1 V^T (W1 D x K row-major, V D x K
// column-major), as column-major U, row-major Ur and 16-bit U16 (NULL: none)
void launch_form_u(int64_t nb, int D, int K, const float* W1, const float* V, float* U, float* Ur, void* u16,
                   int bf16, cudaStream_t st);
template <typename T>
void launch_lu_inverse(int nb, int D, int R, const T* Ablk, const int32_t* diag_idx, double* lu, T* luT,
                       int32_t* piv, T* Ainv, int32_t* status, int level, cudaStream_t st);
// the FP16/BF16 factorizations' a3 in FP64: FP32 blocks in, FP64 LU and
// inverse (scratch lu, inv: nb * R * R each), FP32 inverse out
void launch_lu_inverse_f64_for_f32(int nb, int D, int R, const float* Ablk, const int32_t* diag_idx, double* lu,
                                   double* inv, int32_t* piv, float* Ainv, int32_t* status, int level,
                                   cudaStream_t st);
template <typename T>
void launch_merge(int D, int K, int64_t NP, const T* Ahat, const int32_t* ni, const int32_t* nj,
                  const int32_t* ndst, int64_t FP, const T* Shat, const int32_t* fi, const int32_t* fj,
                  const int32_t* fdst, T* Apar, cudaStream_t st);

// kernels_tc.cu: tensor-core (tcgen05 + TMA) batched GEMM
//   C_b = alpha * (*alpha_dev) * A_b B_b^T, A_b = matrix ia[b] (rowsA x K,
//   K-major, 16-bit) of the nA-matrix array A, B_b likewise, FP32
//   accumulation; out_mode 0: FP32 row-major C, 1: 16-bit C^T, 3: FP32
//   C += result (read-modify-write).
// gemm_tc returns false (and launches nothing) for unsupported shapes.
bool gemm_tc_supported(int M, int N, int K, int lda, int ldb, int ldc);
bool gemm_tc(int ab_bf16, int M, int N, int K, const void* A, int64_t nA, int rowsA, int lda, const int32_t* ia,
             const void* B, int64_t nB, int rowsB, int ldb, const int32_t* ib, void* C, int64_t sC,
             const int32_t* ic, int ldc, int out_mode, int out_bf16, float alpha, const float* alpha_dev,
             int64_t batch, int32_t* err, cudaStream_t st, void* C2 = nullptr, int qsplit = -1,
             const int32_t* qi = nullptr, const int32_t* qj = nullptr, unsigned int* amax_ss = nullptr,
             int64_t rowsA_total = 0,  // rowsA_total > 0: the rows A's tensor map spans (else nA * rowsA)
             int form = -1);           // kernel form 0 / 1 / 2 (g_tc_kernel's meaning); -1: g_tc_kernel
void launch_inv_scale_pair(const float* a, const float* b, float* out, cudaStream_t st);  // out = 1 / (a b)
// 2-D tensor map over a rows x cols 16-bit array (row stride ld elements)
// with box_rows x box_cols tiles, no swizzle (dense row-major tiles in
// shared memory).  False if the driver or the shape does not allow it.
bool make_tile_map(CUtensorMap* tm, const void* base, int bf16, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows, uint32_t box_cols);
// One CTA whose thread 0 waits (bounded by timeout_ns) on an mbarrier that
// nothing completes, then sets *flag = 1: the self-test of the bounded waits.
void launch_wait_selftest(unsigned long long timeout_ns, int32_t* flag, cudaStream_t st);
template <typename S>
void launch_amax_blocks(const S* base, int64_t nblk, int64_t stride, int rows, int cols, int ld, unsigned int* out,
                        cudaStream_t st, const int32_t* idx = nullptr);  // idx: block q is base + idx[q] stride
void launch_pow2_scale(const unsigned int* amax_bits, float target, float* scale, cudaStream_t st,
                       const unsigned int* amax2 = nullptr);
void launch_inv_scale_product(const float* a, const float* b, float* out, cudaStream_t st);
template <typename S>
void launch_to_lowp(int bf16, const S* in, void* out, int64_t n, const float* scale, cudaStream_t st);
void launch_merge_lowp(int D, int K, int64_t NP, const float* Ahat, const int32_t* ni, const int32_t* nj,
                       const int32_t* ndst, int64_t FP, const float* Shat, const int32_t* fi, const int32_t* fj,
                       const int32_t* fdst, void* Apar, const float* scale, int bf16, cudaStream_t st,
                       const int32_t* mirror = nullptr, int skip_lower = 0);
// 16-bit D x D blocks dst[k] = (block src[k])^T outside the SS quadrant
void launch_transpose16_blocks(int D, int R, int64_t n, const int32_t* dst, const int32_t* src, void* A,
                               cudaStream_t st);

// kernels_solve.cu: substitution (Eq. 24-31 and its mirror), H^2 matvec,
// refinement vector operations
// Ahat of level L in storage type TS (T itself, or 16-bit scaled by s with
// iscale -> 1/s on the device; iscale NULL means 1)
// The children of a level's boxes as the first forward step reads them:
// c (nb_c * D), the SR pair sums in part, the near-pair ranges ptr, the
// 16-bit scale of Ahat (NULL: 1) and the child level's D, R, K.  c NULL:
// the input is the level's own vin (leaf level).
template <typename T>
struct ChildIn {
  const T* c = nullptr;
  const T* part = nullptr;
  const int64_t* ptr = nullptr;
  const float* iscale = nullptr;
  int D = 0, R = 0, K = 0;
};
template <typename T>
void launch_fwd1(const DevLevel& L, const FacLevel<T>& F, const ChildIn<T>& ch, cudaStream_t st);

template <typename T, typename TS>
void launch_fwd2(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, cudaStream_t st);
template <typename T, typename TS>
void launch_fwd3(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, T* parent_vin,
                 cudaStream_t st);
template <typename T, typename TS>
void launch_bwd1(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, const T* parent_x,
                 cudaStream_t st);
template <typename T, typename TS>
void launch_bwd2(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, const T* parent_x,
                 cudaStream_t st);
template <typename T>
void launch_gemv_rows(int nb, int n, const T* M, const T* x, T* y, cudaStream_t st);
template <typename T>
void launch_transpose_pairs(int D, int64_t n, const int32_t* dst, const int32_t* src, T* A, cudaStream_t st);
template <typename T>
void launch_transpose_blocks(int64_t nb, int D, const T* in, T* out, cudaStream_t st);  // out_b = in_b^T (D x D)  // y = M x, M n x n row-major

template <typename T>
void launch_matvec_up(const DevLevel& L, const T* X, const T* x, T* xh, cudaStream_t st);
template <typename T>
void launch_matvec_far(const DevLevel& L, const T* S, const T* xh, T* yh, cudaStream_t st);
template <typename T>
void launch_matvec_down(const DevLevel& L, const T* X, const T* yh, T* yh_child, cudaStream_t st);
template <typename T>
void launch_matvec_leaf(const DevLevel& L, const T* A, const T* X, const T* x, const T* yh, T* y, cudaStream_t st);
// The FP64 matvec with each FP64 matrix held as an FP32 pair (hi = fl32, lo
// = fl32 of the rest) and FP32-pair arithmetic throughout: the input vector
// is split once (launch_split_df), the basis coefficients xhat / yhat of
// every level and the leaf partial products stay FP32 pairs, and only the
// leaf output is converted to FP64.
// up: xhat_i = X_i^T z_i (z: the leaf input or the children's xhat)
void launch_matvec_up_df(const DevLevel& L, const float* Xh, const float* Xl, const float* zh, const float* zl,
                         float* oh, float* ol, cudaStream_t st);
// couplings of all levels in one launch: per level its far lists, the
// couplings S (hi / lo), xhat and yhat pairs; CTAs cta0 .. cta0 + nb nch - 1
// (nch 64-row chunks per box)
struct FarDfLevel {
  const int64_t* ptr;
  const int32_t* fj;
  const float *Sh, *Sl, *xh, *xl;
  float *yh, *yl;
  int nb, K, nch, cta0;
};
constexpr int kMaxFarDfLevels = 32;
struct FarDfArgs {
  int nlev;
  FarDfLevel lv[kMaxFarDfLevels];
};
void launch_matvec_far_df_all(const FarDfArgs& a, cudaStream_t st);
// down: [yhat_2p; yhat_2p+1] += X_p yhat_p
void launch_matvec_down_df(const DevLevel& L, const float* Xh, const float* Xl, const float* yh, const float* yl,
                           float* ych, float* ycl, cudaStream_t st);
// leaf, general near lists: y_i = X_i yhat_i + sum_{near j} A_ij x_j
void launch_matvec_leaf_df(const DevLevel& L, const float* Ah, const float* Al, const float* Xh, const float* Xl,
                           const float* xh, const float* xl, const float* yhh, const float* yhl, double* y,
                           cudaStream_t st);
// leaf, symmetric storage: y_i = X_i yhat_i + box i's partial products
void launch_matvec_sym_sum_df(int nb, int D, int K, const int64_t* ptr, const int32_t* ent, const float* Xh,
                              const float* Xl, const float* yhh, const float* yhl, const float* ph, const float* pl,
                              double* y, cudaStream_t st);
void launch_split_lo(const double* a, const float* hi, float* lo, int64_t n, cudaStream_t st);  // lo = fl32(a - hi)
void launch_split_df(const double* v, float* h, float* l, int64_t n, cudaStream_t st);  // h = fl32(v), l = fl32(v - h)
// Leaf matvec on the stored (i <= j) halves of symmetric leaf near blocks:
// per stored pair k = (ui[k], uj[k]) the partial products [A x_j; A^T x_i]
// into part (2 D per pair), then per box y = X yh + its partial products.
bool sym_leaf_supported(int D);  // D = 128 or 256
// Downward step [yh_2p; yh_2p+1] = X_p yh_p + (the children's coupling
// products summed over their CSR lists cptr / cent into part, Kc = D / 2
// entries per product; cptr NULL: none)
template <typename T>
void launch_matvec_down_far(const DevLevel& L, const T* X, const T* yh, T* yh_child, const int64_t* cptr,
                            const int32_t* cent, const T* part, cudaStream_t st);
// (pdl: launched to overlap its predecessor; off where events bracket it)
void launch_matvec_sym_pairs(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* A, const float* x,
                             float* part, bool pdl, cudaStream_t st);
void launch_matvec_sym_pairs_df(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* Ah,
                                const float* Al, const float* xh, const float* xl, float* ph, float* pl,
                                cudaStream_t st);
template <typename T>
void launch_matvec_sym_sum(int nb, int D, int K, const int64_t* ptr, const int32_t* ent, const T* X, const T* yh,
                           const T* part, T* y, cudaStream_t st, bool pdl = true);
// out[k] = fl32(in[idx[k]]), lo[k] = fl32(in[idx[k]] - hi[k]) for blocks of n entries
void launch_gather_blocks(const double* in, const int32_t* idx, int64_t n, int64_t nblk, float* out, cudaStream_t st);
void launch_gather_split_lo(const double* in, const int32_t* idx, int64_t n, int64_t nblk, const float* hi, float* lo,
                            cudaStream_t st);

void launch_gather(const int64_t* slot, const double* src, double* dst, int64_t nslots, cudaStream_t st);
void launch_scatter(const int64_t* slot, const double* src, double* dst, int64_t nslots, cudaStream_t st);
void launch_residual(const double* b, const double* y, double* r, int64_t n, cudaStream_t st);
template <typename T>
void launch_norm2(const T* v, int64_t n, double* out, cudaStream_t st);  // out[0] = sum v^2 (FP64), out[1..256] scratch
template <typename Ti, typename To>
void launch_scaled_copy(const Ti* in, const double* nrm2, bool inverse, To* out, int64_t n, cudaStream_t st);
template <typename T>
void launch_scale_to(const double* in, const double* norm2, T* out, int64_t n, cudaStream_t st);
template <typename T>
void launch_axpy_from(const T* d, const double* norm2, double* x, int64_t n, cudaStream_t st);
// GMRES: out[v] (+)= V_v . w for v < nv (part: nv * 128 scratch); w += sign sum_v coef[v] V_v;
// w = src / sqrt(nrm2[0])
template <typename T>
void launch_multi_dot(const T* V, int64_t ldv, int nv, const T* w, int64_t n, double* part, double* out,
                      bool accumulate, cudaStream_t st);
template <typename T, typename TW>
void launch_multi_axpy(const T* V, int64_t ldv, int nv, const double* coef, double sign, TW* w, int64_t n,
                       cudaStream_t st);

}  // namespace h2
