// Substitution, H^2 matvec and refinement kernels (sm_103a).
//
// Parallel substitution (Eq. 24-31, Section 3.7) and its mirror image for the
// backward pass.  With Ainv_i = (Ahat_ii^RR)^-1 = U'_ii^-1 (P_i L_ii)^-1, the
// product form of L^-1 in Eq. 31 needs only whole-block inverses and
// matrix-vector products, so every step below is a batched GEMV over all
// boxes of a level (one CTA per box), with no serial triangular solve:
//   fwd1  c_i = U_i^T b_i;                  u_i = Ainv_i c_i^R
//   fwd2  v_i = Ainv_i (c_i^R - sum_{j<i near} Ahat_ij^RR u_j)
//   fwd3  s_i = c_i^S - sum_{j near} Ahat_ij^SR v_j   -> parent input
//   bwd1  om_i = v_i - Ainv_i sum_{j near} Ahat_ij^RS x_j^S
//   bwd2  x_i^R = om_i - Ainv_i sum_{j>i near} Ahat_ij^RR om_j;
//         x_i = U_i [x_i^R; x_i^S]
// (fwd2 is L_ii^-1 (b_i^R - sum L(r)_ij L_jj^-1 b_j) followed by U'_ii^-1;
// bwd1/bwd2 are the mirror with U(s)_ij = (P_i L_ii)^-1 Ahat_ij^RS and
// U(r)_ij = (P_i L_ii)^-1 Ahat_ij^RR, multiplied through by U'_ii^-1.)
//
// H^2 matvec (FP64): upward pass x^_i = X_i^T x_i, couplings y^_i +=
// S_ij x^_j on every level, downward pass, leaf y_i = X_i y^_i +
// sum_near A_ij x_j.
#include "h2_internal.h"
#include "kernels.h"

namespace h2 {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ys[r] += sign * sum_c M[r*ld + c] xs[c], r < nr, c < nc; row r is owned by
// warp r % nwarps (so successive calls with the same nr never race).
template <typename T>
__device__ __forceinline__ void warp_rows_gemv(const T* __restrict__ M, int64_t ld, int nr, int nc,
                                               const T* xs, T* ys, T sign) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int r = warp;
  for (; r + 3 * nw < nr; r += 4 * nw) {
    const T* m0 = M + (int64_t)r * ld;
    const T* m1 = m0 + nw * ld;
    const T* m2 = m1 + nw * ld;
    const T* m3 = m2 + nw * ld;
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int c = lane; c < nc; c += 32) {
      T x = xs[c];
      s0 += m0[c] * x;
      s1 += m1[c] * x;
      s2 += m2[c] * x;
      s3 += m3[c] * x;
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    s3 = warp_sum(s3);
    if (lane == 0) {
      ys[r] += sign * s0;
      ys[r + nw] += sign * s1;
      ys[r + 2 * nw] += sign * s2;
      ys[r + 3 * nw] += sign * s3;
    }
  }
  for (; r < nr; r += nw) {
    const T* m0 = M + (int64_t)r * ld;
    T s0 = 0;
    for (int c = lane; c < nc; c += 32) s0 += m0[c] * xs[c];
    s0 = warp_sum(s0);
    if (lane == 0) ys[r] += sign * s0;
  }
}

// ------------------------------------------------------------------------
// Block-row GEMV core.  Warp w owns rows w, w + 8, ... (at most 8 * RPW
// rows); each lane holds a partial sum per owned row over its column chunks
// and keeps accumulating over all blocks of the block row, so the warp
// reduction happens once per row at the end.  Rows are read with 16-byte
// vector loads when the layout allows.
// ------------------------------------------------------------------------
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static float fma4(const V& a, const V& x, float s) {
    s = fmaf(a.x, x.x, s);
    s = fmaf(a.y, x.y, s);
    s = fmaf(a.z, x.z, s);
    return fmaf(a.w, x.w, s);
  }
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ static V zero() { return make_double2(0.0, 0.0); }
  __device__ static double fma4(const V& a, const V& x, double s) { return fma(a.y, x.y, fma(a.x, x.x, s)); }
};

// acc[t] += sum_c M[r_t * ld + c] xs[c] for the rows r_t = r0 + warp + 8 t < nr.
// For each column chunk every lane first issues the loads of all its rows,
// then does the multiply-adds, so RPW independent 16-byte loads per lane are
// in flight at once.
template <typename T, int RPW>
__device__ __forceinline__ void rows_acc(int r0, const T* __restrict__ M, int64_t ld, int nr, int nc,
                                         const T* __restrict__ xs, T (&acc)[RPW]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  using VT = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::n;
  const bool vec = ((ld % VN) == 0) && ((nc % (32 * VN)) == 0) && ((reinterpret_cast<uintptr_t>(M) & 15) == 0);
  const int rbase = r0 + warp;
  if (vec) {
    for (int c = lane; c < nc / VN; c += 32) {
      VT v[RPW];
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        const int r = rbase + 8 * t;
        v[t] = (r < nr) ? __ldg(reinterpret_cast<const VT*>(M + r * ld) + c) : Vec16<T>::zero();
      }
      const VT x = *reinterpret_cast<const VT*>(xs + c * VN);
#pragma unroll
      for (int t = 0; t < RPW; ++t) acc[t] = Vec16<T>::fma4(v[t], x, acc[t]);
    }
  } else {
    for (int c = lane; c < nc; c += 32) {
      T v[RPW];
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        const int r = rbase + 8 * t;
        v[t] = (r < nr) ? __ldg(M + r * ld + c) : T(0);
      }
      const T x = xs[c];
#pragma unroll
      for (int t = 0; t < RPW; ++t) acc[t] = fma(v[t], x, acc[t]);
    }
  }
}

// out[r] = base[r] + sign * sum over lanes of acc (rows owned by this warp)
template <typename T, int RPW>
__device__ __forceinline__ void rows_finish(int r0, int nr, const T (&acc)[RPW], T sign, const T* base, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < RPW; ++t) {
    const int r = r0 + warp + 8 * t;
    T v = warp_sum(acc[t]);
    if (lane == 0 && r < nr) out[r] = (base ? base[r] : T(0)) + sign * v;
  }
}

template <typename T, int RPW>
__device__ __forceinline__ void zero(T (&acc)[RPW]) {
#pragma unroll
  for (int t = 0; t < RPW; ++t) acc[t] = T(0);
}

constexpr int kRPW = 16;  // rows per warp per pass: 128-row chunks with 8 warps
constexpr int kChunk = 8 * kRPW;

// ---------------------------------------------------------------- fwd1 ---
template <typename T>
__global__ void __launch_bounds__(256, 2) fwd1_kernel(int D, int R, const T* __restrict__ U, const T* __restrict__ Ainv,
                                                   const T* __restrict__ vin, T* __restrict__ c, T* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sv = reinterpret_cast<T*>(sm_raw);  // D
  T* sc = sv + D;                        // D
  const int i = blockIdx.x, tid = threadIdx.x;
  for (int e = tid; e < D; e += blockDim.x) sv[e] = vin[(int64_t)i * D + e];
  __syncthreads();
  T acc[kRPW];
  // c[n] = sum_k U(k, n) v[k]; U column-major: column n is contiguous
  for (int r0 = 0; r0 < D; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, U + (int64_t)i * D * D, D, D, D, sv, acc);
    rows_finish<T, kRPW>(r0, D, acc, T(1), nullptr, sc);
  }
  __syncthreads();
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, Ainv + (int64_t)i * R * R, R, R, R, sc, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(1), nullptr, u + (int64_t)i * R);
  }
  for (int e = tid; e < D; e += blockDim.x) c[(int64_t)i * D + e] = sc[e];
}

// ---------------------------------------------------------------- fwd2 ---
// v_i = Ainv_i (c_i^R - sum_{j<i near} Ahat_ij^RR u_j)
template <typename T>
__global__ void __launch_bounds__(256, 2) fwd2_kernel(int D, int R, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ nj, const T* __restrict__ Ahat,
                                                   const T* __restrict__ Ainv, const T* __restrict__ c,
                                                   const T* __restrict__ u, T* __restrict__ v) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sb = reinterpret_cast<T*>(sm_raw);  // R
  T* sx = sb + R;                        // nn * R
  const int i = blockIdx.x, tid = threadIdx.x;
  const int64_t p0 = ptr[i];
  int nlow = 0;
  while (p0 + nlow < ptr[i + 1] && nj[p0 + nlow] < i) ++nlow;  // sorted neighbours: the j < i ones lead
  for (int e = tid; e < nlow * R; e += blockDim.x) sx[e] = u[(int64_t)nj[p0 + e / R] * R + e % R];
  __syncthreads();
  T acc[kRPW];
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    for (int q = 0; q < nlow; ++q) rows_acc<T, kRPW>(r0, Ahat + (p0 + q) * D * D, D, R, R, sx + q * R, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(-1), c + (int64_t)i * D, sb);
  }
  __syncthreads();
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, Ainv + (int64_t)i * R * R, R, R, R, sb, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(1), nullptr, v + (int64_t)i * R);
  }
}

// ---------------------------------------------------------------- fwd3 ---
// s_i = c_i^S - sum_{j near} Ahat_ij^SR v_j  -> parent input slot
template <typename T>
__global__ void __launch_bounds__(256, 2) fwd3_kernel(int D, int R, int K, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ nj, const T* __restrict__ Ahat,
                                                   const T* __restrict__ c, const T* __restrict__ v,
                                                   T* __restrict__ pvin) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sx = reinterpret_cast<T*>(sm_raw);  // nn * R
  const int i = blockIdx.x, tid = threadIdx.x;
  const int64_t p0 = ptr[i];
  const int nn = (int)(ptr[i + 1] - p0);
  for (int e = tid; e < nn * R; e += blockDim.x) sx[e] = v[(int64_t)nj[p0 + e / R] * R + e % R];
  __syncthreads();
  T acc[kRPW];
  const int Dp = 2 * K;
  for (int r0 = 0; r0 < K; r0 += kChunk) {
    zero(acc);
    for (int q = 0; q < nn; ++q)
      rows_acc<T, kRPW>(r0, Ahat + (p0 + q) * D * D + (int64_t)R * D, D, K, R, sx + q * R, acc);
    rows_finish<T, kRPW>(r0, K, acc, T(-1), c + (int64_t)i * D + R, pvin + (int64_t)(i >> 1) * Dp + (i & 1) * K);
  }
}

// ---------------------------------------------------------------- bwd1 ---
// om_i = v_i - Ainv_i sum_{j near} Ahat_ij^RS x_j^S
template <typename T>
__global__ void __launch_bounds__(256, 2) bwd1_kernel(int D, int R, int K, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ nj, const T* __restrict__ Ahat,
                                                   const T* __restrict__ Ainv, const T* __restrict__ v,
                                                   const T* __restrict__ px, T* __restrict__ om) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* st = reinterpret_cast<T*>(sm_raw);  // R
  T* sx = st + R;                        // nn * K
  const int i = blockIdx.x, tid = threadIdx.x, Dp = 2 * K;
  const int64_t p0 = ptr[i];
  const int nn = (int)(ptr[i + 1] - p0);
  for (int e = tid; e < nn * K; e += blockDim.x) {
    const int j = nj[p0 + e / K];
    sx[e] = px[(int64_t)(j >> 1) * Dp + (j & 1) * K + e % K];
  }
  __syncthreads();
  T acc[kRPW];
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    for (int q = 0; q < nn; ++q) rows_acc<T, kRPW>(r0, Ahat + (p0 + q) * D * D + R, D, R, K, sx + q * K, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(1), nullptr, st);
  }
  __syncthreads();
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, Ainv + (int64_t)i * R * R, R, R, R, st, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(-1), v + (int64_t)i * R, om + (int64_t)i * R);
  }
}

// ---------------------------------------------------------------- bwd2 ---
// x_i^R = om_i - Ainv_i sum_{j>i near} Ahat_ij^RR om_j;  x_i = U_i [x_i^R; x_i^S]
template <typename T>
__global__ void __launch_bounds__(256, 2) bwd2_kernel(int D, int R, int K, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ nj, const T* __restrict__ Ahat,
                                                   const T* __restrict__ Ainv, const T* __restrict__ U,
                                                   const T* __restrict__ om, const T* __restrict__ px,
                                                   T* __restrict__ xs) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sq = reinterpret_cast<T*>(sm_raw);  // R
  T* sz = sq + R;                        // D
  T* sx = sz + D;                        // nn * R
  const int i = blockIdx.x, tid = threadIdx.x, Dp = 2 * K;
  const int64_t p0 = ptr[i], p1 = ptr[i + 1];
  int first = 0;
  while (p0 + first < p1 && nj[p0 + first] <= i) ++first;  // neighbours j > i trail
  const int nhi = (int)(p1 - p0) - first;
  for (int e = tid; e < nhi * R; e += blockDim.x) sx[e] = om[(int64_t)nj[p0 + first + e / R] * R + e % R];
  for (int e = tid; e < K; e += blockDim.x) sz[R + e] = px[(int64_t)(i >> 1) * Dp + (i & 1) * K + e];
  __syncthreads();
  T acc[kRPW];
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    for (int q = 0; q < nhi; ++q)
      rows_acc<T, kRPW>(r0, Ahat + (p0 + first + q) * D * D, D, R, R, sx + q * R, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(1), nullptr, sq);
  }
  __syncthreads();
  for (int r0 = 0; r0 < R; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, Ainv + (int64_t)i * R * R, R, R, R, sq, acc);
    rows_finish<T, kRPW>(r0, R, acc, T(-1), om + (int64_t)i * R, sz);
  }
  __syncthreads();
  // x = U z, U column-major: x[m] = sum_n U[n*D + m] z[n] (coalesced over m)
  const T* Ub = U + (int64_t)i * D * D;
  for (int m = tid; m < D; m += blockDim.x) {
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int n = 0;
    for (; n + 3 < D; n += 4) {
      s0 = fma(Ub[(int64_t)n * D + m], sz[n], s0);
      s1 = fma(Ub[(int64_t)(n + 1) * D + m], sz[n + 1], s1);
      s2 = fma(Ub[(int64_t)(n + 2) * D + m], sz[n + 2], s2);
      s3 = fma(Ub[(int64_t)(n + 3) * D + m], sz[n + 3], s3);
    }
    for (; n < D; ++n) s0 = fma(Ub[(int64_t)n * D + m], sz[n], s0);
    xs[(int64_t)i * D + m] = (s0 + s1) + (s2 + s3);
  }
}

static void set_smem(const void* f, size_t sm) {
  if (sm > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename T>
void launch_fwd1(const DevLevel& L, const FacLevel<T>& F, const T* Ainv, cudaStream_t st) {
  size_t sm = sizeof(T) * 2 * L.D;
  ++g_launches;
  fwd1_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.R, F.U, Ainv, F.vin, F.c, F.u);
}
template <typename T>
void launch_fwd2(const DevLevel& L, const FacLevel<T>& F, const T* Ainv, cudaStream_t st) {
  size_t sm = sizeof(T) * (size_t)L.R * (1 + L.max_near);
  set_smem((const void*)fwd2_kernel<T>, sm);
  ++g_launches;
  fwd2_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.R, L.near_ptr, L.near_j, F.Ahat, Ainv, F.c, F.u, F.v);
}
template <typename T>
void launch_fwd3(const DevLevel& L, const FacLevel<T>& F, T* parent_vin, cudaStream_t st) {
  size_t sm = sizeof(T) * (size_t)L.R * L.max_near;
  set_smem((const void*)fwd3_kernel<T>, sm);
  ++g_launches;
  fwd3_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.R, L.K, L.near_ptr, L.near_j, F.Ahat, F.c, F.v, parent_vin);
}
template <typename T>
void launch_bwd1(const DevLevel& L, const FacLevel<T>& F, const T* Ainv, const T* parent_x, cudaStream_t st) {
  size_t sm = sizeof(T) * ((size_t)L.R + (size_t)L.K * L.max_near);
  set_smem((const void*)bwd1_kernel<T>, sm);
  ++g_launches;
  bwd1_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.R, L.K, L.near_ptr, L.near_j, F.Ahat, Ainv, F.v, parent_x, F.om);
}
template <typename T>
void launch_bwd2(const DevLevel& L, const FacLevel<T>& F, const T* Ainv, const T* parent_x, cudaStream_t st) {
  size_t sm = sizeof(T) * ((size_t)L.R + L.D + (size_t)L.R * L.max_near);
  set_smem((const void*)bwd2_kernel<T>, sm);
  ++g_launches;
  bwd2_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.R, L.K, L.near_ptr, L.near_j, F.Ahat, Ainv, F.U, F.om, parent_x,
                                        F.xs);
}

// y = M x for one n x n row-major matrix (root solve with the explicit inverse)
template <typename T>
__global__ void gemv_rows_kernel(int n, const T* __restrict__ M, const T* __restrict__ x, T* __restrict__ y) {
  extern __shared__ unsigned char sm_raw[];
  T* sx = reinterpret_cast<T*>(sm_raw);
  T* sy = sx + n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) { sx[e] = x[e]; sy[e] = 0; }
  __syncthreads();
  warp_rows_gemv<T>(M, n, n, n, sx, sy, T(1));
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) y[e] = sy[e];
}
template <typename T>
void launch_gemv_rows(int n, const T* M, const T* x, T* y, cudaStream_t st) {
  if (n == 0) return;
  const size_t sm = sizeof(T) * 2 * (size_t)n;
  if (sm > 48 * 1024) cudaFuncSetAttribute(gemv_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  gemv_rows_kernel<T><<<1, 256, sm, st>>>(n, M, x, y);
}

#define H2_INST_SOLVE(T)                                                                              \
  template void launch_fwd1<T>(const DevLevel&, const FacLevel<T>&, const T*, cudaStream_t);          \
  template void launch_fwd2<T>(const DevLevel&, const FacLevel<T>&, const T*, cudaStream_t);          \
  template void launch_fwd3<T>(const DevLevel&, const FacLevel<T>&, T*, cudaStream_t);                \
  template void launch_bwd1<T>(const DevLevel&, const FacLevel<T>&, const T*, const T*, cudaStream_t); \
  template void launch_bwd2<T>(const DevLevel&, const FacLevel<T>&, const T*, const T*, cudaStream_t); \
  template void launch_gemv_rows<T>(int, const T*, const T*, T*, cudaStream_t);
H2_INST_SOLVE(double)
H2_INST_SOLVE(float)

// ------------------------------------------------------------- matvec ---
// Element type T: double for the refinement residual, float for the inner
// solver of the mixed-precision refinement.  X, S and A are that level's
// bases, couplings and leaf near blocks in T.

// upward: xh_i[a] = sum_d X_i[d*K + a] x_i[d] (x_i: the box's D inputs).
// Warp w takes the rows d = w, w + 8, ...; lanes take the columns a; each
// warp accumulates its partial sums in its own row of shared memory, then
// the 8 partial rows are added.
template <typename T>
__global__ void __launch_bounds__(256) mv_up_kernel(int D, int K, const T* __restrict__ X, const T* __restrict__ x,
                                                    T* __restrict__ xh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* part = reinterpret_cast<T*>(smraw);  // 8 * K
  T* sx = part + 8 * K;                   // D
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* Xb = X + (int64_t)i * D * K;
  for (int e = tid; e < D; e += 256) sx[e] = x[(int64_t)i * D + e];
  for (int e = tid; e < 8 * K; e += 256) part[e] = T(0);
  __syncthreads();
  T* mine = part + warp * K;
  for (int a0 = 0; a0 < K; a0 += 128) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int d = warp; d < D; d += 8) {
      const T xd = sx[d];
      const T* row = Xb + (int64_t)d * K + a0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = a0 + lane + 32 * q;
        if (a < K) acc[q] = fma(__ldg(row + lane + 32 * q), xd, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = a0 + lane + 32 * q;
      if (a < K) mine[a] = acc[q];
    }
  }
  __syncthreads();
  for (int a = tid; a < K; a += 256) {
    T s = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) s += part[w * K + a];
    xh[(int64_t)i * K + a] = s;
  }
}
template <typename T>
void launch_matvec_up(const DevLevel& L, const T* X, const T* x, T* xh, cudaStream_t st) {
  const size_t sm = sizeof(T) * (8 * (size_t)L.K + L.D);
  set_smem((const void*)mv_up_kernel<T>, sm);
  ++g_launches;
  mv_up_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.K, X, x, xh);
}

// couplings: yh_i = sum_{far j} S_f xh_j   (overwrites yh_i)
template <typename T>
__global__ void __launch_bounds__(256, 2) mv_far_kernel(int K, const int64_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ fj, const T* __restrict__ S,
                                                        const T* __restrict__ xh, T* __restrict__ yh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* smv = reinterpret_cast<T*>(smraw);  // nf * K
  const int i = blockIdx.x, tid = threadIdx.x;
  const int64_t p0 = ptr[i];
  const int nf = (int)(ptr[i + 1] - p0);
  for (int e = tid; e < nf * K; e += blockDim.x) smv[e] = xh[(int64_t)fj[p0 + e / K] * K + e % K];
  __syncthreads();
  T acc[kRPW];
  for (int r0 = 0; r0 < K; r0 += kChunk) {
    zero(acc);
    for (int q = 0; q < nf; ++q) rows_acc<T, kRPW>(r0, S + (p0 + q) * K * K, K, K, K, smv + q * K, acc);
    rows_finish<T, kRPW>(r0, K, acc, T(1), nullptr, yh + (int64_t)i * K);
  }
}
template <typename T>
void launch_matvec_far(const DevLevel& L, const T* S, const T* xh, T* yh, cudaStream_t st) {
  size_t sm = sizeof(T) * (size_t)L.K * std::max(L.max_far, 1);
  set_smem((const void*)mv_far_kernel<T>, sm);
  ++g_launches;
  mv_far_kernel<T><<<L.nb, 256, sm, st>>>(L.K, L.far_ptr, L.far_j, S, xh, yh);
}

// downward: [yh_2p; yh_2p+1] += X_p yh_p   (rows d of X_p, D = 2 Kc): a
// block-row GEMV per parent box
template <typename T>
__global__ void __launch_bounds__(256, 2) mv_down_kernel(int D, int K, const T* __restrict__ X,
                                                         const T* __restrict__ yh, T* __restrict__ yhc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sy = reinterpret_cast<T*>(smraw);  // K
  const int p = blockIdx.x;
  for (int e = threadIdx.x; e < K; e += 256) sy[e] = yh[(int64_t)p * K + e];
  __syncthreads();
  T acc[kRPW];
  T* out = yhc + (int64_t)p * D;
  for (int r0 = 0; r0 < D; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, X + (int64_t)p * D * K, K, D, K, sy, acc);
    rows_finish<T, kRPW>(r0, D, acc, T(1), out, out);
  }
}
template <typename T>
void launch_matvec_down(const DevLevel& L, const T* X, const T* yh, T* yh_child, cudaStream_t st) {
  ++g_launches;
  mv_down_kernel<T><<<L.nb, 256, sizeof(T) * ((L.K + 3) & ~3), st>>>(L.D, L.K, X, yh, yh_child);
}

// leaf: y_i = X_i yh_i + sum_{near j} A_ij x_j
template <typename T>
__global__ void __launch_bounds__(256, 2) mv_leaf_kernel(int D, int K, const int64_t* __restrict__ ptr,
                                                         const int32_t* __restrict__ nj, const T* __restrict__ A,
                                                         const T* __restrict__ X, const T* __restrict__ x,
                                                         const T* __restrict__ yh, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* smv = reinterpret_cast<T*>(smraw);  // K (rounded up to 16 bytes) + nn * D
  const int i = blockIdx.x, tid = threadIdx.x;
  const int64_t p0 = ptr[i];
  const int nn = (int)(ptr[i + 1] - p0);
  const int kpad = (K + 3) & ~3;
  T* sh = smv;
  T* sx = smv + kpad;
  if (yh)
    for (int e = tid; e < K; e += blockDim.x) sh[e] = yh[(int64_t)i * K + e];
  for (int e = tid; e < nn * D; e += blockDim.x) sx[e] = x[(int64_t)nj[p0 + e / D] * D + e % D];
  __syncthreads();
  T acc[kRPW];
  for (int r0 = 0; r0 < D; r0 += kChunk) {
    zero(acc);
    if (yh) rows_acc<T, kRPW>(r0, X + (int64_t)i * D * K, K, D, K, sh, acc);
    for (int q = 0; q < nn; ++q) rows_acc<T, kRPW>(r0, A + (p0 + q) * D * D, D, D, D, sx + q * D, acc);
    rows_finish<T, kRPW>(r0, D, acc, T(1), nullptr, y + (int64_t)i * D);
  }
}
template <typename T>
void launch_matvec_leaf(const DevLevel& L, const T* A, const T* X, const T* x, const T* yh, T* y, cudaStream_t st) {
  const size_t sm = sizeof(T) * ((size_t)((L.K + 3) & ~3) + (size_t)L.D * L.max_near);
  set_smem((const void*)mv_leaf_kernel<T>, sm);
  ++g_launches;
  mv_leaf_kernel<T><<<L.nb, 256, sm, st>>>(L.D, L.K, L.near_ptr, L.near_j, A, X, x, yh, y);
}

#define H2_INST_MV(T)                                                                                           \
  template void launch_matvec_up<T>(const DevLevel&, const T*, const T*, T*, cudaStream_t);                      \
  template void launch_matvec_far<T>(const DevLevel&, const T*, const T*, T*, cudaStream_t);                     \
  template void launch_matvec_down<T>(const DevLevel&, const T*, const T*, T*, cudaStream_t);                    \
  template void launch_matvec_leaf<T>(const DevLevel&, const T*, const T*, const T*, const T*, T*, cudaStream_t);
H2_INST_MV(double)
H2_INST_MV(float)

// ------------------------------------------------------------ vectors ---
__global__ void gather_kernel(const int64_t* __restrict__ slot, const double* __restrict__ src,
                              double* __restrict__ dst, int64_t n) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = slot[s];
    dst[s] = o >= 0 ? src[o] : 0.0;
  }
}
__global__ void scatter_kernel(const int64_t* __restrict__ slot, const double* __restrict__ src,
                               double* __restrict__ dst, int64_t n) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = slot[s];
    if (o >= 0) dst[o] = src[s];
  }
}
static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }
void launch_gather(const int64_t* slot, const double* src, double* dst, int64_t n, cudaStream_t st) {
  ++g_launches;
  gather_kernel<<<grid_for(n), 256, 0, st>>>(slot, src, dst, n);
}
void launch_scatter(const int64_t* slot, const double* src, double* dst, int64_t n, cudaStream_t st) {
  ++g_launches;
  scatter_kernel<<<grid_for(n), 256, 0, st>>>(slot, src, dst, n);
}
__global__ void residual_kernel(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                                int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - y[e];
}
void launch_residual(const double* b, const double* y, double* r, int64_t n, cudaStream_t st) {
  ++g_launches;
  residual_kernel<<<grid_for(n), 256, 0, st>>>(b, y, r, n);
}
// deterministic two-pass sum of squares (accumulated in FP64): 256 partials,
// then one block
template <typename T>
__global__ void norm2_part_kernel(const T* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double sb[8];
  double s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[e];
    s = fma(x, x, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += sb[w];
    part[blockIdx.x] = t;
  }
}
__global__ void norm2_final_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sb[8];
  double s = 0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) s += part[e];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += sb[w];
    out[0] = t;
  }
}
template <typename T>
void launch_norm2(const T* v, int64_t n, double* out, cudaStream_t st) {
  ++g_launches;
  norm2_part_kernel<T><<<256, 256, 0, st>>>(v, n, out + 1);
  ++g_launches;
  norm2_final_kernel<<<1, 256, 0, st>>>(out + 1, 256, out);
}
template void launch_norm2<double>(const double*, int64_t, double*, cudaStream_t);
template void launch_norm2<float>(const float*, int64_t, double*, cudaStream_t);

// out[e] = (To)(in[e] * scale), scale = 1/sqrt(nrm2[0]) (or sqrt(nrm2[0]) when
// inverse == 0); nrm2 == NULL: plain conversion
template <typename Ti, typename To>
__global__ void scaled_copy_kernel(const Ti* __restrict__ in, const double* __restrict__ nrm2, int inverse,
                                   To* __restrict__ out, int64_t n) {
  double s = 1.0;
  if (nrm2) {
    const double r = sqrt(nrm2[0]);
    s = inverse ? (r > 0 ? 1.0 / r : 0.0) : r;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (To)((double)in[e] * s);
}
template <typename Ti, typename To>
void launch_scaled_copy(const Ti* in, const double* nrm2, bool inverse, To* out, int64_t n, cudaStream_t st) {
  ++g_launches;
  scaled_copy_kernel<Ti, To><<<grid_for(n), 256, 0, st>>>(in, nrm2, inverse ? 1 : 0, out, n);
}
template void launch_scaled_copy<double, float>(const double*, const double*, bool, float*, int64_t, cudaStream_t);
template void launch_scaled_copy<float, double>(const float*, const double*, bool, double*, int64_t, cudaStream_t);
template void launch_scaled_copy<float, float>(const float*, const double*, bool, float*, int64_t, cudaStream_t);
template void launch_scaled_copy<double, double>(const double*, const double*, bool, double*, int64_t,
                                                 cudaStream_t);
template <typename T>
__global__ void scale_to_kernel(const double* __restrict__ in, const double* __restrict__ nrm2, T* __restrict__ out,
                                int64_t n) {
  const double s = nrm2[0] > 0 ? 1.0 / sqrt(nrm2[0]) : 1.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)(in[e] * s);
}
template <typename T>
__global__ void axpy_from_kernel(const T* __restrict__ d, const double* __restrict__ nrm2, double* __restrict__ x,
                                 int64_t n) {
  const double s = nrm2[0] > 0 ? sqrt(nrm2[0]) : 1.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += s * (double)d[e];
}
template <typename T>
void launch_scale_to(const double* in, const double* norm2, T* out, int64_t n, cudaStream_t st) {
  ++g_launches;
  scale_to_kernel<T><<<grid_for(n), 256, 0, st>>>(in, norm2, out, n);
}
template <typename T>
void launch_axpy_from(const T* d, const double* norm2, double* x, int64_t n, cudaStream_t st) {
  ++g_launches;
  axpy_from_kernel<T><<<grid_for(n), 256, 0, st>>>(d, norm2, x, n);
}
// ---------------------------------------------------------- GMRES blocks ---
// part[v * nblk + blk] = partial sums of V_v . w (FP64); out[v] (+)= the sum
template <typename T>
__global__ void multi_dot_part_kernel(const T* __restrict__ V, int64_t ldv, const T* __restrict__ w, int64_t n,
                                      double* __restrict__ part) {
  __shared__ double sb[8];
  const int v = blockIdx.y;
  const T* Vv = V + (int64_t)v * ldv;
  double s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)Vv[e], (double)w[e], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < 8; ++k) t += sb[k];
    part[(int64_t)v * gridDim.x + blockIdx.x] = t;
  }
}
__global__ void multi_dot_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out,
                                       int accumulate) {
  __shared__ double sb[8];
  const int v = blockIdx.x;
  double s = 0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += part[(int64_t)v * nblk + k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < 8; ++k) t += sb[k];
    out[v] = accumulate ? out[v] + t : t;
  }
}
template <typename T>
void launch_multi_dot(const T* V, int64_t ldv, int nv, const T* w, int64_t n, double* part, double* out,
                      bool accumulate, cudaStream_t st) {
  if (nv == 0) return;
  const int nblk = 128;
  ++g_launches;
  multi_dot_part_kernel<T><<<dim3(nblk, nv), 256, 0, st>>>(V, ldv, w, n, part);
  ++g_launches;
  multi_dot_final_kernel<<<nv, 256, 0, st>>>(part, nblk, out, accumulate ? 1 : 0);
}
// w += sign * sum_v coef[v] V_v   (coefficients in FP64)
template <typename T, typename TW>
__global__ void multi_axpy_kernel(const T* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ coef,
                                  double sign, TW* __restrict__ w, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int v = 0; v < nv; ++v) s = fma(coef[v], (double)V[(int64_t)v * ldv + e], s);
    w[e] = (TW)((double)w[e] + sign * s);
  }
}
template <typename T, typename TW>
void launch_multi_axpy(const T* V, int64_t ldv, int nv, const double* coef, double sign, TW* w, int64_t n,
                       cudaStream_t st) {
  if (nv == 0) return;
  ++g_launches;
  multi_axpy_kernel<T, TW><<<grid_for(n), 256, 0, st>>>(V, ldv, nv, coef, sign, w, n);
}
template void launch_multi_dot<double>(const double*, int64_t, int, const double*, int64_t, double*, double*, bool,
                                       cudaStream_t);
template void launch_multi_dot<float>(const float*, int64_t, int, const float*, int64_t, double*, double*, bool,
                                      cudaStream_t);
template void launch_multi_axpy<double, double>(const double*, int64_t, int, const double*, double, double*, int64_t,
                                                cudaStream_t);
template void launch_multi_axpy<float, float>(const float*, int64_t, int, const double*, double, float*, int64_t,
                                              cudaStream_t);
template void launch_multi_axpy<float, double>(const float*, int64_t, int, const double*, double, double*, int64_t,
                                               cudaStream_t);

template void launch_scale_to<double>(const double*, const double*, double*, int64_t, cudaStream_t);
template void launch_scale_to<float>(const double*, const double*, float*, int64_t, cudaStream_t);
template void launch_axpy_from<double>(const double*, const double*, double*, int64_t, cudaStream_t);
template void launch_axpy_from<float>(const float*, const double*, double*, int64_t, cudaStream_t);

}  // namespace h2
