// Factorization kernels of the H^2-ULV library (sm_103a).
//
//   eval_blocks_kernel     dense kernel blocks G(B_i, B_j) of the leaf near
//                          pairs and couplings G(SK_i, SK_j) (Algorithm 1),
//                          evaluated from the points
//   gemm_batched_kernel    SIMT batched GEMM C = alpha op(A) op(B) + beta C
//                          (FP64 path: the projection and Schur update
//                          of Algorithm 4, couplings)
//   qr_panel_kernel,       Householder QR of X^orth, its compact WY factor
//   wy_tfactor_kernel      and the explicit U = [U^R U^S] (Eq. 6-7)
//   lu_inverse_kernel      partial-pivot LU of Ahat_ii^RR in FP64 (Algorithm
//                          2, with LU in place of Cholesky) and the
//                          explicit inverse (Ahat_ii^RR)^-1 used by the
//                          Schur update and by the substitution of Eq. 31
//   merge_kernel           children's SS blocks / couplings into the parent
//                          near blocks (the merge of Algorithm 2)
#include <type_traits>

#include "h2_internal.h"
#include "kernels.h"
#include "ptx_util.h"

namespace h2 {

// ------------------------------------------------------------------------
// block evaluation
// ------------------------------------------------------------------------
template <typename T>
__global__ void eval_blocks_kernel(KernelFn G, const double* __restrict__ pts, int64_t npairs,
                                   const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
                                   const int64_t* __restrict__ idx, int idx_stride, int rows, int cols,
                                   T* __restrict__ out) {
  int64_t per = (int64_t)rows * cols;
  int64_t total = npairs * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e / per;
    int64_t rc = e - p * per;
    int r = (int)(rc / cols), c = (int)(rc - (int64_t)r * cols);
    int i = pi[p], j = pj[p];
    int64_t a = idx[(int64_t)i * idx_stride + r], b = idx[(int64_t)j * idx_stride + c];
    out[e] = (T)G.entry(pts, a, b, i == j && r == c);
  }
}

void launch_eval_blocks(const KernelFn& G, const double* pts, int64_t npairs, const int32_t* pi,
                        const int32_t* pj, const int64_t* idx, int idx_stride, int rows, int cols,
                        double* out, cudaStream_t st) {
  if (npairs == 0 || rows == 0 || cols == 0) return;
  int64_t total = npairs * rows * cols;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
  ++g_launches;
  eval_blocks_kernel<double><<<blocks, 256, 0, st>>>(G, pts, npairs, pi, pj, idx, idx_stride, rows, cols, out);
}

// ------------------------------------------------------------------------
// conversions
// ------------------------------------------------------------------------
template <typename S, typename T>
__global__ void convert_kernel(const S* __restrict__ in, T* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)in[e];
}
template <typename S, typename T>
void launch_convert(const S* in, T* out, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  ++g_launches;
  convert_kernel<S, T><<<blocks, 256, 0, st>>>(in, out, n);
}
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<float, float>(const float*, float*, int64_t, cudaStream_t);

// ------------------------------------------------------------------------
// SIMT batched GEMM (row-major operands):
//   op(A)(m,k) = tA ? A[k*lda+m] : A[m*lda+k]
//   op(B)(k,n) = tB ? B[n*ldb+k] : B[k*ldb+n]
//   C(m,n)     = C[m*ldc+n]
// Batch b uses A + (ia ? ia[b] : b) * sA, likewise B and C.
// ------------------------------------------------------------------------
template <typename T, typename TB>
__global__ void __launch_bounds__(256)
gemm_batched_kernel(int M, int N, int K, const T* __restrict__ A, int64_t sA, const int32_t* __restrict__ ia,
                    int lda, int tA, const TB* __restrict__ B, int64_t sB, const int32_t* __restrict__ ib,
                    int ldb, int tB, T* __restrict__ C, int64_t sC, const int32_t* __restrict__ ic, int ldc,
                    T alpha, T beta, int64_t batch) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  for (int64_t b = blockIdx.z; b < batch; b += gridDim.z) {
    const T* Ab = A + (ia ? (int64_t)ia[b] : b) * sA;
    const TB* Bb = B + (ib ? (int64_t)ib[b] : b) * sB;
    T* Cb = C + (ic ? (int64_t)ic[b] : b) * sC;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
      for (int e = threadIdx.x; e < BM * BK; e += 256) {
        int mm, kk;
        if (tA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
        int gm = m0 + mm, gk = k0 + kk;
        T v = T(0);
        if (gm < M && gk < K) v = tA ? Ab[(int64_t)gk * lda + gm] : Ab[(int64_t)gm * lda + gk];
        As[kk][mm] = v;
      }
      for (int e = threadIdx.x; e < BN * BK; e += 256) {
        int nn, kk;
        if (tB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
        int gn = n0 + nn, gk = k0 + kk;
        T v = T(0);
        if (gn < N && gk < K) v = (T)(tB ? Bb[(int64_t)gn * ldb + gk] : Bb[(int64_t)gk * ldb + gn]);
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 16 * j;
        if (gn >= N) continue;
        T* cp = Cb + (int64_t)gm * ldc + gn;
        T r = alpha * acc[i][j];
        if (beta != T(0)) r = fma(beta, *cp, r);
        *cp = r;
      }
    }
  }
}

// FP32 form for tile-sized problems: 128 x 128 tiles, BK = 8, 256 threads
// each holding an 8 x 8 block of C (rows ty*4 + {0..3, 64..67}, columns
// tx*4 + {0..3, 64..67}) so that every shared-memory read is a 16-byte
// vector; the next k-slice is fetched into registers while the current one
// is used, and two shared buffers leave one barrier per slice.
constexpr int G2_BM = 128, G2_BN = 128, G2_BK = 8, G2_LD = 132;

__device__ __forceinline__ void g2_load_a(const float* __restrict__ Ab, int lda, int tA, int M, int K, int m0, int k0,
                                          bool vec, float (&ra)[4]) {
  const int t = threadIdx.x;
  if (!tA) {  // A[m * lda + k]: 4 consecutive k of row m
    const int m = m0 + (t >> 1), k = k0 + (t & 1) * 4;
    if (vec && m < M && k + 3 < K) {
      const float4 v = *reinterpret_cast<const float4*>(Ab + (int64_t)m * lda + k);
      ra[0] = v.x, ra[1] = v.y, ra[2] = v.z, ra[3] = v.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) ra[e] = (m < M && k + e < K) ? Ab[(int64_t)m * lda + k + e] : 0.0f;
    }
  } else {  // A[k * lda + m]: 4 consecutive m of row k
    const int k = k0 + (t >> 5), m = m0 + (t & 31) * 4;
    if (vec && k < K && m + 3 < M) {
      const float4 v = *reinterpret_cast<const float4*>(Ab + (int64_t)k * lda + m);
      ra[0] = v.x, ra[1] = v.y, ra[2] = v.z, ra[3] = v.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) ra[e] = (k < K && m + e < M) ? Ab[(int64_t)k * lda + m + e] : 0.0f;
    }
  }
}
__device__ __forceinline__ void g2_store_a(float (*As)[G2_LD], int tA, const float (&ra)[4]) {
  const int t = threadIdx.x;
  if (!tA) {
    const int m = t >> 1, k = (t & 1) * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) As[k + e][m] = ra[e];
  } else {
    const int k = t >> 5, m = (t & 31) * 4;
    *reinterpret_cast<float4*>(&As[k][m]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
  }
}

// acc = op(A)[m0.., :] op(B)[:, n0..] for one 128 x 128 tile (thread layout
// of the tile kernel below); As / Bs are the CTA's two shared buffers.
template <typename TB>
__device__ __forceinline__ void g2_mainloop(int M, int N, int K, const float* __restrict__ Ab, int lda, int tA,
                                            const TB* __restrict__ Bb, int ldb, int tB, int m0, int n0, int vecA,
                                            int vecB, float (*As)[G2_BK][G2_LD], float (*Bs)[G2_BK][G2_LD],
                                            float (&acc)[8][8]) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  // op(B)(k, n) tile: B[k * ldb + n] (!tB) or B[n * ldb + k] (tB), stored as
  // Bs[k][n]; the same code as A with the roles of m and n exchanged
  auto load_b = [&](int k0, float (&rb)[4]) {
    if (tB) {  // B[n * ldb + k]: 4 consecutive k of row n
      const int n = n0 + (t >> 1), k = k0 + (t & 1) * 4;
      if (vecB && n < N && k + 3 < K) {
        const float4 v = *reinterpret_cast<const float4*>(Bb + (int64_t)n * ldb + k);
        rb[0] = v.x, rb[1] = v.y, rb[2] = v.z, rb[3] = v.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) rb[e] = (n < N && k + e < K) ? (float)Bb[(int64_t)n * ldb + k + e] : 0.0f;
      }
    } else {  // B[k * ldb + n]: 4 consecutive n of row k
      const int k = k0 + (t >> 5), n = n0 + (t & 31) * 4;
      if (vecB && k < K && n + 3 < N) {
        const float4 v = *reinterpret_cast<const float4*>(Bb + (int64_t)k * ldb + n);
        rb[0] = v.x, rb[1] = v.y, rb[2] = v.z, rb[3] = v.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) rb[e] = (k < K && n + e < N) ? (float)Bb[(int64_t)k * ldb + n + e] : 0.0f;
      }
    }
  };
  auto store_b = [&](float (*Bsb)[G2_LD], const float (&rb)[4]) {
    if (tB) {
      const int n = t >> 1, k = (t & 1) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) Bsb[k + e][n] = rb[e];
    } else {
      const int k = t >> 5, n = (t & 31) * 4;
      *reinterpret_cast<float4*>(&Bsb[k][n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    }
  };
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  float ra[4], rb[4];
  g2_load_a(Ab, lda, tA, M, K, m0, 0, vecA, ra);
  load_b(0, rb);
  g2_store_a(As[0], tA, ra);
  store_b(Bs[0], rb);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += G2_BK) {
    const bool more = k0 + G2_BK < K;
    if (more) {
      g2_load_a(Ab, lda, tA, M, K, m0, k0 + G2_BK, vecA, ra);
      load_b(k0 + G2_BK, rb);
    }
#pragma unroll
    for (int kk = 0; kk < G2_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4 + 64]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      g2_store_a(As[buf ^ 1], tA, ra);
      store_b(Bs[buf ^ 1], rb);
    }
    __syncthreads();
    buf ^= 1;
  }
}

template <typename TB>
__global__ void __launch_bounds__(256, 2)
gemm_f32_tile_kernel(int M, int N, int K, const float* __restrict__ A, int64_t sA, const int32_t* __restrict__ ia,
                     int lda, int tA, const TB* __restrict__ B, int64_t sB, const int32_t* __restrict__ ib, int ldb,
                     int tB, float* __restrict__ C, int64_t sC, const int32_t* __restrict__ ic, int ldc, float alpha,
                     float beta, int64_t batch, int vecA, int vecB, int vecC) {
  __shared__ __align__(16) float As[2][G2_BK][G2_LD];
  __shared__ __align__(16) float Bs[2][G2_BK][G2_LD];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * G2_BM, n0 = blockIdx.x * G2_BN;
  for (int64_t b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + (ia ? (int64_t)ia[b] : b) * sA;
    const TB* Bb = B + (ib ? (int64_t)ib[b] : b) * sB;
    float* Cb = C + (ic ? (int64_t)ic[b] : b) * sC;
    float acc[8][8];
    g2_mainloop<TB>(M, N, K, Ab, lda, tA, Bb, ldb, tB, m0, n0, vecA, vecB, As, Bs, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
      if (m >= M) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n = n0 + tx * 4 + h * 64;
        float* cp = Cb + (int64_t)m * ldc + n;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = alpha * acc[i][h * 4 + e];
        if (vecC && n + 3 < N) {
          if (beta != 0.0f) {
            const float4 o = *reinterpret_cast<const float4*>(cp);
            v[0] = fmaf(beta, o.x, v[0]), v[1] = fmaf(beta, o.y, v[1]), v[2] = fmaf(beta, o.z, v[2]),
            v[3] = fmaf(beta, o.w, v[3]);
          }
          *reinterpret_cast<float4*>(cp) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (n + e < N) cp[e] = (beta != 0.0f) ? fmaf(beta, cp[e], v[e]) : v[e];
        }
      }
    }
  }
}

// U from the compact WY form in one pass: Q = I - W1 V^T (W1 = V Tw, D x K
// row-major; V column-major D x K) and U = [Q[:, K:] Q[:, :K]] written three
// ways: column-major U, row-major Ur and the 16-bit column-major copy U16
// (u16 NULL: none).  Tiles and main loop of the tile GEMM; column n of Q is
// column n - K of U for n >= K and n + R otherwise.  D and K are multiples
// of 4, so each thread's 4 x 4 groups lie wholly inside or outside the
// block and on one side of column K.
__global__ void __launch_bounds__(256, 2) form_u_kernel(int D, int K, const float* __restrict__ W1,
                                                        const float* __restrict__ V, float* __restrict__ U,
                                                        float* __restrict__ Ur, void* __restrict__ u16, int bf16,
                                                        int64_t nb) {
  __shared__ __align__(16) float As[2][G2_BK][G2_LD];
  __shared__ __align__(16) float Bs[2][G2_BK][G2_LD];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * G2_BM, n0 = blockIdx.x * G2_BN;
  const int R = D - K;
  for (int64_t b = blockIdx.z; b < nb; b += gridDim.z) {
    const float* Ab = W1 + b * (int64_t)D * K;
    const float* Bb = V + b * (int64_t)D * K;  // V^T row-major K x D
    float acc[8][8];
    g2_mainloop<float>(D, D, K, Ab, K, 0, Bb, D, 0, m0, n0, 1, 1, As, Bs, acc);
    float* Ub = U + b * (int64_t)D * D;
    float* Urb = Ur + b * (int64_t)D * D;
    uint16_t* U16b = u16 ? reinterpret_cast<uint16_t*>(u16) + b * (int64_t)D * D : nullptr;
    // three passes over the thread's four 4 x 4 groups (rows mb.., columns
    // nbase..), one output each, to keep few addresses live
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
      if (pass == 2 && !U16b) break;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int q4 = g >> 1, h = g & 1;
        const int mb = m0 + ty * 4 + q4 * 64, nbase = n0 + tx * 4 + h * 64;
        if (mb >= D || nbase >= D) continue;
        const int cb = nbase >= K ? nbase - K : nbase + R;  // U column of Q column nbase
        auto q = [&](int r, int e) {
          return (mb + r == nbase + e ? 1.0f : 0.0f) - acc[q4 * 4 + r][h * 4 + e];
        };
        if (pass == 0) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
            *reinterpret_cast<float4*>(Urb + (int64_t)(mb + r) * D + cb) =
                make_float4(q(r, 0), q(r, 1), q(r, 2), q(r, 3));
        } else if (pass == 1) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            *reinterpret_cast<float4*>(Ub + (int64_t)(cb + e) * D + mb) = make_float4(q(0, e), q(1, e), q(2, e), q(3, e));
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint32_t w0, w1;
            if (bf16) {
              __nv_bfloat162 x0 = __floats2bfloat162_rn(q(0, e), q(1, e)), x1 = __floats2bfloat162_rn(q(2, e), q(3, e));
              w0 = *reinterpret_cast<uint32_t*>(&x0), w1 = *reinterpret_cast<uint32_t*>(&x1);
            } else {
              __half2 x0 = __floats2half2_rn(q(0, e), q(1, e)), x1 = __floats2half2_rn(q(2, e), q(3, e));
              w0 = *reinterpret_cast<uint32_t*>(&x0), w1 = *reinterpret_cast<uint32_t*>(&x1);
            }
            *reinterpret_cast<uint2*>(U16b + (int64_t)(cb + e) * D + mb) = make_uint2(w0, w1);
          }
        }
      }
    }
  }
}
void launch_form_u(int64_t nb, int D, int K, const float* W1, const float* V, float* U, float* Ur, void* u16,
                   int bf16, cudaStream_t st) {
  if (nb == 0 || D == 0) return;
  dim3 g((D + G2_BN - 1) / G2_BN, (D + G2_BM - 1) / G2_BM, (unsigned)std::min<int64_t>(nb, 65535));
  ++g_launches;
  form_u_kernel<<<g, 256, 0, st>>>(D, K, W1, V, U, Ur, u16, bf16, nb);
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename T, typename TB>
void gemm_simt(int M, int N, int K, const T* A, int64_t sA, const int32_t* ia, int lda, bool tA, const TB* B,
               int64_t sB, const int32_t* ib, int ldb, bool tB, T* C, int64_t sC, const int32_t* ic, int ldc,
               T alpha, T beta, int64_t batch, cudaStream_t st) {
  if (batch == 0 || M == 0 || N == 0) return;
  if constexpr (std::is_same<T, float>::value && std::is_same<TB, float>::value) {
    // 16-byte vector access needs 4-element strides and aligned bases
    const int vecA = (lda % 4 == 0) && (sA % 4 == 0) && aligned16(A);
    const int vecB = (ldb % 4 == 0) && (sB % 4 == 0) && aligned16(B);
    const int vecC = (ldc % 4 == 0) && (sC % 4 == 0) && aligned16(C);
    dim3 g2((N + G2_BN - 1) / G2_BN, (M + G2_BM - 1) / G2_BM, (unsigned)std::min<int64_t>(batch, 65535));
    ++g_launches;
    gemm_f32_tile_kernel<float><<<g2, 256, 0, st>>>(M, N, K, A, sA, ia, lda, tA, B, sB, ib, ldb, tB, C, sC, ic, ldc,
                                                    alpha, beta, batch, vecA, vecB, vecC);
    return;
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64, (unsigned)std::min<int64_t>(batch, 65535));
  ++g_launches;
  gemm_batched_kernel<T, TB><<<grid, 256, 0, st>>>(M, N, K, A, sA, ia, lda, tA, B, sB, ib, ldb, tB, C, sC, ic, ldc,
                                                   alpha, beta, batch);
}
template void gemm_simt<double, double>(int, int, int, const double*, int64_t, const int32_t*, int, bool,
                                        const double*, int64_t, const int32_t*, int, bool, double*, int64_t,
                                        const int32_t*, int, double, double, int64_t, cudaStream_t);
template void gemm_simt<float, float>(int, int, int, const float*, int64_t, const int32_t*, int, bool,
                                      const float*, int64_t, const int32_t*, int, bool, float*, int64_t,
                                      const int32_t*, int, float, float, int64_t, cudaStream_t);
template void gemm_simt<float, double>(int, int, int, const float*, int64_t, const int32_t*, int, bool,
                                       const double*, int64_t, const int32_t*, int, bool, float*, int64_t,
                                       const int32_t*, int, float, float, int64_t, cudaStream_t);

// ------------------------------------------------------------------------
// block-wide sum
// ------------------------------------------------------------------------
template <typename T>
__device__ T block_sum(T v, T* sbuf) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  T t = T(0);
  for (int w = 0; w < nw; ++w) t += sbuf[w];
  return t;
}

// ------------------------------------------------------------------------
// a1: complement bases (Eq. 6-7) in three steps:
//   qr_panel_kernel   Householder QR of X^orth (LAPACK geqr2 conventions:
//                     beta = -sign(alpha) |x|), one CTA per box, the panel in
//                     shared memory when it fits.  Writes the reflectors V
//                     (column-major D x K, unit diagonal stored), tau and
//                     T_i = R (row-major K x K, X^orth = U^S T_i).
//   wy_tfactor_kernel the triangular factor of the compact WY form
//                     H_0 ... H_{K-1} = I - V Tw V^T (LAPACK larft, forward,
//                     columnwise) from S = V^T V.
//   identity + GEMMs  U = [Q[:, K:] Q[:, :K]] with Q = I - V Tw V^T, formed
//                     by batched GEMMs (in the caller).
// ------------------------------------------------------------------------
template <typename T>
__device__ T block_sum2(T v, T* sbuf) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  T t = T(0);
  for (int w = 0; w < nw; ++w) t += sbuf[w];
  __syncthreads();
  return t;
}

// Xin: row-major D x K per box.  Vout: column-major D x K per box.
template <typename T>
__global__ void __launch_bounds__(512) qr_panel_kernel(int D, int K, const T* __restrict__ Xin, T* __restrict__ Vout,
                                                       T* __restrict__ tau_out, T* __restrict__ Tm, T* __restrict__ gscr,
                                                       int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T red[32];
  __shared__ T s_tau, s_scal, s_beta;
  const int box = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  T* X = use_smem ? reinterpret_cast<T*>(smraw) : gscr + (size_t)box * D * K;  // column-major, ld = D
  const T* src = Xin + (size_t)box * D * K;
  for (int e = tid; e < D * K; e += blockDim.x) {
    const int r = e / K, a = e - r * K;
    X[a * D + r] = src[e];
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    T* xk = X + k * D;
    T part = T(0);
    for (int r = k + 1 + tid; r < D; r += blockDim.x) part += xk[r] * xk[r];
    const T xn2 = block_sum2(part, red);
    if (tid == 0) {
      const T alpha = xk[k];
      if (xn2 == T(0)) {
        s_tau = T(0);
      } else {
        const T beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        s_tau = (beta - alpha) / beta;
        s_scal = T(1) / (alpha - beta);
        s_beta = beta;
      }
    }
    __syncthreads();
    const T tk = s_tau;
    if (tk != T(0)) {
      const T scal = s_scal;
      for (int r = k + 1 + tid; r < D; r += blockDim.x) xk[r] *= scal;
      __syncthreads();
      for (int j = k + 1 + warp; j < K; j += nw) {
        T* xj = X + j * D;
        const T xjk = xj[k];
        T w = T(0);
        for (int r = k + 1 + lane; r < D; r += 32) w += xk[r] * xj[r];
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w = tk * (w + xjk);
        if (lane == 0) xj[k] = xjk - w;
        for (int r = k + 1 + lane; r < D; r += 32) xj[r] -= w * xk[r];
      }
      if (tid == 0) xk[k] = s_beta;
    }
    if (tid == 0) tau_out[(size_t)box * K + k] = tk;
    __syncthreads();
  }
  // R (row-major, upper) and V (column-major, unit diagonal, zeros above)
  T* Rb = Tm + (size_t)box * K * K;
  for (int e = tid; e < K * K; e += blockDim.x) {
    const int a = e / K, b = e - a * K;
    Rb[e] = (b >= a) ? X[b * D + a] : T(0);
  }
  T* Vb = Vout + (size_t)box * D * K;
  for (int e = tid; e < D * K; e += blockDim.x) {
    const int a = e / D, r = e - a * D;
    Vb[e] = (r > a) ? X[a * D + r] : (r == a ? T(1) : T(0));
  }
}

// Tw (row-major K x K, upper): for i = 0..K-1:
//   Tw[0:i, i] = -tau_i Tw[0:i, 0:i] S[0:i, i];  Tw[i, i] = tau_i
// S = V^T V (row-major K x K per box).  Step i: warp w computes the rows
// r = w, w + nwarps, ... of the new column, its lanes splitting the dot
// product over c in [r, i) (Tw is upper triangular).
template <typename T>
__global__ void __launch_bounds__(256) wy_tfactor_kernel(int K, const T* __restrict__ S, const T* __restrict__ tau,
                                                         T* __restrict__ Tw, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int box = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // K x K row-major working triangle: shared memory when it fits, else the
  // output block itself; w (K entries) always in shared memory
  T* Ts = use_smem ? reinterpret_cast<T*>(smraw) : Tw + (size_t)box * K * K;
  T* w = use_smem ? Ts + K * K : reinterpret_cast<T*>(smraw);
  const T* Sb = S + (size_t)box * K * K;
  const T* tb = tau + (size_t)box * K;
  for (int e = tid; e < K * K; e += blockDim.x) Ts[e] = T(0);
  __syncthreads();
  for (int i = 0; i < K; ++i) {
    for (int r = tid; r < i; r += blockDim.x) w[r] = Sb[r * K + i];
    __syncthreads();
    const T ti = tb[i];
    for (int r = warp; r < i; r += nw) {
      T sacc = T(0);
      for (int c = r + lane; c < i; c += 32) sacc += Ts[r * K + c] * w[c];
      for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) Ts[r * K + i] = -ti * sacc;
    }
    if (tid == 0) Ts[i * K + i] = ti;
    __syncthreads();
  }
  T* out = Tw + (size_t)box * K * K;
  if (use_smem)
    for (int e = tid; e < K * K; e += blockDim.x) out[e] = Ts[e];
}

// C[r0.., c0..] = alpha A B for the 4 x 4 tile at (r0, c0) of an h x h
// product of shared-memory operands (row-major, leading dimensions lda, ldb,
// ldc).
template <typename T>
__device__ __forceinline__ void smem_mm4(const T* A, int lda, const T* B, int ldb, T* C, int ldc, int h, T alpha,
                                         int r0, int c0) {
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 4
  for (int k = 0; k < h; ++k) {
    T a[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = A[(r0 + i) * lda + k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = B[k * ldb + c0 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) C[(r0 + i) * ldc + c0 + j] = alpha * acc[i][j];
}

// The same factor from the identity Tw^-1 = striu(S) + diag(1 / tau) of the
// compact WY form (tau_k = 0, a reflector equal to I, gives a zero row and
// column k of Tw: M is made the identity there and Tw_kk set to 0).  M is
// padded to Kp (a power of two, 8 <= Kp <= 128) with the identity and
// inverted in shared memory by recursive 2 x 2 blocking: the 8 x 8
// diagonal blocks by back substitution (one thread per column), then for
// b = 16 .. Kp every diagonal block [T11 T12; 0 T22] gets
// T12 = -T11 (M12 T22) from its two already inverted halves (dense 4 x 4
// register-tiled products; the zeros of the triangles are multiplied too).
// In place: Ms (Kp x Kp upper triangular, leading dimension Kp + 1) becomes
// its inverse; Xs is Kp * Kp / 4 scratch; every thread of the CTA calls it
// (Kp a power of two, 8 <= Kp <= 128; at least Kp threads).
template <typename T>
__device__ void tri_inverse_smem(int Kp, T* Ms, T* Xs) {
  const int ld = Kp + 1, tid = threadIdx.x;
  // 8 x 8 diagonal blocks: thread (q, j) solves M_qq x = e_j
  {
    const int nq = Kp / 8;
    T x[8];
    const int q = tid >> 3, j = tid & 7;
    if (q < nq) {
      const T* Mq = Ms + (size_t)(q * 8) * ld + q * 8;
#pragma unroll
      for (int i = 7; i >= 0; --i) {
        T acc = (i == j) ? T(1) : T(0);
#pragma unroll
        for (int k = i + 1; k < 8; ++k) acc -= Mq[i * ld + k] * x[k];
        x[i] = (i <= j) ? acc / Mq[i * ld + i] : T(0);
      }
    }
    __syncthreads();
    if (q < nq) {
      T* Mq = Ms + (size_t)(q * 8) * ld + q * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) Mq[i * ld + j] = x[i];
    }
    __syncthreads();
  }
  // the block products in 4 x 4 register tiles, one per thread
  for (int b = 16; b <= Kp; b *= 2) {
    const int h = b / 2, nb = Kp / b, hh = h * h, tw = h / 4, tpb = tw * tw;
    // X_q = M12 T22
    for (int e = tid; e < nb * tpb; e += blockDim.x) {
      const int q = e / tpb, rc = e - q * tpb, r0 = (rc / tw) * 4, c0 = (rc % tw) * 4;
      smem_mm4<T>(Ms + (size_t)(q * b) * ld + q * b + h, ld, Ms + (size_t)(q * b + h) * ld + q * b + h, ld,
                  Xs + (size_t)q * hh, h, h, T(1), r0, c0);
    }
    __syncthreads();
    // T12 = -T11 X_q, in place of M12
    for (int e = tid; e < nb * tpb; e += blockDim.x) {
      const int q = e / tpb, rc = e - q * tpb, r0 = (rc / tw) * 4, c0 = (rc % tw) * 4;
      smem_mm4<T>(Ms + (size_t)(q * b) * ld + q * b, ld, Xs + (size_t)q * hh, h,
                  Ms + (size_t)(q * b) * ld + q * b + h, ld, h, T(-1), r0, c0);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) wy_tinv_kernel(int K, int Kp, const T* __restrict__ S,
                                                      const T* __restrict__ tau, T* __restrict__ Tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = Kp + 1;
  T* Ms = reinterpret_cast<T*>(smraw);  // Kp x ld
  T* Xs = Ms + (size_t)Kp * ld;           // Kp * Kp / 4 scratch
  const int box = blockIdx.x, tid = threadIdx.x;
  const T* Sb = S + (size_t)box * K * K;
  const T* tb = tau + (size_t)box * K;
  for (int e = tid; e < Kp * Kp; e += blockDim.x) {
    const int r = e / Kp, c = e - r * Kp;
    T v = T(0);
    if (r >= K || c >= K) {
      v = (r == c) ? T(1) : T(0);
    } else {
      const bool zr = tb[r] == T(0), zc = tb[c] == T(0);
      if (r == c) v = zr ? T(1) : T(1) / tb[r];
      else if (c > r && !zr && !zc) v = Sb[r * K + c];
    }
    Ms[r * ld + c] = v;
  }
  __syncthreads();
  tri_inverse_smem<T>(Kp, Ms, Xs);
  T* out = Tw + (size_t)box * K * K;
  for (int e = tid; e < K * K; e += blockDim.x) {
    const int r = e / K, c = e - r * K;
    out[e] = (r == c && tb[r] == T(0)) ? T(0) : Ms[r * ld + c];
  }
}

// U (column-major D x D): column c' holds e_{perm(c')}, perm(c') = K + c'
// for c' < R = D - K, c' - R otherwise ([Q[:, K:] Q[:, :K]] of Q = I).
template <typename T>
__global__ void perm_identity_kernel(int nb, int D, int K, T* __restrict__ U) {
  const int R = D - K;
  const int64_t n = (int64_t)nb * D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e % ((int64_t)D * D);
    const int cp = (int)(q / D), r = (int)(q % D);
    const int src = cp < R ? K + cp : cp - R;
    U[e] = (r == src) ? T(1) : T(0);
  }
}

// Sums of CPW (8) per-lane values over the warp, left in d in every lane.  A transposed butterfly: at xor-distance 16, 8 and 4
// each lane keeps half of its remaining values and adds its partner's copy
// of them (4 + 2 + 1 shuffles), two plain steps finish one column per group
// of four lanes, and one shuffle per column brings every sum back.
template <int CPW>
__device__ __forceinline__ void qr_reduce_cols(float (&d)[CPW]) {
  static_assert(CPW == 8, "the butterfly is written for 8 columns");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool up = lane & 16;
    const float mine = up ? d[q + 4] : d[q], other = up ? d[q] : d[q + 4];
    d[q] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool up = lane & 8;
    const float mine = up ? d[q + 2] : d[q], other = up ? d[q] : d[q + 2];
    d[q] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
  }
  {
    const bool up = lane & 4;
    const float mine = up ? d[1] : d[0], other = up ? d[0] : d[1];
    d[0] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
  }
  d[0] += __shfl_xor_sync(0xffffffffu, d[0], 2);
  d[0] += __shfl_xor_sync(0xffffffffu, d[0], 1);
  // lane l now holds the sum of column 4 * bit4(l) + 2 * bit3(l) + bit2(l)
  const float t = d[0];
#pragma unroll
  for (int c = 0; c < 8; ++c) d[c] = __shfl_sync(0xffffffffu, t, ((c >> 2) << 4) | (((c >> 1) & 1) << 3) | ((c & 1) << 2));
}

// Householder reflector of one register-held column (rows lane + 32 s) at
// pivot row k, by the warp that owns it: the column becomes beta at row k and
// v below it (v_k = 1 implied); v (zeros above k) goes to vb, tau to *stau.
template <int RPL>
__device__ __forceinline__ void qr_reflector(float (&xc)[RPL], int k, int lane, float* vb, float* stau) {
  float alpha = 0.0f, part = 0.0f;
#pragma unroll
  for (int s = 0; s < RPL; ++s) {
    const int r = lane + 32 * s;
    if (r == k) alpha = xc[s];
    if (r > k) part += xc[s] * xc[s];
  }
  for (int o = 16; o; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
  }
  float tau = 0.0f, beta = alpha, scal = 0.0f;
  if (part != 0.0f) {
    beta = -copysignf(sqrtf(alpha * alpha + part), alpha);
    tau = (beta - alpha) / beta;
    scal = 1.0f / (alpha - beta);
  }
#pragma unroll
  for (int s = 0; s < RPL; ++s) {
    const int r = lane + 32 * s;
    float vv = 0.0f;
    if (r == k) {
      vv = 1.0f;
      xc[s] = beta;
    } else if (r > k && tau != 0.0f) {
      vv = xc[s] * scal;
      xc[s] = vv;
    }
    vb[r] = vv;
  }
  if (lane == 0) *stau = tau;
}

// The same factorization in FP32 with the panel in registers: warp w owns
// the contiguous columns 8 w .. 8 w + 7 and lane l rows l, l + 32, ...
// (D <= 32 RPL, K <= 128).  Step k: the owner warp of column k forms the
// reflector (warp reductions only) and publishes v and tau through a
// double-buffered shared vector; after one barrier the warps that still
// hold columns j > k update them: w = tau v^T x_j (lane-local products, one
// warp reduction), x_j -= w v.  The warps whose columns are finished
// reflectors (j < k) form the Gram entries v_j^T v_k instead, so that after
// the last step the compact-WY factor Tw = (striu(V^T V) + diag(1 / tau))^-1
// (zero-tau rows and columns masked, as in wy_tinv_kernel) is inverted in
// shared memory by the same CTA (Tw NULL: no factor).  The rank-1 updates
// stay in registers; shared memory carries v, the Gram matrix and Tw.
template <int RPL>
__global__ void __launch_bounds__(512) qr_reg_kernel(int D, int K, int Kp, const float* __restrict__ Xin,
                                                     float* __restrict__ Vout, float* __restrict__ tau_out,
                                                     float* __restrict__ Tm, float* __restrict__ Tw) {
  constexpr int NW = 16, CPW = 8;
  extern __shared__ __align__(16) unsigned char qsm[];
  float* vsb = reinterpret_cast<float*>(qsm);          // 2 x RPL * 32
  float* s_tau = vsb + 2 * RPL * 32;                    // 2 (+2 pad)
  float* tau_s = s_tau + 4;                             // Kp
  float* scr = tau_s + Kp;                              // max(32 x 129, Kp^2 / 4): load tile, then Xs
  const int nscr = (32 * 129 > Kp * Kp / 4) ? 32 * 129 : Kp * Kp / 4;
  float* Gm = scr + nscr;                               // Kp x (Kp + 1): Gram entries, then Tw
  const int ldg = Kp + 1;
  float(*tile)[NW * CPW + 1] = reinterpret_cast<float(*)[NW * CPW + 1]>(scr);
  const int box = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* src = Xin + (size_t)box * D * K;  // row-major D x K
  float x[CPW][RPL];
  // load through shared memory, 32 rows at a time (coalesced reads)
#pragma unroll
  for (int s = 0; s < RPL; ++s) {
    for (int e = threadIdx.x; e < 32 * K; e += blockDim.x) {
      const int rr = e / K, cc = e - rr * K, r = 32 * s + rr;
      tile[rr][cc] = (r < D) ? src[(size_t)r * K + cc] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = CPW * warp + c;
      x[c][s] = (j < K) ? tile[lane][j] : 0.0f;
    }
    __syncthreads();
  }
  // columns c >= c_lo of this warp take the update with reflector (vb, tk);
  // columns c < c_gram (finished reflectors j < k) give G[j][k] = v_j^T v_k
  auto update = [&](int c_lo, int c_gram, const float* vb, float tk, int k) {
    float v[RPL];
#pragma unroll
    for (int s = 0; s < RPL; ++s) v[s] = vb[lane + 32 * s];
    float d[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      d[c] = 0.0f;
      if ((c >= c_lo || c < c_gram) && CPW * warp + c < K) {
#pragma unroll
        for (int s = 0; s < RPL; ++s) d[c] = fmaf(v[s], x[c][s], d[c]);
      }
    }
    qr_reduce_cols<CPW>(d);
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      if (c >= c_lo && CPW * warp + c < K) {
        const float dj = d[c] * tk;
#pragma unroll
        for (int s = 0; s < RPL; ++s) x[c][s] = fmaf(-dj, v[s], x[c][s]);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < CPW; ++c)
        if (c < c_gram && CPW * warp + c < K) Gm[(CPW * warp + c) * ldg + k] = d[c];
    }
  };
  const bool gram = Tw != nullptr;
  int buf = 0;
  for (int cw = 0; cw < NW; ++cw) {
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) {
      const int k = CPW * cw + cc;
      if (k >= K) break;
      float* vb = vsb + buf * RPL * 32;
      if (warp == cw) qr_reflector<RPL>(x[cc], k, lane, vb, &s_tau[buf]);
      __syncthreads();
      const float tk = s_tau[buf];
      if (tk != 0.0f) {
        if (warp > cw) update(0, 0, vb, tk, k);
        else if (warp == cw) update(cc + 1, gram ? cc : 0, vb, tk, k);
        else if (gram) update(CPW, CPW, vb, tk, k);
      }
      if (threadIdx.x == 0) tau_out[(size_t)box * K + k] = tk, tau_s[k] = tk;
      buf ^= 1;
    }
  }
  // R (row-major, upper) and V (column-major, unit diagonal, zeros above)
  float* Rb = Tm + (size_t)box * K * K;
  float* Vb = Vout + (size_t)box * D * K;
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = CPW * warp + c;
    if (j >= K) continue;
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int r = lane + 32 * s;
      if (r < K) Rb[(size_t)r * K + j] = (r <= j) ? x[c][s] : 0.0f;
      if (r < D) Vb[(size_t)j * D + r] = (r > j) ? x[c][s] : (r == j ? 1.0f : 0.0f);
    }
  }
  if (!gram) return;
  // M = striu(G) + diag(1 / tau), padded to Kp with the identity, in place
  __syncthreads();
  for (int e = threadIdx.x; e < Kp * Kp; e += blockDim.x) {
    const int r = e / Kp, c = e - r * Kp;
    float v = 0.0f;
    if (r >= K || c >= K) {
      v = (r == c) ? 1.0f : 0.0f;
    } else {
      const bool zr = tau_s[r] == 0.0f, zc = tau_s[c] == 0.0f;
      if (r == c) v = zr ? 1.0f : 1.0f / tau_s[r];
      else if (c > r && !zr && !zc) v = Gm[r * ldg + c];
    }
    Gm[r * ldg + c] = v;
  }
  __syncthreads();
  tri_inverse_smem<float>(Kp, Gm, scr);
  float* out = Tw + (size_t)box * K * K;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int r = e / K, c = e - r * K;
    out[e] = (r == c && tau_s[r] == 0.0f) ? 0.0f : Gm[r * ldg + c];
  }
}

template <typename T>
bool launch_qr_panel(int nb, int D, int K, const T* Xin, T* Vout, T* tau, T* Tm, T* gscr, cudaStream_t st, T* Tw) {
  if (nb == 0 || K == 0) return false;
  if (std::is_same<T, float>::value && D <= 256 && K <= 128) {
    int Kp = 8;
    while (Kp < K) Kp *= 2;
    const size_t nscr = std::max<size_t>(32 * 129, (size_t)Kp * Kp / 4);
    const size_t sm = sizeof(float) * (2 * 256 + 4 + Kp + nscr + (Tw ? (size_t)Kp * (Kp + 1) : 0));
    if (sm > 48 * 1024) cudaFuncSetAttribute(qr_reg_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ++g_launches;
    qr_reg_kernel<8><<<nb, 512, sm, st>>>(D, K, Kp, reinterpret_cast<const float*>(Xin),
                                          reinterpret_cast<float*>(Vout), reinterpret_cast<float*>(tau),
                                          reinterpret_cast<float*>(Tm), reinterpret_cast<float*>(Tw));
    return Tw != nullptr;
  }
  const size_t sm = sizeof(T) * (size_t)D * K;
  const int use = sm <= 200 * 1024;
  if (use) cudaFuncSetAttribute(qr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  qr_panel_kernel<T><<<nb, 512, use ? sm : 0, st>>>(D, K, Xin, Vout, tau, Tm, gscr, use);
  return false;
}
template <typename T>
void launch_wy_tfactor(int nb, int K, const T* S, const T* tau, T* Tw, cudaStream_t st) {
  if (nb == 0 || K == 0) return;
  if (K <= 128) {
    int Kp = 8;
    while (Kp < K) Kp *= 2;
    const size_t sm = sizeof(T) * ((size_t)Kp * (Kp + 1) + (size_t)Kp * Kp / 4);
    if (sm > 48 * 1024) cudaFuncSetAttribute(wy_tinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ++g_launches;
    wy_tinv_kernel<T><<<nb, 256, sm, st>>>(K, Kp, S, tau, Tw);
    return;
  }
  size_t sm = sizeof(T) * ((size_t)K * K + K);
  const int use = sm <= 200 * 1024;
  if (!use) sm = sizeof(T) * (size_t)K;
  if (sm > 48 * 1024) cudaFuncSetAttribute(wy_tfactor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  wy_tfactor_kernel<T><<<nb, 256, sm, st>>>(K, S, tau, Tw, use);
}
template <typename T>
void launch_perm_identity(int nb, int D, int K, T* U, cudaStream_t st) {
  const int64_t n = (int64_t)nb * D * D;
  if (n == 0) return;
  ++g_launches;
  perm_identity_kernel<T><<<(int)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(nb, D, K, U);
}
#define H2_INST_QR(T)                                                                                         \
  template bool launch_qr_panel<T>(int, int, int, const T*, T*, T*, T*, T*, cudaStream_t, T*);                \
  template void launch_wy_tfactor<T>(int, int, const T*, const T*, T*, cudaStream_t);                          \
  template void launch_perm_identity<T>(int, int, int, T*, cudaStream_t);
H2_INST_QR(double)
H2_INST_QR(float)

// ------------------------------------------------------------------------
// a3: partial-pivot LU of Ahat_ii^RR (rows/cols 0..R of a D x D row-major
// block), LAPACK getf2 conventions (the first largest |pivot|; whole-row
// interchanges), in the factorization's precision T (FP64 for the FP64
// factorization, FP32 for the mixed-precision one).
//   luT  column-major R x R in T (L unit lower, U upper), piv LAPACK-style
//        (for T = double this is the lu array itself)
//   M    working copy: shared memory (ld = R + 1) when it fits, else luT
// A zero pivot records (level, box) in status[0..1]; the rest of that box's
// factorization is then undefined.
// ------------------------------------------------------------------------
// (TI: the type Ablk is stored in; the factorization runs in T)
template <typename T, typename TI = T>
__global__ void __launch_bounds__(256)
lu_factor_kernel(int D, int R, const TI* __restrict__ Ablk, const int32_t* __restrict__ diag_idx,
                 T* __restrict__ luT, int32_t* __restrict__ piv, int32_t* __restrict__ status, int level,
                 int use_smem) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_p;
  __shared__ T s_inv;
  const int box = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TI* A = Ablk + (size_t)(diag_idx ? diag_idx[box] : box) * D * D;
  T* G = luT + (size_t)box * R * R;
  T* M = use_smem ? reinterpret_cast<T*>(sm_raw) : G;
  const int ld = use_smem ? R + 1 : R;
  int32_t* pv = piv + (size_t)box * R;
  for (int r = warp; r < R; r += 8)
    for (int c = lane; c < R; c += 32) M[c * ld + r] = static_cast<T>(A[(size_t)r * D + c]);
  __syncthreads();
  int bad = 0;
  for (int k = 0; k < R; ++k) {
    if (warp == 0) {
      T best = T(-1);
      int bi = k;
      for (int r = k + lane; r < R; r += 32) {
        T a = fabs(M[k * ld + r]);
        if (a > best) { best = a; bi = r; }
      }
      for (int o = 16; o; o >>= 1) {
        T ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_p = bi;
        pv[k] = bi;
        T d = M[k * ld + bi];
        s_inv = d != T(0) ? T(1) / d : T(0);
      }
    }
    __syncthreads();
    const int p = s_p;
    const T inv = s_inv;
    if (inv == T(0)) {
      bad = 1;
      break;
    }
    if (p != k)
      for (int c = tid; c < R; c += 256) {
        T t = M[c * ld + k];
        M[c * ld + k] = M[c * ld + p];
        M[c * ld + p] = t;
      }
    __syncthreads();
    for (int r = k + 1 + tid; r < R; r += 256) M[k * ld + r] *= inv;
    __syncthreads();
    for (int c = k + 1 + warp; c < R; c += 8) {
      const T f = M[c * ld + k];
      if (f != T(0))
        for (int r = k + 1 + lane; r < R; r += 32) M[c * ld + r] = fma(-M[k * ld + r], f, M[c * ld + r]);
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0 && atomicCAS(status, 0, level + 1) == 0) status[1] = box;
    return;
  }
  if (use_smem)
    for (int c = warp; c < R; c += 8)
      for (int r = lane; r < R; r += 32) G[c * R + r] = M[c * ld + r];
}

// ------------------------------------------------------------------------
// a3 (cont.): Ainv = (P L U)^-1 = U^-1 L^-1 P^T in T, from the factors luT.
// Y starts as P^T (row r = e_perm[r]), then the unit-lower forward sweep and
// the upper backward sweep over all columns at once (row k is final when
// step k starts; the division by U(k,k) is applied to every row at the end).
// mode 2: factors and Y in shared memory; 1: factors only; 0: neither.
// ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
lu_inverse_kernel(int R, const T* __restrict__ luT, const int32_t* __restrict__ piv, T* __restrict__ Ainv, int mode) {
  extern __shared__ unsigned char sm_raw[];
  __shared__ int s_perm[1024];
  const int box = blockIdx.x, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const T* src = luT + (size_t)box * R * R;
  const int ld = mode ? R + 1 : R;
  T* F = mode ? reinterpret_cast<T*>(sm_raw) : const_cast<T*>(src);
  T* Yg = Ainv + (size_t)box * R * R;
  T* Y = (mode == 2) ? F + R * (R + 1) : Yg;
  if (mode)
    for (int c = ty; c < R; c += 8)
      for (int r = tx; r < R; r += 32) F[c * ld + r] = src[c * R + r];
  if (tid == 0) {
    for (int r = 0; r < R; ++r) s_perm[r] = r;
    for (int k = 0; k < R; ++k) {
      int p = piv[(size_t)box * R + k];
      int t = s_perm[k];
      s_perm[k] = s_perm[p];
      s_perm[p] = t;
    }
  }
  __syncthreads();
  for (int r = ty; r < R; r += 8)
    for (int b = tx; b < R; b += 32) Y[r * R + b] = (b == s_perm[r]) ? T(1) : T(0);
  for (int k = 0; k < R - 1; ++k) {
    __syncthreads();
    for (int r = k + 1 + ty; r < R; r += 8) {
      const T l = F[k * ld + r];
      if (l != T(0))
        for (int b = tx; b < R; b += 32) Y[r * R + b] = fma(-l, Y[k * R + b], Y[r * R + b]);
    }
  }
  for (int k = R - 1; k > 0; --k) {
    __syncthreads();
    const T dk = T(1) / F[k * ld + k];
    for (int r = ty; r < k; r += 8) {
      const T u = F[k * ld + r] * dk;
      if (u != T(0))
        for (int b = tx; b < R; b += 32) Y[r * R + b] = fma(-u, Y[k * R + b], Y[r * R + b]);
    }
  }
  __syncthreads();
  for (int r = ty; r < R; r += 8) {
    const T dr = T(1) / F[r * ld + r];
    for (int b = tx; b < R; b += 32) Yg[r * R + b] = Y[r * R + b] * dr;
  }
}

// ------------------------------------------------------------------------
// a3 (cont., FP32 storage): Ainv from the factors with one thread per column
// b of the inverse.  Column b of P^T is e_{perm^-1(b)}; each thread runs the
// unit-lower forward and the upper backward substitution on its own column,
// left-looking in blocks of 32 rows held in registers, reading the factors
// (row-major in shared memory, identity-padded to Rp = 32 ceil(R/32)) with
// 16-byte broadcast loads.  No barrier is needed between columns.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) lu_inverse_f32_kernel(int R, int Rp, const float* __restrict__ luT,
                                                              const int32_t* __restrict__ piv,
                                                              float* __restrict__ Ainv) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_perm[1024];
  float* F = smf;            // Rp x Rp row-major factors
  float* Y = F + Rp * Rp;    // Rp x Rp row-major; column b belongs to thread b
  const int box = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const float* src = luT + (size_t)box * R * R;
  for (int e = tid; e < Rp * Rp; e += nt) {
    const int r = e / Rp, cc = e - r * Rp;
    F[e] = (r < R && cc < R) ? src[cc * R + r] : (r == cc ? 1.f : 0.f);
  }
  if (tid == 0) {
    for (int r = 0; r < Rp; ++r) s_perm[r] = r;
    for (int k = 0; k < R; ++k) {
      const int p = piv[(size_t)box * R + k];
      const int t = s_perm[k];
      s_perm[k] = s_perm[p];
      s_perm[p] = t;
    }
  }
  __syncthreads();
  const int b = tid;
  for (int r = 0; r < Rp; ++r) Y[r * Rp + b] = (s_perm[r] == b) ? 1.f : 0.f;
  float y[32];
  // forward: L unit lower
  for (int i0 = 0; i0 < Rp; i0 += 32) {
#pragma unroll
    for (int q = 0; q < 32; ++q) y[q] = Y[(i0 + q) * Rp + b];
    for (int k = 0; k < i0; k += 4) {
      const float y0 = Y[k * Rp + b], y1 = Y[(k + 1) * Rp + b], y2 = Y[(k + 2) * Rp + b], y3 = Y[(k + 3) * Rp + b];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float4 l = *reinterpret_cast<const float4*>(F + (i0 + q) * Rp + k);
        y[q] = fmaf(-l.x, y0, fmaf(-l.y, y1, fmaf(-l.z, y2, fmaf(-l.w, y3, y[q]))));
      }
    }
#pragma unroll
    for (int q = 1; q < 32; ++q) {
#pragma unroll
      for (int c = 0; c < q; ++c) y[q] = fmaf(-F[(i0 + q) * Rp + i0 + c], y[c], y[q]);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) Y[(i0 + q) * Rp + b] = y[q];
  }
  // backward: U upper
  for (int i0 = Rp - 32; i0 >= 0; i0 -= 32) {
#pragma unroll
    for (int q = 0; q < 32; ++q) y[q] = Y[(i0 + q) * Rp + b];
    for (int k = i0 + 32; k < Rp; k += 4) {
      const float y0 = Y[k * Rp + b], y1 = Y[(k + 1) * Rp + b], y2 = Y[(k + 2) * Rp + b], y3 = Y[(k + 3) * Rp + b];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float4 u = *reinterpret_cast<const float4*>(F + (i0 + q) * Rp + k);
        y[q] = fmaf(-u.x, y0, fmaf(-u.y, y1, fmaf(-u.z, y2, fmaf(-u.w, y3, y[q]))));
      }
    }
#pragma unroll
    for (int q = 31; q >= 0; --q) {
#pragma unroll
      for (int c = q + 1; c < 32; ++c) y[q] = fmaf(-F[(i0 + q) * Rp + i0 + c], y[c], y[q]);
      y[q] = y[q] / F[(i0 + q) * Rp + i0 + q];
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) Y[(i0 + q) * Rp + b] = y[q];
  }
  if (b < R) {
    float* out = Ainv + (size_t)box * R * R;
    for (int r = 0; r < R; ++r) out[(size_t)r * R + b] = Y[r * Rp + b];
  }
}

// ------------------------------------------------------------------------
// a3, mixed precision: (Ahat_ii^RR)^-1 by Gauss-Jordan elimination with
// partial pivoting, in FP32, with the block held in registers.  Thread
// (tr, tc) of an (Rp/TR) x (Rp/TC) grid keeps the TR x TC tile at rows
// TR tr.., columns TC tc.. (Rp = R rounded up to the tile sizes; padding
// rows never pivot).  Step k: the owners of column k propose their largest
// |entry| among rows not yet used as pivots (LAPACK's choice: the first
// largest); the chosen row p is scaled so that its column-k entry becomes
// 1 / a_pk (the in-place form that stores the inverse where the eliminated
// column was), and every other row r takes a_r -= a_rk * (scaled row p)
// with its column-k entry zeroed first.  Rows are never moved, so at the end
//   Ainv[k][pivot(j)] = a[pivot(k)][j],  pivot(k) = the row chosen at step k.
// The row-interchange sequence LAPACK's getrf would record (the same pivots:
// the unused rows of column k are the Schur complement column) is written to
// piv.  A zero or non-finite pivot column records (level, box) in
// status[0..1] and leaves the box's output undefined.
// Tiles: 8 x 8 (256 threads) for R <= 128, 12 x 6 (512 threads) for
// R <= 192; the register file of one SM sub-partition bounds both.
// ------------------------------------------------------------------------
constexpr int kGjMaxR = 192;

struct GjShared {
  float P[kGjMaxR];
  float fcol[kGjMaxR];
  int prow[kGjMaxR], pinv[kGjMaxR], rowat[kGjMaxR];
  int p;
  float pv;
};

// Thread t holds tile (tr, tc) = (t % G, t / G) with G = ntr rounded up to a
// power of two (G divides 32): the owners of a tile column are one lane
// group of one warp, so the pivot search is a shuffle reduction in that
// warp.  One elimination step for column k = TC kc + J (J fixed at compile
// time so that the tile stays in registers); false on a zero pivot column.
template <int TR, int TC, int J>
__device__ __forceinline__ bool gj_step(GjShared& sh, float (&a)[TR][TC], unsigned& used, int kc, int G,
                                        bool has, int tr, int tc, int r0, int c0) {
  const int t = threadIdx.x, k = kc * TC + J;
  // (a) the owner warp of column k finds the pivot: the first largest |a_rk|
  // over rows not yet used
  if ((t >> 5) == ((kc * G) >> 5)) {
    float best = -1.0f, sv = 0.0f;
    int bi = -1;
    if (has && tc == kc) {
#pragma unroll
      for (int i = 0; i < TR; ++i) {
        const float v = fabsf(a[i][J]);
        if (!((used >> i) & 1u) && v > best) best = v, sv = a[i][J], bi = r0 + i;
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o), os = __shfl_xor_sync(0xffffffffu, sv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) best = ob, sv = os, bi = oi;
    }
    if (tc == kc && tr == 0) {
      sh.p = bi, sh.pv = sv;
      if (bi >= 0) sh.prow[k] = bi;
    }
  }
  __syncthreads();
  const int p = sh.p;
  const float pv = sh.pv;
  if (p < 0 || pv == 0.0f || !isfinite(pv)) return false;
  const float inv = __frcp_rn(pv);
  // (b) scaled pivot row -> P, column k -> fcol
  if (has && tr == p / TR) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
      if (r0 + i == p) {
#pragma unroll
        for (int jj = 0; jj < TC; ++jj) {
          const float v = ((jj == J && c0 + jj == k) ? 1.0f : a[i][jj]) * inv;
          a[i][jj] = v;
          sh.P[c0 + jj] = v;
        }
        used |= 1u << i;
      }
  }
  if (has && tc == kc) {
#pragma unroll
    for (int i = 0; i < TR; ++i) sh.fcol[r0 + i] = a[i][J];
  }
  __syncthreads();
  // (c) eliminate column k from every other row
  if (has) {
    float pr[TC];
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) pr[jj] = sh.P[c0 + jj];
    const bool own = (tc == kc);
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      const float f = (r0 + i == p) ? 0.0f : sh.fcol[r0 + i];
      if (own && r0 + i != p) a[i][J] = 0.0f;
#pragma unroll
      for (int jj = 0; jj < TC; ++jj) a[i][jj] = fmaf(-f, pr[jj], a[i][jj]);
    }
  }
  return true;
}

template <int TR, int TC, int J>
__device__ __forceinline__ void gj_steps(bool& ok, GjShared& sh, float (&a)[TR][TC], unsigned& used, int kc, int G,
                                         int left, bool has, int tr, int tc, int r0, int c0) {
  if constexpr (J < TC) {
    if (ok && left > J) ok = gj_step<TR, TC, J>(sh, a, used, kc, G, has, tr, tc, r0, c0);
    gj_steps<TR, TC, J + 1>(ok, sh, a, used, kc, G, left, has, tr, tc, r0, c0);
  }
}

// group size of the kernel's thread mapping (a power of two >= ntr, <= 32)
__host__ __device__ inline int gj_group(int ntr) {
  int g = 1;
  while (g < ntr) g <<= 1;
  return g;
}

template <int TR, int TC, int NT>
__global__ void __launch_bounds__(NT) gj_inverse_kernel(int D, int R, const float* __restrict__ Ablk,
                                                        const int32_t* __restrict__ diag_idx,
                                                        float* __restrict__ Ainv, int32_t* __restrict__ piv,
                                                        int32_t* __restrict__ status, int level) {
  __shared__ GjShared sh;
  constexpr int TL = (TR > TC ? TR : TC);  // Rp is a multiple of both tile edges
  static_assert(TL % TR == 0 && TL % TC == 0, "tile edges must divide the larger one");
  const int box = blockIdx.x, t = threadIdx.x;
  const int Rp = (R + TL - 1) / TL * TL, ntr = Rp / TR, ntc = Rp / TC, G = gj_group(ntr);
  const int tr = t % G, tc = t / G;
  const bool has = tr < ntr && tc < ntc;
  const int r0 = tr * TR, c0 = tc * TC;
  const float* A = Ablk + (size_t)(diag_idx ? diag_idx[box] : box) * D * D;
  float a[TR][TC];
  unsigned used = 0;
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = r0 + i;
    if (!has || r >= R) used |= 1u << i;
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      const int c = c0 + j;
      a[i][j] = (has && r < R && c < R) ? A[(size_t)r * D + c] : 0.0f;
    }
  }
  bool ok = true;
  for (int kc = 0; kc < ntc && ok; ++kc)
    gj_steps<TR, TC, 0>(ok, sh, a, used, kc, G, R - kc * TC, has, tr, tc, r0, c0);
  if (!ok) {
    if (t == 0 && atomicCAS(status, 0, level + 1) == 0) status[1] = box;
    return;
  }
  // unscramble: Ainv[k][prow[j]] = a[prow[k]][j]
  for (int k = t; k < R; k += blockDim.x) sh.pinv[sh.prow[k]] = k;
  __syncthreads();
  if (has) {
    float* out = Ainv + (size_t)box * R * R;
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      const int r = r0 + i;
      if (r >= R) continue;
      const size_t row = (size_t)sh.pinv[r] * R;
#pragma unroll
      for (int jj = 0; jj < TC; ++jj)
        if (c0 + jj < R) out[row + sh.prow[c0 + jj]] = a[i][jj];
    }
  }
  // LAPACK-style interchange sequence of the same pivots: pos[r] is the
  // current position of original row r, rowat[q] the row at position q
  __syncthreads();
  if (t == 0) {
    int* pos = sh.pinv;
    for (int q = 0; q < R; ++q) pos[q] = q, sh.rowat[q] = q;
    int32_t* pv_out = piv + (size_t)box * R;
    for (int k = 0; k < R; ++k) {
      const int r = sh.prow[k], q = pos[r], rk = sh.rowat[k];
      pv_out[k] = q;
      sh.rowat[k] = r, sh.rowat[q] = rk;
      pos[r] = k, pos[rk] = q;
    }
  }
}

// ------------------------------------------------------------------------
// The same in-place elimination for blocks too large for the registers of
// one CTA (FP32 192 < R <= 512, FP64 128 < R <= 256): the columns are split
// over a cluster of CL CTAs (thread-block cluster, distributed shared
// memory).  CTA q of a box holds the columns [q W, (q + 1) W), W = Rp / CL,
// as TR x TC register tiles, thread t at tile (t % G, q W / TC + t / G)
// (16 x 4 tiles of FP32 or 16 x 2 of FP64: 64 registers of data).
// Step k: the CTA owning column k picks the pivot row among the unused rows
// and publishes (p, a_pk) and column k in its shared memory, in the buffer
// of the step's parity; one cluster barrier; every CTA reads them from the
// owner, scales its part of row p and eliminates column k from its other
// rows.  The owner rewrites a buffer two steps later, after every CTA has
// passed the next barrier, so one cluster barrier per step suffices.  A
// failed pivot is seen by every CTA at the same step; all of them leave
// after one more cluster barrier, so that no CTA exits while another may
// still read its shared memory.
// ------------------------------------------------------------------------
template <typename T>
struct __align__(16) GjcShared {
  T fcol[2][512];  // the owner's column k, by step parity
  T fl[512];       // this CTA's copy of it
  T P[512];        // the scaled pivot row (this CTA's columns)
  T pvs[2];        // a_pk, by step parity
  int ps[2];       // p, by step parity
  int prow[512], pinv[512], rowat[512];
};

__device__ __forceinline__ float rcp_pivot(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_pivot(double v) { return 1.0 / v; }

template <typename T, int TR, int TC, int J>
__device__ __forceinline__ bool gjc_step(GjcShared<T>& sh, T (&a)[TR][TC], unsigned& used, int kc, int oq, int kcl,
                                         int q, int G, int Rp, bool has, int tr, int tc, int tcl, int r0, int c0) {
  const int t = threadIdx.x, k = kc * TC + J, b = k & 1;
  if (q == oq) {
    // (a) the owner warp of column k: the first largest |a_rk| over unused rows
    if ((t >> 5) == ((kcl * G) >> 5)) {
      T best = T(-1), sv = T(0);
      int bi = -1;
      if (has && tcl == kcl) {
#pragma unroll
        for (int i = 0; i < TR; ++i) {
          const T v = fabs(a[i][J]);
          if (!((used >> i) & 1u) && v > best) best = v, sv = a[i][J], bi = r0 + i;
        }
      }
      for (int o = G >> 1; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o), os = __shfl_xor_sync(0xffffffffu, sv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) best = ob, sv = os, bi = oi;
      }
      if (tcl == kcl && tr == 0) sh.ps[b] = bi, sh.pvs[b] = sv;
    }
    if (has && tcl == kcl) {
#pragma unroll
      for (int i = 0; i < TR; ++i) sh.fcol[b][r0 + i] = a[i][J];
    }
  }
  cluster_sync();
  const int p = ld_cluster(cluster_map(&sh.ps[b], (uint32_t)oq), int());
  const T pv = ld_cluster(cluster_map(&sh.pvs[b], (uint32_t)oq), T());
  if (p < 0 || pv == T(0) || !isfinite(pv)) return false;
  const T inv = rcp_pivot(pv);
  if (t == 0) sh.prow[k] = p;
  // (b) column k from the owner; this CTA's part of the scaled pivot row
  {
    constexpr int PER = 16 / (int)sizeof(T);
    const uint32_t src = cluster_map(&sh.fcol[b][0], (uint32_t)oq);
    for (int e = t; e < Rp / PER; e += blockDim.x)
      *reinterpret_cast<uint4*>(&sh.fl[e * PER]) = ld_cluster_v4(src + 16u * (uint32_t)e);
  }
  if (has && tr == p / TR) {
#pragma unroll
    for (int i = 0; i < TR; ++i)
      if (r0 + i == p) {
#pragma unroll
        for (int jj = 0; jj < TC; ++jj) {
          const T v = ((jj == J && c0 + jj == k) ? T(1) : a[i][jj]) * inv;
          a[i][jj] = v;
          sh.P[c0 + jj] = v;
        }
        used |= 1u << i;
      }
  }
  __syncthreads();
  // (c) eliminate column k from every other row
  if (has) {
    T pr[TC];
#pragma unroll
    for (int jj = 0; jj < TC; ++jj) pr[jj] = sh.P[c0 + jj];
    const bool own = (tc == kc);
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      const T f = (r0 + i == p) ? T(0) : sh.fl[r0 + i];
      if (own && r0 + i != p) a[i][J] = T(0);
#pragma unroll
      for (int jj = 0; jj < TC; ++jj) a[i][jj] = fma(-f, pr[jj], a[i][jj]);
    }
  }
  return true;
}

template <typename T, int TR, int TC, int J>
__device__ __forceinline__ void gjc_steps(bool& ok, GjcShared<T>& sh, T (&a)[TR][TC], unsigned& used, int kc, int oq,
                                          int kcl, int q, int G, int Rp, int left, bool has, int tr, int tc, int tcl,
                                          int r0, int c0) {
  if constexpr (J < TC) {
    if (ok && left > J) ok = gjc_step<T, TR, TC, J>(sh, a, used, kc, oq, kcl, q, G, Rp, has, tr, tc, tcl, r0, c0);
    gjc_steps<T, TR, TC, J + 1>(ok, sh, a, used, kc, oq, kcl, q, G, Rp, left, has, tr, tc, tcl, r0, c0);
  }
}

template <typename T, int TR, int TC, int CL, int NT>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 1)
    gj_cluster_kernel(int D, int R, int Rp, const float* __restrict__ Ablk, const int32_t* __restrict__ diag_idx,
                      float* __restrict__ Ainv, int32_t* __restrict__ piv, int32_t* __restrict__ status, int level) {
  __shared__ GjcShared<T> sh;
  const int q = (int)cluster_rank();
  const int box = blockIdx.x / CL, t = threadIdx.x;
  const int W = Rp / CL, ntr = Rp / TR, ntcl = W / TC, G = gj_group(ntr);
  const int tr = t % G, tcl = t / G;
  const bool has = tr < ntr && tcl < ntcl;
  const int tc = q * ntcl + tcl;
  const int r0 = tr * TR, c0 = tc * TC;
  const float* A = Ablk + (size_t)(diag_idx ? diag_idx[box] : box) * D * D;
  T a[TR][TC];
  unsigned used = 0;
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int r = r0 + i;
    if (!has || r >= R) used |= 1u << i;
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      const int c = c0 + j;
      a[i][j] = (has && r < R && c < R) ? static_cast<T>(A[(size_t)r * D + c]) : T(0);
    }
  }
  bool ok = true;
  const int nkc = (R + TC - 1) / TC;
  for (int kc = 0; kc < nkc && ok; ++kc) {
    const int oq = kc / ntcl;
    gjc_steps<T, TR, TC, 0>(ok, sh, a, used, kc, oq, kc - oq * ntcl, q, G, Rp, R - kc * TC, has, tr, tc, tcl, r0,
                            c0);
  }
  cluster_sync();
  if (!ok) {
    if (q == 0 && t == 0 && atomicCAS(status, 0, level + 1) == 0) status[1] = box;
    return;
  }
  // unscramble this CTA's columns: Ainv[k][prow[j]] = a[prow[k]][j]
  for (int k = t; k < R; k += blockDim.x) sh.pinv[sh.prow[k]] = k;
  __syncthreads();
  if (has) {
    float* out = Ainv + (size_t)box * R * R;
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      const int r = r0 + i;
      if (r >= R) continue;
      const size_t row = (size_t)sh.pinv[r] * R;
#pragma unroll
      for (int jj = 0; jj < TC; ++jj)
        if (c0 + jj < R) out[row + sh.prow[c0 + jj]] = static_cast<float>(a[i][jj]);
    }
  }
  if (q == 0) {
    // LAPACK-style interchange sequence of the same pivots
    __syncthreads();
    if (t == 0) {
      int* pos = sh.pinv;
      for (int r = 0; r < R; ++r) pos[r] = r, sh.rowat[r] = r;
      int32_t* pv_out = piv + (size_t)box * R;
      for (int k = 0; k < R; ++k) {
        const int r = sh.prow[k], qq = pos[r], rk = sh.rowat[k];
        pv_out[k] = qq;
        sh.rowat[k] = r, sh.rowat[qq] = rk;
        pos[r] = k, pos[rk] = qq;
      }
    }
  }
}

// Inverses of nb blocks by the cluster kernel: FP32 elimination (fp64 = 0)
// for 192 < R <= 512, FP64 for 128 < R <= 256.  False: R not covered.
static bool launch_gj_cluster(bool fp64, int nb, int D, int R, const float* Ablk, const int32_t* diag_idx,
                              float* Ainv, int32_t* piv, int32_t* status, int level, cudaStream_t st) {
  if (!fp64 && R > 192 && R <= 256) {
    ++g_launches;
    gj_cluster_kernel<float, 16, 4, 4, 256><<<nb * 4, 256, 0, st>>>(D, R, (R + 15) / 16 * 16, Ablk, diag_idx, Ainv,
                                                                     piv, status, level);
    return true;
  }
  if (!fp64 && R > 256 && R <= 512) {
    ++g_launches;
    gj_cluster_kernel<float, 16, 4, 8, 512><<<nb * 8, 512, 0, st>>>(D, R, (R + 31) / 32 * 32, Ablk, diag_idx, Ainv,
                                                                     piv, status, level);
    return true;
  }
  if (fp64 && R > 128 && R <= 256) {
    ++g_launches;
    gj_cluster_kernel<double, 16, 2, 8, 256><<<nb * 8, 256, 0, st>>>(D, R, (R + 15) / 16 * 16, Ablk, diag_idx,
                                                                      Ainv, piv, status, level);
    return true;
  }
  return false;
}

// The same elimination for R <= 128 in 16-column panels.  Thread t of warp
// w holds the 8 x 8 tile at rows 8 (lane % 16), columns 16 w + 8 (lane / 16),
// so warp w holds panel w (columns 16 w .. 16 w + 15) for every row.  Per
// panel: (1) its warp runs the 16 in-place steps on the panel columns only
// (pivot search, pivot row and column multipliers by shuffles and a
// warp-private shared row), leaving in column 16 w + a the column p_a of
// the combined elimination E of the 16 steps (p_a: pivot row of step a);
// (2) the rows p_a of every other column are published; (3) every other
// column takes E's effect at once, a_c += (E - I)[:, P] a_old[P, c]: a rank-16
// update.  The pivots are those of the one-column form (the same row order
// of choice); the sums are grouped differently.
constexpr int kGbP = 16;  // panel width

struct GbShared {
  float WmT[2][kGbP][128];   // (E - I)[:, p_a], transposed: WmT[a][r]
  float Prow[2][kGbP][128];  // rows p_a of the matrix before the panel
  float pan[128][kGbP + 1];   // the panel warp's columns, moved between its tile and row layouts
  int pidx[2][128];          // panel slot a of row r, -1 for rows that are no pivot of the panel
  unsigned char used[128];   // rows already chosen as pivots
  int prow[128], pinv[128], rowat[128];
  int bad;
};

__global__ void __launch_bounds__(256, 2) gj_blocked_kernel(int D, int R, const float* __restrict__ Ablk,
                                                            const int32_t* __restrict__ diag_idx,
                                                            float* __restrict__ Ainv, int32_t* __restrict__ piv,
                                                            int32_t* __restrict__ status, int level) {
  __shared__ __align__(16) GbShared sh;
  const int box = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int tr = lane & 15, h = lane >> 4;
  const int r0 = 8 * tr, c0 = 16 * warp + 8 * h;
  const int npan = (R + kGbP - 1) / kGbP;
  const float* A = Ablk + (size_t)(diag_idx ? diag_idx[box] : box) * D * D;
  float x[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + j;
      x[i][j] = (r < R && c < R) ? A[(size_t)r * D + c] : 0.0f;
    }
  }
  for (int e = t; e < 128; e += blockDim.x) sh.used[e] = (e >= R);
  if (t == 0) sh.bad = 0;
  __syncthreads();
  for (int pn = 0; pn < npan; ++pn) {
    const int b = pn & 1;
    if (warp == pn) {
      // (1) the panel's 16 steps, in a row layout: lane l holds rows
      // l + 32 k (k < 4) of the 16 panel columns
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sh.pan[r0 + i][8 * h + j] = x[i][j], x[i][j] = 0.0f;  // (x reloaded below)
      for (int e = lane; e < 128; e += 32) sh.pidx[b][e] = -1;
      __syncwarp();
      float y[4][kGbP];
      unsigned used = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        used |= (unsigned)sh.used[lane + 32 * k] << k;
#pragma unroll
        for (int c = 0; c < kGbP; ++c) y[k][c] = sh.pan[lane + 32 * k][c];
      }
      bool bad = false;
#pragma unroll
      for (int a = 0; a < kGbP; ++a) {
        const int kcol = kGbP * pn + a;
        if (kcol >= R || bad) break;
        // pivot: the first largest |y| of column a over unused rows
        float best = -1.0f, sv = 0.0f;
        int bi = -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float v = fabsf(y[k][a]);
          if (!((used >> k) & 1u) && v > best) best = v, sv = y[k][a], bi = lane + 32 * k;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o), os = __shfl_xor_sync(0xffffffffu, sv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) best = ob, sv = os, bi = oi;
        }
        const int p = bi;
        if (p < 0 || sv == 0.0f || !isfinite(sv)) {
          bad = true;
          break;
        }
        const float inv = __frcp_rn(sv);
        const int owner = p & 31, slot = p >> 5;
        float f[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) f[k] = y[k][a];
        // eight columns at a time: the pivot row's entries from its owner lane
        // (slot p / 32 picked by selects), scaled (its column-a entry
        // becomes 1 / pv), then every row updated
#pragma unroll
        for (int hc = 0; hc < kGbP / 8; ++hc) {
          float pr[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = 8 * hc + q;
            const float t01 = (slot & 1) ? y[1][cc] : y[0][cc], t23 = (slot & 1) ? y[3][cc] : y[2][cc];
            const float v = __shfl_sync(0xffffffffu, (slot & 2) ? t23 : t01, owner);
            pr[q] = (cc == a) ? inv : v * inv;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const bool piv = (lane + 32 * k == p);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int cc = 8 * hc + q;
              y[k][cc] = piv ? pr[q] : fmaf(-f[k], pr[q], cc == a ? 0.0f : y[k][cc]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (lane + 32 * k == p) used |= 1u << k;
        if (lane == 0) {
          sh.prow[kcol] = p;
          sh.used[p] = 1;
          sh.pidx[b][p] = a;
        }
      }
      if (bad && lane == 0) sh.bad = 1;
      __syncwarp();
      // (E - I)[:, p_a] = the panel columns minus 1 at the pivot rows; the
      // panel back to the tile layout
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = lane + 32 * k;
        const int pa = sh.pidx[b][r];
#pragma unroll
        for (int c = 0; c < kGbP; ++c) {
          sh.WmT[b][c][r] = y[k][c] - (pa == c ? 1.0f : 0.0f);
          sh.pan[r][c] = y[k][c];
        }
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[i][j] = sh.pan[r0 + i][8 * h + j];
    }
    __syncthreads();
    if (sh.bad) break;
    const int kn = min(kGbP, R - kGbP * pn);  // steps of this panel
    // (2) rows p_a of the other columns, before the update
    if (warp != pn) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = sh.pidx[b][r0 + i];
        if (a >= 0) {
          float4* dst = reinterpret_cast<float4*>(&sh.Prow[b][a][c0]);
          dst[0] = make_float4(x[i][0], x[i][1], x[i][2], x[i][3]);
          dst[1] = make_float4(x[i][4], x[i][5], x[i][6], x[i][7]);
        }
      }
    }
    __syncthreads();
    // (3) rank-kn update of the other columns
    if (warp != pn) {
#pragma unroll 1
      for (int a = 0; a < kn; ++a) {
        const float4 w0 = *reinterpret_cast<const float4*>(&sh.WmT[b][a][r0]);
        const float4 w1 = *reinterpret_cast<const float4*>(&sh.WmT[b][a][r0 + 4]);
        const float4 p0 = *reinterpret_cast<const float4*>(&sh.Prow[b][a][c0]);
        const float4 p1 = *reinterpret_cast<const float4*>(&sh.Prow[b][a][c0 + 4]);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float q[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) x[i][j] = fmaf(w[i], q[j], x[i][j]);
      }
    }
  }
  if (sh.bad) {
    if (t == 0 && atomicCAS(status, 0, level + 1) == 0) status[1] = box;
    return;
  }
  // unscramble: Ainv[k][prow[j]] = a[prow[k]][j]
  for (int k = t; k < R; k += blockDim.x) sh.pinv[sh.prow[k]] = k;
  __syncthreads();
  float* out = Ainv + (size_t)box * R * R;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + i;
    if (r >= R) continue;
    const size_t row = (size_t)sh.pinv[r] * R;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (c0 + j < R) out[row + sh.prow[c0 + j]] = x[i][j];
  }
  // LAPACK-style interchange sequence of the same pivots
  __syncthreads();
  if (t == 0) {
    int* pos = sh.pinv;
    for (int q = 0; q < R; ++q) pos[q] = q, sh.rowat[q] = q;
    int32_t* pv_out = piv + (size_t)box * R;
    for (int k = 0; k < R; ++k) {
      const int r = sh.prow[k], q = pos[r], rk = sh.rowat[k];
      pv_out[k] = q;
      sh.rowat[k] = r, sh.rowat[q] = rk;
      pos[r] = k, pos[rk] = q;
    }
  }
}

template <typename T>
void launch_lu_inverse(int nb, int D, int R, const T* Ablk, const int32_t* diag_idx, double* lu, T* luT,
                       int32_t* piv, T* Ainv, int32_t* status, int level, cudaStream_t st) {
  if (nb == 0 || R == 0) return;
  (void)lu;  // for T = double, luT is the lu array
  if (std::is_same<T, float>::value && R <= kGjMaxR) {
    // mixed precision: the inverse directly, no LU factors kept
    const float* Af = reinterpret_cast<const float*>(Ablk);
    float* Af_inv = reinterpret_cast<float*>(Ainv);
    ++g_launches;
    if (R <= 128) {
      const int warps = (R + kGbP - 1) / kGbP;
      gj_blocked_kernel<<<nb, 32 * warps, 0, st>>>(D, R, Af, diag_idx, Af_inv, piv, status, level);
    } else {
      const int Rp = (R + 11) / 12 * 12, threads = gj_group(Rp / 12) * (Rp / 6);
      gj_inverse_kernel<12, 6, 512><<<nb, (threads + 31) / 32 * 32, 0, st>>>(D, R, Af, diag_idx, Af_inv, piv, status,
                                                                               level);
    }
    return;
  }
  if (std::is_same<T, float>::value &&
      launch_gj_cluster(false, nb, D, R, reinterpret_cast<const float*>(Ablk), diag_idx, reinterpret_cast<float*>(Ainv),
                        piv, status, level, st))
    return;
  const size_t cap = 220 * 1024;
  size_t sm1 = sizeof(T) * (size_t)R * (R + 1);
  int use = sm1 <= cap;
  if (use) cudaFuncSetAttribute(lu_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  ++g_launches;
  lu_factor_kernel<T><<<nb, 256, use ? sm1 : 0, st>>>(D, R, Ablk, diag_idx, luT, piv, status, level, use);
  if (R > 1024) return;  // the permutation table holds 1024 rows; larger blocks are rejected by the caller
  if (std::is_same<T, float>::value) {
    const int Rp = (R + 31) / 32 * 32;
    const size_t smf = sizeof(float) * 2 * (size_t)Rp * Rp;
    if (smf <= 200 * 1024 && Rp <= 256) {
      cudaFuncSetAttribute(lu_inverse_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
      ++g_launches;
      lu_inverse_f32_kernel<<<nb, Rp, smf, st>>>(R, Rp, reinterpret_cast<const float*>(luT), piv,
                                                  reinterpret_cast<float*>(Ainv));
      return;
    }
  }
  size_t f = sizeof(T) * (size_t)R * (R + 1), y = sizeof(T) * (size_t)R * R;
  int mode = (f + y <= cap) ? 2 : (f <= cap ? 1 : 0);
  size_t sm = mode == 2 ? f + y : (mode == 1 ? f : 0);
  if (sm) cudaFuncSetAttribute(lu_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  lu_inverse_kernel<T><<<nb, 256, sm, st>>>(R, luT, piv, Ainv, mode);
}
// ------------------------------------------------------------------------
// a3 in FP64 for R <= 128: in-place Gauss-Jordan inversion with partial
// pivoting, the matrix in registers.  The R x R block (identity-padded to
// 128 x 128) is spread over 16 x 16 threads; thread (ty, tx) owns rows
// 8 ty .. 8 ty + 7 and columns 8 tx .. 8 tx + 7.  Step k:
//   (a) the owners of column k publish it (f_i = a_ik) and the owners of
//       row k publish that row; barrier;
//   (b) warp 0 picks the pivot row p >= k of largest |a_pk| (the first on
//       ties: LAPACK's choice, which Gauss-Jordan shares with LU because the
//       entries below the diagonal are those of the Schur complement);
//       barrier;
//   (c) the owners of row p publish the scaled pivot row
//       w_j = a_pj / a_pk (j != k), w_k = 1 / a_pk; barrier;
//   (d) rows k and p trade places and every row i != k becomes
//       a_ij - f_i w_j (with a_ik read as 0); row k becomes w.
// After step R-1 the array holds (P A)^-1 = A^-1 P^T; the interchanges
// applied to the columns in reverse order give A^-1, which is written in
// FP32 (one rounding).  Work: R^3 FP64 multiply-adds, bound by the FP64
// pipe; three barriers per step.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1) gj64_reg_kernel(int D, int R, const float* __restrict__ Ablk,
                                                          const int32_t* __restrict__ diag_idx,
                                                          float* __restrict__ Ainv, int32_t* __restrict__ piv,
                                                          int32_t* __restrict__ status, int level) {
  __shared__ double colk[2][128], oldk[2][128], rowk[2][128];
  __shared__ int s_p[2], s_bad;
  __shared__ int src[128], dst[128], pv[128];
  const int box = blockIdx.x, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* A = Ablk + (size_t)(diag_idx ? diag_idx[box] : box) * D * D;
  double a[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = ty * 8 + r;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = tx * 8 + c;
      a[r][c] = (i < R && j < R) ? (double)__ldg(A + (size_t)i * D + j) : (i == j ? 1.0 : 0.0);
    }
  }
  if (tid == 0) s_bad = 0;
  for (int k = 0; k < R; ++k) {
    const int b = k & 1;
    const int kt = k >> 3, kc = k & 7;
    // (a) column k and row k
    if (tx == kt) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        double v = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) v = (c == kc) ? a[r][c] : v;
        colk[b][ty * 8 + r] = v;
      }
    }
    if (ty == kt) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r == kc) {
#pragma unroll
          for (int c = 0; c < 8; ++c) oldk[b][tx * 8 + c] = a[r][c];
        }
    }
    __syncthreads();
    // (b) pivot row
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < R; i += 32) {
        const double v = fabs(colk[b][i]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_p[b] = bi;
        pv[k] = bi;
        if (!(best > 0.0)) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_p[b];
    const double dinv = 1.0 / colk[b][p];
    // (c) scaled pivot row
    if (ty == (p >> 3)) {
      const int pr = p & 7;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r == pr) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int j = tx * 8 + c;
            rowk[b][j] = (j == k) ? dinv : a[r][c] * dinv;
          }
        }
    }
    __syncthreads();
    // (d) swap rows k and p, eliminate column k from every other row
    double w[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = rowk[b][tx * 8 + c];
    const double fk = colk[b][k];  // row k's entry, which moves to row p
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = ty * 8 + r;
      if (i == k) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[r][c] = w[c];
      } else {
        const bool isp = (i == p);
        const double f = isp ? fk : colk[b][i];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = tx * 8 + c;
          const double base = isp ? oldk[b][j] : a[r][c];
          a[r][c] = fma(-f, w[c], (j == k) ? 0.0 : base);
        }
      }
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0 && atomicCAS(status, 0, level + 1) == 0) status[1] = box;
    return;
  }
  // column unscramble: A^-1[:, j] = X[:, src[j]] after the swaps k = R-1 .. 0
  if (tid == 0) {
    for (int j = 0; j < R; ++j) src[j] = j;
    for (int k = R - 1; k >= 0; --k) {
      const int t = src[k];
      src[k] = src[pv[k]];
      src[pv[k]] = t;
    }
    for (int j = 0; j < R; ++j) dst[src[j]] = j;
  }
  __syncthreads();
  for (int k = tid; k < R; k += 256) piv[(size_t)box * R + k] = pv[k];
  float* Y = Ainv + (size_t)box * R * R;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = ty * 8 + r;
    if (i >= R) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = tx * 8 + c;
      if (j < R) Y[(size_t)i * R + dst[j]] = (float)a[r][c];
    }
  }
}

// a3 for the FP16/BF16 factorizations with FP64 arithmetic: the FP32
// Ahat_ii^RR are widened as they are read and inverted in FP64, and the
// inverse is rounded once to FP32 (Ainv); the pivots are LAPACK's.  R <= 128:
// the register Gauss-Jordan kernel above; larger R: the FP64 getf2 kernel
// (lu, nb * R * R FP64 scratch) and the FP64 inverse (inv, the same size).
void launch_lu_inverse_f64_for_f32(int nb, int D, int R, const float* Ablk, const int32_t* diag_idx, double* lu,
                                   double* inv, int32_t* piv, float* Ainv, int32_t* status, int level,
                                   cudaStream_t st) {
  if (nb == 0 || R == 0 || R > 1024) return;
  if (R <= 128) {
    ++g_launches;
    gj64_reg_kernel<<<nb, 256, 0, st>>>(D, R, Ablk, diag_idx, Ainv, piv, status, level);
    return;
  }
  if (launch_gj_cluster(true, nb, D, R, Ablk, diag_idx, Ainv, piv, status, level, st)) return;
  const size_t cap = 220 * 1024;
  const size_t sm1 = sizeof(double) * (size_t)R * (R + 1);
  const int use = sm1 <= cap;
  if (use) cudaFuncSetAttribute(lu_factor_kernel<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  ++g_launches;
  lu_factor_kernel<double, float><<<nb, 256, use ? sm1 : 0, st>>>(D, R, Ablk, diag_idx, lu, piv, status, level, use);
  const size_t f = sizeof(double) * (size_t)R * (R + 1), y = sizeof(double) * (size_t)R * R;
  const int mode = (f + y <= cap) ? 2 : (f <= cap ? 1 : 0);
  const size_t sm = mode == 2 ? f + y : (mode == 1 ? f : 0);
  if (sm) cudaFuncSetAttribute(lu_inverse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  lu_inverse_kernel<double><<<nb, 256, sm, st>>>(R, lu, piv, inv, mode);
  launch_convert<double, float>(inv, Ainv, (int64_t)nb * R * R, st);
}

template void launch_lu_inverse<double>(int, int, int, const double*, const int32_t*, double*, double*, int32_t*,
                                        double*, int32_t*, int, cudaStream_t);
template void launch_lu_inverse<float>(int, int, int, const float*, const int32_t*, double*, float*, int32_t*,
                                       float*, int32_t*, int, cudaStream_t);

// ------------------------------------------------------------------------
// a6: merge.  Child pair q of level l (near: its SS part of Ahat; far: Shat)
// goes to quadrant (i%2, j%2) of parent near block dst[q] (D_{l-1} = 2K).
// ------------------------------------------------------------------------
template <typename T>
__global__ void merge_kernel(int D, int K, int64_t NP, const T* __restrict__ Ahat,
                             const int32_t* __restrict__ ni, const int32_t* __restrict__ nj,
                             const int32_t* __restrict__ ndst, int64_t FP, const T* __restrict__ Shat,
                             const int32_t* __restrict__ fi, const int32_t* __restrict__ fj,
                             const int32_t* __restrict__ fdst, T* __restrict__ Apar) {
  const int R = D - K, Dp = 2 * K;
  const int64_t q = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
  if (q >= NP + FP) return;
  const bool nr = q < NP;
  const int64_t qq = nr ? q : q - NP;
  const int i = nr ? ni[qq] : fi[qq], j = nr ? nj[qq] : fj[qq];
  const int64_t dst = nr ? ndst[qq] : fdst[qq];
  T* out = Apar + dst * Dp * Dp + (int64_t)(i & 1) * K * Dp + (j & 1) * K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
    int a = e / K, b = e - a * K;
    T v = nr ? Ahat[qq * D * D + (int64_t)(R + a) * D + R + b] : Shat[qq * K * K + e];
    out[(int64_t)a * Dp + b] = v;
  }
}

template <typename T>
void launch_merge(int D, int K, int64_t NP, const T* Ahat, const int32_t* ni, const int32_t* nj,
                  const int32_t* ndst, int64_t FP, const T* Shat, const int32_t* fi, const int32_t* fj,
                  const int32_t* fdst, T* Apar, cudaStream_t st) {
  int64_t n = NP + FP;
  if (n == 0 || K == 0) return;
  int gx = std::min(64, (K * K + 255) / 256);
  int64_t gy = std::min<int64_t>(n, 65535), gz = (n + gy - 1) / gy;
  ++g_launches;
  merge_kernel<T><<<dim3(gx, (unsigned)gy, (unsigned)gz), 256, 0, st>>>(D, K, NP, Ahat, ni, nj, ndst, FP, Shat, fi,
                                                                         fj, fdst, Apar);
}
template void launch_merge<double>(int, int, int64_t, const double*, const int32_t*, const int32_t*,
                                   const int32_t*, int64_t, const double*, const int32_t*, const int32_t*,
                                   const int32_t*, double*, cudaStream_t);
template void launch_merge<float>(int, int, int64_t, const float*, const int32_t*, const int32_t*, const int32_t*,
                                  int64_t, const float*, const int32_t*, const int32_t*, const int32_t*, float*,
                                  cudaStream_t);

}  // namespace h2
