// Algorithm 1 on the GPU at a level rank K laid out beforehand (by the rank
// predictor, or the rank cap): randomized interpolative decompositions of
// every box of a level, batched, in FP64.
//
// For box i with points B_i (n_i <= 256), far samples S_F(i) and close boxes
// j != i with close samples S_C(j) (<= 64 points each), the composite matrix
// of Algorithm 1 is M_i = [G(B_i, S_F) | G(B_i, S_C(j)) G(S_C(j), S_C(j))^-1 ...].
// Its sketch Y_i = M_i Omega (n_i x m) takes Omega(p, t) = +-1 as a function
// of the sample point p (splitmix64), so the close part factors as
// G(B_i, S_C(j)) W_j with W_j = G(S_C(j), S_C(j))^-1 Omega(S_C(j)), computed
// once per box j and shared by every box that has j close:
//   cc_weights_kernel  per box j: W_j by Gauss-Jordan on [G(S_C, S_C) | Omega]
//                      (partial pivoting), or by `gs` Gauss-Seidel sweeps from
//                      W = 0 (the shortcut of Section 3.5 for the inverse of
//                      the close part in Algorithm 1)
//   sketch_kernel      per box and half of its rows: Y_i = G(B_i, S_F)
//                      Omega(S_F) + sum_j G(B_i, S_C(j)) W_j, kernel entries
//                      evaluated in 32-sample chunks into shared memory
//   pivqr_id_kernel    per box: column-pivoted Householder QR of the first ms
//                      columns of Y_i, transposed (ms x n_i; the rows of Y_i
//                      are its columns), K + 1 steps in global memory; the
//                      first K pivots are the skeleton, X_i = P [I; (R11^-1
//                      R12)^T]; also the pivot ratio |R_K+1,K+1| / |R_11| and
//                      the interpolation error on the q probe columns.
#include "h2_internal.h"
#include "kernels.h"

namespace h2 {
namespace {

constexpr int GC_CHUNK = 32;   // sample points per evaluated chunk
constexpr int GC_ROWS = 128;   // box rows per sketch CTA
constexpr int GC_MAXM = 160;   // sketch + probe columns
constexpr int GC_MAXS = 64;    // close samples per box

__device__ __forceinline__ uint64_t splitmix64_d(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
// Omega(p, t) in {-1, +1}
__device__ __forceinline__ double omega(uint64_t seed, int64_t p, int t) {
  const uint64_t bits = splitmix64_d(seed ^ ((uint64_t)p * 0x100000001B3ull + (uint64_t)(t >> 6)));
  return ((bits >> (t & 63)) & 1ull) ? 1.0 : -1.0;
}

// W_j (s x m, row-major at W + cptr[j] * m) for every box j.
__global__ void __launch_bounds__(256) cc_weights_kernel(KernelFn G, const double* __restrict__ pts,
                                                         const int64_t* __restrict__ cptr,
                                                         const int64_t* __restrict__ cidx, int m, uint64_t seed,
                                                         int gs, double* __restrict__ W) {
  extern __shared__ __align__(16) double smd[];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int64_t c0 = cptr[j];
  const int s = (int)(cptr[j + 1] - c0);
  if (s == 0) return;
  const int ld = s + m;  // augmented row [A_cc | Omega]
  double* Aug = smd;     // s x ld
  __shared__ int s_p;
  __shared__ double s_inv;
  for (int e = tid; e < s * ld; e += blockDim.x) {
    const int r = e / ld, c = e - r * ld;
    Aug[e] = (c < s) ? G.entry(pts, cidx[c0 + r], cidx[c0 + c], r == c) : omega(seed, cidx[c0 + r], c - s);
  }
  __syncthreads();
  if (gs <= 0) {
    // Gauss-Jordan with partial pivoting on the augmented system
    for (int k = 0; k < s; ++k) {
      if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int r = k + tid; r < s; r += 32) {
          const double v = fabs(Aug[r * ld + k]);
          if (v > best) best = v, bi = r;
        }
        for (int o = 16; o; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
        }
        if (tid == 0) {
          s_p = bi;
          s_inv = best > 0.0 ? 1.0 / Aug[bi * ld + k] : 0.0;
        }
      }
      __syncthreads();
      const int p = s_p;
      if (p != k)
        for (int c = tid; c < ld; c += blockDim.x) {
          const double t = Aug[k * ld + c];
          Aug[k * ld + c] = Aug[p * ld + c];
          Aug[p * ld + c] = t;
        }
      __syncthreads();
      for (int c = tid; c < ld; c += blockDim.x) Aug[k * ld + c] *= s_inv;
      __syncthreads();
      for (int e = tid; e < s * ld; e += blockDim.x) {
        const int r = e / ld, c = e - r * ld;
        if (r != k && c != k) Aug[e] = fma(-Aug[r * ld + k], Aug[k * ld + c], Aug[e]);
      }
      __syncthreads();
      for (int r = tid; r < s; r += blockDim.x)
        if (r != k) Aug[r * ld + k] = 0.0;
      __syncthreads();
    }
    double* Wj = W + c0 * m;
    for (int e = tid; e < s * m; e += blockDim.x) Wj[e] = Aug[(e / m) * ld + s + e % m];
    return;
  }
  // Gauss-Seidel: W = 0, then sweeps r = 0 .. s-1 of
  // W[r] = (Omega[r] - sum_{c != r} A[r][c] W[c]) / A[r][r]; thread t owns column t
  double* Wj = W + c0 * m;
  for (int t = tid; t < m; t += blockDim.x) {
    for (int r = 0; r < s; ++r) Wj[r * m + t] = 0.0;
    for (int it = 0; it < gs; ++it)
      for (int r = 0; r < s; ++r) {
        double a = Aug[r * ld + s + t];
        for (int c = 0; c < s; ++c)
          if (c != r) a = fma(-Aug[r * ld + c], Wj[c * m + t], a);
        Wj[r * m + t] = a / Aug[r * ld + r];
      }
  }
}

// Y_i (D x m row-major at Y + i * D * m), rows [128 h, 128 h + 128) of box i.
__global__ void __launch_bounds__(256) sketch_kernel(KernelFn G, const double* __restrict__ pts, int D, int m,
                                                     const int* __restrict__ nbox, const int64_t* __restrict__ bpts,
                                                     const int64_t* __restrict__ fptr,
                                                     const int64_t* __restrict__ fidx,
                                                     const int64_t* __restrict__ nptr,
                                                     const int32_t* __restrict__ nidx,
                                                     const int64_t* __restrict__ cptr,
                                                     const int64_t* __restrict__ cidx,
                                                     const double* __restrict__ W, uint64_t seed,
                                                     double* __restrict__ Y) {
  extern __shared__ __align__(16) double sks[];
  double(*Gs)[GC_CHUNK + 1] = reinterpret_cast<double(*)[GC_CHUNK + 1]>(sks);   // GC_ROWS rows
  double* Om = sks + GC_ROWS * (GC_CHUNK + 1);                                   // GC_CHUNK x m
  double(*Xa)[3] = reinterpret_cast<double(*)[3]>(Om + GC_CHUNK * m);            // GC_ROWS rows
  int64_t* pid = reinterpret_cast<int64_t*>(Xa + GC_ROWS);                       // GC_CHUNK
  const int i = blockIdx.x >> 1, h = blockIdx.x & 1, tid = threadIdx.x;
  const int n = nbox[i];
  const int a0 = h * GC_ROWS;
  if (a0 >= n) return;
  const int rows = min(GC_ROWS, n - a0);
  const int la = tid & (GC_ROWS - 1), half = tid >> 7;
  const int mh = m / 2;  // columns of this thread: [half * mh, half * mh + mh)
  double acc[GC_MAXM / 2];
#pragma unroll
  for (int t = 0; t < GC_MAXM / 2; ++t) acc[t] = 0.0;
  for (int r = tid; r < rows; r += blockDim.x) {
    const int64_t p = bpts[(int64_t)i * D + a0 + r];
    Xa[r][0] = pts[3 * p], Xa[r][1] = pts[3 * p + 1], Xa[r][2] = pts[3 * p + 2];
  }
  // one chunk of sample points q[0 .. cnt): entries G(B_i rows, q) and the
  // chunk's right factor (Omega rows, or W rows when Wsrc is given)
  auto chunk = [&](const int64_t* q, int cnt, const double* Wsrc) {
    __syncthreads();
    if (tid < cnt) pid[tid] = q[tid];
    __syncthreads();
    for (int e = tid; e < GC_ROWS * GC_CHUNK; e += blockDim.x) {
      const int r = e / GC_CHUNK, c = e - r * GC_CHUNK;
      double g = 0.0;
      if (r < rows && c < cnt) {
        const double* y = pts + 3 * pid[c];
        g = G.off(Xa[r], y);
      }
      Gs[r][c] = g;
    }
    for (int e = tid; e < GC_CHUNK * m; e += blockDim.x) {
      const int c = e / m, t = e - c * m;
      Om[e] = (c < cnt) ? (Wsrc ? Wsrc[(int64_t)c * m + t] : omega(seed, pid[c], t)) : 0.0;
    }
    __syncthreads();
    if (la < rows) {
      for (int c = 0; c < cnt; ++c) {
        const double g = Gs[la][c];
        const double* o = Om + c * m + half * mh;
#pragma unroll
        for (int t = 0; t < GC_MAXM / 2; ++t)
          if (t < mh) acc[t] = fma(g, o[t], acc[t]);
      }
    }
  };
  for (int64_t f = fptr[i]; f < fptr[i + 1]; f += GC_CHUNK)
    chunk(fidx + f, (int)(fptr[i + 1] - f < GC_CHUNK ? fptr[i + 1] - f : GC_CHUNK), nullptr);
  for (int64_t e = nptr[i]; e < nptr[i + 1]; ++e) {
    const int j = nidx[e];
    if (j == i) continue;
    for (int64_t f = cptr[j]; f < cptr[j + 1]; f += GC_CHUNK)
      chunk(cidx + f, (int)(cptr[j + 1] - f < GC_CHUNK ? cptr[j + 1] - f : GC_CHUNK), W + f * m);
  }
  if (la < rows) {
    double* yr = Y + ((int64_t)i * D + a0 + la) * m + half * mh;
#pragma unroll
    for (int t = 0; t < GC_MAXM / 2; ++t)
      if (t < mh) yr[t] = acc[t];
  }
}

// Column-pivoted QR of Z = Y_i^T[0 .. ms) (column a of Z = row a of Y_i, ld
// m), K + 1 steps, then X_i, the skeleton, the pivot ratio and probe error.
// piv (D per box) and T (in place of R12) use Y_i's storage.
__global__ void __launch_bounds__(512) pivqr_id_kernel(int D, int m, int ms, int q, int K,
                                                        const int* __restrict__ nbox, const int64_t* __restrict__ bpts,
                                                        double* __restrict__ Y, int32_t* __restrict__ piv_out,
                                                        double* __restrict__ X, int64_t* __restrict__ SK,
                                                        double* __restrict__ rho_out, double* __restrict__ err_out) {
  __shared__ double cn[256];
  __shared__ int perm[256];
  __shared__ double s_beta, s_tau, s_scal;
  __shared__ int s_pc;
  __shared__ double red[32];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int n = nbox[i];
  double* Z = Y + (int64_t)i * D * m;  // column a at Z + a * m
  for (int a = tid; a < n; a += blockDim.x) perm[a] = a;
  const int steps = min(K + 1, min(ms, n));
  for (int k = 0; k < steps; ++k) {
    __syncthreads();
    // squared norms of columns k .. n-1 over rows k .. ms-1
    for (int a = k + warp; a < n; a += nw) {
      const double* z = Z + (int64_t)a * m;
      double s2 = 0.0;
      for (int t = k + lane; t < ms; t += 32) s2 = fma(z[t], z[t], s2);
      for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) cn[a] = s2;
    }
    __syncthreads();
    if (tid == 0) {
      int pc = k;
      double best = -1.0;
      for (int a = k; a < n; ++a)
        if (cn[a] > best) best = cn[a], pc = a;
      s_pc = pc;
    }
    __syncthreads();
    const int pc = s_pc;
    if (pc != k) {
      for (int t = tid; t < ms; t += blockDim.x) {
        const double u = Z[(int64_t)k * m + t];
        Z[(int64_t)k * m + t] = Z[(int64_t)pc * m + t];
        Z[(int64_t)pc * m + t] = u;
      }
      if (tid == 0) {
        const int u = perm[k];
        perm[k] = perm[pc];
        perm[pc] = u;
      }
    }
    __syncthreads();
    // Householder reflector of column k, rows k .. ms-1
    double* zk = Z + (int64_t)k * m;
    double part = 0.0;
    for (int t = k + 1 + tid; t < ms; t += blockDim.x) part = fma(zk[t], zk[t], part);
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      double xn2 = 0.0;
      for (int w = 0; w < nw; ++w) xn2 += red[w];
      const double alpha = zk[k];
      if (xn2 == 0.0) {
        s_tau = 0.0, s_beta = alpha, s_scal = 0.0;
      } else {
        const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        s_tau = (beta - alpha) / beta, s_scal = 1.0 / (alpha - beta), s_beta = beta;
      }
    }
    __syncthreads();
    const double tau = s_tau, scal = s_scal;
    if (tau != 0.0)
      for (int t = k + 1 + tid; t < ms; t += blockDim.x) zk[t] *= scal;
    __syncthreads();
    if (tid == 0) zk[k] = s_beta;
    if (tau != 0.0) {
      for (int a = k + 1 + warp; a < n; a += nw) {
        double* z = Z + (int64_t)a * m;
        double w = 0.0;
        for (int t = k + 1 + lane; t < ms; t += 32) w = fma(zk[t], z[t], w);
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w = tau * (w + z[k]);
        if (lane == 0) z[k] -= w;
        for (int t = k + 1 + lane; t < ms; t += 32) z[t] = fma(-w, zk[t], z[t]);
      }
    }
  }
  __syncthreads();
  const double rr0 = fabs(Z[0]);
  if (tid == 0) rho_out[i] = (steps > K && rr0 > 0.0) ? fabs(Z[(int64_t)K * m + K]) / rr0 : 0.0;
  // T = R11^-1 R12 in place of R12 (column K + b of Z, rows 0 .. K-1)
  for (int b = tid; b < n - K; b += blockDim.x) {
    double* zc = Z + (int64_t)(K + b) * m;
    for (int t = K - 1; t >= 0; --t) {
      double s = zc[t];
      for (int u = t + 1; u < K; ++u) s = fma(-Z[(int64_t)u * m + t], zc[u], s);
      const double d = Z[(int64_t)t * m + t];
      zc[t] = (fabs(d) > 1e-15 * rr0 && d != 0.0) ? s / d : 0.0;
    }
  }
  __syncthreads();
  // X (D x K row-major), skeleton, pivots
  double* Xi = X + (int64_t)i * D * K;
  for (int e = tid; e < D * K; e += blockDim.x) Xi[e] = 0.0;
  __syncthreads();
  for (int a = tid; a < K; a += blockDim.x) {
    Xi[(int64_t)perm[a] * K + a] = 1.0;
    SK[(int64_t)i * K + a] = bpts[(int64_t)i * D + perm[a]];
  }
  for (int e = tid; e < (n - K) * K; e += blockDim.x) {
    const int b = e / K, a = e - b * K;
    Xi[(int64_t)perm[K + b] * K + a] = Z[(int64_t)(K + b) * m + a];
  }
  for (int a = tid; a < n; a += blockDim.x) piv_out[(int64_t)i * D + a] = perm[a];
  // probe error ||Yq - X Yq[SK]|| / ||Yq|| (probe columns ms .. ms+q-1 are
  // untouched, rows in the original order)
  double e2 = 0.0, y2 = 0.0;
  for (int e = tid; e < n * q; e += blockDim.x) {
    const int a = e / q, c = ms + (e - a * q);
    const double v = Z[(int64_t)a * m + c];
    y2 = fma(v, v, y2);
  }
  for (int e = tid; e < (n - K) * q; e += blockDim.x) {
    const int b = e / q, c = ms + (e - b * q);
    double v = Z[(int64_t)perm[K + b] * m + c];
    for (int u = 0; u < K; ++u) v = fma(-Z[(int64_t)(K + b) * m + u], Z[(int64_t)perm[u] * m + c], v);
    e2 = fma(v, v, e2);
  }
  for (int o = 16; o; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  __syncthreads();
  if (lane == 0) red[warp] = e2, cn[warp] = y2;
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) a += red[w], b += cn[w];
    err_out[i] = sqrt(a / fmax(b, 1e-300));
  }
}

}  // namespace

void launch_cc_weights(const KernelFn& G, const double* pts, int nb, const int64_t* cptr, const int64_t* cidx, int m,
                       uint64_t seed, int gs, double* W, cudaStream_t st) {
  const size_t sm = sizeof(double) * (size_t)GC_MAXS * (GC_MAXS + m);
  cudaFuncSetAttribute(cc_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  cc_weights_kernel<<<nb, 256, sm, st>>>(G, pts, cptr, cidx, m, seed, gs, W);
}

void launch_sketch(const KernelFn& G, const double* pts, int nb, int D, int m, const int* nbox, const int64_t* bpts,
                   const int64_t* fptr, const int64_t* fidx, const int64_t* nptr, const int32_t* nidx,
                   const int64_t* cptr, const int64_t* cidx, const double* W, uint64_t seed, double* Y,
                   cudaStream_t st) {
  const size_t sm = sizeof(double) * ((size_t)GC_ROWS * (GC_CHUNK + 1) + (size_t)GC_CHUNK * m + GC_ROWS * 3) +
                    sizeof(int64_t) * GC_CHUNK;
  cudaFuncSetAttribute(sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  sketch_kernel<<<2 * nb, 256, sm, st>>>(G, pts, D, m, nbox, bpts, fptr, fidx, nptr, nidx, cptr, cidx, W, seed, Y);
}

void launch_pivqr_id(int nb, int D, int m, int ms, int q, int K, const int* nbox, const int64_t* bpts, double* Y,
                     int32_t* piv, double* X, int64_t* SK, double* rho, double* err, cudaStream_t st) {
  ++g_launches;
  pivqr_id_kernel<<<nb, 512, 0, st>>>(D, m, ms, q, K, nbox, bpts, Y, piv, X, SK, rho, err);
}

// ---------------------------------------------------------------------------
// host side: one level at a time; device buffers grow as needed
// ---------------------------------------------------------------------------
namespace {

struct DeviceGpuCompressor : GpuCompressor {
  KernelFn G;
  int gs = 0;
  double* pts = nullptr;
  std::vector<void*> bufs;  // freed at destruction
  ~DeviceGpuCompressor() override {
    for (void* b : bufs) cudaFree(b);
    cudaFree(pts);
  }
  bool supported(int D, int K) const override { return D <= 2 * GC_ROWS && K >= 1 && K + 32 <= GC_MAXM; }
  template <typename V>
  cudaError_t put(V** d, const std::vector<V>& h) {
    *d = nullptr;
    cudaError_t e = cudaMalloc(d, sizeof(V) * std::max<size_t>(h.size(), 1));
    if (e != cudaSuccess) return e;
    bufs.push_back(*d);
    if (!h.empty()) e = cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice);
    return e;
  }
  template <typename V>
  cudaError_t make(V** d, size_t n) {
    cudaError_t e = cudaMalloc(d, sizeof(V) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) bufs.push_back(*d);
    return e;
  }
  std::string run(GpuLevelJob& j) override {
    j.gs = gs;
    const size_t nb = j.nb, D = j.D, K = j.K, m = j.m;
    int* d_nbox;
    int64_t *d_bpts, *d_fptr, *d_fidx, *d_nptr, *d_cptr, *d_cidx, *d_SK;
    int32_t *d_nidx, *d_piv;
    double *d_W, *d_Y, *d_X, *d_rho, *d_err;
    cudaError_t e = cudaSuccess;
#define GC_TRY(x) \
  if ((e = (x)) != cudaSuccess) return std::string(#x) + ": " + cudaGetErrorString(e)
    const size_t nbufs = bufs.size();
    GC_TRY(put(&d_nbox, j.nbox));
    GC_TRY(put(&d_bpts, j.bpts));
    GC_TRY(put(&d_fptr, j.fptr));
    GC_TRY(put(&d_fidx, j.fidx));
    GC_TRY(put(&d_nptr, j.nptr));
    GC_TRY(put(&d_nidx, j.nidx));
    GC_TRY(put(&d_cptr, j.cptr));
    GC_TRY(put(&d_cidx, j.cidx));
    GC_TRY(make(&d_W, j.cidx.size() * m));
    GC_TRY(make(&d_Y, nb * D * m));
    GC_TRY(make(&d_X, nb * D * K));
    GC_TRY(make(&d_SK, nb * K));
    GC_TRY(make(&d_piv, nb * D));
    GC_TRY(make(&d_rho, nb));
    GC_TRY(make(&d_err, nb));
    launch_cc_weights(G, pts, j.nb, d_cptr, d_cidx, j.m, j.seed, j.gs, d_W, 0);
    launch_sketch(G, pts, j.nb, j.D, j.m, d_nbox, d_bpts, d_fptr, d_fidx, d_nptr, d_nidx, d_cptr, d_cidx, d_W, j.seed,
                  d_Y, 0);
    launch_pivqr_id(j.nb, j.D, j.m, j.ms, j.q, j.K, d_nbox, d_bpts, d_Y, d_piv, d_X, d_SK, d_rho, d_err, 0);
    GC_TRY(cudaGetLastError());
    j.X.resize(nb * D * K);
    j.SK.resize(nb * K);
    j.piv.resize(nb * D);
    j.rho.resize(nb);
    j.err.resize(nb);
    GC_TRY(cudaMemcpy(j.X.data(), d_X, sizeof(double) * j.X.size(), cudaMemcpyDeviceToHost));
    GC_TRY(cudaMemcpy(j.SK.data(), d_SK, sizeof(int64_t) * j.SK.size(), cudaMemcpyDeviceToHost));
    GC_TRY(cudaMemcpy(j.piv.data(), d_piv, sizeof(int32_t) * j.piv.size(), cudaMemcpyDeviceToHost));
    GC_TRY(cudaMemcpy(j.rho.data(), d_rho, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    GC_TRY(cudaMemcpy(j.err.data(), d_err, sizeof(double) * nb, cudaMemcpyDeviceToHost));
#undef GC_TRY
    for (size_t b = nbufs; b < bufs.size(); ++b) cudaFree(bufs[b]);
    bufs.resize(nbufs);
    // flops (2 per multiply-add; kernel evaluations not counted): the
    // close-field part (W_j and the close sketch terms) and the far part
    for (size_t jb = 0; jb < nb; ++jb) {
      const double sj = (double)(j.cptr[jb + 1] - j.cptr[jb]);
      j.flops_prefactor += 2.0 * sj * sj * (sj + (double)m);
    }
    for (size_t i = 0; i < nb; ++i) {
      const double ni = j.nbox[i];
      j.flops_far += 2.0 * ni * (double)(j.fptr[i + 1] - j.fptr[i]) * (double)m;
      for (int64_t e2 = j.nptr[i]; e2 < j.nptr[i + 1]; ++e2) {
        const int jj = j.nidx[e2];
        if ((size_t)jj == i) continue;
        j.flops_prefactor += 2.0 * ni * (double)(j.cptr[jj + 1] - j.cptr[jj]) * (double)m;
      }
    }
    return "";
  }
};

}  // namespace

GpuCompressor* make_gpu_compressor(const KernelFn& G, const double* pts, int64_t N, int gs_sweeps) {
  DeviceGpuCompressor* c = new DeviceGpuCompressor();
  c->G = G;
  c->gs = gs_sweeps;
  if (cudaMalloc(&c->pts, sizeof(double) * 3 * (size_t)N) != cudaSuccess ||
      cudaMemcpy(c->pts, pts, sizeof(double) * 3 * (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return nullptr;
  }
  return c;
}

}  // namespace h2
