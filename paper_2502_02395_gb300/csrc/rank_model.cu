// Learned rank predictor: a 16 -> 64 -> 64 -> 1 multilayer perceptron with
// ReLU activations that maps a cluster's geometry features to the fraction
// k / n of its dimension the rank-revealing compression of Algorithm 1
// keeps.  Trained on the GPU by the kernels below (BF16 weights, inputs and
// hidden activations, FP32 accumulation, FP32 master weights and Adam
// moments); used by h2_build_predicted to lay out every level's rank before
// any compression.  The paper has no counterpart: this is the north-star
// extension of the construction.
//
// Parameters, flat (the order of include/h2ulv.h): W1 (64 x 16 row-major),
// b1 (64), W2 (64 x 64 row-major), b2 (64), w3 (64), b3 (1); 5313 numbers.
// Every group starts on a multiple of 64, which the gradient kernel uses.
//
// Kernels (all tiny and latency bound: a few thousand samples, 5313
// parameters):
//   rm_prepare_kernel   (raw - mean) / std -> BF16 network inputs
//   rm_grad_kernel      forward + backward for chunks of 64 samples per CTA
//                       (one thread per sample for the per-sample vectors,
//                       then one thread per 84 parameter slots for the sums over
//                       the chunk), per-CTA partial gradients and loss
//   rm_adam_kernel      sums the partials in a fixed order (deterministic)
//                       and applies Adam; rounds the new weights to BF16
//   rm_reduce_kernel    the same sums without an update (gradient check)
//   rm_forward_kernel   inference
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "h2_internal.h"
#include "kernels.h"

namespace {

constexpr int NIN = 16, NH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248, OFF_B3 = 5312;
constexpr int NPAR = 5313;
constexpr int CH = 64;             // samples per chunk (= threads per CTA)
constexpr int PER_T = 84;          // parameter slots per thread: p = tid + 64 kk, kk < 84
constexpr int LDH = NH + 1;        // padded row length of the per-sample tiles
constexpr int MAX_CTAS = 152 * 4;  // partial-gradient rows

struct GradSmem {
  float W[NPAR];
  float G[NPAR];  // this CTA's gradient sums (entry p owned by thread p % 64)
  float X[CH][NIN + 1];
  float H1[CH][LDH], H2[CH][LDH], DZ1[CH][LDH], DZ2[CH][LDH];
  float DO[CH];
  float red[CH];
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__global__ void __launch_bounds__(256) rm_prepare_kernel(const float* __restrict__ raw, int64_t n,
                                                         const float* __restrict__ mean,
                                                         const float* __restrict__ istd,
                                                         __nv_bfloat16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * NIN; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e % NIN);
    out[e] = __float2bfloat16_rn((raw[e] - mean[f]) * istd[f]);
  }
}

// Forward and backward over chunks of CH samples; partial[cta][p] receives
// this CTA's gradient sums and partial[cta][NPAR] its sum of squared errors.
// step (may be NULL) is incremented once by CTA 0: the Adam step counter.
__global__ void __launch_bounds__(CH) rm_grad_kernel(const __nv_bfloat16* __restrict__ X, const float* __restrict__ y,
                                                     int64_t n, const __nv_bfloat16* __restrict__ w,
                                                     float* __restrict__ partial, float inv_n, int* step) {
  extern __shared__ __align__(16) unsigned char smraw[];
  GradSmem& s = *reinterpret_cast<GradSmem*>(smraw);
  const int t = threadIdx.x;
  if (step && blockIdx.x == 0 && t == 0) atomicAdd(step, 1);
  for (int p = t; p < NPAR; p += CH) s.W[p] = __bfloat162float(w[p]), s.G[p] = 0.f;
  float sse = 0.f;
  const int64_t nchunk = (n + CH - 1) / CH;
  for (int64_t ck = blockIdx.x; ck < nchunk; ck += gridDim.x) {
    const int64_t smp = ck * CH + t;
    const bool valid = smp < n;
    __syncthreads();  // the previous chunk's tiles are no longer read
#pragma unroll
    for (int f = 0; f < NIN; ++f) s.X[t][f] = valid ? __bfloat162float(X[smp * NIN + f]) : 0.f;
    // layer 1: h1 = bf16(relu(W1 x + b1))
    for (int j = 0; j < NH; ++j) {
      float z = s.W[OFF_B1 + j];
#pragma unroll
      for (int f = 0; f < NIN; ++f) z = fmaf(s.W[OFF_W1 + j * NIN + f], s.X[t][f], z);
      s.H1[t][j] = bf16r(fmaxf(z, 0.f));
    }
    // layer 2: h2 = bf16(relu(W2 h1 + b2)); output o = w3 . h2 + b3
    float o = s.W[OFF_B3];
    for (int j = 0; j < NH; ++j) {
      float z = s.W[OFF_B2 + j];
#pragma unroll 16
      for (int k = 0; k < NH; ++k) z = fmaf(s.W[OFF_W2 + j * NH + k], s.H1[t][k], z);
      const float h = bf16r(fmaxf(z, 0.f));
      s.H2[t][j] = h;
      o = fmaf(s.W[OFF_W3 + j], h, o);
    }
    const float e = valid ? o - y[smp] : 0.f;
    sse = fmaf(e, e, sse);
    const float d_o = 2.f * e * inv_n;  // d loss / d o
    s.DO[t] = d_o;
    for (int j = 0; j < NH; ++j) s.DZ2[t][j] = (s.H2[t][j] > 0.f) ? d_o * s.W[OFF_W3 + j] : 0.f;
    for (int k = 0; k < NH; ++k) {
      float a = 0.f;
#pragma unroll 16
      for (int j = 0; j < NH; ++j) a = fmaf(s.DZ2[t][j], s.W[OFF_W2 + j * NH + k], a);
      s.DZ1[t][k] = (s.H1[t][k] > 0.f) ? a : 0.f;
    }
    __syncthreads();
    // sums over the chunk: parameter p = t + 64 kk; the groups start on
    // multiples of 64, so kk alone says which group
    for (int kk = 0; kk < PER_T; ++kk) {
      const int p = t + CH * kk;
      if (p >= NPAR) continue;
      float a = 0.f;
      if (p < OFF_B1) {  // W1[j][f]: sum dz1_j x_f
        const int j = p / NIN, f = p % NIN;
        for (int u = 0; u < CH; ++u) a = fmaf(s.DZ1[u][j], s.X[u][f], a);
      } else if (p < OFF_W2) {  // b1
        const int j = p - OFF_B1;
        for (int u = 0; u < CH; ++u) a += s.DZ1[u][j];
      } else if (p < OFF_B2) {  // W2[j][k]: sum dz2_j h1_k
        const int j = (p - OFF_W2) / NH, k = (p - OFF_W2) % NH;
        for (int u = 0; u < CH; ++u) a = fmaf(s.DZ2[u][j], s.H1[u][k], a);
      } else if (p < OFF_W3) {  // b2
        const int j = p - OFF_B2;
        for (int u = 0; u < CH; ++u) a += s.DZ2[u][j];
      } else if (p < OFF_B3) {  // w3[j]: sum do h2_j
        const int j = p - OFF_W3;
        for (int u = 0; u < CH; ++u) a = fmaf(s.DO[u], s.H2[u][j], a);
      } else {  // b3
        for (int u = 0; u < CH; ++u) a += s.DO[u];
      }
      s.G[p] += a;
    }
  }
  float* out = partial + (size_t)blockIdx.x * (NPAR + 1);
  for (int p = t; p < NPAR; p += CH) out[p] = s.G[p];
  s.red[t] = sse;
  __syncthreads();
  if (t == 0) {
    float a = 0.f;
    for (int u = 0; u < CH; ++u) a += s.red[u];
    out[NPAR] = a;
  }
}

// grad[p] = sum over CTAs of partial[.][p]; loss[0] = sum of squared errors * inv_n.
__global__ void __launch_bounds__(256) rm_reduce_kernel(const float* __restrict__ partial, int nblk, float inv_n,
                                                        float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPAR) return;
  float a = 0.f;
  for (int b = 0; b < nblk; ++b) a += partial[(size_t)b * (NPAR + 1) + p];
  if (p < NPAR) grad[p] = a;
  else loss[0] = a * inv_n;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master weights; the
// step number is *step (incremented by rm_grad_kernel).
__global__ void __launch_bounds__(256) rm_adam_kernel(const float* __restrict__ partial, int nblk, float inv_n,
                                                      float* __restrict__ master, __nv_bfloat16* __restrict__ wb,
                                                      float* __restrict__ m1, float* __restrict__ m2,
                                                      const int* __restrict__ step, float lr, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPAR) return;
  float a = 0.f;
  for (int b = 0; b < nblk; ++b) a += partial[(size_t)b * (NPAR + 1) + p];
  if (p == NPAR) {
    loss[0] = a * inv_n;
    return;
  }
  const float b1 = 0.9f, b2 = 0.999f;
  const int k = *step;
  const float m = b1 * m1[p] + (1.f - b1) * a;
  const float v = b2 * m2[p] + (1.f - b2) * a * a;
  m1[p] = m;
  m2[p] = v;
  const float mh = m / (1.f - powf(b1, (float)k)), vh = v / (1.f - powf(b2, (float)k));
  const float wnew = master[p] - lr * mh / (sqrtf(vh) + 1e-8f);
  master[p] = wnew;
  wb[p] = __float2bfloat16_rn(wnew);
}

// Inference: one thread per sample, weights in shared memory.
__global__ void __launch_bounds__(128) rm_forward_kernel(const __nv_bfloat16* __restrict__ X, int64_t n,
                                                         const __nv_bfloat16* __restrict__ w, float* __restrict__ out) {
  __shared__ float W[NPAR];
  for (int p = threadIdx.x; p < NPAR; p += blockDim.x) W[p] = __bfloat162float(w[p]);
  __syncthreads();
  const int64_t smp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (smp >= n) return;
  float x[NIN], h1[NH];
#pragma unroll
  for (int f = 0; f < NIN; ++f) x[f] = __bfloat162float(X[smp * NIN + f]);
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float z = W[OFF_B1 + j];
#pragma unroll
    for (int f = 0; f < NIN; ++f) z = fmaf(W[OFF_W1 + j * NIN + f], x[f], z);
    h1[j] = bf16r(fmaxf(z, 0.f));
  }
  float o = W[OFF_B3];
#pragma unroll 1
  for (int j = 0; j < NH; ++j) {
    float z = W[OFF_B2 + j];
#pragma unroll
    for (int k = 0; k < NH; ++k) z = fmaf(W[OFF_W2 + j * NH + k], h1[k], z);
    o = fmaf(W[OFF_W3 + j], bf16r(fmaxf(z, 0.f)), o);
  }
  out[smp] = o;
}

// splitmix64 (Steele, Lea, Flood 2014): the counter-based generator of the
// initial weights.
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

struct h2_rank_model {
  int dev = 0;
  cudaStream_t st = nullptr;
  float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *partial = nullptr, *loss = nullptr, *grad = nullptr;
  __nv_bfloat16* wb = nullptr;
  int* step = nullptr;
  float *d_mean = nullptr, *d_istd = nullptr, *d_zero = nullptr, *d_one = nullptr;
  float mean[NIN], istd[NIN];
  bool normalized = false;
  // data buffers (grown on demand)
  int64_t cap = 0;
  float *raw = nullptr, *y = nullptr, *out = nullptr;
  __nv_bfloat16* X = nullptr;
  std::string err;
};

namespace {

#define RM_CK(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_);    \
      return e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA; \
    }                                                                 \
  } while (0)

h2_status ensure_cap(h2_rank_model* m, int64_t n) {
  if (n <= m->cap) return H2_OK;
  cudaFree(m->raw);
  cudaFree(m->y);
  cudaFree(m->out);
  cudaFree(m->X);
  m->raw = m->y = m->out = nullptr;
  m->X = nullptr;
  m->cap = 0;
  RM_CK(cudaMalloc(&m->raw, sizeof(float) * n * NIN));
  RM_CK(cudaMalloc(&m->y, sizeof(float) * n));
  RM_CK(cudaMalloc(&m->out, sizeof(float) * n));
  RM_CK(cudaMalloc(&m->X, sizeof(__nv_bfloat16) * n * NIN));
  m->cap = n;
  return H2_OK;
}

// Copy n x 16 features (host or device) into m->raw and make BF16 network
// inputs with the given normalization (device vectors mean, istd).
h2_status stage_inputs(h2_rank_model* m, const float* feats, int64_t n, const float* mean, const float* istd) {
  h2_status s = ensure_cap(m, n);
  if (s != H2_OK) return s;
  RM_CK(cudaMemcpyAsync(m->raw, feats, sizeof(float) * n * NIN, cudaMemcpyDefault, m->st));
  const int grid = (int)std::min<int64_t>((n * NIN + 255) / 256, 1024);
  ++h2::g_launches;
  rm_prepare_kernel<<<grid, 256, 0, m->st>>>(m->raw, n, mean, istd, m->X);
  RM_CK(cudaGetLastError());
  return H2_OK;
}

h2_status stage_targets(h2_rank_model* m, const float* y, int64_t n) {
  RM_CK(cudaMemcpyAsync(m->y, y, sizeof(float) * n, cudaMemcpyDefault, m->st));
  return H2_OK;
}

int grad_ctas(int64_t n) { return (int)std::min<int64_t>((n + CH - 1) / CH, MAX_CTAS); }

void launch_grad(h2_rank_model* m, int64_t n, int nblk, bool count_step) {
  ++h2::g_launches;
  rm_grad_kernel<<<nblk, CH, sizeof(GradSmem), m->st>>>(m->X, m->y, n, m->wb, m->partial, 1.f / (float)n,
                                                         count_step ? m->step : nullptr);
}

void launch_adam(h2_rank_model* m, int64_t n, int nblk, float lr) {
  ++h2::g_launches;
  rm_adam_kernel<<<(NPAR + 1 + 255) / 256, 256, 0, m->st>>>(m->partial, nblk, 1.f / (float)n, m->master, m->wb,
                                                             m->m1, m->m2, m->step, lr, m->loss);
}

}  // namespace

extern "C" {

h2_status h2_rank_model_create(h2_rank_model** out, uint64_t seed) {
  if (!out) return H2_ERR_INVALID_ARG;
  *out = nullptr;
  h2_rank_model* m = new h2_rank_model();
  cudaGetDevice(&m->dev);
  auto fail = [&](h2_status s) {
    h2_rank_model_destroy(m);
    return s;
  };
#define RM_ALLOC(p, n)                                            \
  if (cudaMalloc(&(p), (n)) != cudaSuccess) return fail(H2_ERR_OOM)
  RM_ALLOC(m->master, sizeof(float) * NPAR);
  RM_ALLOC(m->m1, sizeof(float) * NPAR);
  RM_ALLOC(m->m2, sizeof(float) * NPAR);
  RM_ALLOC(m->grad, sizeof(float) * NPAR);
  RM_ALLOC(m->wb, sizeof(__nv_bfloat16) * NPAR);
  RM_ALLOC(m->partial, sizeof(float) * (size_t)MAX_CTAS * (NPAR + 1));
  RM_ALLOC(m->loss, sizeof(float) * 2);
  RM_ALLOC(m->step, sizeof(int));
  RM_ALLOC(m->d_mean, sizeof(float) * NIN);
  RM_ALLOC(m->d_istd, sizeof(float) * NIN);
  RM_ALLOC(m->d_zero, sizeof(float) * NIN);
  RM_ALLOC(m->d_one, sizeof(float) * NIN);
#undef RM_ALLOC
  // He-uniform initial weights from splitmix64(seed, index); zero biases
  std::vector<float> w(NPAR, 0.f), zero(NIN, 0.f), one(NIN, 1.f);
  auto uni = [&](int p) { return (float)((splitmix64(seed * 0x100000001B3ull + (uint64_t)p) >> 11) * 0x1.0p-53); };
  for (int p = OFF_W1; p < OFF_B1; ++p) w[p] = (2.f * uni(p) - 1.f) * std::sqrt(6.f / NIN);
  for (int p = OFF_W2; p < OFF_B2; ++p) w[p] = (2.f * uni(p) - 1.f) * std::sqrt(6.f / NH);
  for (int p = OFF_W3; p < OFF_B3; ++p) w[p] = (2.f * uni(p) - 1.f) * std::sqrt(6.f / NH);
  for (int f = 0; f < NIN; ++f) m->mean[f] = 0.f, m->istd[f] = 1.f;
  if (cudaFuncSetAttribute(rm_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)) !=
      cudaSuccess)
    return fail(H2_ERR_CUDA);
  h2_status s = h2_rank_model_set_weights(m, w.data());
  if (s != H2_OK) return fail(s);
  if (cudaMemcpy(m->d_zero, zero.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_one, one.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_mean, zero.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_istd, one.data(), sizeof(float) * NIN, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(H2_ERR_CUDA);
  *out = m;
  return H2_OK;
}

h2_status h2_rank_model_set_weights(h2_rank_model* m, const float* theta) {
  if (!m || !theta) return H2_ERR_INVALID_ARG;
  m->err.clear();
  std::vector<float> h(NPAR);
  std::memcpy(h.data(), theta, sizeof(float) * NPAR);
  std::vector<__nv_bfloat16> hb(NPAR);
  for (int p = 0; p < NPAR; ++p) hb[p] = __float2bfloat16_rn(h[p]);
  RM_CK(cudaMemcpy(m->master, h.data(), sizeof(float) * NPAR, cudaMemcpyHostToDevice));
  RM_CK(cudaMemcpy(m->wb, hb.data(), sizeof(__nv_bfloat16) * NPAR, cudaMemcpyHostToDevice));
  RM_CK(cudaMemset(m->m1, 0, sizeof(float) * NPAR));
  RM_CK(cudaMemset(m->m2, 0, sizeof(float) * NPAR));
  RM_CK(cudaMemset(m->step, 0, sizeof(int)));
  return H2_OK;
}

h2_status h2_rank_model_get_weights(h2_rank_model* m, float* theta, float* mean, float* istd) {
  if (!m || !theta) return H2_ERR_INVALID_ARG;
  m->err.clear();
  RM_CK(cudaMemcpy(theta, m->master, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
  if (mean) std::memcpy(mean, m->mean, sizeof(float) * NIN);
  if (istd) std::memcpy(istd, m->istd, sizeof(float) * NIN);
  return H2_OK;
}

h2_status h2_rank_model_grad(h2_rank_model* m, const float* inputs, const float* targets, int64_t n, float* loss,
                             float* grad) {
  if (!m || !inputs || !targets || n < 1 || !grad) return H2_ERR_INVALID_ARG;
  m->err.clear();
  h2_status s = stage_inputs(m, inputs, n, m->d_zero, m->d_one);
  if (s != H2_OK) return s;
  if ((s = stage_targets(m, targets, n)) != H2_OK) return s;
  const int nblk = grad_ctas(n);
  launch_grad(m, n, nblk, false);
  ++h2::g_launches;
  rm_reduce_kernel<<<(NPAR + 1 + 255) / 256, 256, 0, m->st>>>(m->partial, nblk, 1.f / (float)n, m->grad, m->loss);
  RM_CK(cudaGetLastError());
  RM_CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, m->st));
  float l = 0.f;
  RM_CK(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
  RM_CK(cudaStreamSynchronize(m->st));
  if (loss) *loss = l;
  return H2_OK;
}

h2_status h2_rank_model_train(h2_rank_model* m, const float* feats, const float* targets, int64_t n, int32_t steps,
                              float lr, float* loss_out) {
  if (!m || !feats || !targets || n < 1 || steps < 0 || !(lr > 0.f)) return H2_ERR_INVALID_ARG;
  m->err.clear();
  // normalization of the features: mean and 1 / standard deviation over the
  // training set (host copy of the features)
  std::vector<float> h((size_t)n * NIN);
  RM_CK(cudaMemcpy(h.data(), feats, sizeof(float) * n * NIN, cudaMemcpyDefault));
  for (int f = 0; f < NIN; ++f) {
    double a = 0, b = 0;
    for (int64_t i = 0; i < n; ++i) a += h[(size_t)i * NIN + f];
    a /= (double)n;
    for (int64_t i = 0; i < n; ++i) {
      const double d = h[(size_t)i * NIN + f] - a;
      b += d * d;
    }
    const double sd = std::sqrt(b / (double)n);
    m->mean[f] = (float)a;
    m->istd[f] = sd > 1e-6 ? (float)(1.0 / sd) : 1.f;
  }
  m->normalized = true;
  RM_CK(cudaMemcpy(m->d_mean, m->mean, sizeof(float) * NIN, cudaMemcpyHostToDevice));
  RM_CK(cudaMemcpy(m->d_istd, m->istd, sizeof(float) * NIN, cudaMemcpyHostToDevice));
  h2_status s = stage_inputs(m, feats, n, m->d_mean, m->d_istd);
  if (s != H2_OK) return s;
  if ((s = stage_targets(m, targets, n)) != H2_OK) return s;
  const int nblk = grad_ctas(n);
  // full-batch Adam; 64 steps (two launches each) per CUDA graph
  const int per_graph = 64;
  cudaGraphExec_t exec = nullptr;
  if (steps >= per_graph) {
    cudaStream_t cap = nullptr;
    RM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t keep = m->st;
    m->st = cap;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < per_graph; ++k) {
        launch_grad(m, n, nblk, true);
        launch_adam(m, n, nblk, lr);
      }
      e = cudaStreamEndCapture(cap, &graph);
    }
    m->st = keep;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      m->err = std::string("training graph: ") + cudaGetErrorString(e);
      return H2_ERR_CUDA;
    }
  }
  RM_CK(cudaStreamSynchronize(m->st));
  int done = 0;
  for (; exec && done + per_graph <= steps; done += per_graph) RM_CK(cudaGraphLaunch(exec, m->st));
  for (; done < steps; ++done) {
    launch_grad(m, n, nblk, true);
    launch_adam(m, n, nblk, lr);
  }
  RM_CK(cudaGetLastError());
  float l = 0.f;
  RM_CK(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
  RM_CK(cudaStreamSynchronize(m->st));
  if (exec) cudaGraphExecDestroy(exec);
  if (loss_out) *loss_out = l;
  return H2_OK;
}

h2_status h2_rank_model_predict(h2_rank_model* m, const float* feats, int64_t n, float* out) {
  if (!m || !feats || n < 0 || !out) return H2_ERR_INVALID_ARG;
  m->err.clear();
  if (n == 0) return H2_OK;
  h2_status s = stage_inputs(m, feats, n, m->d_mean, m->d_istd);
  if (s != H2_OK) return s;
  ++h2::g_launches;
  rm_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, m->st>>>(m->X, n, m->wb, m->out);
  RM_CK(cudaGetLastError());
  RM_CK(cudaMemcpyAsync(out, m->out, sizeof(float) * n, cudaMemcpyDefault, m->st));
  RM_CK(cudaStreamSynchronize(m->st));
  return H2_OK;
}

const char* h2_rank_model_last_error(const h2_rank_model* m) { return m ? m->err.c_str() : ""; }

void h2_rank_model_destroy(h2_rank_model* m) {
  if (!m) return;
  for (void* p : {(void*)m->master, (void*)m->m1, (void*)m->m2, (void*)m->partial, (void*)m->loss, (void*)m->grad,
                  (void*)m->wb, (void*)m->step, (void*)m->d_mean, (void*)m->d_istd, (void*)m->d_zero,
                  (void*)m->d_one, (void*)m->raw, (void*)m->y, (void*)m->out, (void*)m->X})
    if (p) cudaFree(p);
  delete m;
}

}  // extern "C"
