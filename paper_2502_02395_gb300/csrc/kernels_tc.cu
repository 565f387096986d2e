// Tensor-core batched GEMM for the mixed-precision contractions (sm_103a,
// tcgen05 + TMA), and the FP16/BF16 operand preparation around it.
//
//   C_b (M x N) = alpha * A_b (M x K) * B_b (N x K)^T
//
// A and B are K-major (row-major with K contiguous) FP16 or BF16 matrices
// inside larger 2-D arrays; batch b uses matrix ia[b] of A and ib[b] of B.
// One CTA computes a 128 x N tile (N <= 256) of one batch entry:
//   * warp 0 (one thread) streams 64-wide K slices of A and B into shared
//     memory with TMA (128-byte swizzle), two stages, mbarrier handshakes;
//   * warp 1 allocates the FP32 accumulator in tensor memory (N columns) and
//     one thread issues tcgen05.mma (M = 128, N, K = 16 per instruction);
//     tcgen05.commit releases each stage and finally signals the epilogue;
//   * all four warps read the accumulator back (tcgen05.ld, one TMEM lane per
//     output row) and store it as FP32 row-major, or as FP16/BF16 transposed
//     (C^T, K-major for a following GEMM), scaled by alpha * (*alpha_dev).
// Every wait is bounded (2 s of global time); on expiry the CTA records the
// failure in err[0], drains its own copies in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "h2_internal.h"
#include "kernels.h"
#include "ptx_util.h"

namespace h2 {

std::atomic<int> g_tc_kernel{2};

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;  // one 128-byte swizzle atom of 16-bit elements
constexpr int TC_STAGES = 2;
constexpr unsigned long long TC_TIMEOUT_NS = 2000000000ull;

// Wait for the phase of the given parity; false after TC_TIMEOUT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return h2::mbar_wait(bar, parity, TC_TIMEOUT_NS);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand, 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024
// bytes apart (stride byte offset), descriptor version 1, layout type 2.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;            // leading byte offset (16 B; unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;            // descriptor version
  d |= (uint64_t)2u << 61;            // SWIZZLE_128B
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A/B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int ab_bf16, int M, int N) {
  return (1u << 4) | ((uint32_t)ab_bf16 << 7) | ((uint32_t)ab_bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct TcArgs {
  int M, N, K;
  int rowsA, rowsB;  // rows per matrix inside the A / B tensors
  const int32_t* ia;
  const int32_t* ib;
  void* C;
  int64_t sC;
  const int32_t* ic;
  int ldc;
  int out_mode;  // 0: FP32 row-major; 1: 16-bit transposed (C^T row-major, ld = ldc); 3: FP32 C += result
  int out_bf16;  // 16-bit output type for out_mode 1
  float alpha;
  const float* alpha_dev;
  int32_t* err;
  int ab_bf16;
  uint32_t tmem_cols;
  void* C2;  // optional second output for out_mode 0: 16-bit copy of the raw accumulator (row-major, ldc)
  int c2_bf16;
  // Quadrant split (out_mode 0 with C2): rows and columns >= qsplit form the
  // SS quadrant.  For a batch entry whose pair (qi[b], qj[b]) is off the
  // diagonal, the FP32 output keeps only SS and C2 everything but SS; a
  // diagonal entry gets the full FP32 output.  qsplit < 0: no split.
  int qsplit;
  const int32_t* qi;
  const int32_t* qj;
  // optional: max |FP32 output| over the SS quadrants of the off-diagonal
  // entries, accumulated by atomicMax on the float bits (the merge's scale)
  unsigned int* amax_ss;
};

// Row-major stores of a warp's 32 consecutive rows through shared memory:
// every lane holds 16 values (FP32) or 8 packed pairs (16 bits) of its row
// m0 + lane at columns n0 .. n0 + 15; they are transposed in stg (32 x 17
// words, this warp's) and written as whole row segments, 4 lanes per FP32
// row (8 rows per store) or 2 lanes per 16-bit row (16 rows per store),
// instead of one 16-byte piece of 32 different rows per store.  add: C +=
// (read-modify-write).  Warp-collective.
__device__ __forceinline__ void tc_rows_store_f32(float* stg, const float (&v)[16], float* C, int64_t ldc, bool add) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = v[j];
  __syncwarp();
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int r = it * 8 + (lane >> 2), c4 = (lane & 3) * 4;
    const float* q = stg + r * 17 + c4;
    float4 w = make_float4(q[0], q[1], q[2], q[3]);
    float4* o = reinterpret_cast<float4*>(C + (int64_t)r * ldc + c4);
    if (add) {
      const float4 old = *o;
      w.x += old.x, w.y += old.y, w.z += old.z, w.w += old.w;
    }
    *o = w;
  }
  __syncwarp();
}
__device__ __forceinline__ void tc_rows_store_u16(float* stg, const uint32_t (&h)[8], uint16_t* C, int64_t ldc) {
  const int lane = threadIdx.x & 31;
  uint32_t* su = reinterpret_cast<uint32_t*>(stg);
#pragma unroll
  for (int j = 0; j < 8; ++j) su[lane * 9 + j] = h[j];
  __syncwarp();
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int r = it * 16 + (lane >> 1), c = (lane & 1) * 4;
    const uint32_t* q = su + r * 9 + c;
    *reinterpret_cast<uint4*>(C + (int64_t)r * ldc + 2 * c) = make_uint4(q[0], q[1], q[2], q[3]);
  }
  __syncwarp();
}

// Epilogue of one output row m of batch entry b: reads the row's N
// accumulator columns from TMEM (lane_addr: this warp's lane quarter) in
// 16-column chunks and stores them in the output mode of p.  Every lane of
// the warp must call it (tcgen05.ld is warp-collective); rows m >= M and
// failed tiles (ok false) store nothing.  Returns max |FP32 output| over the
// SS quadrant of an off-diagonal split entry (0 otherwise).  With stg (this
// warp's 32 x 17 words of shared memory), the warp's rows are m - lane ..
// m - lane + 31, and the row-major outputs (modes 0 and 3) go through
// tc_rows_store_*.
__device__ __forceinline__ float tc_epilogue_row(const TcArgs& p, int64_t b, int m, uint32_t lane_addr, bool ok,
                                                 float* stg = nullptr) {
  const float alpha = p.alpha * (p.alpha_dev ? *p.alpha_dev : 1.0f);
  char* Cb = reinterpret_cast<char*>(p.C);
  const int64_t cbase = (int64_t)(p.ic ? p.ic[b] : (int)b) * p.sC;
  const bool split = p.qsplit >= 0 && p.qi[b] != p.qj[b];
  float ss_max = 0.0f;
  for (int n0 = 0; n0 < p.N; n0 += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(lane_addr + (uint32_t)n0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!ok || m >= p.M) continue;
    // the staged stores need warp-uniform quadrant tests: rows of a warp on
    // one side of qsplit (true for a multiple of 32)
    const int lane = threadIdx.x & 31;
    if (stg && (p.out_mode == 0 || p.out_mode == 3) && (p.qsplit < 0 || p.qsplit % 32 == 0)) {
      const int64_t row0 = (int64_t)(m - lane) * p.ldc + n0;
      if (p.out_mode == 3) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) * alpha;
        tc_rows_store_f32(stg, v, reinterpret_cast<float*>(Cb) + cbase + row0, p.ldc, true);
        continue;
      }
      const bool ss = (m >= p.qsplit) && (n0 >= p.qsplit);
      if (!split || ss) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = __uint_as_float(r[j]) * alpha;
          if (split) ss_max = fmaxf(ss_max, fabsf(v[j]));
        }
        tc_rows_store_f32(stg, v, reinterpret_cast<float*>(Cb) + cbase + row0, p.ldc, false);
      }
      if (p.C2 && !(p.qsplit >= 0 && ss)) {
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const float a0 = __uint_as_float(r[j]), a1 = __uint_as_float(r[j + 1]);
          if (p.c2_bf16) {
            __nv_bfloat162 t = __floats2bfloat162_rn(a0, a1);
            h[j / 2] = *reinterpret_cast<uint32_t*>(&t);
          } else {
            __half2 t = __floats2half2_rn(a0, a1);
            h[j / 2] = *reinterpret_cast<uint32_t*>(&t);
          }
        }
        tc_rows_store_u16(stg, h, reinterpret_cast<uint16_t*>(p.C2) + cbase + row0, p.ldc);
      }
      continue;
    }
    if (p.out_mode == 0) {
      const bool ss = (m >= p.qsplit) && (n0 >= p.qsplit);
      if (!split || ss) {
        float* out = reinterpret_cast<float*>(Cb) + cbase + (int64_t)m * p.ldc + n0;
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          float4 v = make_float4(__uint_as_float(r[j]) * alpha, __uint_as_float(r[j + 1]) * alpha,
                                 __uint_as_float(r[j + 2]) * alpha, __uint_as_float(r[j + 3]) * alpha);
          *reinterpret_cast<float4*>(out + j) = v;
          if (split)
            ss_max = fmaxf(ss_max, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      }
      if (p.C2 && !(p.qsplit >= 0 && ss)) {
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const float a0 = __uint_as_float(r[j]), a1 = __uint_as_float(r[j + 1]);
          if (p.c2_bf16) {
            __nv_bfloat162 t = __floats2bfloat162_rn(a0, a1);
            h[j / 2] = *reinterpret_cast<uint32_t*>(&t);
          } else {
            __half2 t = __floats2half2_rn(a0, a1);
            h[j / 2] = *reinterpret_cast<uint32_t*>(&t);
          }
        }
        uint4* o2 = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(p.C2) + cbase + (int64_t)m * p.ldc + n0);
        o2[0] = make_uint4(h[0], h[1], h[2], h[3]);
        o2[1] = make_uint4(h[4], h[5], h[6], h[7]);
      }
    } else if (p.out_mode == 3) {
      float* out = reinterpret_cast<float*>(Cb) + cbase + (int64_t)m * p.ldc + n0;
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        float4 v = *reinterpret_cast<float4*>(out + j);
        v.x = fmaf(__uint_as_float(r[j]), alpha, v.x);
        v.y = fmaf(__uint_as_float(r[j + 1]), alpha, v.y);
        v.z = fmaf(__uint_as_float(r[j + 2]), alpha, v.z);
        v.w = fmaf(__uint_as_float(r[j + 3]), alpha, v.w);
        *reinterpret_cast<float4*>(out + j) = v;
      }
    } else if (p.out_bf16) {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(Cb) + cbase;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        out[(int64_t)(n0 + j) * p.ldc + m] = __float2bfloat16_rn(__uint_as_float(r[j]) * alpha);
    } else {
      __half* out = reinterpret_cast<__half*>(Cb) + cbase;
#pragma unroll
      for (int j = 0; j < 16; ++j) out[(int64_t)(n0 + j) * p.ldc + m] = __float2half_rn(__uint_as_float(r[j]) * alpha);
    }
  }
  return ss_max;
}

__global__ void __launch_bounds__(128) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, TcArgs p,
                                                      int64_t batch) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh;
  __shared__ float stg_sh[4][32 * 17];  // the epilogue's row transposes, one per warp

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned stage buffers
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* base = smem_raw + pad;
  const uint32_t a_bytes = TC_BM * TC_BK * 2;
  const uint32_t b_bytes = (uint32_t)p.N * TC_BK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int kblocks = p.K / TC_BK;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    fail_sh = 0;
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = idesc_f16(p.ab_bf16, TC_BM, p.N);

  uint32_t it_count = 0;  // tiles processed by this CTA (phase bookkeeping)
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y, ++it_count) {
    // (the A / B row coordinates are < 2^31: the caller checks nA * rowsA)
    const int m0 = blockIdx.x * TC_BM;
    const int rowA = (p.ia ? p.ia[b] : (int)b) * p.rowsA + m0;
    const int rowB = (p.ib ? p.ib[b] : (int)b) * p.rowsB;
    // stage s is used kblocks/2 (rounded) times per tile; global use index
    const uint32_t use0 = it_count * (uint32_t)kblocks;
    if (warp == 0 && lane == 0) {
      for (int kb = 0; kb < kblocks; ++kb) {
        const uint32_t u = use0 + kb;
        const int s = u % TC_STAGES;
        if (u >= TC_STAGES) {
          if (!mbar_wait(&empty_bar[s], ((u / TC_STAGES) - 1) & 1)) { fail_sh = 1; break; }
        }
        uint8_t* sa = base + s * stage_bytes;
        mbar_expect_tx(&full_bar[s], stage_bytes);
        tma_load_2d(sa, &tmA, &full_bar[s], kb * TC_BK, rowA);
        tma_load_2d(sa + a_bytes, &tmB, &full_bar[s], kb * TC_BK, rowB);
      }
    } else if (warp == 1 && lane == 0) {
      for (int kb = 0; kb < kblocks; ++kb) {
        const uint32_t u = use0 + kb;
        const int s = u % TC_STAGES;
        if (!mbar_wait(&full_bar[s], (u / TC_STAGES) & 1)) { fail_sh = 1; break; }
        tc_fence_after();
        const uint32_t sa = smem_u32(base + s * stage_bytes);
        const uint64_t da = smem_desc_sw128(sa);
        const uint64_t db = smem_desc_sw128(sa + a_bytes);
#pragma unroll
        for (int k = 0; k < TC_BK / 16; ++k) {
          // advance 16 elements (32 bytes) along K inside the swizzle atom
          const uint64_t off = (uint64_t)((k * 32) >> 4);
          const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty_bar[s]))
                     : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done_bar))
                   : "memory");
    }
    // epilogue: every thread owns output row m0 + tid (TMEM lane tid)
    __syncwarp();
    bool ok = mbar_wait(&done_bar, it_count & 1);
    if (!ok) fail_sh = 1;
    tc_fence_after();
    const int m = m0 + tid;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const bool split = p.qsplit >= 0 && p.qi[b] != p.qj[b];
    float ss_max = tc_epilogue_row(p, b, m, lane_addr, ok, stg_sh[warp]);
    if (p.amax_ss && split) {
      for (int o = 16; o; o >>= 1) ss_max = fmaxf(ss_max, __shfl_xor_sync(0xffffffffu, ss_max, o));
      if (lane == 0 && ss_max > 0.0f) atomicMax(p.amax_ss, __float_as_uint(ss_max));
    }
    tc_fence_before();
    __syncthreads();
    if (fail_sh) break;
  }
  // drain: the producer's last loads must land before the CTA exits
  if (fail_sh && tid == 0) {
    atomicExch(p.err, 1);
    for (int s = 0; s < TC_STAGES; ++s) mbar_wait(&full_bar[s], 0), mbar_wait(&full_bar[s], 1);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// ------------------------------------------------------------------------
// The same GEMM as a persistent, warp-specialized kernel: one CTA per SM
// loops over (M tile, batch entry) tiles.  Warp 0 (one thread) streams the
// K slices with TMA through a WS_STAGES ring; warp 1 allocates two FP32
// accumulators in TMEM (2 x N columns) and one thread issues the MMAs,
// alternating accumulators tile by tile; warps 2-5 run the epilogue of
// tile t (warp w reads TMEM lane quarter w % 4) while the MMAs of tile t + 1
// fill the other accumulator, and release it with 128 arrivals on acc_empty.
// Every wait is bounded as in tc_gemm_kernel; on expiry the role records
// the failure and stops, the MMAs are drained through a final commit, the
// producer's copies in flight are waited for, and TMEM is freed.
// ------------------------------------------------------------------------
constexpr int WS_STAGES = 4;

__global__ void __launch_bounds__(192, 1) tc_gemm_ws_kernel(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB, TcArgs p,
                                                            int64_t batch) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[WS_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[WS_STAGES];
  __shared__ __align__(8) uint64_t accf[2];
  __shared__ __align__(8) uint64_t acce[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh;
  __shared__ uint32_t issued_sh;
  __shared__ float stg_sh[4][32 * 17];  // the epilogue warps' row transposes

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* base = smem_raw + pad;
  const uint32_t a_bytes = TC_BM * TC_BK * 2;
  const uint32_t b_bytes = (uint32_t)p.N * TC_BK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int kblocks = p.K / TC_BK;
  const int mtiles = p.M / TC_BM;
  const int64_t ntiles = batch * mtiles;
  const uint32_t cols = p.tmem_cols;  // one accumulator; two are allocated

  if (tid == 0) {
    for (int s = 0; s < WS_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&accf[k], 1);
      mbar_init(&acce[k], 128);
    }
    mbar_init(&fin_bar, 1);
    fail_sh = 0;
    issued_sh = 0;
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(2 * cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = idesc_f16(p.ab_bf16, TC_BM, p.N);
  volatile int* fail = &fail_sh;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t u = 0;
      for (int64_t t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
        const int64_t b = t / mtiles;
        const int m0 = (int)(t % mtiles) * TC_BM;
        const int rowA = (p.ia ? p.ia[b] : (int)b) * p.rowsA + m0;
        const int rowB = (p.ib ? p.ib[b] : (int)b) * p.rowsB;
        for (int kb = 0; kb < kblocks; ++kb, ++u) {
          const int s = u % WS_STAGES;
          if (u >= WS_STAGES && !mbar_wait(&empty_bar[s], ((u / WS_STAGES) - 1) & 1)) {
            *fail = 1;
            break;
          }
          uint8_t* sa = base + s * stage_bytes;
          mbar_expect_tx(&full_bar[s], stage_bytes);
          tma_load_2d(sa, &tmA, &full_bar[s], kb * TC_BK, rowA);
          tma_load_2d(sa + a_bytes, &tmB, &full_bar[s], kb * TC_BK, rowB);
        }
      }
      issued_sh = u;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t u = 0, lt = 0;
      for (int64_t t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x, ++lt) {
        const uint32_t buf = lt & 1;
        if (lt >= 2 && !mbar_wait(&acce[buf], ((lt / 2) - 1) & 1)) {
          *fail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc_addr = tmem + buf * cols;
        bool ok = true;
        for (int kb = 0; kb < kblocks; ++kb, ++u) {
          const int s = u % WS_STAGES;
          if (!mbar_wait(&full_bar[s], (u / WS_STAGES) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(base + s * stage_bytes);
          const uint64_t da = smem_desc_sw128(sa);
          const uint64_t db = smem_desc_sw128(sa + a_bytes);
#pragma unroll
          for (int k = 0; k < TC_BK / 16; ++k) {
            const uint64_t off = (uint64_t)((k * 32) >> 4);
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
                "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty_bar[s]))
                       : "memory");
        }
        if (!ok) {
          *fail = 1;
          break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&accf[buf]))
                     : "memory");
      }
      // every MMA issued so far completes before fin_bar's first phase
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&fin_bar))
                   : "memory");
      if (!mbar_wait(&fin_bar, 0)) *fail = 1;
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t lt = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const uint32_t buf = lt & 1;
      const bool ok = mbar_wait(&accf[buf], (lt / 2) & 1);
      tc_fence_after();
      const int64_t b = t / mtiles;
      const int m = (int)(t % mtiles) * TC_BM + row;
      float ss_max = tc_epilogue_row(p, b, m, tmem + buf * cols + lane_off, ok, stg_sh[q]);
      if (p.amax_ss && p.qsplit >= 0 && p.qi[b] != p.qj[b]) {
        for (int o = 16; o; o >>= 1) ss_max = fmaxf(ss_max, __shfl_xor_sync(0xffffffffu, ss_max, o));
        if (lane == 0 && ss_max > 0.0f) atomicMax(p.amax_ss, __float_as_uint(ss_max));
      }
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      if (!ok) {
        *fail = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (fail_sh && tid == 0) {
    atomicExch(p.err, 1);
    // wait for the producer's copies in flight: stage s was armed
    // ceil((issued - s) / WS_STAGES) times; its last phase must complete
    const uint32_t issued = issued_sh;
    for (int s = 0; s < WS_STAGES; ++s)
      if (issued > (uint32_t)s) {
        const uint32_t uses = (issued - s + WS_STAGES - 1) / WS_STAGES;
        mbar_wait(&full_bar[s], (uses - 1) & 1);
      }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * cols) : "memory");
  }
}

// ------------------------------------------------------------------------
// host side: tensor maps
// ------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

bool make_map(CUtensorMap* tm, const void* base, int bf16, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool make_tile_map(CUtensorMap* tm, const void* base, int bf16, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows, uint32_t box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  if (box_rows == 0 || box_cols == 0 || box_rows > 256 || box_cols > 256 || (box_cols * 2) % 16 || (ld * 2) % 16 ||
      (reinterpret_cast<uintptr_t>(base) & 15))
    return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool gemm_tc_supported(int M, int N, int K, int lda, int ldb, int ldc) {
  (void)ldc;
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if (M % TC_BM || K % TC_BK || N % 16 || N > 256) return false;
  if (lda % 8 || ldb % 8) return false;  // 16-byte row strides for TMA
  return encode_fn() != nullptr;
}

// A: nA matrices of rowsA x lda (16-bit) starting at A; B likewise.
bool gemm_tc(int ab_bf16, int M, int N, int K, const void* A, int64_t nA, int rowsA, int lda, const int32_t* ia,
             const void* B, int64_t nB, int rowsB, int ldb, const int32_t* ib, void* C, int64_t sC,
             const int32_t* ic, int ldc, int out_mode, int out_bf16, float alpha, const float* alpha_dev,
             int64_t batch, int32_t* err, cudaStream_t st, void* C2, int qsplit, const int32_t* qi,
             const int32_t* qj, unsigned int* amax_ss, int64_t rowsA_total, int form) {
  if (batch == 0) return true;
  if (!gemm_tc_supported(M, N, K, lda, ldb, ldc)) return false;
  const uint64_t ra = rowsA_total > 0 ? (uint64_t)rowsA_total : (uint64_t)nA * rowsA;
  if (ra >= (1ull << 31) || (uint64_t)nB * rowsB >= (1ull << 31)) return false;
  if (out_mode == 3 && (ldc % 4 || (reinterpret_cast<uintptr_t>(C) & 15))) return false;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, ab_bf16, ra, (uint64_t)K, (uint64_t)lda, TC_BM)) return false;
  if (!make_map(&tb, B, ab_bf16, (uint64_t)nB * rowsB, (uint64_t)K, (uint64_t)ldb, (uint32_t)N)) return false;
  TcArgs p{};
  p.M = M;
  p.N = N;
  p.K = K;
  p.rowsA = rowsA;
  p.rowsB = rowsB;
  p.ia = ia;
  p.ib = ib;
  p.C = C;
  p.sC = sC;
  p.ic = ic;
  p.ldc = ldc;
  p.out_mode = out_mode;
  p.out_bf16 = out_bf16;
  p.alpha = alpha;
  p.alpha_dev = alpha_dev;
  p.err = err;
  p.ab_bf16 = ab_bf16;
  p.C2 = (out_mode == 0) ? C2 : nullptr;
  p.c2_bf16 = ab_bf16;
  // the split needs the pair lists, a 16-bit copy and quadrant edges on the
  // epilogue's 16-column chunks
  const bool split = p.C2 && qsplit >= 0 && qsplit % 16 == 0 && qi && qj;
  p.qsplit = split ? qsplit : -1;
  p.qi = split ? qi : nullptr;
  p.qj = split ? qj : nullptr;
  p.amax_ss = split ? amax_ss : nullptr;
  uint32_t cols = 32;
  while (cols < (uint32_t)N) cols <<= 1;
  p.tmem_cols = cols;
  size_t smem = (size_t)TC_STAGES * (TC_BM * TC_BK * 2 + (size_t)N * TC_BK * 2) + 1024;
  // at most 512 / cols CTAs may share an SM's tensor memory: pad shared memory
  // so that no more fit (228 KB per SM)
  const size_t per_sm = 228 * 1024;
  const size_t max_ctas = 512 / cols;
  smem = std::max(smem, per_sm / (max_ctas + 1) + 1024);
  cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int mode = form >= 0 ? form : g_tc_kernel.load();
  if (mode == 2 && 2 * cols <= 512) {
    // persistent warp-specialized kernel: one CTA per SM (TMEM holds two
    // accumulators), WS_STAGES-deep ring
    const size_t sm_ws = (size_t)WS_STAGES * (TC_BM * TC_BK * 2 + (size_t)N * TC_BK * 2) + 1024;
    cudaFuncSetAttribute(tc_gemm_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_ws);
    const int64_t ntiles = batch * (M / TC_BM);
    ++g_launches;
    tc_gemm_ws_kernel<<<(unsigned)std::min<int64_t>(ntiles, nsm), 192, sm_ws, st>>>(ta, tb, p, batch);
    return true;
  }
  // one CTA per batch entry (mode 0), or a persistent grid of two CTAs per
  // SM looping over the entries (mode 1)
  int64_t gy = std::min<int64_t>(batch, 65535);
  if (mode == 1) gy = std::min<int64_t>(gy, std::max<int64_t>(1, (int64_t)nsm * 2 / (M / TC_BM)));
  dim3 grid(M / TC_BM, (unsigned)gy);
  ++g_launches;
  tc_gemm_kernel<<<grid, 128, smem, st>>>(ta, tb, p, batch);
  return true;
}

// ------------------------------------------------------------------------
// self-test of the bounded waits: an mbarrier that expects one arrival which
// never comes.  Thread 0 waits with the same helper the TMA kernels use; when
// the wait gives up it records the failure in *flag (as those kernels record
// theirs in the context's status word) and the CTA returns.  Nothing else
// touches global memory.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(32) wait_selftest_kernel(unsigned long long timeout_ns, int32_t* flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncwarp();
  if (threadIdx.x == 0 && !h2::mbar_wait(&bar, 0, timeout_ns)) atomicExch(flag, 1);
  __syncwarp();
}

void launch_wait_selftest(unsigned long long timeout_ns, int32_t* flag, cudaStream_t st) {
  ++g_launches;
  wait_selftest_kernel<<<1, 32, 0, st>>>(timeout_ns, flag);
}

// ------------------------------------------------------------------------
// operand preparation
// ------------------------------------------------------------------------
// amax[0] = max |x| over nblk strided sub-blocks: block q holds rows x cols
// entries at base + q*stride + r*ld + c.  One CTA per block; warps over
// rows, lanes over columns.
template <typename S>
__global__ void __launch_bounds__(256) amax_blocks_kernel(const S* __restrict__ base, int64_t nblk, int64_t stride,
                                                          int rows, int cols, int ld, const int32_t* __restrict__ idx,
                                                          unsigned int* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float m = 0.0f;
  for (int64_t q = blockIdx.x; q < nblk; q += gridDim.x) {
    const S* B = base + (idx ? (int64_t)idx[q] : q) * stride;
    for (int r = warp; r < rows; r += 8)
      for (int c = lane; c < cols; c += 32) m = fmaxf(m, fabsf((float)__ldg(B + (int64_t)r * ld + c)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}
template <typename S>
void launch_amax_blocks(const S* base, int64_t nblk, int64_t stride, int rows, int cols, int ld, unsigned int* out,
                        cudaStream_t st, const int32_t* idx) {
  if (nblk == 0 || rows == 0 || cols == 0) return;
  const int blocks = (int)std::min<int64_t>(nblk, 152 * 16);
  ++g_launches;
  amax_blocks_kernel<S><<<blocks, 256, 0, st>>>(base, nblk, stride, rows, cols, ld, idx, out);
}
template void launch_amax_blocks<float>(const float*, int64_t, int64_t, int, int, int, unsigned int*, cudaStream_t,
                                        const int32_t*);
template void launch_amax_blocks<double>(const double*, int64_t, int64_t, int, int, int, unsigned int*, cudaStream_t,
                                         const int32_t*);

// scale[0] = 2^e with amax * 2^e <= target (largest such power of two),
// scale[1] = 2^-e.  amax = 0 gives scale 1.  amax is the larger of the two
// accumulators (the second optional).
__global__ void pow2_scale_kernel(const unsigned int* __restrict__ amax_bits, const unsigned int* __restrict__ amax2,
                                  float target, float* __restrict__ scale) {
  float a = __uint_as_float(amax_bits[0]);
  if (amax2) a = fmaxf(a, __uint_as_float(amax2[0]));
  float s = 1.0f;
  if (a > 0.0f && isfinite(a)) {
    int e = (int)floorf(log2f(target / a));
    e = max(-100, min(100, e));
    s = ldexpf(1.0f, e);
    while (a * s > target) s *= 0.5f;
  }
  scale[0] = s;
  scale[1] = 1.0f / s;
}
void launch_pow2_scale(const unsigned int* amax_bits, float target, float* scale, cudaStream_t st,
                       const unsigned int* amax2) {
  ++g_launches;
  pow2_scale_kernel<<<1, 1, 0, st>>>(amax_bits, amax2, target, scale);
}

// out[0] = 1 / (a[0] * b[0] * b[0])  (the inverse scale of a product A B B^T)
__global__ void inv_scale_product_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                         float* __restrict__ out) {
  out[0] = 1.0f / (a[0] * b[0] * b[0]);
}
void launch_inv_scale_product(const float* a, const float* b, float* out, cudaStream_t st) {
  ++g_launches;
  inv_scale_product_kernel<<<1, 1, 0, st>>>(a, b, out);
}

// out[0] = 1 / (a[0] * b[0])  (the inverse scale of a product of two scaled operands)
__global__ void inv_scale_pair_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                      float* __restrict__ out) {
  out[0] = 1.0f / (a[0] * b[0]);
}
void launch_inv_scale_pair(const float* a, const float* b, float* out, cudaStream_t st) {
  ++g_launches;
  inv_scale_pair_kernel<<<1, 1, 0, st>>>(a, b, out);
}

// out16[e] = (16-bit) (in[e] * scale[0])
template <typename S>
__global__ void to_lowp_kernel(const S* __restrict__ in, void* __restrict__ out, int64_t n, const float* __restrict__ scale,
                               int bf16) {
  const float s = scale ? scale[0] : 1.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float v = (float)in[e] * s;
    if (bf16) reinterpret_cast<__nv_bfloat16*>(out)[e] = __float2bfloat16_rn(v);
    else reinterpret_cast<__half*>(out)[e] = __float2half_rn(v);
  }
}
template <typename S>
void launch_to_lowp(int bf16, const S* in, void* out, int64_t n, const float* scale, cudaStream_t st) {
  if (n == 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  ++g_launches;
  to_lowp_kernel<S><<<blocks, 256, 0, st>>>(in, out, n, scale, bf16);
}
template void launch_to_lowp<float>(int, const float*, void*, int64_t, const float*, cudaStream_t);
template void launch_to_lowp<double>(int, const double*, void*, int64_t, const float*, cudaStream_t);

// 16-bit merge (the merge of Algorithm 2 in the scaled low-precision layout):
// child SS blocks (FP32 Ahat, rows/cols R..D) and couplings (FP32 Shat) go
// to the parent's 16-bit near blocks, multiplied by scale[0].  One CTA per
// child pair; warps over rows, lanes over columns.  mirror (non-NULL when
// only the upper pairs were projected): a lower near pair (i > j) takes its
// mirror's SS transposed.  skip_lower: the parent level projects its upper
// pairs only, so pairs bound for a lower parent pair are skipped.
__global__ void __launch_bounds__(256) merge_lowp_kernel(int D, int K, int64_t NP, const float* __restrict__ Ahat,
                                                         const int32_t* __restrict__ ni, const int32_t* __restrict__ nj,
                                                         const int32_t* __restrict__ ndst, int64_t FP,
                                                         const float* __restrict__ Shat, const int32_t* __restrict__ fi,
                                                         const int32_t* __restrict__ fj, const int32_t* __restrict__ fdst,
                                                         void* __restrict__ Apar, const float* __restrict__ scale,
                                                         int bf16, const int32_t* __restrict__ mirror, int skip_lower) {
  const int R = D - K, Dp = 2 * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float s = scale[0];
  for (int64_t q = blockIdx.x; q < NP + FP; q += gridDim.x) {
    const bool nr = q < NP;
    const int64_t qq = nr ? q : q - NP;
    const int i = nr ? ni[qq] : fi[qq], j = nr ? nj[qq] : fj[qq];
    if (skip_lower && (i >> 1) > (j >> 1)) continue;
    const bool tr = nr && mirror && i > j;
    const int64_t dst = nr ? ndst[qq] : fdst[qq];
    const int64_t sq = tr ? (int64_t)mirror[qq] : qq;
    const float* src = nr ? Ahat + sq * D * D + (int64_t)R * D + R : Shat + qq * K * K;
    const int lds = nr ? D : K;
    const int64_t obase = dst * Dp * Dp + (int64_t)(i & 1) * K * Dp + (j & 1) * K;
    for (int a = warp; a < K; a += 8) {
      const int64_t o = obase + (int64_t)a * Dp;
      for (int b = lane; b < K; b += 32) {
        // entry (a, b): the mirror's (b, a) for a lower pair (L1 holds the
        // block's columns across the CTA's rows)
        const float v = __ldg(tr ? src + (int64_t)b * lds + a : src + (int64_t)a * lds + b) * s;
        if (bf16) reinterpret_cast<__nv_bfloat16*>(Apar)[o + b] = __float2bfloat16_rn(v);
        else reinterpret_cast<__half*>(Apar)[o + b] = __float2half_rn(v);
      }
    }
  }
}

// The same merge with vector accesses, for K a multiple of 32 and 16-byte
// aligned rows (R, D multiples of 4): a child quadrant is read as float4
// pairs and written as 8 packed 16-bit entries per thread; a lower pair's
// quadrant (its mirror's SS transposed) goes through 32 x 32 shared-memory
// tiles so that both its reads and its writes stay coalesced.
__device__ __forceinline__ uint32_t pack2_lowp(float a, float b, int bf16) {
  if (bf16) {
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&t);
  }
  __half2 t = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}

__global__ void __launch_bounds__(256) merge_lowp_vec_kernel(int D, int K, int64_t NP, const float* __restrict__ Ahat,
                                                             const int32_t* __restrict__ ni,
                                                             const int32_t* __restrict__ nj,
                                                             const int32_t* __restrict__ ndst, int64_t FP,
                                                             const float* __restrict__ Shat,
                                                             const int32_t* __restrict__ fi,
                                                             const int32_t* __restrict__ fj,
                                                             const int32_t* __restrict__ fdst, void* __restrict__ Apar,
                                                             const float* __restrict__ scale, int bf16,
                                                             const int32_t* __restrict__ mirror, int skip_lower) {
  __shared__ float t[32][33];
  const int R = D - K, Dp = 2 * K;
  const float s = scale[0];
  uint16_t* out16 = reinterpret_cast<uint16_t*>(Apar);
  for (int64_t q = blockIdx.x; q < NP + FP; q += gridDim.x) {
    const bool nr = q < NP;
    const int64_t qq = nr ? q : q - NP;
    const int i = nr ? ni[qq] : fi[qq], j = nr ? nj[qq] : fj[qq];
    if (skip_lower && (i >> 1) > (j >> 1)) continue;
    const bool tr = nr && mirror && i > j;
    const int64_t dst = nr ? ndst[qq] : fdst[qq];
    const int64_t sq = tr ? (int64_t)mirror[qq] : qq;
    const float* src = nr ? Ahat + sq * D * D + (int64_t)R * D + R : Shat + qq * K * K;
    const int lds = nr ? D : K;
    const int64_t obase = dst * Dp * Dp + (int64_t)(i & 1) * K * Dp + (j & 1) * K;
    if (!tr) {
      const int groups = K / 8;
      for (int e = threadIdx.x; e < K * groups; e += blockDim.x) {
        const int a = e / groups, g = e - a * groups;
        const float4 v0 = __ldg(reinterpret_cast<const float4*>(src + (int64_t)a * lds + g * 8));
        const float4 v1 = __ldg(reinterpret_cast<const float4*>(src + (int64_t)a * lds + g * 8 + 4));
        const uint4 w = make_uint4(pack2_lowp(v0.x * s, v0.y * s, bf16), pack2_lowp(v0.z * s, v0.w * s, bf16),
                                   pack2_lowp(v1.x * s, v1.y * s, bf16), pack2_lowp(v1.z * s, v1.w * s, bf16));
        *reinterpret_cast<uint4*>(out16 + obase + (int64_t)a * Dp + g * 8) = w;
      }
    } else {
      const int nt = K / 32, x = threadIdx.x & 31, y0 = threadIdx.x >> 5;
      for (int tile = 0; tile < nt * nt; ++tile) {
        const int ta = tile / nt, tb = tile - ta * nt;  // output rows ta*32.., columns tb*32..
        __syncthreads();
        for (int y = y0; y < 32; y += 8) t[y][x] = __ldg(src + (int64_t)(tb * 32 + y) * lds + ta * 32 + x);
        __syncthreads();
        for (int y = y0; y < 32; y += 8) {
          const float v = t[x][y] * s;
          const uint16_t h = bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
          out16[obase + (int64_t)(ta * 32 + y) * Dp + tb * 32 + x] = h;
        }
      }
    }
  }
}

// 16-bit blocks of the lower pairs as their mirrors transposed:
// A[dst[k]] = A[src[k]]^T (D x D), outside the trailing R.. x R.. (SS)
// quadrant.  32 x 32 tiles through shared memory; blockIdx.x is the tile,
// blockIdx.y + 65535 blockIdx.z the pair.
__global__ void __launch_bounds__(256) transpose16_blocks_kernel(int D, int R, int64_t n, const int32_t* __restrict__ dst,
                                                                 const int32_t* __restrict__ src,
                                                                 uint16_t* __restrict__ A) {
  __shared__ uint16_t t[32][34];
  const int64_t k = blockIdx.y + (int64_t)blockIdx.z * 65535;
  if (k >= n) return;
  const int nt = (D + 31) / 32;
  const int tr = blockIdx.x / nt, tc = blockIdx.x % nt;  // output tile
  if (tr * 32 >= R && tc * 32 >= R) return;              // inside SS (R a multiple of 32) or past it
  const uint16_t* in = A + (int64_t)src[k] * D * D;
  uint16_t* out = A + (int64_t)dst[k] * D * D;
  const int x = threadIdx.x & 31, y0 = threadIdx.x >> 5;
  for (int y = y0; y < 32; y += 8) {  // input tile (tc, tr): rows tc*32 + y, columns tr*32 + x
    const int r = tc * 32 + y, c = tr * 32 + x;
    t[y][x] = (r < D && c < D) ? in[(int64_t)r * D + c] : 0;
  }
  __syncthreads();
  for (int y = y0; y < 32; y += 8) {
    const int r = tr * 32 + y, c = tc * 32 + x;
    if (r < D && c < D && !(r >= R && c >= R)) out[(int64_t)r * D + c] = t[x][y];
  }
}
// The same with 64 x 64 tiles moved as 32-bit words (two 16-bit entries),
// for D and R multiples of 64: word x of shared row y holds input entries
// (y, 2x), (y, 2x + 1); an output word takes entry y of input rows 2x and
// 2x + 1.
__global__ void __launch_bounds__(256) transpose16_blocks64_kernel(int D, int R, int64_t n,
                                                                   const int32_t* __restrict__ dst,
                                                                   const int32_t* __restrict__ src,
                                                                   uint16_t* __restrict__ A) {
  __shared__ uint32_t t[64][33];
  const int64_t k = blockIdx.y + (int64_t)blockIdx.z * 65535;
  if (k >= n) return;
  const int nt = D / 64;
  const int tr = blockIdx.x / nt, tc = blockIdx.x % nt;  // output tile
  if (tr * 64 >= R && tc * 64 >= R) return;              // the SS quadrant
  const uint32_t* in = reinterpret_cast<const uint32_t*>(A + (int64_t)src[k] * D * D);
  uint32_t* out = reinterpret_cast<uint32_t*>(A + (int64_t)dst[k] * D * D);
  const int x = threadIdx.x & 31, y0 = threadIdx.x >> 5;
  const int Dw = D / 2;  // words per row
  for (int y = y0; y < 64; y += 8) t[y][x] = in[(int64_t)(tc * 64 + y) * Dw + tr * 32 + x];
  __syncthreads();
  for (int y = y0; y < 64; y += 8) {
    const uint32_t a = t[2 * x][y >> 1], b = t[2 * x + 1][y >> 1];
    const uint32_t lo = (y & 1) ? (a >> 16) : (a & 0xffffu), hi = (y & 1) ? (b >> 16) : (b & 0xffffu);
    out[(int64_t)(tr * 64 + y) * Dw + tc * 32 + x] = lo | (hi << 16);
  }
}

void launch_transpose16_blocks(int D, int R, int64_t n, const int32_t* dst, const int32_t* src, void* A,
                               cudaStream_t st) {
  if (n <= 0) return;
  if (D % 64 == 0 && R % 64 == 0) {
    const int nt = D / 64;
    dim3 grid(nt * nt, (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
    ++g_launches;
    transpose16_blocks64_kernel<<<grid, 256, 0, st>>>(D, R, n, dst, src, reinterpret_cast<uint16_t*>(A));
    return;
  }
  const int nt = (D + 31) / 32;
  dim3 grid(nt * nt, (unsigned)std::min<int64_t>(n, 65535), (unsigned)((n + 65534) / 65535));
  ++g_launches;
  transpose16_blocks_kernel<<<grid, 256, 0, st>>>(D, R, n, dst, src, reinterpret_cast<uint16_t*>(A));
}
// rows of Ahat's SS quadrant start on 16 bytes: D and R = D - K multiples of 4
static bool R_aligned(int D, int K) { return D % 4 == 0 && (D - K) % 4 == 0; }

void launch_merge_lowp(int D, int K, int64_t NP, const float* Ahat, const int32_t* ni, const int32_t* nj,
                       const int32_t* ndst, int64_t FP, const float* Shat, const int32_t* fi, const int32_t* fj,
                       const int32_t* fdst, void* Apar, const float* scale, int bf16, cudaStream_t st,
                       const int32_t* mirror, int skip_lower) {
  const int64_t n = NP + FP;
  if (n == 0 || K == 0) return;
  const int blocks = (int)std::min<int64_t>(n, 152 * 16);
  ++g_launches;
  if (K % 32 == 0 && R_aligned(D, K) && (reinterpret_cast<uintptr_t>(Apar) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(Ahat) & 15) == 0 && (reinterpret_cast<uintptr_t>(Shat) & 15) == 0) {
    merge_lowp_vec_kernel<<<blocks, 256, 0, st>>>(D, K, NP, Ahat, ni, nj, ndst, FP, Shat, fi, fj, fdst, Apar, scale,
                                                  bf16, mirror, skip_lower);
    return;
  }
  merge_lowp_kernel<<<blocks, 256, 0, st>>>(D, K, NP, Ahat, ni, nj, ndst, FP, Shat, fi, fj, fdst, Apar, scale, bf16,
                                            mirror, skip_lower);
}

}  // namespace h2
