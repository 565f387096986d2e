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
#include <atomic>

#include "h2_internal.h"
#include "kernels.h"
#include "ptx_util.h"

namespace h2 {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Transposed warp sum: every lane holds N values (N a power of two no larger
// than G, the width of an aligned lane group, a power of two <= 32).  At
// xor-distance G/2, G/4, ... each lane keeps half of its remaining values
// and adds its partner's copies of them, then plain steps finish: lane l
// ends with the group sum of value tsum_index<N, G>(l), after N - 1 + the
// remaining plain shuffles (instead of N log2 G for N separate sums).
template <int N, int G, typename T>
__device__ __forceinline__ T tsum(const T (&v)[N]) {
  if constexpr (N == 1) {
    T x = v[0];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  } else {
    const bool up = threadIdx.x & (G / 2);
    T w[N / 2];
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const T mine = up ? v[q + N / 2] : v[q], other = up ? v[q] : v[q + N / 2];
      w[q] = mine + __shfl_xor_sync(0xffffffffu, other, G / 2);
    }
    return tsum<N / 2, G / 2, T>(w);
  }
}
template <int N, int G>
__device__ __forceinline__ int tsum_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int n = N, g = G; n > 1; n >>= 1, g >>= 1)
    if (lane & (g / 2)) idx += n / 2;
  return idx;
}
// lanes holding a distinct tsum result: the first lane of each group of
// G / N lanes with equal index
template <int N, int G>
__device__ __forceinline__ bool tsum_leader(int lane) {
  return (lane & (G / N - 1)) == 0;
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
// Vector loads of the stored matrix entries, converted to the compute type:
// 16 bytes of FP32 / FP64, 8 bytes (4 entries) of FP16 / BF16.
template <typename TS>
struct Ld;
template <>
struct Ld<float> {
  static constexpr int VN = 4;
  template <typename T>
  __device__ static void get(const float* p, T (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
  }
};
template <>
struct Ld<double> {
  static constexpr int VN = 2;
  template <typename T>
  __device__ static void get(const double* p, T (&o)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x, o[1] = v.y;
  }
};
template <>
struct Ld<__half> {
  static constexpr int VN = 4;
  template <typename T>
  __device__ static void get(const __half* p, T (&o)[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
  }
};
template <>
struct Ld<__nv_bfloat16> {
  static constexpr int VN = 4;
  template <typename T>
  __device__ static void get(const __nv_bfloat16* p, T (&o)[4]) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
    o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
  }
};
// exact conversion of one stored entry to the compute type
template <typename T, typename TS>
struct Cvt {
  __device__ static T go(TS v) { return (T)v; }
};
template <typename T>
struct Cvt<T, __half> {
  __device__ static T go(__half v) { return (T)__half2float(v); }
};
template <typename T>
struct Cvt<T, __nv_bfloat16> {
  __device__ static T go(__nv_bfloat16 v) { return (T)__bfloat162float(v); }
};

// acc[t] += sum_{c0 <= c < c1} M[r_t * ld + c] xs[c], one column per lane
template <typename TS, typename T, int RPW>
__device__ __forceinline__ void rows_acc_scalar(int rbase, int c0, int c1, const TS* __restrict__ M, int64_t ld,
                                                int nr, const T* __restrict__ xs, T (&acc)[RPW]) {
  const int lane = threadIdx.x & 31;
  for (int c = c0 + lane; c < c1; c += 32) {
    T v[RPW];
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int r = rbase + 8 * t;
      v[t] = (r < nr) ? Cvt<T, TS>::go(M[r * ld + c]) : T(0);
    }
    const T x = xs[c];
#pragma unroll
    for (int t = 0; t < RPW; ++t) acc[t] = fma(v[t], x, acc[t]);
  }
}

// acc[t] += sum_c M[r_t * ld + c] xs[c] for the rows r_t = r0 + warp + 8 t < nr
// (M stored as TS, accumulation in T).  Columns are read with vector loads
// (a few leading and trailing columns one by one where M's alignment or nc
// asks for it).  For each column chunk every lane first issues the loads of
// all its rows, then does the multiply-adds, so RPW independent vector loads
// per lane are in flight at once.
template <typename TS, typename T, int RPW>
__device__ __forceinline__ void rows_acc2(int r0, const TS* __restrict__ M, int64_t ld, int nr, int nc,
                                          const T* __restrict__ xs, T (&acc)[RPW]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int VN = Ld<TS>::VN;
  const int rbase = r0 + warp;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(M);
  if ((ld % VN) != 0 || (addr % sizeof(TS)) != 0) {
    rows_acc_scalar<TS, T, RPW>(rbase, 0, nc, M, ld, nr, xs, acc);
    return;
  }
  const int mis = (int)((addr / sizeof(TS)) % VN);
  const int head = min(nc, (VN - mis) % VN);
  const int cv1 = head + (nc - head) / VN * VN;
  if (head > 0) rows_acc_scalar<TS, T, RPW>(rbase, 0, head, M, ld, nr, xs, acc);
  for (int c = head + lane * VN; c < cv1; c += 32 * VN) {
    T v[RPW][VN];
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int r = rbase + 8 * t;
      if (r < nr) {
        Ld<TS>::get(M + r * ld + c, v[t]);
      } else {
#pragma unroll
        for (int e = 0; e < VN; ++e) v[t][e] = T(0);
      }
    }
    T x[VN];
#pragma unroll
    for (int e = 0; e < VN; ++e) x[e] = xs[c + e];
#pragma unroll
    for (int t = 0; t < RPW; ++t)
#pragma unroll
      for (int e = 0; e < VN; ++e) acc[t] = fma(v[t][e], x[e], acc[t]);
  }
  if (cv1 < nc) rows_acc_scalar<TS, T, RPW>(rbase, cv1, nc, M, ld, nr, xs, acc);
}

template <typename T, int RPW>
__device__ __forceinline__ void rows_acc(int r0, const T* __restrict__ M, int64_t ld, int nr, int nc,
                                         const T* __restrict__ xs, T (&acc)[RPW]) {
  rows_acc2<T, T, RPW>(r0, M, ld, nr, nc, xs, acc);
}

// out[r] = base[r] + sign * sum over lanes of acc (rows owned by this warp)
template <typename T, int RPW>
__device__ __forceinline__ void rows_finish(int r0, int nr, const T (&acc)[RPW], T sign, const T* base, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (RPW == 16 || RPW == 8) {
    const T v = tsum<RPW, 32, T>(acc);
    const int t = tsum_index<RPW, 32>(lane), r = r0 + warp + 8 * t;
    if (tsum_leader<RPW, 32>(lane) && r < nr) out[r] = (base ? base[r] : T(0)) + sign * v;
  } else {
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int r = r0 + warp + 8 * t;
      T v = warp_sum(acc[t]);
      if (lane == 0 && r < nr) out[r] = (base ? base[r] : T(0)) + sign * v;
    }
  }
}

template <typename T, int RPW>
__device__ __forceinline__ void zero(T (&acc)[RPW]) {
#pragma unroll
  for (int t = 0; t < RPW; ++t) acc[t] = T(0);
}

constexpr int kRPW = 16;  // rows per warp per pass: 128-row chunks with 8 warps
constexpr int kChunk = 8 * kRPW;

// ------------------------------------------------------------------------
// CTA-wide GEMV on 16-byte chunks.
// ------------------------------------------------------------------------
// One 16-byte chunk of stored entries (VN of them) converted to T.
template <typename TS>
struct Chunk;
template <>
struct Chunk<float> {
  static constexpr int VN = 4;
  template <typename T>
  __device__ static void cvt(const uint4& u, T (&o)[4]) {
    o[0] = __uint_as_float(u.x), o[1] = __uint_as_float(u.y), o[2] = __uint_as_float(u.z), o[3] = __uint_as_float(u.w);
  }
};
template <>
struct Chunk<double> {
  static constexpr int VN = 2;
  template <typename T>
  __device__ static void cvt(const uint4& u, T (&o)[2]) {
    o[0] = __hiloint2double((int)u.y, (int)u.x), o[1] = __hiloint2double((int)u.w, (int)u.z);
  }
};
template <>
struct Chunk<__half> {
  static constexpr int VN = 8;
  template <typename T>
  __device__ static void cvt(const uint4& u, T (&o)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      o[2 * k] = f.x, o[2 * k + 1] = f.y;
    }
  }
};
template <>
struct Chunk<__nv_bfloat16> {
  static constexpr int VN = 8;
  template <typename T>
  __device__ static void cvt(const uint4& u, T (&o)[8]) {
    // a BF16 value is the upper half of the FP32 with the same bits
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};

// 16-byte loads each lane keeps in flight: 128 rows of 256 bytes per pass
// of a 256-thread CTA (a 128 x 128 block in 16 bits or a 128 x 64 one in
// 32 bits) ...
template <typename TS>
struct Unr {
  static constexpr int v = 8;
};
// ... and 128 rows of 512 bytes for 4- and 8-byte entries
template <>
struct Unr<float> {
  static constexpr int v = 16;
};
template <>
struct Unr<double> {
  static constexpr int v = 16;
};

struct NoHook {
  __device__ void operator()() const {}
};

// y[r] = (base ? base[r] : 0) + alpha * sum_{c < nc} M[r * ld + c] xs[c] for
// r < nr, by all threads of the CTA (M stored as TS, arithmetic in T; xs in
// shared memory; nc <= ld).  A row's 16-byte chunks are spread over cpr lanes
// (the smallest power of two covering them, at most 32), so one warp load
// covers 32 / cpr rows; each lane issues UNR such loads before it uses them.
// A chunk that runs past column nc (but, as nc <= ld and ld is a multiple of
// the chunk, not past the row) is loaded whole and its extra entries are
// zeroed.  hook() runs once, in every thread, after the first loads have been
// issued and before xs is read: it is where the caller fills xs (and
// synchronizes), so that filling xs overlaps the first round trip to memory.
// Rows of a misaligned M are read entry by entry.  y is written by one lane
// per row, with no barrier afterwards.  base and y may be global or shared
// (generic loads and stores).
template <typename TS, typename T, int UNR, typename Hook = NoHook>
__device__ __forceinline__ void cta_gemv(const TS* __restrict__ M, int64_t ld, int nr, int nc,
                                         const T* xs, T alpha, const T* base, T* y, Hook hook = Hook()) {
  constexpr int VN = Chunk<TS>::VN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool vec = ((reinterpret_cast<uintptr_t>(M) & 15) == 0) && ((ld * (int64_t)sizeof(TS)) % 16 == 0);
  if (!vec || nr <= 0 || nc <= 0) {
    hook();
    for (int r = warp; r < nr; r += nw) {
      T s = T(0);
      for (int c = lane; c < nc; c += 32) s = fma(Cvt<T, TS>::go(M[r * ld + c]), xs[c], s);
      s = warp_sum(s);
      if (lane == 0) y[r] = (base ? base[r] : T(0)) + alpha * s;
    }
    return;
  }
  const int nch = (nc + VN - 1) / VN;
  int cpr = 32;
  while (cpr > 1 && cpr / 2 >= nch) cpr >>= 1;
  const int rpi = 32 / cpr, sub = lane / cpr, cl = lane & (cpr - 1);
  const int rows_pass = nw * UNR * rpi;
  const int nit = (nch + cpr - 1) / cpr;  // chunk rounds per pass (the same in every lane)
  bool first = true;
  for (int rb = 0; rb < nr; rb += rows_pass) {
    T acc[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u] = T(0);
    for (int it = 0; it < nit; ++it) {
      const int ch = cl + it * cpr;
      const int c = ch * VN;
      uint4 raw[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int r = rb + (u * nw + warp) * rpi + sub;
        raw[u] = (ch < nch && r < nr) ? __ldg(reinterpret_cast<const uint4*>(M + r * ld + c)) : make_uint4(0, 0, 0, 0);
      }
      if (first) {
        hook();
        first = false;
      }
      if (ch < nch) {
        const int lim = nc - c;  // valid entries of this chunk
        T xv[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) xv[e] = (e < lim) ? xs[c + e] : T(0);
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          T v[VN];
          Chunk<TS>::cvt(raw[u], v);
          if (lim < VN) {
#pragma unroll
            for (int e = 0; e < VN; ++e) v[e] = (e < lim) ? v[e] : T(0);
          }
#pragma unroll
          for (int e = 0; e < VN; ++e) acc[u] = fma(v[e], xv[e], acc[u]);
        }
      }
    }
    if (cpr == 32) {
      const T v = tsum<UNR, 32, T>(acc);
      const int r = rb + tsum_index<UNR, 32>(lane) * nw + warp;
      if (tsum_leader<UNR, 32>(lane) && r < nr) y[r] = (base ? base[r] : T(0)) + alpha * v;
    } else if (cpr == 16 && UNR <= 16) {
      const T v = tsum<UNR, 16, T>(acc);
      const int r = rb + (tsum_index<UNR, 16>(lane) * nw + warp) * 2 + sub;
      if (tsum_leader<UNR, 16>(lane) && r < nr) y[r] = (base ? base[r] : T(0)) + alpha * v;
    } else {
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        for (int o = cpr >> 1; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        const int r = rb + (u * nw + warp) * rpi + sub;
        if (cl == 0 && r < nr) y[r] = (base ? base[r] : T(0)) + alpha * acc[u];
      }
    }
  }
}

// y[m] = sum_{n < nn} M[n * ld + m] z[n] for m < nm (M column-major: the
// columns are contiguous).  Warps take columns n, lanes take 16-byte chunks
// of m; the per-warp partial vectors (part: nwarps * nm entries of shared
// memory) are added at the end.  Ends with the result in y and a barrier.
template <typename TS, typename T>
__device__ __forceinline__ void cta_gemv_cols(const TS* __restrict__ M, int64_t ld, int nm, int nn,
                                              const T* __restrict__ z, T* part, T* y) {
  constexpr int VN = Chunk<TS>::VN;
  constexpr int NU = 8;  // columns in flight per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool vec = ((reinterpret_cast<uintptr_t>(M) & 15) == 0) && ((ld * (int64_t)sizeof(TS)) % 16 == 0);
  for (int m0 = lane * VN; m0 < nm; m0 += 32 * VN) {
    T acc[VN];
#pragma unroll
    for (int e = 0; e < VN; ++e) acc[e] = T(0);
    if (vec && m0 + VN <= nm) {
      int n = warp;
      for (; n + (NU - 1) * nw < nn; n += NU * nw) {
        uint4 raw[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) raw[u] = __ldg(reinterpret_cast<const uint4*>(M + (int64_t)(n + u * nw) * ld + m0));
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          T v[VN];
          Chunk<TS>::cvt(raw[u], v);
          const T zn = z[n + u * nw];
#pragma unroll
          for (int e = 0; e < VN; ++e) acc[e] = fma(v[e], zn, acc[e]);
        }
      }
      for (; n < nn; n += nw) {
        T v[VN];
        Chunk<TS>::cvt(__ldg(reinterpret_cast<const uint4*>(M + (int64_t)n * ld + m0)), v);
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[e] = fma(v[e], z[n], acc[e]);
      }
    } else {
      for (int n = warp; n < nn; n += nw) {
#pragma unroll
        for (int e = 0; e < VN; ++e)
          if (m0 + e < nm) acc[e] = fma(Cvt<T, TS>::go(M[(int64_t)n * ld + m0 + e]), z[n], acc[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < VN; ++e)
      if (m0 + e < nm) part[warp * nm + m0 + e] = acc[e];
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += part[w * nm + m];
    y[m] = s;
  }
  __syncthreads();
}

// sum over the pairs q in [q0, q1) of part[q][r], in pair order; eight
// independent loads are issued before they are added
template <typename T>
__device__ __forceinline__ T sum_pairs(const T* part, int nr, int64_t q0, int64_t q1, int r) {
  T s = T(0);
  int64_t q = q0;
  for (; q + 8 <= q1; q += 8) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = part[(q + k) * nr + r];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; q < q1; ++q) s += part[q * nr + r];
  return s;
}

// Programmatic dependent launch: the substitution kernels are launched so
// that they may start while their predecessor in the stream drains.  Each
// issues its loads of factorization data (fixed during a solve) first, then
// waits here until the predecessor has finished and its writes are visible,
// and only then reads vectors or writes anything.  (Launched without the
// attribute, the wait returns at once.)
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next kernel in the stream begin launching once every CTA of this
// one has started
__device__ __forceinline__ void griddep_launch_next() { asm volatile("griddepcontrol.launch_dependents;" :::); }
// asks L2 for the 128-byte lines of [p, p + bytes) (the CTA's threads share
// the lines): a kernel whose second matrix is read only after a dependent
// step has it on chip by then
__device__ __forceinline__ void prefetch_l2(const void* p, int64_t bytes) {
  const char* b = static_cast<const char*>(p);
  for (int64_t o = (int64_t)threadIdx.x * 128; o < bytes; o += (int64_t)blockDim.x * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(b + o));
}

// The pair kernel runs one CTA per near pair p = (i, j) of a level (or of a
// sub-list of them) and writes one block-vector product into part[p]:
//   PH_RR: Ahat_ij^RR x_j (x_j = xv[j R ..], R entries)        fwd2 / bwd2
//   PH_SR: Ahat_ij^SR x_j (x_j = xv[j R ..], R entries)        fwd3
//   PH_RS: Ahat_ij^RS x_j^S (x_j^S: box j's slot of the parent
//          vector xv, K entries)                                bwd1
// Ahat is stored as TS: T itself, or 16 bits holding s * Ahat (the per-box
// kernels apply 1 / s to the sums).  The block's loads are issued before the
// pair's indices and x_j are read.
enum { PH_RR = 0, PH_SR = 1, PH_RS = 2 };

// One pair's product (entry t of list, or pair t); dep: launched as a
// programmatic dependent (wait for the predecessor before reading x).
template <typename T, typename TS, int PH>
__device__ __forceinline__ void pair_body(int64_t t, int D, int R, int K, const int32_t* __restrict__ list,
                                          const int32_t* __restrict__ nj, const TS* __restrict__ Ahat,
                                          const T* xv, T* part, bool dep) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sx = reinterpret_cast<T*>(sm_raw);  // nc
  const int64_t p = list ? list[t] : t;
  const int nr = (PH == PH_SR) ? K : R;
  const int nc = (PH == PH_RS) ? K : R;
  const TS* M = Ahat + p * D * D + (PH == PH_SR ? (int64_t)R * D : (PH == PH_RS ? R : 0));
  cta_gemv<TS, T, Unr<TS>::v>(M, D, nr, nc, sx, T(1), nullptr, part + p * nr, [&] {
    const int j = nj[p];
    if (dep) {
      griddep_wait();
      griddep_launch_next();
    }
    const T* x = (PH == PH_RS) ? xv + (int64_t)(j >> 1) * 2 * K + (j & 1) * K : xv + (int64_t)j * R;
    for (int e = threadIdx.x; e < nc; e += blockDim.x) sx[e] = x[e];
    __syncthreads();
  });
}
template <typename T, typename TS, int PH>
__global__ void __launch_bounds__(256, sizeof(TS) == 2 ? 3 : 2) pair_kernel(int D, int R, int K, const int32_t* __restrict__ list,
                                                   const int32_t* __restrict__ nj, const TS* __restrict__ Ahat,
                                                   const T* __restrict__ xv, T* __restrict__ part) {
  pair_body<T, TS, PH>(blockIdx.x, D, R, K, list, nj, Ahat, xv, part, true);
}

// Persistent form of the pair kernel for blocks that one pass of the CTA
// covers (rows <= 8 * UNR * 32 / cpr, a row's chunks <= 32): each CTA walks
// the pairs t = blockIdx.x, + gridDim.x, ... and issues the block loads of
// its next pair before it reduces and stores the current one, so that every
// CTA keeps a block's worth of loads in flight.  x_j is staged in a
// double-buffered shared vector.
template <typename T, typename TS, int PH>
__global__ void __launch_bounds__(256, sizeof(TS) == 2 ? 3 : 2)
    pair_persist_kernel(int D, int R, int K, int64_t n, const int32_t* __restrict__ list,
                        const int32_t* __restrict__ nj, const TS* __restrict__ Ahat, const T* __restrict__ xv,
                        T* __restrict__ part) {
  constexpr int VN = Chunk<TS>::VN;
  constexpr int UNR = Unr<TS>::v;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nr = (PH == PH_SR) ? K : R;
  const int nc = (PH == PH_RS) ? K : R;
  const int ncp = (nc + 3) & ~3;
  T* sxb[2] = {reinterpret_cast<T*>(sm_raw), reinterpret_cast<T*>(sm_raw) + ncp};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nch = (nc + VN - 1) / VN;
  int cpr = 32;
  while (cpr > 1 && cpr / 2 >= nch) cpr >>= 1;
  const int rpi = 32 / cpr, sub = lane / cpr, cl = lane & (cpr - 1);
  const int c = cl * VN;
  const bool chunk_ok = cl < nch;
  const int lim = nc - c;
  const int64_t off = (PH == PH_SR ? (int64_t)R * D : (PH == PH_RS ? R : 0));
  int64_t t = blockIdx.x;
  if (t >= n) return;
  int64_t p = list ? list[t] : t;
  uint4 raw[UNR];
  auto issue = [&](int64_t pp) {
    const TS* M = Ahat + pp * D * D + off;
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int r = (u * nw + warp) * rpi + sub;
      raw[u] = (chunk_ok && r < nr) ? __ldg(reinterpret_cast<const uint4*>(M + (int64_t)r * D + c))
                                    : make_uint4(0, 0, 0, 0);
    }
  };
  issue(p);
  griddep_wait();
  griddep_launch_next();
  int buf = 0;
  while (true) {
    const int j = nj[p];
    T* sx = sxb[buf];
    const T* x = (PH == PH_RS) ? xv + (int64_t)(j >> 1) * 2 * K + (j & 1) * K : xv + (int64_t)j * R;
    for (int e = threadIdx.x; e < nc; e += blockDim.x) sx[e] = x[e];
    __syncthreads();
    T acc[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u] = T(0);
    if (chunk_ok) {
      T xvv[VN];
#pragma unroll
      for (int e = 0; e < VN; ++e) xvv[e] = (e < lim) ? sx[c + e] : T(0);
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        T v[VN];
        Chunk<TS>::cvt(raw[u], v);
        if (lim < VN) {
#pragma unroll
          for (int e = 0; e < VN; ++e) v[e] = (e < lim) ? v[e] : T(0);
        }
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[u] = fma(v[e], xvv[e], acc[u]);
      }
    }
    // the next pair's loads go out before this pair's reduction and stores
    const int64_t tn = t + gridDim.x;
    int64_t pn = -1;
    if (tn < n) {
      pn = list ? list[tn] : tn;
      issue(pn);
    }
    T* out = part + p * nr;
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      for (int o = cpr >> 1; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      const int r = (u * nw + warp) * rpi + sub;
      if (cl == 0 && r < nr) out[r] = acc[u];
    }
    if (tn >= n) break;
    t = tn, p = pn, buf ^= 1;
  }
}

// TMA-fed form for 16-bit blocks: a persistent CTA keeps kPairStages tiles
// (the quadrant of s * Ahat_ij, nr x nc, dense row-major) in flight in a
// shared-memory ring; thread 0 issues one 2-D tensor copy per tile.  A tile
// is consumed as in the register form (cpr lanes per row, 16-byte chunks)
// with this lane's x_j chunk in registers, then its stage is refilled with
// the tile kPairStages pairs ahead.  Waits are bounded (2 s); on expiry
// every thread leaves together, thread 0 having waited (bounded) for the
// copies still in flight and set *err.
constexpr int kPairStages = 2;
constexpr unsigned long long kPairTimeoutNs = 2000000000ull;

template <typename TS, int PH>
__global__ void __launch_bounds__(256, 3)
    pair_tma_kernel(const __grid_constant__ CUtensorMap tm, int D, int R, int K, int64_t n,
                    const int32_t* __restrict__ list, const int32_t* __restrict__ nj, const float* __restrict__ xv,
                    float* __restrict__ part, int32_t* __restrict__ err) {
  constexpr int VN = 8;
  constexpr int UNR = 8;  // rows per lane: nr <= 8 warps * UNR * (32 / cpr)
  extern __shared__ __align__(128) unsigned char sm_dyn[];
  __shared__ __align__(8) uint64_t full[kPairStages];
  const int nr = (PH == PH_SR) ? K : R;
  const int nc = (PH == PH_RS) ? K : R;
  const uint32_t tile_bytes = (uint32_t)nr * nc * 2;
  const uint32_t stage_stride = (tile_bytes + 127u) & ~127u;
  // tensor copies need 128-byte aligned destinations: the ring starts at the
  // first such address (the launch adds 128 bytes of room)
  unsigned char* sm_raw = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
  if (smem_u32(sm_raw) & 127u) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int row_off = (PH == PH_SR) ? R : 0, col_off = (PH == PH_RS) ? R : 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nch = nc / VN;
  int cpr = 32;
  while (cpr > 1 && cpr / 2 >= nch) cpr >>= 1;
  const int rpi = 32 / cpr, sub = lane / cpr, cl = lane & (cpr - 1);
  const int64_t G = gridDim.x;
  if (tid == 0) {
    for (int s = 0; s < kPairStages; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int s, int64_t t) {
    const int64_t p = list ? list[t] : t;
    mbar_expect_tx(&full[s], tile_bytes);
    tma_load_2d(sm_raw + s * stage_stride, &tm, &full[s], col_off, (int)(p * D + row_off));
  };
  if (tid == 0)
    for (int s = 0; s < kPairStages; ++s)
      if (blockIdx.x + s * G < n) issue(s, blockIdx.x + s * G);
  // x_j of a pair: this lane's 8-entry chunk, in registers
  auto load_x = [&](int j, float (&xr)[VN]) {
    const float* x = (PH == PH_RS) ? xv + (int64_t)(j >> 1) * 2 * K + (j & 1) * K : xv + (int64_t)j * R;
    if (cl < nch) {
      const float4 a = *reinterpret_cast<const float4*>(x + cl * VN);
      const float4 b = *reinterpret_cast<const float4*>(x + cl * VN + 4);
      xr[0] = a.x, xr[1] = a.y, xr[2] = a.z, xr[3] = a.w, xr[4] = b.x, xr[5] = b.y, xr[6] = b.z, xr[7] = b.w;
    } else {
#pragma unroll
      for (int e = 0; e < VN; ++e) xr[e] = 0.0f;
    }
  };
  // a pair's x_j is loaded one pair ahead of its use and the pair indices
  // two pairs ahead, so that no dependent load sits between two tiles
  int64_t t = blockIdx.x;
  int64_t p = list ? list[t] : t;
  int j = nj[p];
  int64_t p1 = -1;
  int j1 = 0;
  if (t + G < n) p1 = list ? list[t + G] : t + G, j1 = nj[p1];
  griddep_wait();
  griddep_launch_next();
  float xr[VN];
  load_x(j, xr);
  for (int it = 0; t < n; t += G, ++it) {
    const int s = it % kPairStages;
    int64_t p2 = -1;
    int j2 = 0;
    if (t + 2 * G < n) p2 = list ? list[t + 2 * G] : t + 2 * G, j2 = nj[p2];
    // thread 0 waits (bounded) while the others sit at the barrier; then
    // every thread observes the completed phase itself (one poll) before
    // it reads the tile
    const uint32_t par = (uint32_t)(it / kPairStages) & 1u;
    bool ok = true;
    if (tid == 0) ok = mbar_wait(&full[s], par, kPairTimeoutNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, 1);
        // copies issued for this and the next stages may still be in flight
        for (int k = 0; k < kPairStages; ++k) {
          const int64_t tk = t + k * G;
          if (tk < n) mbar_wait(&full[(it + k) % kPairStages], (uint32_t)((it + k) / kPairStages) & 1u, kPairTimeoutNs);
        }
      }
      __syncthreads();
      return;
    }
    // (the phase stays complete until thread 0 re-arms the stage after the
    // next barrier, so this poll succeeds at once)
    if (!mbar_test(&full[s], par)) mbar_wait(&full[s], par, kPairTimeoutNs);
    const unsigned char* tile = sm_raw + s * stage_stride;
    float acc[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      acc[u] = 0.0f;
      const int r = (u * nw + warp) * rpi + sub;
      if (r < nr && cl < nch) {
        const uint4 v4 = *reinterpret_cast<const uint4*>(tile + ((size_t)r * nc + cl * VN) * 2);
        float v[VN];
        Chunk<TS>::cvt(v4, v);
#pragma unroll
        for (int e = 0; e < VN; ++e) acc[u] = fmaf(v[e], xr[e], acc[u]);
      }
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0 && t + kPairStages * G < n) issue(s, t + kPairStages * G);
    if (p1 >= 0) load_x(j1, xr);  // the next pair's x_j, before this pair's reduction
    float* out = part + p * nr;
    if (cpr == 16) {
      // transposed butterfly over the 16 lanes of a row group: at xor 8, 4
      // and 2 each lane keeps half of its remaining rows and adds its
      // partner's copies of them; xor 1 finishes.  Lane bits (3, 2, 1) then
      // name the row u the lane holds.
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool up = lane & 8;
        const float mine = up ? acc[q + 4] : acc[q], other = up ? acc[q] : acc[q + 4];
        acc[q] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const bool up = lane & 4;
        const float mine = up ? acc[q + 2] : acc[q], other = up ? acc[q] : acc[q + 2];
        acc[q] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
      }
      {
        const bool up = lane & 2;
        const float mine = up ? acc[1] : acc[0], other = up ? acc[0] : acc[1];
        acc[0] = mine + __shfl_xor_sync(0xffffffffu, other, 2);
      }
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
      const int u = (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) | ((lane >> 1) & 1);
      const int r = (u * nw + warp) * rpi + sub;
      if ((lane & 1) == 0 && r < nr) out[r] = acc[0];
    } else {
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        for (int o = cpr >> 1; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        const int r = (u * nw + warp) * rpi + sub;
        if (cl == 0 && r < nr) out[r] = acc[u];
      }
    }
    p = p1, j = j1, p1 = p2, j1 = j2;
  }
}


// The per-box kernels below split a box's output rows over ns CTAs
// (grid = nb * ns; CTA b takes box b / ns and row slice b % ns), so that a
// level with few boxes still spreads its rows over the GPU.
struct Slice {
  int i, r0, nr;
};
__device__ __forceinline__ Slice slice_of(int64_t b, int ns, int nrows) {
  const int i = (int)(b / ns), s = (int)(b % ns);
  const int per = ((nrows + ns - 1) / ns + 7) & ~7;
  const int r0 = min(s * per, nrows);
  return {i, r0, min(per, nrows - r0)};
}

// ---------------------------------------------------------------- fwd1 ---
// [u_i; c_i^S]: u_i = Ainv_i c_i^R = M1_i b_i with M1_i = Ainv_i (U_i^R)^T
// (row-major R x D, formed by the factorization) and c_i^S = (U_i^S)^T b_i
// (rows R.. of U^T, i.e. columns R.. of the column-major U).  Above the leaf
// level the box input b_i is assembled first from its two children c:
// b_i = [s_2i; s_2i+1], s_c = c_c^S - sum_{j near c} Ahat_cj^SR v_j (the
// pair sums of the children's SR products).
// Each step below is a body over one work item (box and row slice, or
// pair) called by its kernel (dep: launched as a programmatic dependent, so
// wait for the predecessor before reading its output).
template <typename T>
__device__ __forceinline__ void fwd1_body(int64_t t, int D, int R, int ns, const T* __restrict__ M1,
                                          const T* __restrict__ U, const T* vin, const ChildIn<T>& ch, T* u, T* c,
                                          bool dep) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sv = reinterpret_cast<T*>(sm_raw);  // D
  const Slice sl = slice_of(t, ns, D);
  const int i = sl.i;
  bool loaded = false;
  auto hook = [&] {
    if (loaded) return;
    loaded = true;
    if (dep) {
      griddep_wait();
      griddep_launch_next();
    }
    if (ch.c) {
      const T isc = ch.iscale ? T(ch.iscale[0]) : T(1);
      for (int e = threadIdx.x; e < D; e += blockDim.x) {
        const int cc = 2 * i + e / ch.K, r = e % ch.K;
        sv[e] = ch.c[(int64_t)cc * ch.D + ch.R + r] - isc * sum_pairs(ch.part, ch.K, ch.ptr[cc], ch.ptr[cc + 1], r);
      }
    } else {
      for (int e = threadIdx.x; e < D; e += blockDim.x) sv[e] = vin[(int64_t)i * D + e];
    }
    __syncthreads();
  };
  const int a0 = sl.r0, a1 = min(sl.r0 + sl.nr, R), b0 = max(sl.r0, R), b1 = sl.r0 + sl.nr;
  if (a1 > a0 && b1 > b0) prefetch_l2(U + ((int64_t)i * D + b0) * D, (int64_t)(b1 - b0) * D * sizeof(T));
  if (a1 > a0)
    cta_gemv<T, T, Unr<T>::v>(M1 + ((int64_t)i * R + a0) * D, D, a1 - a0, D, sv, T(1), nullptr,
                              u + (int64_t)i * R + a0, hook);
  if (b1 > b0)
    cta_gemv<T, T, Unr<T>::v>(U + ((int64_t)i * D + b0) * D, D, b1 - b0, D, sv, T(1), nullptr,
                              c + (int64_t)i * D + b0, hook);
}
// (two CTAs per SM: the register cap spills a few bytes of the assembly of b
// but doubles the loads in flight per SM; the substitution took 21.5 ms
// per step instead of 22.0 ms at 162 registers and one CTA per SM)
template <typename T>
__global__ void __launch_bounds__(256, 2) fwd1_kernel(int D, int R, int ns, const T* __restrict__ M1,
                                                   const T* __restrict__ U, const T* __restrict__ vin,
                                                   ChildIn<T> ch, T* __restrict__ u, T* __restrict__ c) {
  fwd1_body<T>(blockIdx.x, D, R, ns, M1, U, vin, ch, u, c, true);
}

// ---------------------------------------------------------------- fwd2 ---
// v_i = Ainv_i (c_i^R - sum_{j<i near} Ahat_ij^RR u_j)
//     = u_i - Ainv_i sum_{j<i near} Ahat_ij^RR u_j
template <typename T>
__device__ __forceinline__ void fwd2_body(int64_t t, int R, int ns, const int64_t* __restrict__ ptr,
                                          const int32_t* __restrict__ lo_cnt, const float* __restrict__ iscale,
                                          const T* __restrict__ Ainv, const T* u, const T* part, T* v,
                                          bool dep) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sb = reinterpret_cast<T*>(sm_raw);  // R
  const Slice sl = slice_of(t, ns, R);
  const int i = sl.i;
  cta_gemv<T, T, Unr<T>::v>(Ainv + ((int64_t)i * R + sl.r0) * R, R, sl.nr, R, sb, T(-1), u + (int64_t)i * R + sl.r0,
                            v + (int64_t)i * R + sl.r0, [&] {
                              const T isc = iscale ? T(iscale[0]) : T(1);
                              // the pairs j < i lead the box's sorted range
                              const int64_t q0 = ptr[i], q1 = q0 + lo_cnt[i];
                              if (dep) {
                                griddep_wait();
                                griddep_launch_next();
                              }
                              for (int r = threadIdx.x; r < R; r += blockDim.x)
                                sb[r] = isc * sum_pairs(part, R, q0, q1, r);
                              __syncthreads();
                            });
}
template <typename T>
__global__ void __launch_bounds__(256) fwd2_kernel(int R, int ns, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ lo_cnt, const float* __restrict__ iscale,
                                                   const T* __restrict__ Ainv, const T* __restrict__ u,
                                                   const T* __restrict__ part, T* __restrict__ v) {
  fwd2_body<T>(blockIdx.x, R, ns, ptr, lo_cnt, iscale, Ainv, u, part, v, true);
}

// ---------------------------------------------------------------- fwd3 ---
// s_i = c_i^S - sum_{j near} Ahat_ij^SR v_j  -> parent input slot
template <typename T>
__device__ __forceinline__ void fwd3_body(int i, int D, int R, int K, const int64_t* __restrict__ ptr,
                                          const float* __restrict__ iscale, const T* c, const T* part, T* pvin,
                                          bool dep) {
  const T isc = iscale ? T(iscale[0]) : T(1);
  const int64_t q0 = ptr[i], q1 = ptr[i + 1];
  T* out = pvin + (int64_t)(i >> 1) * 2 * K + (i & 1) * K;
  if (dep) {
    griddep_wait();
    griddep_launch_next();
  }
  for (int r = threadIdx.x; r < K; r += blockDim.x)
    out[r] = c[(int64_t)i * D + R + r] - isc * sum_pairs(part, K, q0, q1, r);
}
template <typename T>
__global__ void __launch_bounds__(128) fwd3_kernel(int D, int R, int K, const int64_t* __restrict__ ptr,
                                                   const float* __restrict__ iscale, const T* __restrict__ c,
                                                   const T* __restrict__ part, T* __restrict__ pvin) {
  fwd3_body<T>(blockIdx.x, D, R, K, ptr, iscale, c, part, pvin, true);
}

// ---------------------------------------------------------------- bwd1 ---
// om_i = v_i - Ainv_i sum_{j near} Ahat_ij^RS x_j^S
template <typename T>
__device__ __forceinline__ void bwd1_body(int64_t t, int R, int ns, const int64_t* __restrict__ ptr,
                                          const float* __restrict__ iscale, const T* __restrict__ Ainv,
                                          const T* v, const T* part, T* om, bool dep) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* st = reinterpret_cast<T*>(sm_raw);  // R
  const Slice sl = slice_of(t, ns, R);
  const int i = sl.i;
  cta_gemv<T, T, Unr<T>::v>(Ainv + ((int64_t)i * R + sl.r0) * R, R, sl.nr, R, st, T(-1), v + (int64_t)i * R + sl.r0,
                            om + (int64_t)i * R + sl.r0, [&] {
                              const T isc = iscale ? T(iscale[0]) : T(1);
                              const int64_t q0 = ptr[i], q1 = ptr[i + 1];
                              if (dep) {
                                griddep_wait();
                                griddep_launch_next();
                              }
                              for (int r = threadIdx.x; r < R; r += blockDim.x) st[r] = isc * sum_pairs(part, R, q0, q1, r);
                              __syncthreads();
                            });
}
template <typename T>
__global__ void __launch_bounds__(256) bwd1_kernel(int R, int ns, const int64_t* __restrict__ ptr,
                                                   const float* __restrict__ iscale, const T* __restrict__ Ainv,
                                                   const T* __restrict__ v, const T* __restrict__ part,
                                                   T* __restrict__ om) {
  bwd1_body<T>(blockIdx.x, R, ns, ptr, iscale, Ainv, v, part, om, true);
}

// ---------------------------------------------------------------- bwd2 ---
// x_i = U_i z_i, z_i = [x_i^R; x_i^S] with
// x_i^R = om_i - Ainv_i sum_{j>i near} Ahat_ij^RR om_j and x_i^S from the
// parent.  Every CTA of box i forms the whole x_i^R (Ainv_i is read once
// from memory and then from L2 when the rows are split), then its slice of
// the rows of U_i z_i (Ur: U_i row-major).
template <typename T>
__device__ __forceinline__ void bwd2_body(int64_t t, int D, int R, int K, int ns, const int64_t* __restrict__ ptr,
                                          const int32_t* __restrict__ hi_cnt, const float* __restrict__ iscale,
                                          const T* __restrict__ Ainv, const T* om, const T* px, const T* part,
                                          const T* __restrict__ Ur, T* xs, bool dep) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* zs = reinterpret_cast<T*>(sm_raw);  // D
  T* sq = zs + ((D + 3) & ~3);           // R
  const Slice sl = slice_of(t, ns, D);
  const int i = sl.i;
  prefetch_l2(Ur + ((int64_t)i * D + sl.r0) * D, (int64_t)sl.nr * D * sizeof(T));
  cta_gemv<T, T, Unr<T>::v>(Ainv + (int64_t)i * R * R, R, R, R, sq, T(-1), om + (int64_t)i * R, zs, [&] {
    const T isc = iscale ? T(iscale[0]) : T(1);
    // the pairs j > i trail the box's sorted range
    const int64_t q1 = ptr[i + 1], q0 = q1 - hi_cnt[i];
    if (dep) {
      griddep_wait();
      griddep_launch_next();
    }
    const T* xi = px + (int64_t)(i >> 1) * 2 * K + (i & 1) * K;
    for (int e = threadIdx.x; e < K; e += blockDim.x) zs[R + e] = xi[e];
    for (int r = threadIdx.x; r < R; r += blockDim.x) sq[r] = isc * sum_pairs(part, R, q0, q1, r);
    __syncthreads();
  });
  cta_gemv<T, T, Unr<T>::v>(Ur + ((int64_t)i * D + sl.r0) * D, D, sl.nr, D, zs, T(1), nullptr,
                            xs + (int64_t)i * D + sl.r0, [] { __syncthreads(); });
}
template <typename T>
__global__ void __launch_bounds__(256) bwd2_kernel(int D, int R, int K, int ns, const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ hi_cnt, const float* __restrict__ iscale,
                                                   const T* __restrict__ Ainv, const T* __restrict__ om,
                                                   const T* __restrict__ px, const T* __restrict__ part,
                                                   const T* __restrict__ Ur, T* __restrict__ xs) {
  bwd2_body<T>(blockIdx.x, D, R, K, ns, ptr, hi_cnt, iscale, Ainv, om, px, part, Ur, xs, true);
}

// out_b = (in_b)^T for nb square D x D blocks (32 x 32 tiles through shared memory)
template <typename T>
__global__ void transpose_blocks_kernel(int D, const T* __restrict__ in, T* __restrict__ out) {
  __shared__ T tile[32][33];
  const int64_t b = blockIdx.z;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const T* src = in + b * D * D;
  T* dst = out + b * D * D;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = by + y, c = bx + threadIdx.x;
    if (r < D && c < D) tile[y][threadIdx.x] = src[(int64_t)r * D + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = bx + y, c = by + threadIdx.x;
    if (r < D && c < D) dst[(int64_t)r * D + c] = tile[threadIdx.x][y];
  }
}
template <typename T>
void launch_transpose_blocks(int64_t nb, int D, const T* in, T* out, cudaStream_t st) {
  if (nb == 0 || D == 0) return;
  ++g_launches;
  dim3 grid((D + 31) / 32, (D + 31) / 32, (unsigned)nb);
  transpose_blocks_kernel<T><<<grid, dim3(32, 8), 0, st>>>(D, in, out);
}

// A[dst[k]] = A[src[k]]^T for D x D blocks of one array (the lower near
// pairs of a symmetric level from their mirrors); blocks by z, grid-strided.
template <typename T>
__global__ void transpose_pairs_kernel(int D, int64_t n, const int32_t* __restrict__ dsti,
                                       const int32_t* __restrict__ srci, T* __restrict__ A) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int64_t k = blockIdx.z; k < n; k += gridDim.z) {
    const T* src = A + (int64_t)srci[k] * D * D;
    T* dst = A + (int64_t)dsti[k] * D * D;
    for (int y = threadIdx.y; y < 32; y += 8) {
      const int r = by + y, c = bx + threadIdx.x;
      if (r < D && c < D) tile[y][threadIdx.x] = src[(int64_t)r * D + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
      const int r = bx + y, c = by + threadIdx.x;
      if (r < D && c < D) dst[(int64_t)r * D + c] = tile[threadIdx.x][y];
    }
    __syncthreads();
  }
}
template <typename T>
void launch_transpose_pairs(int D, int64_t n, const int32_t* dst, const int32_t* src, T* A, cudaStream_t st) {
  if (n == 0 || D == 0) return;
  ++g_launches;
  dim3 grid((D + 31) / 32, (D + 31) / 32, (unsigned)std::min<int64_t>(n, 65535));
  transpose_pairs_kernel<T><<<grid, dim3(32, 8), 0, st>>>(D, n, dst, src, A);
}

static void set_smem(const void* f, size_t sm) {
  if (sm > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

// Launch with programmatic stream serialization (see griddep_wait).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++g_launches;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

static int num_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
  }
  return nsm;
}

// row slices per box: enough CTAs for two per SM, at least 32 rows each
// a launch of at most one CTA per SM: its CTAs stream their blocks alone,
// so they ask L2 for them before waiting on the previous kernel
static bool small_level(int64_t nblocks) { return nblocks <= num_sms(); }

// launch shapes the autotuner (h2_autotune) sets: per-box CTAs per SM and
// TMA pair-kernel CTAs per SM (process-wide)
std::atomic<int> g_box_ctas_per_sm{1};
std::atomic<int> g_pair_ctas_per_sm{3};

static int row_splits(int nb, int nrows) {
  const int nsm = num_sms();
  if (nb <= 0) return 1;
  int ns = (g_box_ctas_per_sm.load() * nsm + nb - 1) / nb;
  ns = std::min(ns, std::max(1, nrows / 32));
  return std::max(ns, 1);
}

template <typename T, typename TS, int PH>
static void launch_pairs(const DevLevel& L, const FacLevel<T>& F, const int32_t* list, int64_t n, const TS* Ahat,
                         const T* xv, T* part, cudaStream_t st) {
  if (n <= 0) return;
  const int nr = (PH == PH_SR) ? L.K : L.R;
  const int nc = (PH == PH_RS) ? L.K : L.R;
  if constexpr (sizeof(TS) == 2 && std::is_same<T, float>::value) {
    if (F.tma) {
      const CUtensorMap& tm = (PH == PH_RR) ? F.tm_rr : (PH == PH_SR ? F.tm_sr : F.tm_rs);
      const size_t stage = ((size_t)nr * nc * 2 + 127) & ~(size_t)127;
      const size_t sm = kPairStages * stage + 128;  // + room to align the ring
      const int64_t grid = std::min<int64_t>(n, (int64_t)g_pair_ctas_per_sm.load() * num_sms());
      set_smem((const void*)pair_tma_kernel<TS, PH>, sm);
      launch_pdl(pair_tma_kernel<TS, PH>, (unsigned)grid, 256, sm, st, tm, L.D, L.R, L.K, n, list, L.near_j,
                 reinterpret_cast<const float*>(xv), reinterpret_cast<float*>(part), F.err);
      return;
    }
  }
  // the persistent form when one pass covers the block and its rows load as
  // aligned 16-byte chunks
  constexpr int VN = Chunk<TS>::VN;
  const int nch = (nc + VN - 1) / VN;
  int cpr = 32;
  while (cpr > 1 && cpr / 2 >= nch) cpr >>= 1;
  const int64_t off = (PH == PH_SR ? (int64_t)L.R * L.D : (PH == PH_RS ? L.R : 0));
  const bool aligned = ((L.D * sizeof(TS)) % 16 == 0) && ((off * (int64_t)sizeof(TS)) % 16 == 0) &&
                       ((reinterpret_cast<uintptr_t>(Ahat) & 15) == 0);
  if (aligned && nch <= 32 && nr <= 8 * Unr<TS>::v * (32 / cpr) && nc > 0) {
    const int per_sm = sizeof(TS) == 2 ? 3 : 2;
    const int64_t grid = std::min<int64_t>(n, (int64_t)per_sm * num_sms());
    const size_t sm = sizeof(T) * 2 * (size_t)((nc + 3) & ~3);
    set_smem((const void*)pair_persist_kernel<T, TS, PH>, sm);
    launch_pdl(pair_persist_kernel<T, TS, PH>, (unsigned)grid, 256, sm, st, L.D, L.R, L.K, n, list, L.near_j, Ahat,
               xv, part);
    return;
  }
  const size_t sm = sizeof(T) * (size_t)std::max(nc, 1);
  set_smem((const void*)pair_kernel<T, TS, PH>, sm);
  launch_pdl(pair_kernel<T, TS, PH>, (unsigned)n, 256, sm, st, L.D, L.R, L.K, list, L.near_j, Ahat, xv, part);
}

// ------------------------------------------------------------------------
// Streamed per-box steps for levels with many boxes (D = 256, R = 128 or
// D = 128, R = 64; FP32 factors).  A persistent CTA (one per SM) walks its
// boxes i = blockIdx.x, + gridDim.x, ..., and each box's factor rows flow
// through a shared-memory ring of kBoxStages 16 KB stages, filled by
// one-dimensional bulk copies that thread 0 issues kBoxStages stages ahead,
// across box boundaries, so that the copies of the next box overlap the
// reductions of this one.  A stage holds whole rows (16 KB / row bytes of
// them); warp w takes rows w, w + 8, ..., each lane RW / 32 consecutive
// entries of a row, with its part of the box's input vector in registers,
// and the rows of a warp meet in one transposed butterfly.
//   BX_FWD1: [u_i; c_i^S] = [M1_i; (U_i^S)^T] b_i, b_i as fwd1 forms it;
//   BX_FWD2: v_i = u_i - Ainv_i (s^-1 sum_{j<i near} part);
//   BX_BWD1: om_i = v_i - Ainv_i (s^-1 sum_{j near} part);
//   BX_BWD2: x_i^R = om_i - Ainv_i (s^-1 sum_{j>i near} part), then
//            x_i = U_i [x_i^R; x_i^S] from the row-major copy Ur.
// The same products as fwd1..bwd2 with the sums grouped differently.
// Waits are bounded (2 s); on expiry every thread leaves together, thread 0
// having waited (bounded) for the copies still in flight and set *err.
// ------------------------------------------------------------------------
enum { BX_FWD1 = 0, BX_FWD2 = 1, BX_BWD1 = 2, BX_BWD2 = 3 };
constexpr int kBoxStages = 8;
constexpr uint32_t kBoxStageBytes = 16384;

struct BoxArgs {
  int64_t nb;
  const int64_t* ptr;    // near-pair CSR of the level
  const int32_t* cnt;    // pairs j < i (FWD2) or j > i (BWD2) of each box
  const float* iscale;   // 1 / s of the 16-bit Ahat, or NULL
  const float* Ainv;     // nb x R x R
  const float* M1;       // nb x R x D
  const float* U;        // nb x D x D, column-major (rows R.. of U^T: (U^S)^T)
  const float* Ur;       // nb x D x D, row-major
  const float* vin;      // leaf input (FWD1 without children)
  ChildIn<float> ch;     // children's SR sums (FWD1 above the leaf)
  float* u;
  float* c;
  float* v;
  float* om;
  const float* px;       // parent's solution slots (BWD2)
  float* xs;
  const float* part;
  int32_t* err;
};

template <int MODE, int D, int R>
struct BoxShape {
  static constexpr int K = D - R;
  static constexpr int RWA = (MODE == BX_FWD1) ? D : R;              // row width of the first matrix
  static constexpr int RPA = (int)kBoxStageBytes / (4 * RWA);          // its rows per stage
  static constexpr int NA = ((MODE == BX_FWD1) ? D : R) / RPA;         // its stages
  static constexpr int RPB = (int)kBoxStageBytes / (4 * D);            // BWD2's Ur rows per stage
  static constexpr int NB = (MODE == BX_BWD2) ? D / RPB : 0;
  static constexpr int NS = NA + NB;
  static_assert(R % RPA == 0 && D % RPB == 0 && RPA % 8 == 0 && RPB % 8 == 0, "stage rows");
};

template <int MODE, int D, int R>
__device__ __forceinline__ const float* box_stage_src(const BoxArgs& a, int64_t i, int j) {
  using S = BoxShape<MODE, D, R>;
  if constexpr (MODE == BX_FWD1) {
    const int r0 = j * S::RPA;
    return r0 < R ? a.M1 + ((size_t)i * R + r0) * D : a.U + ((size_t)i * D + r0) * D;
  } else {
    if (j < S::NA) return a.Ainv + ((size_t)i * R + (size_t)j * S::RPA) * R;
    return a.Ur + ((size_t)i * D + (size_t)(j - S::NA) * S::RPB) * D;
  }
}

// One stage: RPS rows of width RW at tile (rows j * RPS .. of the box's
// current matrix); out(row, value) stores a finished row.
template <int RW, int RPS, typename Out>
__device__ __forceinline__ void box_stage_rows(const float* tile, const float (&xr)[RW / 32], int row0, Out out) {
  constexpr int VL = RW / 32, NR = RPS / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NR];
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    const float* rowp = tile + (size_t)(warp + 8 * t) * RW + lane * VL;
    float s = 0.0f;
    if constexpr (VL % 4 == 0) {
#pragma unroll
      for (int e = 0; e < VL; e += 4) {
        const float4 m = *reinterpret_cast<const float4*>(rowp + e);
        s = fmaf(m.x, xr[e], s);
        s = fmaf(m.y, xr[e + 1], s);
        s = fmaf(m.z, xr[e + 2], s);
        s = fmaf(m.w, xr[e + 3], s);
      }
    } else {
#pragma unroll
      for (int e = 0; e < VL; e += 2) {
        const float2 m = *reinterpret_cast<const float2*>(rowp + e);
        s = fmaf(m.x, xr[e], s);
        s = fmaf(m.y, xr[e + 1], s);
      }
    }
    acc[t] = s;
  }
  const float v = tsum<NR, 32, float>(acc);
  if (tsum_leader<NR, 32>(lane)) out(row0 + warp + 8 * tsum_index<NR, 32>(lane), v);
}

template <int MODE, int D, int R>
__global__ void __launch_bounds__(256, 1) box_stream_kernel(BoxArgs a) {
  using S = BoxShape<MODE, D, R>;
  constexpr int K = S::K;
  extern __shared__ __align__(128) unsigned char sm_dyn[];
  __shared__ __align__(8) uint64_t full[kBoxStages];
  unsigned char* ring = sm_dyn + ((128u - (smem_u32(sm_dyn) & 127u)) & 127u);
  float* xv = reinterpret_cast<float*>(ring + (size_t)kBoxStages * kBoxStageBytes);  // D
  float* zs = xv + D;                                                                  // D
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t G = gridDim.x;
  const int64_t nmine = (blockIdx.x < a.nb) ? (a.nb - blockIdx.x + G - 1) / G : 0;
  const int64_t total = nmine * S::NS;  // this CTA's stages
  if (tid == 0) {
    for (int s = 0; s < kBoxStages; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int64_t g) {
    const int s = (int)(g % kBoxStages);
    const int64_t i = blockIdx.x + (g / S::NS) * G;
    mbar_expect_tx(&full[s], kBoxStageBytes);
    bulk_load(ring + (size_t)s * kBoxStageBytes, box_stage_src<MODE, D, R>(a, i, (int)(g % S::NS)), kBoxStageBytes,
              &full[s]);
  };
  // factor rows are fixed during a solve: their copies start before the
  // wait for the previous kernel
  if (tid == 0)
    for (int64_t g = 0; g < kBoxStages && g < total; ++g) issue(g);
  griddep_wait();
  griddep_launch_next();
  const float isc = a.iscale ? a.iscale[0] : 1.0f;
  int64_t g = 0;
  for (int64_t k = 0; k < nmine; ++k) {
    const int64_t i = blockIdx.x + k * G;
    // the box's input vector
    if constexpr (MODE == BX_FWD1) {
      if (a.ch.c) {
        const float cs = a.ch.iscale ? a.ch.iscale[0] : 1.0f;
        for (int e = tid; e < D; e += blockDim.x) {
          const int64_t cc = 2 * i + e / a.ch.K;
          const int r = e % a.ch.K;
          xv[e] = a.ch.c[cc * a.ch.D + a.ch.R + r] - cs * sum_pairs(a.ch.part, a.ch.K, a.ch.ptr[cc], a.ch.ptr[cc + 1], r);
        }
      } else {
        for (int e = tid; e < D; e += blockDim.x) xv[e] = a.vin[i * D + e];
      }
    } else {
      int64_t q0 = a.ptr[i], q1 = a.ptr[i + 1];
      if (MODE == BX_FWD2) q1 = q0 + a.cnt[i];
      if (MODE == BX_BWD2) q0 = q1 - a.cnt[i];
      for (int r = tid; r < R; r += blockDim.x) xv[r] = isc * sum_pairs(a.part, R, q0, q1, r);
      if (MODE == BX_BWD2) {
        const float* xp = a.px + (i >> 1) * 2 * K + (i & 1) * K;
        for (int e = tid; e < K; e += blockDim.x) zs[R + e] = xp[e];
      }
    }
    __syncthreads();
    float xa[S::RWA / 32];
#pragma unroll
    for (int e = 0; e < S::RWA / 32; ++e) xa[e] = xv[lane * (S::RWA / 32) + e];
    float xb[D / 32];
    for (int j = 0; j < S::NS; ++j, ++g) {
      if (MODE == BX_BWD2 && j == S::NA) {
        // x_i^R is complete (the stage loop ends in a barrier)
#pragma unroll
        for (int e = 0; e < D / 32; ++e) xb[e] = zs[lane * (D / 32) + e];
      }
      const int s = (int)(g % kBoxStages);
      const uint32_t par = (uint32_t)(g / kBoxStages) & 1u;
      bool ok = true;
      if (tid == 0) ok = mbar_wait(&full[s], par, kPairTimeoutNs);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(a.err, 1);
          for (int64_t h = g; h < g + kBoxStages && h < total; ++h)
            mbar_wait(&full[h % kBoxStages], (uint32_t)(h / kBoxStages) & 1u, kPairTimeoutNs);
        }
        __syncthreads();
        return;
      }
      if (!mbar_test(&full[s], par)) mbar_wait(&full[s], par, kPairTimeoutNs);
      const float* tile = reinterpret_cast<const float*>(ring + (size_t)s * kBoxStageBytes);
      if (j < S::NA) {
        box_stage_rows<S::RWA, S::RPA>(tile, xa, j * S::RPA, [&](int r, float val) {
          if constexpr (MODE == BX_FWD1) {
            if (r < R) a.u[i * R + r] = val;
            else a.c[i * D + r] = val;
          } else if constexpr (MODE == BX_FWD2) {
            a.v[i * R + r] = a.u[i * R + r] - val;
          } else if constexpr (MODE == BX_BWD1) {
            a.om[i * R + r] = a.v[i * R + r] - val;
          } else {
            zs[r] = a.om[i * R + r] - val;
          }
        });
      } else if constexpr (MODE == BX_BWD2) {
        box_stage_rows<D, S::RPB>(tile, xb, (j - S::NA) * S::RPB, [&](int r, float val) { a.xs[i * D + r] = val; });
      }
      __syncthreads();  // every thread is done with stage s (and zs / xv of this box)
      if (tid == 0 && g + kBoxStages < total) issue(g + kBoxStages);
    }
  }
}

// The streamed form for a level: D = 256 with R = 128, or D = 128 with
// R = 64, FP32 factors with 16-byte aligned rows, and enough boxes to give
// every SM some (false: use the row-split kernels).
std::atomic<int> g_box_stream{0};  // H2_OPT_BOX_STREAM (process-wide)

template <int MODE>
static bool launch_box_stream(const DevLevel& L, const BoxArgs& a, cudaStream_t st) {
  const int nsm = num_sms();
  const int mode = g_box_stream.load();
  if (mode == 0 || (mode == 1 && L.nb < nsm) || a.err == nullptr) return false;
  if (!((L.D == 256 && L.R == 128) || (L.D == 128 && L.R == 64))) return false;
  const size_t sm = (size_t)kBoxStages * kBoxStageBytes + 2 * sizeof(float) * L.D + 128;
  const unsigned grid = (unsigned)std::min<int64_t>(L.nb, nsm);
  if (L.D == 256) {
    set_smem((const void*)box_stream_kernel<MODE, 256, 128>, sm);
    launch_pdl(box_stream_kernel<MODE, 256, 128>, grid, 256, sm, st, a);
  } else {
    set_smem((const void*)box_stream_kernel<MODE, 128, 64>, sm);
    launch_pdl(box_stream_kernel<MODE, 128, 64>, grid, 256, sm, st, a);
  }
  return true;
}

// the streamed per-box form's arguments for a level
template <typename T>
static BoxArgs box_args(const DevLevel& L, const FacLevel<T>& F, const float* iscale) {
  BoxArgs a{};
  a.nb = L.nb;
  a.ptr = L.near_ptr;
  a.iscale = iscale;
  a.Ainv = reinterpret_cast<const float*>(F.Ainv);
  a.M1 = reinterpret_cast<const float*>(F.M1);
  a.U = reinterpret_cast<const float*>(F.U);
  a.Ur = reinterpret_cast<const float*>(F.Ur);
  a.vin = reinterpret_cast<const float*>(F.vin);
  a.u = reinterpret_cast<float*>(F.u);
  a.c = reinterpret_cast<float*>(F.c);
  a.v = reinterpret_cast<float*>(F.v);
  a.om = reinterpret_cast<float*>(F.om);
  a.xs = reinterpret_cast<float*>(F.xs);
  a.part = reinterpret_cast<const float*>(F.part);
  a.err = F.err;
  return a;
}

template <typename T>
void launch_fwd1(const DevLevel& L, const FacLevel<T>& F, const ChildIn<T>& ch, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    BoxArgs a = box_args(L, F, nullptr);
    a.ch = ch;
    if (launch_box_stream<BX_FWD1>(L, a, st)) return;
  }
  const int ns = row_splits(L.nb, L.D);
  launch_pdl(fwd1_kernel<T>, L.nb * ns, 256, sizeof(T) * L.D, st, L.D, L.R, ns, F.M1, F.U, F.vin, ch, F.u, F.c);
}
template <typename T, typename TS>
void launch_fwd2(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, cudaStream_t st) {
  if (L.R == 0) return;
  launch_pairs<T, TS, PH_RR>(L, F, L.lo_pairs, L.n_lo, Ahat, F.u, F.part, st);
  if constexpr (std::is_same<T, float>::value) {
    BoxArgs a = box_args(L, F, iscale);
    a.cnt = L.lo_cnt;
    if (launch_box_stream<BX_FWD2>(L, a, st)) return;
  }
  const int ns = row_splits(L.nb, L.R);
  launch_pdl(fwd2_kernel<T>, L.nb * ns, 256, sizeof(T) * L.R, st, L.R, ns, L.near_ptr, L.lo_cnt, iscale, F.Ainv, F.u,
             F.part, F.v);
}
template <typename T, typename TS>
void launch_fwd3(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, T* parent_vin,
                 cudaStream_t st) {
  if (L.K == 0) return;
  launch_pairs<T, TS, PH_SR>(L, F, nullptr, L.NP, Ahat, F.v, F.part, st);
  // above level 1 the parent's fwd1 sums these pair products itself
  if (parent_vin) launch_pdl(fwd3_kernel<T>, L.nb, 128, 0, st, L.D, L.R, L.K, L.near_ptr, iscale, F.c, F.part, parent_vin);
}
template <typename T, typename TS>
void launch_bwd1(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, const T* parent_x,
                 cudaStream_t st) {
  if (L.R == 0) return;
  launch_pairs<T, TS, PH_RS>(L, F, nullptr, L.NP, Ahat, parent_x, F.part, st);
  if constexpr (std::is_same<T, float>::value) {
    if (launch_box_stream<BX_BWD1>(L, box_args(L, F, iscale), st)) return;
  }
  const int ns = row_splits(L.nb, L.R);
  launch_pdl(bwd1_kernel<T>, L.nb * ns, 256, sizeof(T) * L.R, st, L.R, ns, L.near_ptr, iscale, F.Ainv, F.v, F.part,
             F.om);
}
template <typename T, typename TS>
void launch_bwd2(const DevLevel& L, const FacLevel<T>& F, const TS* Ahat, const float* iscale, const T* parent_x,
                 cudaStream_t st) {
  if (L.R > 0) launch_pairs<T, TS, PH_RR>(L, F, L.hi_pairs, L.n_hi, Ahat, F.om, F.part, st);
  if constexpr (std::is_same<T, float>::value) {
    BoxArgs a = box_args(L, F, iscale);
    a.cnt = L.hi_cnt;
    a.px = reinterpret_cast<const float*>(parent_x);
    if (launch_box_stream<BX_BWD2>(L, a, st)) return;
  }
  const int ns = row_splits(L.nb, L.D);
  const size_t sm = sizeof(T) * ((size_t)((L.D + 3) & ~3) + std::max(L.R, 1));
  launch_pdl(bwd2_kernel<T>, L.nb * ns, 256, sm, st, L.D, L.R, L.K, ns, L.near_ptr, L.hi_cnt, iscale, F.Ainv, F.om,
             parent_x, F.part, F.Ur, F.xs);
}

// y_b = M_b x_b for nb n x n row-major matrices, one CTA each (root solves
// with the explicit inverses: one root, or one per system of a forest)
template <typename T>
__global__ void gemv_rows_kernel(int n, const T* __restrict__ M, const T* __restrict__ x, T* __restrict__ y) {
  extern __shared__ unsigned char sm_raw[];
  M += (size_t)blockIdx.x * n * n;
  x += (size_t)blockIdx.x * n;
  y += (size_t)blockIdx.x * n;
  T* sx = reinterpret_cast<T*>(sm_raw);
  T* sy = sx + n;
  for (int e = threadIdx.x; e < n; e += blockDim.x) { sx[e] = x[e]; sy[e] = 0; }
  __syncthreads();
  warp_rows_gemv<T>(M, n, n, n, sx, sy, T(1));
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) y[e] = sy[e];
}
template <typename T>
void launch_gemv_rows(int nb, int n, const T* M, const T* x, T* y, cudaStream_t st) {
  if (n == 0 || nb == 0) return;
  const size_t sm = sizeof(T) * 2 * (size_t)n;
  if (sm > 48 * 1024) cudaFuncSetAttribute(gemv_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  ++g_launches;
  gemv_rows_kernel<T><<<nb, 256, sm, st>>>(n, M, x, y);
}

#define H2_INST_SOLVE(T)                                                                     \
  template void launch_fwd1<T>(const DevLevel&, const FacLevel<T>&, const ChildIn<T>&, cudaStream_t); \
  template void launch_transpose_blocks<T>(int64_t, int, const T*, T*, cudaStream_t);         \
  template void launch_transpose_pairs<T>(int, int64_t, const int32_t*, const int32_t*, T*, cudaStream_t); \
  template void launch_gemv_rows<T>(int, int, const T*, const T*, T*, cudaStream_t);
H2_INST_SOLVE(double)
H2_INST_SOLVE(float)
#define H2_INST_SUBST(T, TS)                                                                                   \
  template void launch_fwd2<T, TS>(const DevLevel&, const FacLevel<T>&, const TS*, const float*, cudaStream_t); \
  template void launch_fwd3<T, TS>(const DevLevel&, const FacLevel<T>&, const TS*, const float*, T*,            \
                                   cudaStream_t);                                                              \
  template void launch_bwd1<T, TS>(const DevLevel&, const FacLevel<T>&, const TS*, const float*, const T*,      \
                                   cudaStream_t);                                                              \
  template void launch_bwd2<T, TS>(const DevLevel&, const FacLevel<T>&, const TS*, const float*, const T*,      \
                                   cudaStream_t);
H2_INST_SUBST(double, double)
H2_INST_SUBST(float, float)
H2_INST_SUBST(float, __half)
H2_INST_SUBST(float, __nv_bfloat16)

// ------------------------------------------------------------- matvec ---
// Element type T: double for the refinement residual, float for the inner
// solver of the mixed-precision refinement.  X, S and A are that level's
// bases, couplings and leaf near blocks in T.

// upward: xh_i[a] = sum_d X_i[d*K + a] x_i[d] (x_i: the box's D inputs):
// the column form of the CTA GEMV (warps over d, lanes over 16-byte chunks
// of a, eight rows of X in flight per lane).
template <typename T>
__global__ void __launch_bounds__(256) mv_up_kernel(int D, int K, const T* __restrict__ X, const T* __restrict__ x,
                                                    T* __restrict__ xh, int pf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* part = reinterpret_cast<T*>(smraw);  // 8 * K
  T* sx = part + 8 * K;                   // D
  const int i = blockIdx.x, tid = threadIdx.x;
  if (pf) prefetch_l2(X + (int64_t)i * D * K, (int64_t)D * K * sizeof(T));
  griddep_wait();
  griddep_launch_next();
  for (int e = tid; e < D; e += 256) sx[e] = x[(int64_t)i * D + e];
  __syncthreads();
  cta_gemv_cols<T, T>(X + (int64_t)i * D * K, K, K, D, sx, part, xh + (int64_t)i * K);
}
template <typename T>
void launch_matvec_up(const DevLevel& L, const T* X, const T* x, T* xh, cudaStream_t st) {
  const size_t sm = sizeof(T) * (8 * (size_t)L.K + L.D);
  set_smem((const void*)mv_up_kernel<T>, sm);
  launch_pdl(mv_up_kernel<T>, L.nb, 256, sm, st, L.D, L.K, X, x, xh, small_level(L.nb) ? 1 : 0);
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
  griddep_wait();
  griddep_launch_next();
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
  launch_pdl(mv_far_kernel<T>, L.nb, 256, sm, st, L.K, L.far_ptr, L.far_j, S, xh, yh);
}

// downward: [yh_2p; yh_2p+1] += X_p yh_p   (rows d of X_p, D = 2 Kc): a
// block-row GEMV per parent box
template <typename T>
__global__ void __launch_bounds__(256, 2) mv_down_kernel(int D, int K, const T* __restrict__ X,
                                                         const T* __restrict__ yh, T* __restrict__ yhc, int pf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sy = reinterpret_cast<T*>(smraw);  // K
  const int p = blockIdx.x;
  if (pf) prefetch_l2(X + (int64_t)p * D * K, (int64_t)D * K * sizeof(T));
  griddep_wait();
  griddep_launch_next();
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
  launch_pdl(mv_down_kernel<T>, L.nb, 256, sizeof(T) * ((L.K + 3) & ~3), st, L.D, L.K, X, yh, yh_child,
             small_level(L.nb) ? 1 : 0);
}

// downward step that also adds the children's coupling products:
// [yh_2p; yh_2p+1] = X_p yh_p + f, f[h Kc + r] = sum over the partial
// products of child c = 2p + h (CSR cptr / cent over the child level; entry
// e = 2k (+1) is part[(2k (+1)) Kc ..]).  cptr NULL: f = 0.  Overwrites the
// children's yh (the per-level sums of the coupling products are folded in).
template <typename T>
__global__ void __launch_bounds__(256, 2) mv_down_far_kernel(int D, int K, const T* __restrict__ X,
                                                             const T* __restrict__ yh, T* __restrict__ yhc,
                                                             const int64_t* __restrict__ cptr,
                                                             const int32_t* __restrict__ cent,
                                                             const T* __restrict__ part, int pf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sy = reinterpret_cast<T*>(smraw);  // K
  T* sf = sy + ((K + 3) & ~3);          // D
  const int p = blockIdx.x;
  const int Kc = D / 2;
  if (pf) prefetch_l2(X + (int64_t)p * D * K, (int64_t)D * K * sizeof(T));
  griddep_wait();
  griddep_launch_next();
  for (int e = threadIdx.x; e < K; e += 256) sy[e] = yh[(int64_t)p * K + e];
  for (int r = threadIdx.x; r < D; r += 256) {
    T s = T(0);
    if (cptr) {
      const int c = 2 * p + r / Kc, rr = r % Kc;
      for (int64_t q = cptr[c]; q < cptr[c + 1]; ++q) s += part[(int64_t)cent[q] * Kc + rr];
    }
    sf[r] = s;
  }
  __syncthreads();
  T acc[kRPW];
  T* out = yhc + (int64_t)p * D;
  for (int r0 = 0; r0 < D; r0 += kChunk) {
    zero(acc);
    rows_acc<T, kRPW>(r0, X + (int64_t)p * D * K, K, D, K, sy, acc);
    rows_finish<T, kRPW>(r0, D, acc, T(1), sf, out);
  }
}
template <typename T>
void launch_matvec_down_far(const DevLevel& L, const T* X, const T* yh, T* yh_child, const int64_t* cptr,
                            const int32_t* cent, const T* part, cudaStream_t st) {
  const size_t sm = sizeof(T) * ((size_t)((L.K + 3) & ~3) + L.D);
  launch_pdl(mv_down_far_kernel<T>, L.nb, 256, sm, st, L.D, L.K, X, yh, yh_child, cptr, cent, part,
             small_level(L.nb) ? 1 : 0);
}
template void launch_matvec_down_far<float>(const DevLevel&, const float*, const float*, float*, const int64_t*,
                                            const int32_t*, const float*, cudaStream_t);

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
  griddep_wait();
  griddep_launch_next();
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

// ---------------------------------------------------- FP64 by FP32 pairs ---
// The FP64 matvec of the mixed refinement's residual, on GB300's FP32 units:
// every FP64 matrix entry m is held as m_h + m_l (m_h = fl32(m),
// m_l = fl32(m - m_h): m to about 2^-48 relative) and every FP64 input x as
// x_h + x_l likewise.  m x = m_h x_h + (m_h x_l + m_l x_h) + O(2^-48 m x);
// the first product is split exactly into p + e by a fused multiply-add,
// and the running sum is an FP32 pair (H, L): H += p by an error-free
// two-sum whose error joins L with e and the cross terms.  Sums over lanes,
// warps and blocks stay FP32 pairs (df_add, df_tsum) and each output is
// converted to FP64 once: GB300's FP64 pipe is too slow for per-entry work.
// The kernels then read 8 bytes per entry, as the FP64 ones do, but spend
// FP32 instructions on them.
// (the _rn intrinsics keep the compiler from fusing the two-sum's operations)
__device__ __forceinline__ void df_fma(float& H, float& L, float mh, float ml, float xh, float xl) {
  const float p = __fmul_rn(mh, xh);
  const float e = fmaf(mh, xh, -p);
  const float small = fmaf(mh, xl, fmaf(ml, xh, e));
  const float s = __fadd_rn(H, p);
  const float bb = __fsub_rn(s, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  H = s;
  L = __fadd_rn(L, __fadd_rn(small, err));
}

// (H, L) += (h, l) for FP32 pairs: an error-free two-sum of the high parts
// (exact in either operand order) with its error joining the low parts
__device__ __forceinline__ void df_add(float& H, float& L, float h, float l) {
  const float s = __fadd_rn(H, h);
  const float bb = __fsub_rn(s, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bb)), __fsub_rn(h, bb));
  H = s;
  L = __fadd_rn(L, __fadd_rn(l, err));
}
// The transposed warp sum (tsum) of N FP32 pairs per lane, in FP32-pair
// arithmetic: lane l ends with the pair sum of value tsum_index<N, G>(l).
// GB300 runs FP64 instructions at a small fraction of the FP32 rate, so the
// FP32-pair kernels reduce in pairs and convert to FP64 once per result.
template <int N, int G>
__device__ __forceinline__ void df_tsum(const float (&h)[N], const float (&l)[N], float& H, float& L) {
  if constexpr (N == 1) {
    H = h[0], L = l[0];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, H, o), ol = __shfl_xor_sync(0xffffffffu, L, o);
      df_add(H, L, oh, ol);
    }
  } else {
    const bool up = threadIdx.x & (G / 2);
    float wh[N / 2], wl[N / 2];
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      wh[q] = up ? h[q + N / 2] : h[q];
      wl[q] = up ? l[q + N / 2] : l[q];
      const float xh = up ? h[q] : h[q + N / 2], xl = up ? l[q] : l[q + N / 2];
      const float oh = __shfl_xor_sync(0xffffffffu, xh, G / 2), ol = __shfl_xor_sync(0xffffffffu, xl, G / 2);
      df_add(wh[q], wl[q], oh, ol);
    }
    df_tsum<N / 2, G / 2>(wh, wl, H, L);
  }
}

constexpr int kRPWdf = 8;  // rows per warp per pass: 64-row chunks

// H[t] + L[t] += sum_c (Mh + Ml)[r_t * ld + c] (xh + xl)[c], rows r_t = r0 + warp + 8 t < nr
template <int RPW>
__device__ __forceinline__ void rows_acc_df(int r0, const float* __restrict__ Mh, const float* __restrict__ Ml,
                                            int64_t ld, int nr, int nc, const float* __restrict__ xh,
                                            const float* __restrict__ xl, float (&H)[RPW], float (&L)[RPW]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = r0 + warp;
  const bool vec = (ld % 4 == 0) && (nc % 4 == 0) && ((reinterpret_cast<uintptr_t>(Mh) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(Ml) & 15) == 0) && ((reinterpret_cast<uintptr_t>(xh) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(xl) & 15) == 0);
  if (vec) {
    for (int c = lane * 4; c < nc; c += 128) {
      float4 vh[RPW], vl[RPW];
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        const int r = rbase + 8 * t;
        if (r < nr) {
          vh[t] = __ldg(reinterpret_cast<const float4*>(Mh + r * ld + c));
          vl[t] = __ldg(reinterpret_cast<const float4*>(Ml + r * ld + c));
        } else {
          vh[t] = make_float4(0.f, 0.f, 0.f, 0.f);
          vl[t] = vh[t];
        }
      }
      const float4 ah = *reinterpret_cast<const float4*>(xh + c);
      const float4 al = *reinterpret_cast<const float4*>(xl + c);
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        df_fma(H[t], L[t], vh[t].x, vl[t].x, ah.x, al.x);
        df_fma(H[t], L[t], vh[t].y, vl[t].y, ah.y, al.y);
        df_fma(H[t], L[t], vh[t].z, vl[t].z, ah.z, al.z);
        df_fma(H[t], L[t], vh[t].w, vl[t].w, ah.w, al.w);
      }
    }
  } else {
    for (int c = lane; c < nc; c += 32) {
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        const int r = rbase + 8 * t;
        if (r < nr) df_fma(H[t], L[t], Mh[r * ld + c], Ml[r * ld + c], xh[c], xl[c]);
      }
    }
  }
}

// out[r] = base[r] + sum over lanes of (H + L): the lanes' pairs added in
// FP32-pair arithmetic, the result converted to FP64 once
template <int RPW>
__device__ __forceinline__ void rows_finish_df(int r0, int nr, const float (&H)[RPW], const float (&L)[RPW],
                                               const double* base, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float sh, sl;
  df_tsum<RPW, 32>(H, L, sh, sl);
  const int r = r0 + warp + 8 * tsum_index<RPW, 32>(lane);
  if (tsum_leader<RPW, 32>(lane) && r < nr) out[r] = (base ? base[r] : 0.0) + ((double)sh + (double)sl);
}

__device__ __forceinline__ void df_split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// leaf: y_i = X_i yh_i + sum_{near j} A_ij x_j
__global__ void __launch_bounds__(256, 2) mv_leaf_df_kernel(int D, int K, const int64_t* __restrict__ ptr,
                                                            const int32_t* __restrict__ nj, const float* __restrict__ Ah,
                                                            const float* __restrict__ Al, const float* __restrict__ Xh,
                                                            const float* __restrict__ Xl, const float* __restrict__ xh,
                                                            const float* __restrict__ xl, const float* __restrict__ yhh,
                                                            const float* __restrict__ yhl, double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int i = blockIdx.x, tid = threadIdx.x;
  const int64_t p0 = ptr[i];
  const int nn = (int)(ptr[i + 1] - p0);
  const int Kp = (K + 3) & ~3, Dp = (D + 3) & ~3;
  float* hh = reinterpret_cast<float*>(smraw);  // Kp
  float* hl = hh + Kp;                          // Kp
  float* xsh = hl + Kp;                         // nn * Dp
  float* xsl = xsh + (size_t)nn * Dp;           // nn * Dp
  if (yhh)
    for (int e = tid; e < K; e += blockDim.x) hh[e] = yhh[(int64_t)i * K + e], hl[e] = yhl[(int64_t)i * K + e];
  for (int e = tid; e < nn * D; e += blockDim.x) {
    const int q = e / D, d = e - q * D;
    const int64_t g = (int64_t)nj[p0 + q] * D + d;
    xsh[q * Dp + d] = xh[g];
    xsl[q * Dp + d] = xl[g];
  }
  __syncthreads();
  float H[kRPWdf], L[kRPWdf];
  for (int r0 = 0; r0 < D; r0 += 8 * kRPWdf) {
    zero(H);
    zero(L);
    if (yhh) rows_acc_df<kRPWdf>(r0, Xh + (int64_t)i * D * K, Xl + (int64_t)i * D * K, K, D, K, hh, hl, H, L);
    for (int q = 0; q < nn; ++q)
      rows_acc_df<kRPWdf>(r0, Ah + (p0 + q) * D * D, Al + (p0 + q) * D * D, D, D, D, xsh + q * Dp, xsl + q * Dp, H,
                          L);
    rows_finish_df<kRPWdf>(r0, D, H, L, nullptr, y + (int64_t)i * D);
  }
}
void launch_matvec_leaf_df(const DevLevel& L, const float* Ah, const float* Al, const float* Xh, const float* Xl,
                           const float* xh, const float* xl, const float* yhh, const float* yhl, double* y,
                           cudaStream_t st) {
  const size_t Kp = (L.K + 3) & ~3, Dp = (L.D + 3) & ~3;
  const size_t sm = 2 * sizeof(float) * (Kp + Dp * (size_t)L.max_near);
  set_smem((const void*)mv_leaf_df_kernel, sm);
  ++g_launches;
  mv_leaf_df_kernel<<<L.nb, 256, sm, st>>>(L.D, L.K, L.near_ptr, L.near_j, Ah, Al, Xh, Xl, xh, xl, yhh, yhl, y);
}

// h = fl32(v), l = fl32(v - h): an FP64 vector as FP32 pairs, once per use
// of the vector rather than once per block that reads it
__global__ void split_df_kernel(const double* __restrict__ v, float* __restrict__ h, float* __restrict__ l,
                                int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    df_split(v[e], h[e], l[e]);
}
void launch_split_df(const double* v, float* h, float* l, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ++g_launches;
  split_df_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(v, h, l, n);
}

// The residual's passes through the bases and couplings with every vector
// held as FP32 pairs (xhat and yhat of all levels, the leaf partial
// products), so that no FP64 instruction runs per matrix entry or per
// vector element until the leaf output y is formed.

// the row sums of (H, L) over the lanes (df_tsum), written as pairs by the
// leader lanes (add: added to the pair already there)
template <int RPW>
__device__ __forceinline__ void rows_finish_pair(int r0, int nr, const float (&H)[RPW], const float (&L)[RPW],
                                                 float* oh, float* ol, bool add) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float sh, sl;
  df_tsum<RPW, 32>(H, L, sh, sl);
  const int r = r0 + warp + 8 * tsum_index<RPW, 32>(lane);
  if (tsum_leader<RPW, 32>(lane) && r < nr) {
    if (add) df_add(sh, sl, oh[r], ol[r]);
    oh[r] = sh;
    ol[r] = sl;
  }
}

// upward: xhat_i = X_i^T z_i (X_i: D x K row-major as Xh + Xl; z_i: the
// leaf input or the children's xhat, D pairs).  Warps take rows n, lanes
// 4-column chunks of the output; the 8 warps' pairs are added at the end.
__global__ void __launch_bounds__(256, 2) mv_up_df_kernel(int D, int K, const float* __restrict__ Xh,
                                                          const float* __restrict__ Xl, const float* __restrict__ zh,
                                                          const float* __restrict__ zl, float* __restrict__ oh,
                                                          float* __restrict__ ol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* szh = reinterpret_cast<float*>(smraw);  // D
  float* szl = szh + D;                          // D
  float* ph = szl + D;                           // 8 * K
  float* pl = ph + 8 * K;                        // 8 * K
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < D; e += blockDim.x) szh[e] = zh[(int64_t)i * D + e], szl[e] = zl[(int64_t)i * D + e];
  __syncthreads();
  const float* Mh = Xh + (int64_t)i * D * K;
  const float* Ml = Xl + (int64_t)i * D * K;
  if (K % 4 == 0) {
    for (int m0 = lane * 4; m0 < K; m0 += 128) {
      float H[4] = {0.f, 0.f, 0.f, 0.f}, L[4] = {0.f, 0.f, 0.f, 0.f};
      constexpr int NU = 8;  // rows in flight per lane
      int n = warp;
      for (; n + 8 * (NU - 1) < D; n += 8 * NU) {
        float4 vh[NU], vl[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          vh[u] = __ldg(reinterpret_cast<const float4*>(Mh + (int64_t)(n + 8 * u) * K + m0));
          vl[u] = __ldg(reinterpret_cast<const float4*>(Ml + (int64_t)(n + 8 * u) * K + m0));
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const float a = szh[n + 8 * u], b = szl[n + 8 * u];
          df_fma(H[0], L[0], vh[u].x, vl[u].x, a, b);
          df_fma(H[1], L[1], vh[u].y, vl[u].y, a, b);
          df_fma(H[2], L[2], vh[u].z, vl[u].z, a, b);
          df_fma(H[3], L[3], vh[u].w, vl[u].w, a, b);
        }
      }
      for (; n < D; n += 8) {
        const float4 vh = __ldg(reinterpret_cast<const float4*>(Mh + (int64_t)n * K + m0));
        const float4 vl = __ldg(reinterpret_cast<const float4*>(Ml + (int64_t)n * K + m0));
        const float a = szh[n], b = szl[n];
        df_fma(H[0], L[0], vh.x, vl.x, a, b);
        df_fma(H[1], L[1], vh.y, vl.y, a, b);
        df_fma(H[2], L[2], vh.z, vl.z, a, b);
        df_fma(H[3], L[3], vh.w, vl.w, a, b);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) ph[warp * K + m0 + e] = H[e], pl[warp * K + m0 + e] = L[e];
    }
  } else {
    for (int m = lane; m < K; m += 32) {
      float H = 0.f, L = 0.f;
      for (int n = warp; n < D; n += 8) df_fma(H, L, Mh[(int64_t)n * K + m], Ml[(int64_t)n * K + m], szh[n], szl[n]);
      ph[warp * K + m] = H, pl[warp * K + m] = L;
    }
  }
  __syncthreads();
  for (int m = tid; m < K; m += blockDim.x) {
    float H = ph[m], L = pl[m];
#pragma unroll
    for (int w = 1; w < 8; ++w) df_add(H, L, ph[w * K + m], pl[w * K + m]);
    oh[(int64_t)i * K + m] = H;
    ol[(int64_t)i * K + m] = L;
  }
}
void launch_matvec_up_df(const DevLevel& L, const float* Xh, const float* Xl, const float* zh, const float* zl,
                         float* oh, float* ol, cudaStream_t st) {
  const size_t sm = sizeof(float) * (2 * (size_t)L.D + 16 * (size_t)L.K);
  set_smem((const void*)mv_up_df_kernel, sm);
  ++g_launches;
  mv_up_df_kernel<<<L.nb, 256, sm, st>>>(L.D, L.K, Xh, Xl, zh, zl, oh, ol);
}

// couplings of every level in one launch: CTA (box i of level l, rows
// 64 c .. 64 c + 63) forms those rows of yhat_i = sum_{far j} S_ij xhat_j;
// the levels run in the order given (longest far lists first)
__global__ void __launch_bounds__(256, 2) mv_far_df_all_kernel(const __grid_constant__ FarDfArgs a) {
  const int b = blockIdx.x;
  int l = 0;
  while (l + 1 < a.nlev && b >= a.lv[l + 1].cta0) ++l;
  const FarDfLevel& f = a.lv[l];
  const int loc = b - f.cta0, i = loc / f.nch, r0 = (loc % f.nch) * 8 * kRPWdf;
  const int64_t p0 = f.ptr[i], p1 = f.ptr[i + 1];
  const int K = f.K;
  float H[kRPWdf], L[kRPWdf];
  zero(H);
  zero(L);
  for (int64_t q = p0; q < p1; ++q) {
    const int j = f.fj[q];
    rows_acc_df<kRPWdf>(r0, f.Sh + q * K * K, f.Sl + q * K * K, K, K, K, f.xh + (int64_t)j * K, f.xl + (int64_t)j * K,
                        H, L);
  }
  rows_finish_pair<kRPWdf>(r0, K, H, L, f.yh + (int64_t)i * K, f.yl + (int64_t)i * K, false);
}
void launch_matvec_far_df_all(const FarDfArgs& a, cudaStream_t st) {
  if (a.nlev <= 0) return;
  const FarDfLevel& last = a.lv[a.nlev - 1];
  const int grid = last.cta0 + last.nb * last.nch;
  if (grid <= 0) return;
  ++g_launches;
  mv_far_df_all_kernel<<<grid, 256, 0, st>>>(a);
}

// downward: [yhat_2p; yhat_2p+1] += X_p yhat_p in pairs
__global__ void __launch_bounds__(256, 2) mv_down_df_kernel(int D, int K, const float* __restrict__ Xh,
                                                            const float* __restrict__ Xl, const float* __restrict__ yh,
                                                            const float* __restrict__ yl, float* __restrict__ ych,
                                                            float* __restrict__ ycl) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Kp = (K + 3) & ~3;
  float* sh = reinterpret_cast<float*>(smraw);  // Kp
  float* sl = sh + Kp;                          // Kp
  const int p = blockIdx.x;
  for (int e = threadIdx.x; e < K; e += blockDim.x) sh[e] = yh[(int64_t)p * K + e], sl[e] = yl[(int64_t)p * K + e];
  __syncthreads();
  float H[kRPWdf], L[kRPWdf];
  for (int r0 = 0; r0 < D; r0 += 8 * kRPWdf) {
    zero(H);
    zero(L);
    rows_acc_df<kRPWdf>(r0, Xh + (int64_t)p * D * K, Xl + (int64_t)p * D * K, K, D, K, sh, sl, H, L);
    rows_finish_pair<kRPWdf>(r0, D, H, L, ych + (int64_t)p * D, ycl + (int64_t)p * D, true);
  }
}
void launch_matvec_down_df(const DevLevel& L, const float* Xh, const float* Xl, const float* yh, const float* yl,
                           float* ych, float* ycl, cudaStream_t st) {
  const size_t sm = 2 * sizeof(float) * (size_t)((L.K + 3) & ~3);
  ++g_launches;
  mv_down_df_kernel<<<L.nb, 256, sm, st>>>(L.D, L.K, Xh, Xl, yh, yl, ych, ycl);
}

// leaf output of the symmetric form: y_i = X_i yhat_i + box i's partial
// products (pairs, in list order), converted to FP64 once per entry
__global__ void __launch_bounds__(256, 2) mv_sym_sum_df_kernel(int D, int K, const int64_t* __restrict__ ptr,
                                                               const int32_t* __restrict__ ent,
                                                               const float* __restrict__ Xh,
                                                               const float* __restrict__ Xl,
                                                               const float* __restrict__ yhh,
                                                               const float* __restrict__ yhl,
                                                               const float* __restrict__ ph,
                                                               const float* __restrict__ pl, double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Kp = (K + 3) & ~3;
  float* shh = reinterpret_cast<float*>(smraw);  // Kp
  float* shl = shh + Kp;                         // Kp
  float* sbh = shl + Kp;                         // D
  float* sbl = sbh + D;                          // D
  const int i = blockIdx.x;
  const int64_t e0 = ptr[i], e1 = ptr[i + 1];
  if (Xh)
    for (int e = threadIdx.x; e < K; e += blockDim.x) shh[e] = yhh[(int64_t)i * K + e], shl[e] = yhl[(int64_t)i * K + e];
  for (int r = threadIdx.x; r < D; r += blockDim.x) {
    float H = 0.f, L = 0.f;
    for (int64_t q = e0; q < e1; ++q) {
      const int en = ent[q];
      const int64_t g = (int64_t)(en >> 1) * 2 * D + (en & 1) * D + r;
      df_add(H, L, ph[g], pl[g]);
    }
    sbh[r] = H, sbl[r] = L;
  }
  __syncthreads();
  if (Xh) {
    float H[kRPWdf], L[kRPWdf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 0; r0 < D; r0 += 8 * kRPWdf) {
      zero(H);
      zero(L);
      rows_acc_df<kRPWdf>(r0, Xh + (int64_t)i * D * K, Xl + (int64_t)i * D * K, K, D, K, shh, shl, H, L);
      float th, tl;
      df_tsum<kRPWdf, 32>(H, L, th, tl);
      const int r = r0 + warp + 8 * tsum_index<kRPWdf, 32>(lane);
      if (tsum_leader<kRPWdf, 32>(lane) && r < D) {
        df_add(th, tl, sbh[r], sbl[r]);
        y[(int64_t)i * D + r] = (double)th + (double)tl;
      }
    }
  } else {
    for (int r = threadIdx.x; r < D; r += blockDim.x) y[(int64_t)i * D + r] = (double)sbh[r] + (double)sbl[r];
  }
}
void launch_matvec_sym_sum_df(int nb, int D, int K, const int64_t* ptr, const int32_t* ent, const float* Xh,
                              const float* Xl, const float* yhh, const float* yhl, const float* ph, const float* pl,
                              double* y, cudaStream_t st) {
  const size_t sm = sizeof(float) * (2 * (size_t)((K + 3) & ~3) + 2 * (size_t)D);
  ++g_launches;
  mv_sym_sum_df_kernel<<<nb, 256, sm, st>>>(D, K, ptr, ent, Xh, Xl, yhh, yhl, ph, pl, y);
}

// lo[e] = fl32(a[e] - hi[e]) (hi = fl32(a))
__global__ void split_lo_kernel(const double* __restrict__ a, const float* __restrict__ hi, float* __restrict__ lo,
                                int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    lo[e] = (float)(a[e] - (double)hi[e]);
}
void launch_split_lo(const double* a, const float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ++g_launches;
  split_lo_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(a, hi, lo, n);
}

// -------------------------------------------- symmetric leaf near blocks ---
// The leaf near blocks of a symmetric kernel satisfy A_ji = A_ij^T, so the
// inner solver's matvec keeps only the blocks with i <= j ("stored pairs")
// and reads each once: the CTA of stored pair k = (a, b) forms
// u = A_ab x_b (for box a) and, when a != b, w = A_ab^T x_a (for box b)
// into part[k] = [u; w]; a per-box kernel then adds y_i = X_i yh_i + the
// partial products of the box (listed in ent: 2k for a u, 2k + 1 for a w).
// Warp w takes the rows r = w, w + 8, ... of the block, each lane a
// 4-column chunk per 128 columns: u needs one warp reduction per row, w
// stays in the lane's registers and the 8 warps' partial w meet in shared
// memory.
constexpr int kSymRPW = 8;  // rows per warp in flight

template <int CH>  // 4-column chunks per lane: D = 128 CH
__global__ void __launch_bounds__(256, 2) mv_sym_pair_kernel(int D, int64_t npu, const int32_t* __restrict__ ui,
                                                             const int32_t* __restrict__ uj,
                                                             const float* __restrict__ A, const float* __restrict__ x,
                                                             float* __restrict__ part, int pf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* xa = reinterpret_cast<float*>(smraw);  // D
  float* wp = xa + D;                           // 8 * D
  const int64_t k = blockIdx.x;
  const int a = ui[k], b = uj[k], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool both = a != b;
  const float* M = A + k * D * D;
  if (pf) prefetch_l2(M, (int64_t)D * D * sizeof(float));
  griddep_wait();
  griddep_launch_next();
  for (int e = tid; e < D; e += blockDim.x) xa[e] = x[(int64_t)a * D + e];
  float xb[CH][4];
#pragma unroll
  for (int h = 0; h < CH; ++h) {
    const float4 v = *reinterpret_cast<const float4*>(x + (int64_t)b * D + lane * 4 + 128 * h);
    xb[h][0] = v.x, xb[h][1] = v.y, xb[h][2] = v.z, xb[h][3] = v.w;
  }
  float wacc[CH][4];
#pragma unroll
  for (int h = 0; h < CH; ++h)
#pragma unroll
    for (int e = 0; e < 4; ++e) wacc[h][e] = 0.0f;
  __syncthreads();
  float* u = part + k * 2 * D;
  for (int r0 = warp; r0 < D; r0 += 8 * kSymRPW) {
    float4 v[kSymRPW][CH];
#pragma unroll
    for (int t = 0; t < kSymRPW; ++t) {
      const int r = r0 + 8 * t;
#pragma unroll
      for (int h = 0; h < CH; ++h)
        v[t][h] = (r < D) ? __ldg(reinterpret_cast<const float4*>(M + (int64_t)r * D + lane * 4 + 128 * h))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float su[kSymRPW];
#pragma unroll
    for (int t = 0; t < kSymRPW; ++t) {
      const int r = r0 + 8 * t;
      const float xr = (r < D) ? xa[r] : 0.0f;
      float s = 0.0f;
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        s = fmaf(v[t][h].x, xb[h][0], s);
        s = fmaf(v[t][h].y, xb[h][1], s);
        s = fmaf(v[t][h].z, xb[h][2], s);
        s = fmaf(v[t][h].w, xb[h][3], s);
        wacc[h][0] = fmaf(v[t][h].x, xr, wacc[h][0]);
        wacc[h][1] = fmaf(v[t][h].y, xr, wacc[h][1]);
        wacc[h][2] = fmaf(v[t][h].z, xr, wacc[h][2]);
        wacc[h][3] = fmaf(v[t][h].w, xr, wacc[h][3]);
      }
      su[t] = s;
    }
    {
      const float sv = tsum<kSymRPW, 32, float>(su);
      const int r = r0 + 8 * tsum_index<kSymRPW, 32>(lane);
      if (tsum_leader<kSymRPW, 32>(lane) && r < D) u[r] = sv;
    }
  }
  if (!both) return;
#pragma unroll
  for (int h = 0; h < CH; ++h)
    *reinterpret_cast<float4*>(wp + warp * D + lane * 4 + 128 * h) =
        make_float4(wacc[h][0], wacc[h][1], wacc[h][2], wacc[h][3]);
  __syncthreads();
  for (int c = tid; c < D; c += blockDim.x) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += wp[w * D + c];
    u[D + c] = s;
  }
}

// y_i = X_i yh_i + sum of box i's partial products (in list order)
template <typename T>
__global__ void __launch_bounds__(256) mv_sym_sum_kernel(int D, int K, const int64_t* __restrict__ ptr,
                                                         const int32_t* __restrict__ ent, const T* __restrict__ X,
                                                         const T* __restrict__ yh, const T* __restrict__ part,
                                                         T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sh = reinterpret_cast<T*>(smraw);  // K
  T* sb = sh + ((K + 3) & ~3);          // D
  const int i = blockIdx.x;
  const int64_t e0 = ptr[i], e1 = ptr[i + 1];
  auto hook = [&] {
    griddep_wait();
    griddep_launch_next();
    for (int e = threadIdx.x; e < K; e += blockDim.x) sh[e] = yh[(int64_t)i * K + e];
    for (int r = threadIdx.x; r < D; r += blockDim.x) {
      T s = T(0);
      int64_t q = e0;
      for (; q + 4 <= e1; q += 4) {
        T v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int en = ent[q + t];
          v[t] = part[(int64_t)(en >> 1) * 2 * D + (en & 1) * D + r];
        }
        s += (v[0] + v[1]) + (v[2] + v[3]);
      }
      for (; q < e1; ++q) {
        const int en = ent[q];
        s += part[(int64_t)(en >> 1) * 2 * D + (en & 1) * D + r];
      }
      sb[r] = s;
    }
    __syncthreads();
  };
  if (X) {
    cta_gemv<T, T, Unr<T>::v>(X + (int64_t)i * D * K, K, D, K, sh, T(1), sb, y + (int64_t)i * D, hook);
  } else {
    hook();
    for (int r = threadIdx.x; r < D; r += blockDim.x) y[(int64_t)i * D + r] = sb[r];
  }
}

// FP32-pair form for the residual (see df_fma): A as hi + lo, x as FP32
// pairs xh + xl, partial products as FP32 pairs (ph + pl, 2 D per stored
// pair).  A row's lanes are added by df_tsum and the lane that keeps the row
// (lane k keeps the row of pass k mod 16 and half k / 16) stores it after
// the last pass; the column sums of A^T x_i are added over the warps.
template <int CH>
__global__ void __launch_bounds__(256, 2) mv_sym_pair_df_kernel(int D, int64_t npu, const int32_t* __restrict__ ui,
                                                                const int32_t* __restrict__ uj,
                                                                const float* __restrict__ Ah,
                                                                const float* __restrict__ Al,
                                                                const float* __restrict__ xh,
                                                                const float* __restrict__ xl,
                                                                float* __restrict__ ph, float* __restrict__ pl) {
  constexpr int RPW = 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* xah = reinterpret_cast<float*>(smraw);  // D
  float* xal = xah + D;                          // D
  float* wph = xal + D;                          // 8 * D column partials (high parts)
  float* wpl = wph + 8 * D;                      // 8 * D (low parts)
  const int64_t k = blockIdx.x;
  const int a = ui[k], b = uj[k], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool both = a != b;
  const float* Mh = Ah + k * D * D;
  const float* Ml = Al + k * D * D;
  for (int e = tid; e < D; e += blockDim.x) xah[e] = xh[(int64_t)a * D + e], xal[e] = xl[(int64_t)a * D + e];
  float xbh[CH][4], xbl[CH][4];
#pragma unroll
  for (int h = 0; h < CH; ++h) {
    const float4 vh = *reinterpret_cast<const float4*>(xh + (int64_t)b * D + lane * 4 + 128 * h);
    const float4 vl = *reinterpret_cast<const float4*>(xl + (int64_t)b * D + lane * 4 + 128 * h);
    xbh[h][0] = vh.x, xbh[h][1] = vh.y, xbh[h][2] = vh.z, xbh[h][3] = vh.w;
    xbl[h][0] = vl.x, xbl[h][1] = vl.y, xbl[h][2] = vl.z, xbl[h][3] = vl.w;
  }
  float wH[CH][4], wL[CH][4];
#pragma unroll
  for (int h = 0; h < CH; ++h)
#pragma unroll
    for (int e = 0; e < 4; ++e) wH[h][e] = 0.0f, wL[h][e] = 0.0f;
  __syncthreads();
  float* uh = ph + k * 2 * D;
  float* ul = pl + k * 2 * D;
  // rows r0 + 8 t (t < RPW) of this warp; the next group's loads are issued
  // before the current group is used
  auto load_rows = [&](int r0, float4 (&vh)[RPW][CH], float4 (&vl)[RPW][CH]) {
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int r = r0 + 8 * t;
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int64_t off = (int64_t)r * D + lane * 4 + 128 * h;
        vh[t][h] = (r < D) ? __ldg(reinterpret_cast<const float4*>(Mh + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
        vl[t][h] = (r < D) ? __ldg(reinterpret_cast<const float4*>(Ml + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  float4 nh[RPW][CH], nl[RPW][CH];
  load_rows(warp, nh, nl);
  float keep_h = 0.0f, keep_l = 0.0f;  // the row this lane stores at the end
  for (int r0 = warp, it = 0; r0 < D; r0 += 8 * RPW, ++it) {
    float4 vh[RPW][CH], vl[RPW][CH];
#pragma unroll
    for (int t = 0; t < RPW; ++t)
#pragma unroll
      for (int h = 0; h < CH; ++h) vh[t][h] = nh[t][h], vl[t][h] = nl[t][h];
    if (r0 + 8 * RPW < D) load_rows(r0 + 8 * RPW, nh, nl);
    float rh[RPW], rl[RPW];
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int r = r0 + 8 * t;
      const float xrh = (r < D) ? xah[r] : 0.0f, xrl = (r < D) ? xal[r] : 0.0f;
      float H = 0.0f, L = 0.0f;
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const float mh[4] = {vh[t][h].x, vh[t][h].y, vh[t][h].z, vh[t][h].w};
        const float ml[4] = {vl[t][h].x, vl[t][h].y, vl[t][h].z, vl[t][h].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          df_fma(H, L, mh[e], ml[e], xbh[h][e], xbl[h][e]);
          if (both) df_fma(wH[h][e], wL[h][e], mh[e], ml[e], xrh, xrl);
        }
      }
      rh[t] = H, rl[t] = L;
    }
    float sh, sl;
    df_tsum<RPW, 32>(rh, rl, sh, sl);  // lanes 0-15: row r0, lanes 16-31: row r0 + 8
    if ((lane & 15) == it) keep_h = sh, keep_l = sl;
  }
  {
    const int r = warp + 8 * RPW * (lane & 15) + 8 * (lane >> 4);
    if (r < D) uh[r] = keep_h, ul[r] = keep_l;
  }
  if (!both) return;
#pragma unroll
  for (int h = 0; h < CH; ++h)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      wph[warp * D + lane * 4 + 128 * h + e] = wH[h][e];
      wpl[warp * D + lane * 4 + 128 * h + e] = wL[h][e];
    }
  __syncthreads();
  for (int c = tid; c < D; c += blockDim.x) {
    float H = wph[c], L = wpl[c];
#pragma unroll
    for (int w = 1; w < 8; ++w) df_add(H, L, wph[w * D + c], wpl[w * D + c]);
    uh[D + c] = H, ul[D + c] = L;
  }
}

bool sym_leaf_supported(int D) { return D == 128 || D == 256; }

template <int CH>
static void launch_sym_pairs_ch(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* A,
                                const float* x, float* part, bool pdl, cudaStream_t st) {
  const size_t sm = sizeof(float) * 9 * (size_t)D;
  set_smem((const void*)mv_sym_pair_kernel<CH>, sm);
  const int pf = small_level(npu) ? 1 : 0;
  if (pdl) {
    launch_pdl(mv_sym_pair_kernel<CH>, (unsigned)npu, 256, sm, st, D, npu, ui, uj, A, x, part, pf);
  } else {
    ++g_launches;
    mv_sym_pair_kernel<CH><<<(unsigned)npu, 256, sm, st>>>(D, npu, ui, uj, A, x, part, pf);
  }
}
void launch_matvec_sym_pairs(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* A, const float* x,
                             float* part, bool pdl, cudaStream_t st) {
  if (npu <= 0) return;
  switch (D / 128) {
    case 1: launch_sym_pairs_ch<1>(D, npu, ui, uj, A, x, part, pdl, st); break;
    case 2: launch_sym_pairs_ch<2>(D, npu, ui, uj, A, x, part, pdl, st); break;
    default: launch_sym_pairs_ch<2>(D, npu, ui, uj, A, x, part, pdl, st); break;
  }
}
template <int CH>
static void launch_sym_pairs_df_ch(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* Ah,
                                   const float* Al, const float* xh, const float* xl, float* ph, float* pl,
                                   cudaStream_t st) {
  const size_t sm = sizeof(float) * 18 * (size_t)D;
  set_smem((const void*)mv_sym_pair_df_kernel<CH>, sm);
  ++g_launches;
  mv_sym_pair_df_kernel<CH><<<(unsigned)npu, 256, sm, st>>>(D, npu, ui, uj, Ah, Al, xh, xl, ph, pl);
}
void launch_matvec_sym_pairs_df(int D, int64_t npu, const int32_t* ui, const int32_t* uj, const float* Ah,
                                const float* Al, const float* xh, const float* xl, float* ph, float* pl,
                                cudaStream_t st) {
  if (npu <= 0) return;
  switch (D / 128) {
    case 1: launch_sym_pairs_df_ch<1>(D, npu, ui, uj, Ah, Al, xh, xl, ph, pl, st); break;
    case 2: launch_sym_pairs_df_ch<2>(D, npu, ui, uj, Ah, Al, xh, xl, ph, pl, st); break;
    default: launch_sym_pairs_df_ch<2>(D, npu, ui, uj, Ah, Al, xh, xl, ph, pl, st); break;
  }
}
template <typename T>
void launch_matvec_sym_sum(int nb, int D, int K, const int64_t* ptr, const int32_t* ent, const T* X, const T* yh,
                           const T* part, T* y, cudaStream_t st, bool pdl) {
  const size_t sm = sizeof(T) * ((size_t)((K + 3) & ~3) + D);
  if (pdl) {
    launch_pdl(mv_sym_sum_kernel<T>, nb, 256, sm, st, D, K, ptr, ent, X, yh, part, y);
  } else {
    ++g_launches;
    mv_sym_sum_kernel<T><<<nb, 256, sm, st>>>(D, K, ptr, ent, X, yh, part, y);
  }
}
template void launch_matvec_sym_sum<float>(int, int, int, const int64_t*, const int32_t*, const float*, const float*,
                                           const float*, float*, cudaStream_t, bool);

// out[k] = (To) in[idx[k]] for blocks of n entries
template <typename Ti, typename To>
__global__ void gather_blocks_kernel(const Ti* __restrict__ in, const int32_t* __restrict__ idx, int64_t n,
                                     int64_t nblk, To* __restrict__ out) {
  const int64_t total = n * nblk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / n, r = e - k * n;
    out[e] = (To)in[(int64_t)idx[k] * n + r];
  }
}
void launch_gather_blocks(const double* in, const int32_t* idx, int64_t n, int64_t nblk, float* out, cudaStream_t st) {
  if (n * nblk <= 0) return;
  ++g_launches;
  gather_blocks_kernel<double, float><<<(unsigned)std::min<int64_t>((n * nblk + 255) / 256, 152 * 32), 256, 0, st>>>(
      in, idx, n, nblk, out);
}
// lo[k] = fl32(in[idx[k]] - hi[k])
__global__ void gather_split_lo_kernel(const double* __restrict__ in, const int32_t* __restrict__ idx, int64_t n,
                                       int64_t nblk, const float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t total = n * nblk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / n, r = e - k * n;
    lo[e] = (float)(in[(int64_t)idx[k] * n + r] - (double)hi[e]);
  }
}
void launch_gather_split_lo(const double* in, const int32_t* idx, int64_t n, int64_t nblk, const float* hi, float* lo,
                            cudaStream_t st) {
  if (n * nblk <= 0) return;
  ++g_launches;
  gather_split_lo_kernel<<<(unsigned)std::min<int64_t>((n * nblk + 255) / 256, 152 * 32), 256, 0, st>>>(in, idx, n,
                                                                                                        nblk, hi, lo);
}

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
// (a product a b added to the FP32 pair (H, L): a fused multiply-add splits
// it exactly into p + e)
__device__ __forceinline__ void df_acc(float& H, float& L, float a, float b) {
  const float p = __fmul_rn(a, b);
  df_add(H, L, p, fmaf(a, b, -p));
}
// The block's FP32-pair partial (H, L) as one FP64 value, by thread 0: lanes
// and warps are added in FP32 pairs (FP64 instructions are slow on GB300).
__device__ __forceinline__ double block_df_total(float H, float L) {
  __shared__ float bh[8], bl[8];
  float rh[1] = {H}, rl[1] = {L}, sh, sl;
  df_tsum<1, 32>(rh, rl, sh, sl);
  if ((threadIdx.x & 31) == 0) bh[threadIdx.x >> 5] = sh, bl[threadIdx.x >> 5] = sl;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    float th = bh[0], tl = bl[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) df_add(th, tl, bh[w], bl[w]);
    t = (double)th + (double)tl;
  }
  return t;
}

template <typename T>
__global__ void norm2_part_kernel(const T* __restrict__ v, int64_t n, double* __restrict__ part) {
  if constexpr (std::is_same<T, float>::value) {
    float H = 0.0f, L = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
      df_acc(H, L, v[e], v[e]);
    const double t = block_df_total(H, L);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    return;
  }
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
// (the scale is formed once per block: an FP64 square root and division per
// thread would cost more than the copy on GB300; FP32 data are scaled in FP32)
template <typename Ti, typename To>
__global__ void scaled_copy_kernel(const Ti* __restrict__ in, const double* __restrict__ nrm2, int inverse,
                                   To* __restrict__ out, int64_t n) {
  __shared__ double ss;
  if (threadIdx.x == 0) {
    double s = 1.0;
    if (nrm2) {
      const double r = sqrt(nrm2[0]);
      s = inverse ? (r > 0 ? 1.0 / r : 0.0) : r;
    }
    ss = s;
  }
  __syncthreads();
  const double s = ss;
  if constexpr (std::is_same<Ti, float>::value && std::is_same<To, float>::value) {
    const float sf = (float)s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
      out[e] = in[e] * sf;
  } else {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
      out[e] = (To)((double)in[e] * s);
  }
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
  __shared__ double ss;
  if (threadIdx.x == 0) ss = nrm2[0] > 0 ? 1.0 / sqrt(nrm2[0]) : 1.0;
  __syncthreads();
  const double s = ss;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)(in[e] * s);
}
template <typename T>
__global__ void axpy_from_kernel(const T* __restrict__ d, const double* __restrict__ nrm2, double* __restrict__ x,
                                 int64_t n) {
  __shared__ double ss;
  if (threadIdx.x == 0) ss = nrm2[0] > 0 ? sqrt(nrm2[0]) : 1.0;
  __syncthreads();
  const double s = ss;
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
  const int v = blockIdx.y;
  const T* Vv = V + (int64_t)v * ldv;
  if constexpr (std::is_same<T, float>::value) {
    float H = 0.0f, L = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
      df_acc(H, L, Vv[e], w[e]);
    const double t = block_df_total(H, L);
    if (threadIdx.x == 0) part[(int64_t)v * gridDim.x + blockIdx.x] = t;
    return;
  }
  __shared__ double sb[8];
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
// The FP32 form (nv <= kAxpyPairs): the coefficients as FP32 pairs in shared
// memory (split once per block), the combination in FP32-pair arithmetic,
// w rounded to FP32 once.
constexpr int kAxpyPairs = 128;
__global__ void multi_axpy_f32_kernel(const float* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ coef,
                                      float sign, float* __restrict__ w, int64_t n) {
  __shared__ float ch[kAxpyPairs], cl[kAxpyPairs];
  for (int v = threadIdx.x; v < nv; v += blockDim.x) df_split(coef[v], ch[v], cl[v]);
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float H = 0.0f, L = 0.0f;
    for (int v = 0; v < nv; ++v) {
      const float x = V[(int64_t)v * ldv + e];
      df_acc(H, L, ch[v], x);
      L = fmaf(cl[v], x, L);
    }
    float wh = w[e], wl = 0.0f;
    df_add(wh, wl, sign * H, sign * L);
    w[e] = wh + wl;
  }
}
template <typename T, typename TW>
void launch_multi_axpy(const T* V, int64_t ldv, int nv, const double* coef, double sign, TW* w, int64_t n,
                       cudaStream_t st) {
  if (nv == 0) return;
  ++g_launches;
  if constexpr (std::is_same<T, float>::value && std::is_same<TW, float>::value) {
    if (nv <= kAxpyPairs) {
      multi_axpy_f32_kernel<<<grid_for(n), 256, 0, st>>>(V, ldv, nv, coef, (float)sign, w, n);
      return;
    }
  }
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
