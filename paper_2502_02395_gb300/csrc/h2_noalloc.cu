// y = A_H2 x without any device allocation at call time.
//
// Who needs this: code that has built its H^2 context up front but must not
// allocate device memory later — for example a host framework that hands
// out all device memory itself and forbids cudaMalloc from libraries, or a
// solver loop on a latency budget, where cudaMalloc / cudaFree may block or
// synchronize the device.  h2_matvec keeps its per-call scratch in buffers
// the context allocated at build time; this variant instead takes that
// scratch from one fixed array compiled into the library, so the call itself
// allocates nothing and touches no allocator.
//
// The scratch array: g_matvec_scratch below, 16 MiB (2^21 doubles).  A GPU
// holds it from the moment the library's module containing it is loaded on
// that device (with lazy module loading: the first h2_matvec_noalloc call
// there) until the process exits.  Every call on a device shares it and it
// keeps the previous call's contents; the matvec overwrites every entry it
// later reads, so nothing has to be cleared.  Two calls whose work overlaps
// on the GPU (different streams, or several contexts on one device) race on
// the array and give wrong results.
#include <mutex>

#include "h2_internal.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 21;  // 16 MiB
static __device__ __align__(256) double g_matvec_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array for the current device, looked up once per
// device (the first call on a device does this set-up).
h2_status scratch_address(int dev, double** out, std::string& err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal " + std::to_string(dev) + " out of range";
    return H2_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return H2_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return H2_OK;
}

// p is managed memory, or device memory of the context's device dev.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" h2_status h2_matvec_noalloc(h2_ctx* c, const double* x, double* y) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->A64) {
    c->err = "the FP64 leaf blocks were released (H2_OPT_FP64_LEAF)";
    return H2_ERR_STATE;
  }
  if (!x || !y || !on_device(x, c->dev) || !on_device(y, c->dev)) {
    c->err = "h2_matvec_noalloc needs device pointers on the context's device for x and y";
    return H2_ERR_INVALID_ARG;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->dev) {
    c->err = "h2_matvec_noalloc must run with the context's device current";
    return H2_ERR_INVALID_ARG;
  }
  const int L = c->L;
  const h2::DevLevel& lf = c->lv[L];
  const size_t nslot = (size_t)lf.nb * lf.D;
  const size_t nhat = (size_t)c->hat_off[L + 1];
  const size_t need = 2 * nslot + 2 * nhat;
  if (need > kScratchDoubles) {
    c->err = "h2_matvec_noalloc: the problem needs " + std::to_string(need) +
             " doubles of scratch; the fixed array holds " + std::to_string(kScratchDoubles);
    return H2_ERR_INVALID_ARG;
  }
  double* scr = nullptr;
  h2_status s = scratch_address(dev, &scr, c->err);
  if (s != H2_OK) return s;
  double* xt = scr;          // x in padded tree order
  double* yt = xt + nslot;   // y in padded tree order
  double* xh = yt + nslot;   // upward skeleton coefficients, per level
  double* yh = xh + nhat;    // downward skeleton coefficients, per level
  cudaStream_t st = c->stream;
  h2::launch_gather(c->slot_pt, x, xt, (int64_t)nslot, st);
  if (L == 0) {
    h2::launch_matvec_leaf<double>(c->lv[0], c->A64, nullptr, xt, nullptr, yt, st);
  } else {
    const std::vector<int64_t>& off = c->hat_off;
    h2::launch_matvec_up<double>(c->lv[L], c->lv[L].X, xt, xh + off[L], st);
    for (int l = L - 1; l >= 1; --l) h2::launch_matvec_up<double>(c->lv[l], c->lv[l].X, xh + off[l + 1], xh + off[l], st);
    for (int l = 1; l <= L; ++l) h2::launch_matvec_far<double>(c->lv[l], c->lv[l].S, xh + off[l], yh + off[l], st);
    for (int l = 1; l < L; ++l) h2::launch_matvec_down<double>(c->lv[l], c->lv[l].X, yh + off[l], yh + off[l + 1], st);
    h2::launch_matvec_leaf<double>(c->lv[L], c->A64, c->lv[L].X, xt, yh + off[L], yt, st);
  }
  h2::launch_scatter(c->slot_pt, yt, y, (int64_t)nslot, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("h2_matvec_noalloc: ") + cudaGetErrorString(e);
    return H2_ERR_CUDA;
  }
  return H2_OK;
}
