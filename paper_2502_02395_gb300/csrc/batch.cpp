// Batches of independent systems (uneven N, per-cluster ranks): every
// system keeps its own context (instance, factorization, CUDA graphs of its
// substitution), and a pool of host workers, each with its own CUDA stream,
// factors and solves them concurrently, largest first, so that small
// systems that cannot fill the GPU alone share it.  The pool size is chosen
// by measurement (h2_batch_tune).  Built on the C ABI of the single-system
// solver; no counterpart in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/h2ulv.h"

struct h2_batch {
  std::vector<h2_ctx*> ctx;
  std::vector<int64_t> n;  // N of each system
  int workers = 4;
  std::vector<cudaStream_t> streams;
  std::string err;
  double last_seconds = 0;
  std::vector<double> tune_seconds;  // by worker count 1, 2, 4, 8, 16 (0: not tried)
};

namespace {

h2_status ensure_streams(h2_batch* b, int w) {
  while ((int)b->streams.size() < w) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      b->err = "cudaStreamCreate failed";
      return H2_ERR_CUDA;
    }
    b->streams.push_back(s);
  }
  return H2_OK;
}

// Factor (prec >= 0) and/or solve (B != NULL) every system with `w` workers.
h2_status run(h2_batch* b, int w, int32_t prec, const double* const* B, double* const* X, double target,
              int32_t max_iters, double* relres, int32_t* iters) {
  const int ns = (int)b->ctx.size();
  h2_status s = ensure_streams(b, w);
  if (s != H2_OK) return s;
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->n[a] > b->n[c]; });
  std::atomic<int> next{0};
  std::vector<h2_status> st(ns, H2_OK);
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&](int k) {
    cudaSetDevice(dev);
    for (;;) {
      const int t = next.fetch_add(1);
      if (t >= ns) break;
      const int i = order[t];
      h2_ctx* c = b->ctx[i];
      h2_status r = h2_set_stream(c, b->streams[k]);
      if (r == H2_OK && prec >= 0) r = h2_factor(c, prec);
      if (r == H2_OK && B) {
        double rel = 0;
        int32_t its = 0;
        r = h2_solve(c, B[i], X[i], target, max_iters, &rel, &its);
        if (relres) relres[i] = rel;
        if (iters) iters[i] = its;
      }
      if (r == H2_OK) r = cudaStreamSynchronize(b->streams[k]) == cudaSuccess ? H2_OK : H2_ERR_CUDA;
      st[i] = r;
    }
  };
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<std::thread> pool;
  for (int k = 1; k < w; ++k) pool.emplace_back(worker, k);
  worker(0);
  for (auto& th : pool) th.join();
  b->last_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < ns; ++i)
    if (st[i] != H2_OK) {
      b->err = "system " + std::to_string(i) + ": " + h2_last_error(b->ctx[i]);
      return st[i];
    }
  return H2_OK;
}

}  // namespace

extern "C" {

h2_status h2_batch_create(h2_batch** out, h2_ctx* const* ctxs, const int64_t* n, int32_t count) {
  if (!out || !ctxs || !n || count < 1) return H2_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!ctxs[i] || n[i] < 1) return H2_ERR_INVALID_ARG;
  h2_batch* b = new h2_batch();
  b->ctx.assign(ctxs, ctxs + count);
  b->n.assign(n, n + count);
  b->tune_seconds.assign(5, 0.0);
  *out = b;
  return H2_OK;
}

h2_status h2_batch_run(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                       int32_t max_iters, double* relres, int32_t* iters, double* seconds) {
  if (!b || (prec < -1 || prec > H2_PREC_BF16) || (B && !X) || (prec < 0 && !B)) return H2_ERR_INVALID_ARG;
  b->err.clear();
  h2_status s = run(b, b->workers, prec, B, X, target, max_iters, relres, iters);
  if (seconds) *seconds = b->last_seconds;
  return s;
}

h2_status h2_batch_tune(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                        int32_t max_iters, int32_t* workers_out) {
  if (!b || prec < 0 || prec > H2_PREC_BF16 || !B || !X) return H2_ERR_INVALID_ARG;
  b->err.clear();
  const int cand[5] = {1, 2, 4, 8, 16};
  double best = INFINITY;
  int bw = b->workers;
  h2_status last = H2_OK;
  for (int k = 0; k < 5; ++k) {
    if (cand[k] > 2 * (int)b->ctx.size()) break;
    // a system that stops above the target still gives a timing
    h2_status s = run(b, cand[k], prec, B, X, target, max_iters, nullptr, nullptr);
    if (s != H2_OK && s != H2_ERR_NOT_CONVERGED) return s;
    last = s;
    b->tune_seconds[k] = b->last_seconds;
    if (b->last_seconds < best) best = b->last_seconds, bw = cand[k];
  }
  b->workers = bw;
  if (workers_out) *workers_out = bw;
  return last;
}

h2_status h2_batch_stats(const h2_batch* b, char* json, size_t cap) {
  if (!b || !json) return H2_ERR_INVALID_ARG;
  std::string o = "{\"systems\":" + std::to_string(b->ctx.size()) + ",\"workers\":" + std::to_string(b->workers) +
                  ",\"last_seconds\":" + std::to_string(b->last_seconds) + ",\"tune_seconds\":{";
  const int cand[5] = {1, 2, 4, 8, 16};
  bool first = true;
  for (int k = 0; k < 5; ++k) {
    if (b->tune_seconds[k] <= 0) continue;
    o += (first ? "\"" : ",\"") + std::to_string(cand[k]) + "\":" + std::to_string(b->tune_seconds[k]);
    first = false;
  }
  o += "}}";
  if (o.size() + 1 > cap) return H2_ERR_INVALID_ARG;
  std::memcpy(json, o.c_str(), o.size() + 1);
  return H2_OK;
}

const char* h2_batch_last_error(const h2_batch* b) { return b ? b->err.c_str() : ""; }

void h2_batch_destroy(h2_batch* b) {
  if (!b) return;
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  // the contexts go back to the legacy default stream (theirs were the
  // batch's worker streams)
  for (h2_ctx* c : b->ctx) h2_set_stream(c, nullptr);
  delete b;
}

}  // extern "C"
