// Batches of independent systems (uneven N, per-cluster ranks), in one of
// two forms, both built on the C ABI of the single-system solver:
//  * pool: every system keeps its own context (instance, factorization,
//    CUDA graphs of its substitution), and a pool of host workers, each
//    with its own CUDA stream, factors and solves them concurrently,
//    largest first, so that small systems that cannot fill the GPU alone
//    share it;
//  * forest: the systems are grouped by tree depth and each group is one
//    instance (h2_build_forest), so every level of the factorization, the
//    substitution and the matvec is one launch per kernel over all systems
//    of the group, the constant-rank batching of Section 4.1 taken across
//    systems.  A group's systems are solved together: each right-hand side
//    is scaled to unit norm and the group is refined to target / sqrt(m)
//    (m systems), so that every system's residual, |r_s| <= |r|, is at most
//    target; each system's relative residual is then recomputed from one
//    FP64 matvec of the group.  The pool runs the groups.
// The worker count is chosen by measurement (h2_batch_tune).  No
// counterpart in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <condition_variable>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/h2ulv.h"

struct h2_batch {
  std::vector<h2_ctx*> ctx;  // pool: one per system; forest: one per group (owned)
  std::vector<int64_t> n;    // N of each context
  bool forest = false;
  // forest: the systems of group g (in its order), each system's group and
  // offset in the group's vector, and its N
  std::vector<std::vector<int>> group_sys;
  std::vector<int> sys_group;
  std::vector<int64_t> sys_off, sys_n;
  int workers = 4;
  std::string kernels;  // h2_autotune's choices on the largest context (JSON; "" before h2_batch_tune)
  std::vector<cudaStream_t> streams;
  std::string err;
  double last_seconds = 0;
  std::vector<double> tune_seconds;  // by worker count 1, 2, 4, 8, 16 (0: not tried)
};

namespace {

// One forest group's solve (see the file comment).  Host vectors of the
// group's N: the scaled right-hand sides, the solution and A_H2 x.
h2_status solve_group(h2_batch* b, int g, const double* const* B, double* const* X, double target,
                      int32_t max_iters, double* relres, int32_t* iters, std::string& msg) {
  const std::vector<int>& sys = b->group_sys[g];
  const int64_t ng = b->n[g];
  std::vector<double> bg(ng), xg(ng, 0.0), yg(ng);
  std::vector<double> nrm(sys.size(), 0.0);
  for (size_t k = 0; k < sys.size(); ++k) {
    const int s = sys[k];
    const double* bs = B[s];
    double q = 0;
    for (int64_t t = 0; t < b->sys_n[s]; ++t) q += bs[t] * bs[t];
    nrm[k] = std::sqrt(q);
    const double inv = nrm[k] > 0 ? 1.0 / nrm[k] : 0.0;
    for (int64_t t = 0; t < b->sys_n[s]; ++t) bg[b->sys_off[s] + t] = bs[t] * inv;
  }
  h2_ctx* c = b->ctx[g];
  double rel = 0;
  int32_t its = 0;
  const double tg = target > 0 ? target / std::sqrt((double)sys.size()) : target;
  h2_status r = h2_solve(c, bg.data(), xg.data(), tg, max_iters, &rel, &its);
  if (r != H2_OK && r != H2_ERR_NOT_CONVERGED) return r;
  // A_H2 x in FP32-pair arithmetic (about 2^-46 of the row sums; the FP64
  // leaf blocks are released)
  h2_status rm = h2_matvec_arith(c, xg.data(), yg.data(), 2);
  if (rm != H2_OK) return rm;
  int worst = -1;
  double wrel = 0;
  for (size_t k = 0; k < sys.size(); ++k) {
    const int s = sys[k];
    double q = 0;
    for (int64_t t = 0; t < b->sys_n[s]; ++t) {
      const int64_t e = b->sys_off[s] + t;
      q += (bg[e] - yg[e]) * (bg[e] - yg[e]);
      X[s][t] = xg[e] * nrm[k];
    }
    const double rs = nrm[k] > 0 ? std::sqrt(q) : 0.0;
    if (relres) relres[s] = rs;
    if (iters) iters[s] = its;
    if (target > 0 && rs > target && rs > wrel) wrel = rs, worst = s;
  }
  if (worst >= 0) {
    msg = "system " + std::to_string(worst) + " stopped at relative residual " + std::to_string(wrel);
    return H2_ERR_NOT_CONVERGED;
  }
  return H2_OK;
}

// A forest batch scales and splits its vectors on the host: B[s] and X[s]
// must be host memory there (a pool batch takes host or device vectors).
bool host_vectors(h2_batch* b, const double* const* B, double* const* X) {
  if (!b->forest) return true;
  for (size_t s = 0; s < b->sys_n.size(); ++s)
    for (const void* v : {(const void*)B[s], (const void*)X[s]}) {
      cudaPointerAttributes a{};
      if (!v) {
        b->err = "system " + std::to_string(s) + ": NULL vector";
        return false;
      }
      if (cudaPointerGetAttributes(&a, v) != cudaSuccess) {
        cudaGetLastError();
        continue;  // not known to CUDA: host memory
      }
      if (a.type == cudaMemoryTypeDevice) {
        b->err = "system " + std::to_string(s) + ": a forest batch takes host vectors";
        return false;
      }
    }
  return true;
}

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
  std::vector<std::string> msg(ns);
  // forest groups holding a factorization, and releases so far
  std::mutex mu;
  std::condition_variable cv;
  int holding = 0, released = 0;
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
      bool holds = false;
      if (r == H2_OK && prec >= 0) {
        if (b->forest) {
          std::lock_guard<std::mutex> lk(mu);
          ++holding;  // factoring or holding a factorization
          holds = true;
        }
        r = h2_factor(c, prec);
        // a forest group whose factorization does not fit waits until
        // another group releases its arrays (none left: the error stands)
        while (b->forest && r == H2_ERR_OOM) {
          std::unique_lock<std::mutex> lk(mu);
          --holding;
          holds = false;
          if (holding == 0) break;
          const int seen = released;
          cv.wait(lk, [&] { return released != seen || holding == 0; });
          ++holding;
          holds = true;
          lk.unlock();
          r = h2_factor(c, prec);
        }
        if (r != H2_OK && holds) {
          {
            std::lock_guard<std::mutex> lk(mu);
            --holding;
            ++released;
          }
          holds = false;
          cv.notify_all();
        }
      }
      if (r == H2_OK && B && !b->forest) {
        double rel = 0;
        int32_t its = 0;
        r = h2_solve(c, B[i], X[i], target, max_iters, &rel, &its);
        if (relres) relres[i] = rel;
        if (iters) iters[i] = its;
      } else if (r == H2_OK && B) {
        r = solve_group(b, i, B, X, target, max_iters, relres, iters, msg[i]);
      }
      if (r == H2_OK) r = cudaStreamSynchronize(b->streams[k]) == cudaSuccess ? H2_OK : H2_ERR_CUDA;
      if (holds) {
        const h2_status rr = h2_release_factorization(c);
        if (r == H2_OK) r = rr;
        {
          std::lock_guard<std::mutex> lk(mu);
          --holding;
          ++released;
        }
        cv.notify_all();
      }
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
      if (b->forest) b->err = "group " + std::to_string(i) + ": " + (msg[i].empty() ? h2_last_error(b->ctx[i]) : msg[i]);
      else b->err = "system " + std::to_string(i) + ": " + h2_last_error(b->ctx[i]);
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

h2_status h2_batch_create_forest(h2_batch** out, const h2_params* p, const double* const* points, const int64_t* N,
                                 const int32_t* leaf, int32_t count) {
  if (!out || !p || !points || !N || count < 1) return H2_ERR_INVALID_ARG;
  *out = nullptr;
  // group the systems by (leaf size, tree depth), ascending
  std::vector<std::tuple<int, int, int>> key(count);
  for (int32_t s = 0; s < count; ++s) {
    const int lf = leaf ? leaf[s] : p->leaf_size;
    const int d = h2_tree_depth(N[s], lf);
    if (lf < 1 || d < 1 || !points[s]) return H2_ERR_INVALID_ARG;
    key[s] = {lf, d, s};
  }
  std::sort(key.begin(), key.end());
  h2_batch* b = new h2_batch();
  b->forest = true;
  b->sys_group.assign(count, -1);
  b->sys_off.assign(count, 0);
  b->sys_n.assign(N, N + count);
  for (int32_t k = 0; k < count;) {
    int32_t e = k;
    while (e < count && std::get<0>(key[e]) == std::get<0>(key[k]) && std::get<1>(key[e]) == std::get<1>(key[k])) ++e;
    const int g = (int)b->group_sys.size();
    std::vector<int> sys;
    std::vector<const double*> pts;
    std::vector<int64_t> ns;
    int64_t off = 0;
    for (int32_t t = k; t < e; ++t) {
      const int s = std::get<2>(key[t]);
      sys.push_back(s);
      pts.push_back(points[s]);
      ns.push_back(N[s]);
      b->sys_group[s] = g;
      b->sys_off[s] = off;
      off += N[s];
    }
    h2_params pg = *p;
    pg.leaf_size = std::get<0>(key[k]);
    h2_ctx* c = nullptr;
    h2_status st = h2_build_forest(&c, &pg, pts.data(), ns.data(), (int32_t)sys.size());
    // the batch factors in FP16 / BF16 only: the FP64 leaf blocks (8 bytes of
    // the instance's 14 per leaf entry) go before the next group is built
    if (st == H2_OK) st = h2_set_option(c, H2_OPT_FP64_LEAF, 0);
    if (st != H2_OK) {
      if (c) h2_destroy(c);
      h2_batch_destroy(b);
      return st;
    }
    b->ctx.push_back(c);
    b->n.push_back(off);
    b->group_sys.push_back(sys);
    k = e;
  }
  b->tune_seconds.assign(5, 0.0);
  *out = b;
  return H2_OK;
}

h2_status h2_batch_run(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                       int32_t max_iters, double* relres, int32_t* iters, double* seconds) {
  if (!b || (prec < -1 || prec > H2_PREC_BF16) || (B && !X) || (prec < 0 && !B)) return H2_ERR_INVALID_ARG;
  b->err.clear();
  if (B && !host_vectors(b, B, X)) return H2_ERR_INVALID_ARG;
  h2_status s = run(b, b->workers, prec, B, X, target, max_iters, relres, iters);
  if (seconds) *seconds = b->last_seconds;
  return s;
}

h2_status h2_batch_tune(h2_batch* b, int32_t prec, const double* const* B, double* const* X, double target,
                        int32_t max_iters, int32_t* workers_out) {
  if (!b || prec < 0 || prec > H2_PREC_BF16 || !B || !X) return H2_ERR_INVALID_ARG;
  b->err.clear();
  if (!host_vectors(b, B, X)) return H2_ERR_INVALID_ARG;
  // kernel forms and launch shapes first, on the largest context
  {
    size_t big = 0;
    for (size_t k = 1; k < b->ctx.size(); ++k)
      if (b->n[k] > b->n[big]) big = k;
    std::vector<char> js(1 << 14);
    h2_status s = h2_autotune(b->ctx[big], prec, js.data(), js.size());
    if (b->forest) h2_release_factorization(b->ctx[big]);
    if (s != H2_OK) {
      b->err = std::string("autotune: ") + h2_last_error(b->ctx[big]);
      return s;
    }
    b->kernels = js.data();
  }
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
  const size_t nsys = b->forest ? b->sys_n.size() : b->ctx.size();
  std::string o = "{\"systems\":" + std::to_string(nsys) + ",\"mode\":\"" + (b->forest ? "forest" : "pool") +
                  "\",\"groups\":" + std::to_string(b->ctx.size()) + ",\"workers\":" + std::to_string(b->workers) +
                  ",\"last_seconds\":" + std::to_string(b->last_seconds) + ",\"tune_seconds\":{";
  const int cand[5] = {1, 2, 4, 8, 16};
  bool first = true;
  for (int k = 0; k < 5; ++k) {
    if (b->tune_seconds[k] <= 0) continue;
    o += (first ? "\"" : ",\"") + std::to_string(cand[k]) + "\":" + std::to_string(b->tune_seconds[k]);
    first = false;
  }
  o += "}";
  if (!b->kernels.empty()) o += ",\"kernels\":" + b->kernels;
  if (b->forest) {
    o += ",\"group_systems\":[";
    for (size_t g = 0; g < b->group_sys.size(); ++g) o += (g ? "," : "") + std::to_string(b->group_sys[g].size());
    o += "]";
  }
  o += "}";
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
  // batch's worker streams); a forest batch owns its group contexts
  for (h2_ctx* c : b->ctx) {
    if (b->forest) h2_destroy(c);
    else h2_set_stream(c, nullptr);
  }
  delete b;
}

}  // extern "C"
