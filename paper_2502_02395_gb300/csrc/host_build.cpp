// Host-side part of h2_build: cluster tree, near/far lists and the
// interpolative decompositions of Algorithm 1 (construction with the
// pre-factorization basis, Section 3.4-3.5).  Dense kernel blocks are not
// formed here; the GPU evaluates them from the points (h2_api.cu).
//
// Per box i of level l the composite matrix
//     M_i = [ G(B_i, S_F) | G(B_i, S_C^j) G(S_C^j, S_C^j)^-1  (close j != i) ]
// is row-compressed.  M_i^T is streamed in row chunks through a structured
// Householder update of an n x n triangular factor (the R of a tall QR,
// which carries the same column norms and column-pivoting decisions as M_i^T
// itself); a column-pivoted QR of that triangle then gives the skeleton
// pivots and X_i = P [I; (R11^-1 R12)^T].  Boxes of a level are independent
// and run in parallel (OpenMP).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "h2_internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace h2 {

int depth_of(int64_t n, int leaf) {
  int L = 0;
  while ((int64_t)leaf << L < n) ++L;
  return L;
}

namespace {

// Median split along the longest bounding-box axis; ties by original index.
void build_tree(const double* P, int64_t N, int L, std::vector<int64_t>& perm,
                std::vector<int64_t>& leaf_off) {
  perm.resize(N);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<int64_t> off = {0, N};
  for (int l = 0; l < L; ++l) {
    int nb = 1 << l;
    std::vector<int64_t> nxt(2 * nb + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < nb; ++i) {
      int64_t a = off[i], b = off[i + 1];
      double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int64_t t = a; t < b; ++t)
        for (int d = 0; d < 3; ++d) {
          double v = P[3 * perm[t] + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
      int ax = 0;
      for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
      std::sort(perm.begin() + a, perm.begin() + b, [&](int64_t u, int64_t v) {
        double pu = P[3 * u + ax], pv = P[3 * v + ax];
        return pu < pv || (pu == pv && u < v);
      });
      nxt[2 * i] = a;
      nxt[2 * i + 1] = a + (b - a) / 2;
    }
    nxt[2 * nb] = N;
    off.swap(nxt);
  }
  leaf_off = off;
}

struct Geo {
  std::vector<double> c, R;  // centres (3 per box), half-diagonals
};

Geo geometry(const double* P, const std::vector<int64_t>& perm, const std::vector<int64_t>& off) {
  int nb = (int)off.size() - 1;
  Geo g;
  g.c.assign(3 * nb, 0.0);
  g.R.assign(nb, 0.0);
  for (int i = 0; i < nb; ++i) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = off[i]; t < off[i + 1]; ++t)
      for (int d = 0; d < 3; ++d) {
        double v = P[3 * perm[t] + d];
        lo[d] = std::min(lo[d], v);
        hi[d] = std::max(hi[d], v);
      }
    double s = 0;
    for (int d = 0; d < 3; ++d) {
      g.c[3 * i + d] = 0.5 * (lo[d] + hi[d]);
      s += (hi[d] - lo[d]) * (hi[d] - lo[d]);
    }
    g.R[i] = 0.5 * std::sqrt(s);
  }
  return g;
}

// ---- small dense kernels (host) ------------------------------------------

// Stacked QR update: [R; C] = Q [R'; 0], R n x n row-major upper triangular,
// C c x n column-major (column j at C + j*c).  C is destroyed.
void tsqr_update(double* R, int n, double* C, int c) {
  for (int k = 0; k < n; ++k) {
    double* ck = C + (size_t)k * c;
    double alpha = R[(size_t)k * n + k];
    double xn2 = 0.0;
#pragma omp simd reduction(+ : xn2)
    for (int r = 0; r < c; ++r) xn2 += ck[r] * ck[r];
    if (xn2 == 0.0) continue;
    double beta = -std::copysign(std::sqrt(alpha * alpha + xn2), alpha);
    double tau = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
#pragma omp simd
    for (int r = 0; r < c; ++r) ck[r] *= scal;
    R[(size_t)k * n + k] = beta;
    for (int j = k + 1; j < n; ++j) {
      double* cj = C + (size_t)j * c;
      double w = 0.0;
#pragma omp simd reduction(+ : w)
      for (int r = 0; r < c; ++r) w += ck[r] * cj[r];
      w = tau * (w + R[(size_t)k * n + j]);
      R[(size_t)k * n + j] -= w;
#pragma omp simd
      for (int r = 0; r < c; ++r) cj[r] -= w * ck[r];
    }
  }
}

// Column-pivoted Householder QR of the n x n row-major matrix R (in place;
// the result is upper triangular, row-major).  piv[t] = original column.
void pivoted_qr(double* R, int n, std::vector<int>& piv) {
  std::vector<double> A((size_t)n * n);  // column-major working copy
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)j * n + i] = R[(size_t)i * n + j];
  piv.resize(n);
  std::iota(piv.begin(), piv.end(), 0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = -1.0;
    for (int j = k; j < n; ++j) {
      const double* aj = &A[(size_t)j * n];
      double s = 0.0;
      for (int r = k; r < n; ++r) s += aj[r] * aj[r];
      if (s > best) {
        best = s;
        p = j;
      }
    }
    if (p != k) {
      std::swap_ranges(A.begin() + (size_t)k * n, A.begin() + (size_t)(k + 1) * n,
                       A.begin() + (size_t)p * n);
      std::swap(piv[k], piv[p]);
    }
    double* ak = &A[(size_t)k * n];
    double alpha = ak[k], xn2 = 0.0;
    for (int r = k + 1; r < n; ++r) xn2 += ak[r] * ak[r];
    if (xn2 == 0.0) continue;
    double beta = -std::copysign(std::sqrt(alpha * alpha + xn2), alpha);
    double tau = (beta - alpha) / beta, scal = 1.0 / (alpha - beta);
    for (int r = k + 1; r < n; ++r) ak[r] *= scal;
    ak[k] = beta;
    for (int j = k + 1; j < n; ++j) {
      double* aj = &A[(size_t)j * n];
      double w = aj[k];
      for (int r = k + 1; r < n; ++r) w += ak[r] * aj[r];
      w *= tau;
      aj[k] -= w;
      for (int r = k + 1; r < n; ++r) aj[r] -= w * ak[r];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] = (j >= i) ? A[(size_t)j * n + i] : 0.0;
}

// Solve Acc Y = B in place (Acc s x s row-major, destroyed; B s x m
// column-major).  Partial pivoting.  Returns false on a zero pivot.
bool lu_solve_cols(double* Acc, int s, double* B, int m) {
  std::vector<int> ip(s);
  for (int k = 0; k < s; ++k) {
    int p = k;
    for (int r = k + 1; r < s; ++r)
      if (std::fabs(Acc[(size_t)r * s + k]) > std::fabs(Acc[(size_t)p * s + k])) p = r;
    ip[k] = p;
    if (Acc[(size_t)p * s + k] == 0.0) return false;
    if (p != k)
      for (int j = 0; j < s; ++j) std::swap(Acc[(size_t)k * s + j], Acc[(size_t)p * s + j]);
    double d = Acc[(size_t)k * s + k];
    for (int r = k + 1; r < s; ++r) {
      double f = Acc[(size_t)r * s + k] /= d;
      for (int j = k + 1; j < s; ++j) Acc[(size_t)r * s + j] -= f * Acc[(size_t)k * s + j];
    }
  }
  for (int c = 0; c < m; ++c) {
    double* b = B + (size_t)c * s;
    for (int k = 0; k < s; ++k)
      if (ip[k] != k) std::swap(b[k], b[ip[k]]);
    for (int k = 0; k < s; ++k)
      for (int r = k + 1; r < s; ++r) b[r] -= Acc[(size_t)r * s + k] * b[k];
    for (int k = s - 1; k >= 0; --k) {
      b[k] /= Acc[(size_t)k * s + k];
      for (int r = 0; r < k; ++r) b[r] -= Acc[(size_t)r * s + k] * b[k];
    }
  }
  return true;
}

// splitmix64 (Steele, Lea, Flood 2014): the counter-based generator of the
// sketches' random signs.
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// The 16 features of every box of a level (the list in h2ulv.h) into f
// (nb x kRankFeatures row-major); nbox[i] is box i's dimension.
void level_features(const h2_params& p, const double* P, const std::vector<int64_t>& perm,
                    const std::vector<int64_t>& off, const HostLevel& hl, int l, int L, const std::vector<int>& nbox,
                    std::vector<float>& f) {
  const int nb = hl.nb;
  f.assign((size_t)nb * kRankFeatures, 0.f);
  std::vector<double> lo(3 * (size_t)nb, INFINITY), hi(3 * (size_t)nb, -INFINITY), c(3 * (size_t)nb), R(nb);
  for (int i = 0; i < nb; ++i) {
    for (int64_t t = off[i]; t < off[i + 1]; ++t)
      for (int d = 0; d < 3; ++d) {
        const double v = P[3 * perm[t] + d];
        lo[3 * i + d] = std::min(lo[3 * i + d], v);
        hi[3 * i + d] = std::max(hi[3 * i + d], v);
      }
    double s2 = 0;
    for (int d = 0; d < 3; ++d) {
      if (off[i + 1] == off[i]) lo[3 * i + d] = hi[3 * i + d] = 0.0;
      c[3 * i + d] = 0.5 * (lo[3 * i + d] + hi[3 * i + d]);
      s2 += (hi[3 * i + d] - lo[3 * i + d]) * (hi[3 * i + d] - lo[3 * i + d]);
    }
    R[i] = 0.5 * std::sqrt(s2);
  }
  std::vector<int> nnear(nb, 0), nfar(nb, 0);
  std::vector<double> dfar(nb, INFINITY);
  for (size_t q = 0; q < hl.near.size() / 2; ++q) ++nnear[hl.near[2 * q]];
  for (size_t q = 0; q < hl.far.size() / 2; ++q) {
    const int i = hl.far[2 * q], j = hl.far[2 * q + 1];
    ++nfar[i];
    double d2 = 0;
    for (int d = 0; d < 3; ++d) d2 += (c[3 * i + d] - c[3 * j + d]) * (c[3 * i + d] - c[3 * j + d]);
    dfar[i] = std::min(dfar[i], std::sqrt(d2) / std::max(R[i], 1e-12));
  }
  const int k = p.kernel;
  const float fam_lap = (k == H2_K_LAPLACE_EPS || k == H2_K_LAPLACE_PAPER) ? 1.f : 0.f;
  const float fam_yuk = (k == H2_K_YUKAWA_EPS || k == H2_K_YUKAWA_PAPER) ? 1.f : 0.f;
  const float fam_gau = (k == H2_K_GAUSSIAN) ? 1.f : 0.f;
  const double lenp = (k == H2_K_LAPLACE_EPS || k == H2_K_YUKAWA_EPS) ? p.eps : (k == H2_K_GAUSSIAN ? p.ell : 1.0);
  KernelFn G{p.kernel, p.eps, p.ell, p.diag_shift};
  const double origin[3] = {0.0, 0.0, 0.0};
  const double dg = std::fabs(G.diag(origin));
  for (int i = 0; i < nb; ++i) {
    float* fi = &f[(size_t)i * kRankFeatures];
    double e[3] = {hi[3 * i] - lo[3 * i], hi[3 * i + 1] - lo[3 * i + 1], hi[3 * i + 2] - lo[3 * i + 2]};
    std::sort(e, e + 3, [](double a, double b) { return a > b; });
    for (int d = 0; d < 3; ++d) fi[d] = (float)std::log10(std::max(e[d], 1e-12));
    fi[3] = (float)std::log2(std::max<double>(1.0, (double)(off[i + 1] - off[i])));
    fi[4] = (float)std::log2(std::max(1, nbox[i]));
    fi[5] = (float)std::log2(std::max(1, nnear[i]));
    fi[6] = (float)std::log2(1.0 + nfar[i]);
    fi[7] = nfar[i] ? (float)std::log10(std::max(dfar[i], 1e-12)) : 0.f;
    fi[8] = (float)p.eta;
    fi[9] = L ? (float)l / (float)L : 0.f;
    fi[10] = (float)std::log10(p.tol);
    fi[11] = fam_lap;
    fi[12] = fam_yuk;
    fi[13] = fam_gau;
    fi[14] = (float)std::log10(std::max(lenp, 1e-30));
    fi[15] = (float)std::log10(std::max(dg, 1e-30));
  }
}

// A level's rank from the predictions y_i of k_i / n_i: max_i ceil(1.05 y_i
// n_i) + 2 (a 5 % margin), raised to the level's cap (max_rank, else D / 2)
// once it is within 10 % of it, at least 1.
int predicted_rank(const h2_params& p, const std::vector<float>& y, const std::vector<int>& n, int D) {
  int k = 1;
  for (size_t i = 0; i < y.size(); ++i) {
    const double v = std::min(1.0, std::max(0.0, (double)y[i]));
    k = std::max(k, (int)std::ceil(1.05 * v * n[i]) + 2);
  }
  const int cap = p.max_rank > 0 ? p.max_rank : D / 2;
  if (k >= 0.9 * cap) k = cap;
  return std::max(1, std::min(k, cap));
}

// Column-pivoted Householder QR of the m x n column-major matrix Z (in
// place, ld m) for `steps` steps; piv[t] = original column of column t.
void pivoted_qr_rect(std::vector<double>& Z, int m, int n, int steps, std::vector<int>& piv) {
  piv.resize(n);
  std::iota(piv.begin(), piv.end(), 0);
  for (int k = 0; k < steps; ++k) {
    int pc = k;
    double best = -1.0;
    for (int j = k; j < n; ++j) {
      const double* zj = &Z[(size_t)j * m];
      double s = 0.0;
      for (int r = k; r < m; ++r) s += zj[r] * zj[r];
      if (s > best) best = s, pc = j;
    }
    if (pc != k) {
      std::swap_ranges(Z.begin() + (size_t)k * m, Z.begin() + (size_t)(k + 1) * m, Z.begin() + (size_t)pc * m);
      std::swap(piv[k], piv[pc]);
    }
    double* zk = &Z[(size_t)k * m];
    const double alpha = zk[k];
    double xn2 = 0.0;
    for (int r = k + 1; r < m; ++r) xn2 += zk[r] * zk[r];
    if (xn2 == 0.0) continue;
    const double beta = -std::copysign(std::sqrt(alpha * alpha + xn2), alpha);
    const double tau = (beta - alpha) / beta, scal = 1.0 / (alpha - beta);
    for (int r = k + 1; r < m; ++r) zk[r] *= scal;
    zk[k] = beta;
    for (int j = k + 1; j < n; ++j) {
      double* zj = &Z[(size_t)j * m];
      double w = zj[k];
      for (int r = k + 1; r < m; ++r) w += zk[r] * zj[r];
      w *= tau;
      zj[k] -= w;
      for (int r = k + 1; r < m; ++r) zj[r] -= w * zk[r];
    }
  }
}

using RowSink = std::function<void(double*, int)>;
using RowsFn = std::function<bool(int, const RowSink&)>;

// Randomized interpolative decomposition of box i (dimension n) at rank K:
// Y = M_i Omega with K + 26 sketch columns and 6 probe columns (Rademacher
// signs from splitmix64(seed, row, column)); a column-pivoted QR of the
// sketch part of Y^T, K + 1 steps, gives the skeleton (the first K pivots)
// and R11, R12 (written as the first K rows of Rout, n x n row-major, as the
// plain pass leaves them).  Accepted when the sketch's (K+1)-th pivot is at
// most tol of the first (or K is the level's cap) and the interpolation
// error on the probe columns, ||Yq - X Yq[SK]|| / ||Yq||, is at most
// 10 max(tol, that pivot ratio).
bool sketch_box(const RowsFn& rows_of, int i, int n, int K, bool capped, double tol, uint64_t seed,
                std::vector<double>& Rout, std::vector<int>& piv) {
  const int ms = std::min(K + 26, n), q = 6, m = ms + q;
  std::vector<double> Y((size_t)n * m, 0.0), w(m);
  uint64_t g = 0;
  const bool rows_ok = rows_of(i, [&](double* C, int c) {
    for (int r = 0; r < c; ++r, ++g) {
      for (int t0 = 0; t0 < m; t0 += 64) {
        const uint64_t bits = splitmix64(seed ^ (g * 0x100000001B3ull + (uint64_t)t0));
        for (int t = t0; t < std::min(m, t0 + 64); ++t) w[t] = ((bits >> (t - t0)) & 1ull) ? 1.0 : -1.0;
      }
      for (int a = 0; a < n; ++a) {
        const double v = C[(size_t)a * c + r];
        if (v == 0.0) continue;
        double* y = &Y[(size_t)a * m];
#pragma omp simd
        for (int t = 0; t < m; ++t) y[t] += v * w[t];
      }
    }
  });
  if (!rows_ok) return false;
  std::vector<double> Z((size_t)ms * n);
  for (int j = 0; j < n; ++j)
    for (int t = 0; t < ms; ++t) Z[(size_t)j * ms + t] = Y[(size_t)j * m + t];
  const int steps = std::min(K + 1, std::min(ms, n));
  pivoted_qr_rect(Z, ms, n, steps, piv);
  const double r0 = std::fabs(Z[0]);
  if (!(r0 > 0.0)) return false;
  const double rho = (steps > K) ? std::fabs(Z[(size_t)K * ms + K]) / r0 : 0.0;
  Rout.assign((size_t)n * n, 0.0);
  for (int t = 0; t < K; ++t)
    for (int u = t; u < n; ++u) Rout[(size_t)t * n + u] = Z[(size_t)u * ms + t];
  // T = R11^-1 R12 and the probe error
  const int mm = n - K;
  std::vector<double> T((size_t)K * mm, 0.0);
  for (int t = K - 1; t >= 0; --t) {
    const double d = Rout[(size_t)t * n + t];
    if (!(std::fabs(d) > 1e-15 * r0)) continue;
    for (int b = 0; b < mm; ++b) {
      double s = Rout[(size_t)t * n + K + b];
      for (int u = t + 1; u < K; ++u) s -= Rout[(size_t)t * n + u] * T[(size_t)u * mm + b];
      T[(size_t)t * mm + b] = s / d;
    }
  }
  double e2 = 0.0, y2 = 0.0;
  for (int a = 0; a < n; ++a)
    for (int k = 0; k < q; ++k) y2 += Y[(size_t)a * m + ms + k] * Y[(size_t)a * m + ms + k];
  for (int b = 0; b < mm; ++b)
    for (int k = 0; k < q; ++k) {
      double v = Y[(size_t)piv[K + b] * m + ms + k];
      for (int u = 0; u < K; ++u) v -= T[(size_t)u * mm + b] * Y[(size_t)piv[u] * m + ms + k];
      e2 += v * v;
    }
  const double e = std::sqrt(e2 / std::max(y2, 1e-300));
  return (capped || rho <= tol) && e <= 10.0 * std::max(tol, rho);
}

}  // namespace

std::string build_host(const h2_params& p, const double* pts, int64_t N, HostH2& H, RankPredictor* pred,
                       bool layout_only, GpuCompressor* gpu, const std::vector<int>* force_K) {
  KernelFn G{p.kernel, p.eps, p.ell, p.diag_shift};
  H.N = N;
  H.points.assign(pts, pts + 3 * N);
  const double* P = H.points.data();
  int L = depth_of(N, p.leaf_size);
  H.L = L;
  build_tree(P, N, L, H.perm, H.leaf_offsets);
  H.lv.assign(L + 1, HostLevel());

  // box offsets per level (tree positions)
  std::vector<std::vector<int64_t>> off(L + 1);
  for (int l = 0; l <= L; ++l) {
    int nb = 1 << l;
    off[l].resize(nb + 1);
    for (int i = 0; i <= nb; ++i) off[l][i] = H.leaf_offsets[(size_t)i << (L - l)];
  }
  // near / far lists
  H.lv[0].nb = 1;
  H.lv[0].near = {0, 0};
  for (int l = 1; l <= L; ++l) {
    Geo g = geometry(P, H.perm, off[l]);
    std::vector<std::pair<int, int>> nl, fl;
    const auto& pn = H.lv[l - 1].near;
    for (size_t q = 0; q < pn.size() / 2; ++q) {
      int pp = pn[2 * q], qq = pn[2 * q + 1];
      for (int a = 2 * pp; a <= 2 * pp + 1; ++a)
        for (int b = 2 * qq; b <= 2 * qq + 1; ++b) {
          double dx = g.c[3 * a] - g.c[3 * b], dy = g.c[3 * a + 1] - g.c[3 * b + 1],
                 dz = g.c[3 * a + 2] - g.c[3 * b + 2];
          double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
          bool adm = (a != b) && dist > p.eta * (g.R[a] + g.R[b]);
          (adm ? fl : nl).push_back({a, b});
        }
    }
    std::sort(nl.begin(), nl.end());
    std::sort(fl.begin(), fl.end());
    HostLevel& hl = H.lv[l];
    hl.nb = 1 << l;
    for (auto& e : nl) { hl.near.push_back(e.first); hl.near.push_back(e.second); }
    for (auto& e : fl) { hl.far.push_back(e.first); hl.far.push_back(e.second); }
  }

  // leaf dimension and the level points (original indices)
  std::vector<std::vector<std::vector<int64_t>>> bp(L + 1);
  bp[L].resize((size_t)1 << L);
  int Dl = 0;
  for (int i = 0; i < (1 << L); ++i) {
    bp[L][i].assign(H.perm.begin() + off[L][i], H.perm.begin() + off[L][i + 1]);
    Dl = std::max<int>(Dl, (int)bp[L][i].size());
  }
  H.lv[L].D = Dl;
  RankRecord& rec = H.rec;
  rec.feats.assign(L + 1, {});
  rec.ranks.assign(L + 1, {});
  rec.dims.assign(L + 1, {});
  rec.K_pred.assign(L + 1, -1);

  // predicted layout without any compression: each level's dimension is
  // twice the predicted rank of the level below
  if (layout_only) {
    if (!pred) return "layout without a predictor";
    int nprev = 0;
    for (int l = L; l >= 1; --l) {
      HostLevel& hl = H.lv[l];
      std::vector<int> nbox(hl.nb);
      for (int i = 0; i < hl.nb; ++i) nbox[i] = (l == L) ? (int)bp[L][i].size() : 2 * nprev;
      if (l < L) hl.D = 2 * nprev;
      std::vector<float> f;
      level_features(p, P, H.perm, off[l], hl, l, L, nbox, f);
      std::vector<float> yhat;
      if (!pred->predict(f, hl.nb, yhat)) return "rank predictor failed at level " + std::to_string(l);
      hl.K = predicted_rank(p, yhat, nbox, hl.D);
      rec.K_pred[l] = hl.K;
      rec.feats[l].swap(f);
      rec.dims[l] = nbox;
      nprev = hl.K;
    }
    H.lv[0].D = L ? 2 * nprev : (int)N;
    return "";
  }

  const int CH = 256;  // chunk rows of the streamed QR / sketch
  for (int l = L; l >= 1; --l) {
    HostLevel& hl = H.lv[l];
    int nb = hl.nb, D = hl.D;
    std::vector<std::vector<int>> nbrs(nb);
    for (size_t q = 0; q < hl.near.size() / 2; ++q) nbrs[hl.near[2 * q]].push_back(hl.near[2 * q + 1]);
    std::vector<int> nbox(nb);
    for (int i = 0; i < nb; ++i) nbox[i] = (int)bp[l][i].size();
    std::vector<float> feats;
    level_features(p, P, H.perm, off[l], hl, l, L, nbox, feats);
    int cap = p.max_rank > 0 ? p.max_rank : D / 2;
    int nmin = D;
    for (int i = 0; i < nb; ++i) nmin = std::min<int>(nmin, (int)bp[l][i].size());
    const int capK = std::max(1, std::min(cap, nmin));

    // The rows of M_i^T (Algorithm 1): the stride-sampled far field, then
    // G(S_C, S_C)^-1 G(S_C, B_i) for each close box j != i, in chunks of at
    // most CH rows (c x n, column-major), handed to sink(C, c).  False if a
    // close-field sample block is singular.
    auto rows_of = [&](int i, const std::function<void(double*, int)>& sink) -> bool {
      const std::vector<int64_t>& Pi = bp[l][i];
      const int n = (int)Pi.size();
      std::vector<double> C((size_t)CH * n);
      int64_t nearcnt = 0;
      for (int j : nbrs[i]) nearcnt += off[l][j + 1] - off[l][j];
      const int64_t F = N - nearcnt;
      const int64_t s = (p.far_samples <= 0 || p.far_samples >= F) ? F : p.far_samples;
      for (int64_t t0 = 0; t0 < s; t0 += CH) {
        const int c = (int)std::min<int64_t>(CH, s - t0);
        for (int r = 0; r < c; ++r) {
          int64_t q = ((t0 + r) * F) / s;
          for (int j : nbrs[i]) {  // sorted intervals
            if (q < off[l][j]) break;
            q += off[l][j + 1] - off[l][j];
          }
          const int64_t pt = H.perm[q];
          for (int cc = 0; cc < n; ++cc) C[(size_t)cc * c + r] = G.entry(P, pt, Pi[cc], false);
        }
        sink(C.data(), c);
      }
      for (int j : nbrs[i]) {
        if (j == i) continue;
        const std::vector<int64_t>& Pj = bp[l][j];
        const int nj = (int)Pj.size();
        const int sc = (p.near_samples <= 0 || p.near_samples >= nj) ? nj : p.near_samples;
        std::vector<int64_t> SC(sc);
        for (int t = 0; t < sc; ++t) SC[t] = Pj[((int64_t)t * nj) / sc];
        std::vector<double> Acc((size_t)sc * sc), B((size_t)sc * n);
        for (int a = 0; a < sc; ++a)
          for (int b = 0; b < sc; ++b) Acc[(size_t)a * sc + b] = G.entry(P, SC[a], SC[b], a == b);
        for (int cc = 0; cc < n; ++cc)
          for (int a = 0; a < sc; ++a) B[(size_t)cc * sc + a] = G.entry(P, SC[a], Pi[cc], false);
        if (!lu_solve_cols(Acc.data(), sc, B.data(), n)) return false;
        sink(B.data(), sc);
      }
      return true;
    };

    std::vector<std::vector<double>> Rb(nb);
    std::vector<std::vector<int>> pivs(nb);
    std::vector<int> ranks(nb, 0);
    int bad = -1;
    // the plain rank-revealing pass of one box: streamed QR of M_i^T, then a
    // column-pivoted QR of its triangle; ranks[i] = #{|R_tt| > tol |R_11|}
    auto plain_box = [&](int i) {
      const int n = (int)bp[l][i].size();
      std::vector<double> R((size_t)n * n, 0.0);
      if (!rows_of(i, [&](double* C, int c) { tsqr_update(R.data(), n, C, c); })) {
#pragma omp critical
        bad = i;
        return;
      }
      std::vector<int> piv;
      pivoted_qr(R.data(), n, piv);
      const double r0 = n ? std::fabs(R[0]) : 0.0;
      int k = 0;
      if (r0 > 0)
        for (int t = 0; t < n; ++t) k += std::fabs(R[(size_t)t * n + t]) > p.tol * r0;
      ranks[i] = k;
      Rb[i].swap(R);
      pivs[i].swap(piv);
    };

    auto t0 = std::chrono::steady_clock::now();
    int K = 0;
    bool done = false;
    // boxes whose X and skeleton come straight from the GPU construction
    std::vector<char> direct(nb, 0);
    GpuLevelJob job;
    if (pred || gpu) {
      if (pred) {
        std::vector<float> yhat;
        if (!pred->predict(feats, nb, yhat)) return "rank predictor failed at level " + std::to_string(l);
        K = std::min(predicted_rank(p, yhat, nbox, D), capK);
        rec.K_pred[l] = K;
      } else {
        K = capK;  // fixed rank: the level's cap
      }
      std::vector<char> ok(nb, 0);
      bool sketched = false;
      if (gpu && gpu->supported(D, K) && p.near_samples > 0 && p.near_samples <= 64) {
        // the level's sample lists for the GPU sketches
        job.nb = nb, job.D = D, job.K = K;
        job.m = std::min(160, ((K + 32 + 1) / 2) * 2);  // K + 26 sketch columns, 6 probes
        job.q = 6, job.ms = job.m - 6;
        job.seed = splitmix64(0xC0FFEEull + (uint64_t)l);
        job.nbox = nbox;
        job.bpts.assign((size_t)nb * D, -1);
        job.fptr.assign(nb + 1, 0);
        job.nptr.assign(nb + 1, 0);
        job.cptr.assign(nb + 1, 0);
        for (int i = 0; i < nb; ++i) {
          for (size_t a = 0; a < bp[l][i].size(); ++a) job.bpts[(size_t)i * D + a] = bp[l][i][a];
          int64_t nearcnt = 0;
          for (int j : nbrs[i]) nearcnt += off[l][j + 1] - off[l][j];
          const int64_t F = N - nearcnt;
          const int64_t sF = (p.far_samples <= 0 || p.far_samples >= F) ? F : p.far_samples;
          for (int64_t t = 0; t < sF; ++t) {
            int64_t q = (t * F) / sF;
            for (int j : nbrs[i]) {
              if (q < off[l][j]) break;
              q += off[l][j + 1] - off[l][j];
            }
            job.fidx.push_back(H.perm[q]);
          }
          job.fptr[i + 1] = (int64_t)job.fidx.size();
          for (int j : nbrs[i]) job.nidx.push_back(j);
          job.nptr[i + 1] = (int64_t)job.nidx.size();
          const std::vector<int64_t>& Pi = bp[l][i];
          const int ni = (int)Pi.size();
          const int sc = std::min(ni, p.near_samples);
          for (int t = 0; t < sc; ++t) job.cidx.push_back(Pi[((int64_t)t * ni) / sc]);
          job.cptr[i + 1] = (int64_t)job.cidx.size();
        }
        const std::string e = gpu->run(job);
        if (!e.empty()) return "GPU construction at level " + std::to_string(l) + ": " + e;
        for (int i = 0; i < nb; ++i) {
          ranks[i] = -1;
          ok[i] = (K >= capK || job.rho[i] <= p.tol) && job.err[i] <= 10.0 * std::max(p.tol, job.rho[i]);
          direct[i] = ok[i];
        }
        ++rec.gpu_levels;
        rec.flops_prefactor += job.flops_prefactor;
        rec.flops_far += job.flops_far;
        sketched = true;
      } else if (pred) {
        const uint64_t lseed = splitmix64(0x5eedull + (uint64_t)l);
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < nb; ++i) {
          ranks[i] = -1;
          ok[i] = sketch_box(rows_of, i, (int)bp[l][i].size(), K, K >= capK, p.tol, splitmix64(lseed ^ (uint64_t)i),
                             Rb[i], pivs[i]);
        }
        sketched = true;
      }
      if (sketched) {
        int need = K;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : need)
        for (int i = 0; i < nb; ++i) {
          if (ok[i]) continue;
          plain_box(i);
          need = std::max(need, std::min(ranks[i], capK));
        }
        if (bad >= 0)
          return "singular close-field sample block at level " + std::to_string(l) + " box " + std::to_string(bad);
        for (int i = 0; i < nb; ++i) rec.fallback_boxes += !ok[i];
        done = need <= K;
        if (!done) {
          ++rec.fallback_levels;
          std::fill(direct.begin(), direct.end(), 0);
        }
      }
    }
    if (!done) {
#pragma omp parallel for schedule(dynamic, 1)
      for (int i = 0; i < nb; ++i) plain_box(i);
      int kmax = *std::max_element(ranks.begin(), ranks.end());
      K = std::max(1, std::min(kmax, capK));
      // a rank laid out beforehand (the systems of a forest share each
      // level's rank): the pivoted QR's first K pivots, at most the smallest
      // box of the level
      if (force_K && l < (int)force_K->size() && (*force_K)[l] > 0) K = std::min((*force_K)[l], nmin);
    }
    rec.compress_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (bad >= 0)
      return "singular close-field sample block at level " + std::to_string(l) + " box " + std::to_string(bad);
    if (nmin == 0) K = 0;
    hl.K = K;
    if (l == L) H.ranks_leaf = ranks;
    rec.feats[l].swap(feats);
    rec.ranks[l] = ranks;
    rec.dims[l] = nbox;
    hl.X.assign((size_t)nb * D * K, 0.0);
    hl.SK.assign((size_t)nb * K, 0);
    bp[l - 1].resize(nb / 2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < nb; ++i) {
      double* X = &hl.X[(size_t)i * D * K];
      if (direct[i]) {
        std::memcpy(X, &job.X[(size_t)i * D * K], sizeof(double) * (size_t)D * K);
        for (int a = 0; a < K; ++a) hl.SK[(size_t)i * K + a] = job.SK[(size_t)i * K + a];
        continue;
      }
      const std::vector<double>& R = Rb[i];
      const std::vector<int>& piv = pivs[i];
      int n = (int)bp[l][i].size();
      int m = n - K;
      // T = R11^-1 R12 (K x m); rows with a zero pivot are set to 0
      std::vector<double> T((size_t)K * m, 0.0);
      double r0 = n ? std::fabs(R[0]) : 0.0;
      for (int t = K - 1; t >= 0; --t) {
        double d = R[(size_t)t * n + t];
        if (!(std::fabs(d) > 1e-15 * r0) || d == 0.0) continue;
        for (int b = 0; b < m; ++b) {
          double s = R[(size_t)t * n + K + b];
          for (int u = t + 1; u < K; ++u) s -= R[(size_t)t * n + u] * T[(size_t)u * m + b];
          T[(size_t)t * m + b] = s / d;
        }
      }
      for (int a = 0; a < K; ++a) X[(size_t)piv[a] * K + a] = 1.0;
      for (int b = 0; b < m; ++b)
        for (int a = 0; a < K; ++a) X[(size_t)piv[K + b] * K + a] = T[(size_t)a * m + b];
      for (int a = 0; a < K; ++a) hl.SK[(size_t)i * K + a] = bp[l][i][piv[a]];
    }
    for (int q = 0; q < nb / 2; ++q) {
      bp[l - 1][q].assign(hl.SK.begin() + (size_t)(2 * q) * K, hl.SK.begin() + (size_t)(2 * q + 2) * K);
    }
    H.lv[l - 1].D = 2 * K;
  }
  if (L == 0) H.lv[0].D = (int)N;
  return "";
}

// The systems must share each level's rank.  (Padding a smaller rank with
// zero basis columns would keep A_H2, but the complement basis of such an
// X_i keeps complement directions in its skeleton part; their near-field
// couplings at the parent level are not in the parent's pre-factorization
// basis, so eliminating them there drops fill-ins the construction never
// bounded, and the refinement slows or stalls.)  Leaves of fewer points than
// the largest leaf get padding points, as a single instance pads its own.
std::string combine_forest(const std::vector<HostH2>& parts, HostH2& H) {
  const int S = (int)parts.size();
  if (S < 1) return "empty forest";
  const int L = parts[0].L;
  for (const HostH2& P : parts)
    if (P.L != L) return "the systems of a forest must have the same tree depth";
  if (L < 1) return "the systems of a forest need at least one level below the root";
  for (int l = 1; l <= L; ++l)
    for (const HostH2& P : parts)
      if (P.lv[l].K != parts[0].lv[l].K) return "the systems of a forest must share each level's rank";
  H = HostH2();
  H.L = L;
  H.lv.assign(L + 1, HostLevel());
  std::vector<int> K(L + 2, 0), D(L + 1, 0);
  for (int l = 1; l <= L; ++l)
    for (const HostH2& P : parts) K[l] = std::max(K[l], P.lv[l].K);
  for (const HostH2& P : parts) D[L] = std::max(D[L], P.lv[L].D);
  // leaves padded to a multiple of 128 (the tensor-core tile and the
  // symmetric-storage matvec's block widths) while that stays <= 1024
  if ((D[L] + 127) / 128 * 128 <= 1024) D[L] = (D[L] + 127) / 128 * 128;
  for (int l = 0; l < L; ++l) D[l] = 2 * K[l + 1];
  std::vector<int64_t> poff(S + 1, 0);
  H.leaf_offsets.push_back(0);
  for (int s = 0; s < S; ++s) {
    const HostH2& P = parts[s];
    poff[s + 1] = poff[s] + P.N;
    H.points.insert(H.points.end(), P.points.begin(), P.points.end());
    for (int64_t t : P.perm) H.perm.push_back(t + poff[s]);
    for (size_t i = 1; i < P.leaf_offsets.size(); ++i) H.leaf_offsets.push_back(P.leaf_offsets[i] + poff[s]);
    H.ranks_leaf.insert(H.ranks_leaf.end(), P.ranks_leaf.begin(), P.ranks_leaf.end());
    H.rec.compress_s += P.rec.compress_s;
    H.rec.fallback_boxes += P.rec.fallback_boxes;
    H.rec.flops_prefactor += P.rec.flops_prefactor;
    H.rec.flops_far += P.rec.flops_far;
  }
  H.N = poff[S];
  for (int l = 0; l <= L; ++l) {
    HostLevel& h = H.lv[l];
    const int nbs = 1 << l;
    h.nb = S * nbs;
    h.D = D[l];
    h.K = l ? K[l] : 0;
    if (l >= 1) {
      h.X.assign((size_t)h.nb * D[l] * K[l], 0.0);
      h.SK.assign((size_t)h.nb * K[l], -1);
    }
    for (int s = 0; s < S; ++s) {
      const HostLevel& g = parts[s].lv[l];
      const int bo = s * nbs;
      for (int32_t v : g.near) h.near.push_back(v + bo);
      for (int32_t v : g.far) h.far.push_back(v + bo);
      if (l == 0 || g.K == 0) continue;
      const int Ks = g.K, Ds = g.D;
      // leaf rows keep their slot; above, child c's skeleton entry a goes to
      // row c K[l + 1] + a of the padded layout
      const int Kc = (l < L) ? parts[s].lv[l + 1].K : 0;
      if (l < L && Ds != 2 * Kc) return "inconsistent box dimension in a forest system";
      for (int i = 0; i < nbs; ++i) {
        const double* src = &g.X[(size_t)i * Ds * Ks];
        double* dst = &h.X[(size_t)(bo + i) * D[l] * K[l]];
        for (int r = 0; r < Ds; ++r) {
          const int rr = (l == L) ? r : (r / Kc) * K[l + 1] + r % Kc;
          for (int a = 0; a < Ks; ++a) dst[(size_t)rr * K[l] + a] = src[(size_t)r * Ks + a];
        }
        for (int a = 0; a < Ks; ++a) {
          const int64_t v = g.SK[(size_t)i * Ks + a];
          h.SK[(size_t)(bo + i) * K[l] + a] = v < 0 ? -1 : v + poff[s];
        }
      }
    }
  }
  return "";
}

}  // namespace h2
