// C ABI of the H^2-ULV library: context setup, factorization driver,
// substitution / refinement driver, matvec, export and statistics.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <sstream>

#include "h2_internal.h"
#include "kernels.h"

using namespace h2;

std::atomic<long long> h2::g_launches{0};

namespace {

thread_local std::string g_last_error;

#define CKC(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);                       \
      return e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA;                \
    }                                                                                   \
  } while (0)

#define CKS(call)                      \
  do {                                 \
    h2_status s_ = (call);             \
    if (s_ != H2_OK) return s_;        \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

h2_status check_params(const h2_params* p, std::string& err) {
  if (!p) { err = "params is NULL"; return H2_ERR_INVALID_ARG; }
  if (p->kernel < 0 || p->kernel > H2_K_POLY2_TEST) { err = "unknown kernel"; return H2_ERR_INVALID_ARG; }
  if (p->leaf_size < 1 || p->leaf_size > 1024) { err = "leaf_size outside 1..1024"; return H2_ERR_INVALID_ARG; }
  if (!(p->eta >= 0.0)) { err = "eta < 0"; return H2_ERR_INVALID_ARG; }
  if (!(p->tol > 0.0)) { err = "tol <= 0"; return H2_ERR_INVALID_ARG; }
  if (p->max_rank < 0) { err = "max_rank < 0"; return H2_ERR_INVALID_ARG; }
  if ((p->kernel == H2_K_LAPLACE_EPS || p->kernel == H2_K_YUKAWA_EPS) && !(p->eps > 0.0)) {
    err = "eps <= 0";
    return H2_ERR_INVALID_ARG;
  }
  if (p->kernel == H2_K_GAUSSIAN && !(p->ell > 0.0)) { err = "ell <= 0"; return H2_ERR_INVALID_ARG; }
  return H2_OK;
}

// ---------------------------------------------------------------------------
// device setup from the host structure
// ---------------------------------------------------------------------------
template <typename V>
h2_status upload(h2_ctx* c, V** dst, const std::vector<V>& src) {
  CKC(dalloc(c, dst, src.size()));
  if (!src.empty()) CKC(cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice));
  return H2_OK;
}

// The leaf blocks scaled by a power of two into FP16 (bf16 = 0) or BF16
// (bf16 = 1): the operand of the leaf-level projection on the tensor cores.
// Part of the H^2 instance; built once per context and type.
h2_status make_leaf_lowp(h2_ctx* c, int bf16) {
  if (c->A16[bf16]) return H2_OK;
  const DevLevel& lf = c->lv[c->L];
  const int64_t n = (int64_t)lf.NP * lf.D * lf.D;
  unsigned int* amax = nullptr;
  CKC(dalloc(c, &amax, 1));
  CKC(dalloc(c, &c->A16_scale[bf16], 2));
  CKC(dalloc(c, reinterpret_cast<uint16_t**>(&c->A16[bf16]), n));
  CKC(cudaMemsetAsync(amax, 0, sizeof(unsigned int), c->stream));
  launch_amax_blocks<double>(c->A64, lf.NP, (int64_t)lf.D * lf.D, lf.D, lf.D, lf.D, amax, c->stream);
  launch_pow2_scale(amax, 128.0f, c->A16_scale[bf16], c->stream);
  launch_to_lowp<double>(bf16, c->A64, c->A16[bf16], n, c->A16_scale[bf16], c->stream);
  // couplings, per level, with max |S| scaled to sqrt(32768 / K): the
  // tensor-core coupling products then stay inside FP16 (|S T^T| <= 32768)
  for (int l = 1; l <= c->L; ++l) {
    DevLevel& d = c->lv[l];
    if (d.FP == 0 || d.K == 0) continue;
    const int64_t ns = d.FP * (int64_t)d.K * d.K;
    CKC(dalloc(c, &d.S16_scale[bf16], 2));
    CKC(dalloc(c, reinterpret_cast<uint16_t**>(&d.S16[bf16]), ns));
    CKC(cudaMemsetAsync(amax, 0, sizeof(unsigned int), c->stream));
    launch_amax_blocks<double>(d.S, d.FP, (int64_t)d.K * d.K, d.K, d.K, d.K, amax, c->stream);
    launch_pow2_scale(amax, std::sqrt(32768.0f / d.K), d.S16_scale[bf16], c->stream);
    launch_to_lowp<double>(bf16, d.S, d.S16[bf16], ns, d.S16_scale[bf16], c->stream);
  }
  CKC(cudaGetLastError());
  CKC(cudaStreamSynchronize(c->stream));
  return H2_OK;
}

h2_status setup_device(h2_ctx* c) {
  HostH2& H = c->host;
  c->L = H.L;
  c->N = H.N;
  const int L = H.L;
  CKC(cudaGetDevice(&c->dev));
  c->lv.assign(L + 1, DevLevel());
  for (int l = 0; l <= L; ++l) {
    DevLevel& d = c->lv[l];
    const HostLevel& h = H.lv[l];
    d.nb = h.nb;  // 2^l, or 2^l per system of a forest
    d.D = h.D;
    d.K = l ? h.K : 0;
    d.R = d.D - d.K;
    if (d.D > 1024) {
      c->err = "box dimension " + std::to_string(d.D) + " at level " + std::to_string(l) + " exceeds 1024";
      return H2_ERR_INVALID_ARG;
    }
    d.NP = (int64_t)h.near.size() / 2;
    d.FP = (int64_t)h.far.size() / 2;
    d.h_near_ptr.assign(d.nb + 1, 0);
    d.h_far_ptr.assign(d.nb + 1, 0);
    d.h_diag_pair.assign(d.nb, -1);
    for (int64_t q = 0; q < d.NP; ++q) {
      int i = h.near[2 * q], j = h.near[2 * q + 1];
      d.h_near_i.push_back(i);
      d.h_near_j.push_back(j);
      d.h_near_ptr[i + 1]++;
      if (i == j) d.h_diag_pair[i] = (int32_t)q;
    }
    for (int64_t q = 0; q < d.FP; ++q) {
      d.h_far_i.push_back(h.far[2 * q]);
      d.h_far_j.push_back(h.far[2 * q + 1]);
      d.h_far_ptr[h.far[2 * q] + 1]++;
    }
    for (int i = 0; i < d.nb; ++i) {
      d.max_near = std::max<int>(d.max_near, (int)d.h_near_ptr[i + 1]);
      d.max_far = std::max<int>(d.max_far, (int)d.h_far_ptr[i + 1]);
      d.h_near_ptr[i + 1] += d.h_near_ptr[i];
      d.h_far_ptr[i + 1] += d.h_far_ptr[i];
      if (d.h_diag_pair[i] < 0) {
        c->err = "level " + std::to_string(l) + " box " + std::to_string(i) + " lacks its diagonal near pair";
        return H2_ERR_INVALID_ARG;
      }
    }
    CKS(upload(c, &d.near_i, d.h_near_i));
    CKS(upload(c, &d.near_j, d.h_near_j));
    CKS(upload(c, &d.near_ptr, d.h_near_ptr));
    {
      std::vector<int32_t> lo, hi, loc(d.nb, 0), hic(d.nb, 0);
      for (int64_t q = 0; q < d.NP; ++q) {
        const int i = d.h_near_i[q], j = d.h_near_j[q];
        if (j < i) lo.push_back((int32_t)q), ++loc[i];
        if (j > i) hi.push_back((int32_t)q), ++hic[i];
      }
      d.n_lo = (int64_t)lo.size();
      d.n_hi = (int64_t)hi.size();
      CKS(upload(c, &d.lo_pairs, lo));
      CKS(upload(c, &d.hi_pairs, hi));
      CKS(upload(c, &d.lo_cnt, loc));
      CKS(upload(c, &d.hi_cnt, hic));
    }
    CKS(upload(c, &d.diag_pair, d.h_diag_pair));
    CKS(upload(c, &d.far_i, d.h_far_i));
    CKS(upload(c, &d.far_j, d.h_far_j));
    CKS(upload(c, &d.far_ptr, d.h_far_ptr));
    if (l >= 1) {
      CKS(upload(c, &d.X, h.X));
      CKS(upload(c, &d.SK, h.SK));
    }
  }
  // parent near-pair index of every near and far pair (merge destinations)
  for (int l = 1; l <= L; ++l) {
    DevLevel& d = c->lv[l];
    const DevLevel& pd = c->lv[l - 1];
    std::map<std::pair<int, int>, int32_t> pidx;
    for (int64_t q = 0; q < pd.NP; ++q) pidx[{pd.h_near_i[q], pd.h_near_j[q]}] = (int32_t)q;
    auto find = [&](int i, int j, int32_t& out) -> bool {
      auto it = pidx.find({i >> 1, j >> 1});
      if (it == pidx.end()) return false;
      out = it->second;
      return true;
    };
    d.h_near_dst.resize(d.NP);
    d.h_far_dst.resize(d.FP);
    for (int64_t q = 0; q < d.NP; ++q)
      if (!find(d.h_near_i[q], d.h_near_j[q], d.h_near_dst[q])) {
        c->err = "near pair without a near parent pair at level " + std::to_string(l);
        return H2_ERR_INVALID_ARG;
      }
    for (int64_t q = 0; q < d.FP; ++q)
      if (!find(d.h_far_i[q], d.h_far_j[q], d.h_far_dst[q])) {
        c->err = "far pair without a near parent pair at level " + std::to_string(l);
        return H2_ERR_INVALID_ARG;
      }
    CKS(upload(c, &d.near_dst, d.h_near_dst));
    CKS(upload(c, &d.far_dst, d.h_far_dst));
  }
  // points, leaf slots, leaf blocks, couplings
  CKS(upload(c, &c->pts, H.points));
  const DevLevel& lf = c->lv[L];
  std::vector<int64_t> slot((size_t)lf.nb * lf.D, -1);
  for (int i = 0; i < lf.nb; ++i)
    for (int64_t t = H.leaf_offsets[i]; t < H.leaf_offsets[i + 1]; ++t)
      slot[(size_t)i * lf.D + (t - H.leaf_offsets[i])] = H.perm[t];
  CKS(upload(c, &c->slot_pt, slot));
  CKC(dalloc(c, &c->A64, (size_t)lf.NP * lf.D * lf.D));
  launch_eval_blocks(c->kfn, c->pts, lf.NP, lf.near_i, lf.near_j, c->slot_pt, lf.D, lf.D, lf.D, c->A64, 0);
  CKC(cudaGetLastError());
  for (int l = 1; l <= L; ++l) {
    DevLevel& d = c->lv[l];
    CKC(dalloc(c, &d.S, (size_t)std::max<int64_t>(d.FP, 1) * d.K * d.K));
    launch_eval_blocks(c->kfn, c->pts, d.FP, d.far_i, d.far_j, d.SK, d.K, d.K, d.K, d.S, 0);
    CKC(cudaGetLastError());
  }
  // vectors and scratch
  const int64_t nslot = (int64_t)lf.nb * lf.D;
  for (double** p : {&c->b64, &c->x64, &c->r64, &c->y64, &c->t64}) CKC(dalloc(c, p, nslot));
  CKC(dalloc(c, &c->io_a, c->N));
  CKC(dalloc(c, &c->io_b, c->N));
  c->hat_off.assign(L + 2, 0);
  for (int l = 1; l <= L; ++l) c->hat_off[l + 1] = c->hat_off[l] + (int64_t)c->lv[l].nb * c->lv[l].K;
  CKC(dalloc(c, &c->xhat, c->hat_off[L + 1]));
  CKC(dalloc(c, &c->yhat, c->hat_off[L + 1]));
  // FP32 copy of the H^2 matrix: the operator of the inner solver of the
  // mixed-precision refinement (part of the instance)
  CKC(dalloc(c, &c->xhat32, c->hat_off[L + 1]));
  CKC(dalloc(c, &c->yhat32, c->hat_off[L + 1]));
  for (float** p : {&c->xdf_h, &c->xdf_l}) CKC(dalloc(c, p, nslot));
  for (float** p : {&c->hdf_h, &c->hdf_l, &c->ydf_h, &c->ydf_l}) CKC(dalloc(c, p, c->hat_off[L + 1]));
  c->sym = sym_leaf_supported(lf.D);
  if (c->sym) {
    // the kernels' near blocks are symmetric (A_ji = A_ij^T): keep i <= j
    std::vector<int32_t> uq, ui, uj;
    for (int64_t q = 0; q < lf.NP; ++q)
      if (lf.h_near_i[q] <= lf.h_near_j[q])
        uq.push_back((int32_t)q), ui.push_back(lf.h_near_i[q]), uj.push_back(lf.h_near_j[q]);
    c->npu = (int64_t)uq.size();
    std::vector<std::vector<std::pair<int32_t, int32_t>>> lists(lf.nb);  // (partner box, entry)
    for (int64_t k = 0; k < c->npu; ++k) {
      lists[ui[k]].push_back({uj[k], (int32_t)(2 * k)});
      if (ui[k] != uj[k]) lists[uj[k]].push_back({ui[k], (int32_t)(2 * k + 1)});
    }
    std::vector<int64_t> ptr(lf.nb + 1, 0);
    std::vector<int32_t> ent;
    for (int i = 0; i < lf.nb; ++i) {
      std::sort(lists[i].begin(), lists[i].end());
      for (auto& pe : lists[i]) ent.push_back(pe.second);
      ptr[i + 1] = (int64_t)ent.size();
    }
    CKS(upload(c, &c->sym_q, uq));
    CKS(upload(c, &c->sym_i, ui));
    CKS(upload(c, &c->sym_j, uj));
    CKS(upload(c, &c->sym_ptr, ptr));
    CKS(upload(c, &c->sym_ent, ent));
    const int64_t DD = (int64_t)lf.D * lf.D;
    CKC(dalloc(c, &c->A32, (size_t)(c->npu * DD)));
    CKC(dalloc(c, &c->Alo, (size_t)(c->npu * DD)));
    launch_gather_blocks(c->A64, c->sym_q, DD, c->npu, c->A32, 0);
    launch_gather_split_lo(c->A64, c->sym_q, DD, c->npu, c->A32, c->Alo, 0);
  } else {
    CKC(dalloc(c, &c->A32, (size_t)lf.NP * lf.D * lf.D));
    launch_convert<double, float>(c->A64, c->A32, (int64_t)lf.NP * lf.D * lf.D, 0);
    CKC(dalloc(c, &c->Alo, (size_t)lf.NP * lf.D * lf.D));
    launch_split_lo(c->A64, c->A32, c->Alo, (int64_t)lf.NP * lf.D * lf.D, 0);
  }
  // upper / lower split of each level's near list (symmetric kernels)
  for (int l = 1; l <= L && c->sym; ++l) {
    DevLevel& d = c->lv[l];
    std::map<std::pair<int32_t, int32_t>, int32_t> at;
    for (int64_t q = 0; q < d.NP; ++q) at[{d.h_near_i[q], d.h_near_j[q]}] = (int32_t)q;
    d.h_mirror.assign(d.NP, -1);
    bool closed = true;
    std::vector<int32_t> uq, ui, uj, lq, lm;
    for (int64_t q = 0; q < d.NP; ++q) {
      const int32_t i = d.h_near_i[q], j = d.h_near_j[q];
      auto it = at.find({j, i});
      if (it == at.end()) {
        closed = false;
        break;
      }
      d.h_mirror[q] = it->second;
      if (i <= j) uq.push_back((int32_t)q), ui.push_back(i), uj.push_back(j);
      else lq.push_back((int32_t)q), lm.push_back(it->second);
    }
    if (!closed) continue;
    d.near_sym = true;
    d.n_up = (int64_t)uq.size();
    d.n_lw = (int64_t)lq.size();
    CKS(upload(c, &d.su_q, uq));
    CKS(upload(c, &d.su_i, ui));
    CKS(upload(c, &d.su_j, uj));
    CKS(upload(c, &d.mirror, d.h_mirror));
    if (d.n_lw) {
      CKS(upload(c, &d.lw_q, lq));
      CKS(upload(c, &d.lw_m, lm));
    }
  }
  c->X64p.assign(L + 1, nullptr);
  c->S64p.assign(L + 1, nullptr);
  c->X32p.assign(L + 1, nullptr);
  c->S32p.assign(L + 1, nullptr);
  c->Slo.assign(L + 1, nullptr);
  c->Xlo.assign(L + 1, nullptr);
  size_t npart = c->sym ? (size_t)c->npu * 2 * lf.D : 0;
  // one batch of all levels' stored coupling pairs when every level with
  // couplings qualifies for the symmetric form with one common rank
  std::vector<int64_t> goff(L + 1, 0);
  {
    bool ok = true;
    int K0 = -1;
    int64_t tot = 0;
    for (int l = 1; l <= L && ok; ++l) {
      const DevLevel& d = c->lv[l];
      if (d.FP == 0) continue;
      if (!sym_leaf_supported(d.K) || (K0 >= 0 && d.K != K0) || c->hat_off[l] % d.K != 0) ok = false;
      K0 = d.K;
      goff[l] = tot;
      for (int64_t q = 0; q < d.FP; ++q) tot += d.h_far_i[q] < d.h_far_j[q];
    }
    c->cb_ok = ok && tot > 0;
    if (c->cb_ok) {
      c->cb_K = K0;
      c->cb_n = tot;
      CKC(dalloc(c, &c->S32u_all, (size_t)tot * K0 * K0));
    }
  }
  std::vector<int32_t> cbi, cbj;
  for (int l = 1; l <= L; ++l) {
    DevLevel& d = c->lv[l];
    const size_t nx = (size_t)d.nb * d.D * d.K, ns = (size_t)std::max<int64_t>(d.FP, 1) * d.K * d.K;
    CKC(dalloc(c, &d.X32, nx));
    CKC(dalloc(c, &d.S32, ns));
    launch_convert<double, float>(d.X, d.X32, (int64_t)nx, 0);
    launch_convert<double, float>(d.S, d.S32, (int64_t)ns, 0);
    d.far_sym = d.FP > 0 && sym_leaf_supported(d.K);
    if (d.far_sym) {
      // couplings of a symmetric kernel: S_ji = S_ij^T; keep i < j
      std::vector<int32_t> fq, fi, fj;
      for (int64_t q = 0; q < d.FP; ++q)
        if (d.h_far_i[q] < d.h_far_j[q]) fq.push_back((int32_t)q), fi.push_back(d.h_far_i[q]), fj.push_back(d.h_far_j[q]);
      d.fpu = (int64_t)fq.size();
      std::vector<std::vector<std::pair<int32_t, int32_t>>> lists(d.nb);
      for (int64_t k = 0; k < d.fpu; ++k) {
        lists[fi[k]].push_back({fj[k], (int32_t)(2 * k)});
        lists[fj[k]].push_back({fi[k], (int32_t)(2 * k + 1)});
      }
      std::vector<int64_t> ptr(d.nb + 1, 0);
      std::vector<int32_t> ent;
      for (int i = 0; i < d.nb; ++i) {
        std::sort(lists[i].begin(), lists[i].end());
        for (auto& pe : lists[i]) ent.push_back(pe.second);
        ptr[i + 1] = (int64_t)ent.size();
      }
      int32_t* fsq = nullptr;
      CKS(upload(c, &fsq, fq));
      CKS(upload(c, &d.fs_i, fi));
      CKS(upload(c, &d.fs_j, fj));
      CKS(upload(c, &d.fs_ptr, ptr));
      CKS(upload(c, &d.fs_ent, ent));
      const int64_t KK = (int64_t)d.K * d.K;
      if (c->cb_ok) {
        d.fs_goff = goff[l];
        d.S32u = c->S32u_all + goff[l] * KK;
        const int32_t s0 = (int32_t)(c->hat_off[l] / d.K);
        for (int64_t k = 0; k < d.fpu; ++k) cbi.push_back(s0 + fi[k]), cbj.push_back(s0 + fj[k]);
      } else {
        CKC(dalloc(c, &d.S32u, (size_t)(d.fpu * KK)));
      }
      launch_gather_blocks(d.S, fsq, KK, d.fpu, d.S32u, 0);
      npart = std::max(npart, (size_t)d.fpu * 2 * d.K);
    }
    // the residual's FP32-pair matvec reads the couplings in full
    CKC(dalloc(c, &c->Slo[l], ns));
    launch_split_lo(d.S, d.S32, c->Slo[l], (int64_t)d.FP * d.K * d.K, 0);
    CKC(dalloc(c, &c->Xlo[l], nx));
    launch_split_lo(d.X, d.X32, c->Xlo[l], (int64_t)nx, 0);
    c->X64p[l] = d.X;
    c->S64p[l] = d.S;
    c->X32p[l] = d.X32;
    c->S32p[l] = d.S32;
  }
  if (c->cb_ok) {
    CKS(upload(c, &c->cb_i, cbi));
    CKS(upload(c, &c->cb_j, cbj));
    CKC(dalloc(c, &c->part32c, (size_t)c->cb_n * 2 * c->cb_K));
  }
  if (npart) {
    CKC(dalloc(c, &c->part32, npart));
    CKC(dalloc(c, &c->part64, npart));
  }
  CKC(cudaGetLastError());

  CKC(dalloc(c, &c->red, 1024));  // three norm slots of 257 doubles: 0, 300, 600
  CKC(dalloc(c, &c->status, 4));
  CKC(cudaMemset(c->status, 0, 4 * sizeof(int32_t)));
  CKC(cudaDeviceSynchronize());
  // the FP16 copy of the leaf blocks used by mixed-precision factorizations
  if (L >= 1 && gemm_tc_supported(lf.D, lf.D, lf.D, lf.D, lf.D, lf.D)) CKS(make_leaf_lowp(c, 0));
  return H2_OK;
}

// ---------------------------------------------------------------------------
// factorization
// ---------------------------------------------------------------------------
struct Ev {
  cudaEvent_t e[2];
};

template <typename T>
void release_factor(h2_ctx* c, Factor<T>& F);

template <typename T>
h2_status alloc_factor_arrays(h2_ctx* c, Factor<T>& F) {
  AllocSink sink(c, &F.allocs);
  const int L = c->L;
  F.lv.assign(L + 1, FacLevel<T>());
  size_t wk = 0, wk16 = 0, wq = 0, wc = 0, wc16 = 0;
  for (int l = 0; l <= L; ++l) {
    const DevLevel& d = c->lv[l];
    FacLevel<T>& f = F.lv[l];
    const size_t nb = d.nb, D = d.D, K = d.K, R = d.R;
    wk = std::max(wk, (size_t)d.NP * D * D);
    const bool mixed = !std::is_same<T, double>::value;
    f.tc = mixed && l >= 1 && gemm_tc_supported(d.D, d.D, d.D, d.D, d.D, d.D);
    bool leaf64 = (l == L) && !mixed;
    if (!leaf64 && !(f.tc && l == L)) {
      if (f.tc) CKC(dalloc(c, reinterpret_cast<uint16_t**>(&f.Ain16), (size_t)d.NP * D * D));
      else CKC(dalloc(c, &f.Ain, (size_t)d.NP * D * D));
    }
    if (l == 0) continue;
    if (f.tc) {
      CKC(dalloc(c, reinterpret_cast<uint16_t**>(&f.U16), nb * D * D));
      wk16 = std::max(wk16, (size_t)d.NP * D * D);
    }
    f.tc_coup = mixed && d.FP > 0 && gemm_tc_supported(d.K, d.K, d.K, d.K, d.K, d.K);
    if (f.tc_coup) {
      CKC(dalloc(c, reinterpret_cast<uint16_t**>(&f.T16), nb * K * K));
      wc16 = std::max(wc16, (size_t)d.FP * K * K);
    } else {
      wc = std::max(wc, (size_t)d.FP * K * K);
    }
    CKC(dalloc(c, &f.U, nb * D * D));
    CKC(dalloc(c, &f.Ur, nb * D * D));
    CKC(dalloc(c, &f.Tm, nb * K * K));
    CKC(dalloc(c, &f.Xo, nb * D * K));
    CKC(dalloc(c, &f.Vq, nb * D * K));
    CKC(dalloc(c, &f.tau, nb * std::max<size_t>(K, 1)));
    CKC(dalloc(c, &f.Tw, nb * K * K));
    if (sizeof(T) * D * K > 200 * 1024) CKC(dalloc(c, &f.Qs, nb * D * K));
    wq = std::max(wq, nb * (K * K + D * K));
    CKC(dalloc(c, &f.Ahat, (size_t)d.NP * D * D));
    if (f.tc) CKC(dalloc(c, reinterpret_cast<uint16_t**>(&f.Ahat16), (size_t)d.NP * D * D));
    CKC(dalloc(c, &f.Shat, (size_t)std::max<int64_t>(d.FP, 1) * K * K));
    CKC(dalloc(c, &f.Z, nb * R * K));
    // LU factors in the factorization's precision (FP64: the lu array)
    if (std::is_same<T, double>::value) {
      CKC(dalloc(c, &f.lu, nb * R * R));
      f.luT = reinterpret_cast<T*>(f.lu);
    } else {
      CKC(dalloc(c, &f.luT, nb * R * R));
    }
    CKC(dalloc(c, &f.Ainv, nb * R * R));
    CKC(dalloc(c, &f.piv, nb * R));
    for (T** p : {&f.vin, &f.c, &f.xs}) CKC(dalloc(c, p, nb * D));
    CKC(dalloc(c, &f.M1, std::max<size_t>(nb * R * D, 1)));
    for (T** p : {&f.u, &f.v, &f.om}) CKC(dalloc(c, p, nb * std::max<size_t>(R, 1)));
  }
  const int D0 = c->lv[0].D;
  size_t npart = 1;
  for (int l = 1; l <= L; ++l) {
    const DevLevel& d = c->lv[l];
    npart = std::max(npart, (size_t)d.NP * (size_t)std::max(d.R, d.K));
  }
  CKC(dalloc(c, &F.part, npart));
  for (int l = 1; l <= L; ++l) F.lv[l].part = F.part;
  CKC(dalloc(c, &F.Wk, wk));
  if (wk16) CKC(dalloc(c, reinterpret_cast<uint16_t**>(&F.W16), wk16));
  CKC(dalloc(c, &F.Wq, std::max<size_t>(wq, 1)));
  if (wc) CKC(dalloc(c, &F.Wc, wc));
  if (wc16) CKC(dalloc(c, reinterpret_cast<uint16_t**>(&F.W16c), wc16));
  CKC(dalloc(c, &F.scales, 2 * (size_t)(L + 1)));
  CKC(dalloc(c, &F.tscale, 2 * (size_t)(L + 1)));
  CKC(dalloc(c, &F.cscale, (size_t)(L + 1)));
  CKC(dalloc(c, &F.amax, 3 * (size_t)(L + 1)));
  CKC(dalloc(c, &F.sch, 8));
  CKC(dalloc(c, &F.sch_amax, 2));
  // one root block per system (a forest has several)
  const size_t nr = (size_t)c->lv[0].nb;
  if (std::is_same<T, double>::value) {
    CKC(dalloc(c, &F.root_lu, nr * D0 * D0));
    F.root_luT = reinterpret_cast<T*>(F.root_lu);
  } else {
    CKC(dalloc(c, &F.root_luT, nr * D0 * D0));
  }
  CKC(dalloc(c, &F.root_inv, nr * D0 * D0));
  CKC(dalloc(c, &F.root_piv, nr * D0));
  CKC(dalloc(c, &F.root_vec, nr * D0));
  CKC(dalloc(c, &F.root_x, nr * D0));
  return H2_OK;
}

// A factorization's arrays, all or none: a failed allocation frees the
// ones made before it, so that the next h2_factor starts afresh.
template <typename T>
h2_status alloc_factor(h2_ctx* c, Factor<T>& F) {
  if (!F.lv.empty()) return H2_OK;
  const h2_status s = alloc_factor_arrays(c, F);
  if (s != H2_OK) {
    cudaGetLastError();
    release_factor(c, F);
  }
  return s;
}

template <typename T>
void gemm(int prec, int M, int N, int K, const T* A, int64_t sA, const int32_t* ia, int lda, bool tA, const T* B,
          int64_t sB, const int32_t* ib, int ldb, bool tB, T* C, int64_t sC, const int32_t* ic, int ldc, T alpha,
          T beta, int64_t batch, cudaStream_t st) {
  (void)prec;
  gemm_simt<T, T>(M, N, K, A, sA, ia, lda, tA, B, sB, ib, ldb, tB, C, sC, ic, ldc, alpha, beta, batch, st);
}

// The factorization runs on two streams.  The basis stream computes, level
// by level, what depends only on the bases: the complement bases (a1: QR of
// X^orth, which needs the children's T only), their 16-bit copy and the
// projected couplings (a2': T_i S_ij T_j^T).  The context's stream runs the
// chain through the matrix entries (a2 projection, a3 inverses, a4/a5
// Schur updates, a6 merge), waiting for level l's bases before a2 and for
// its couplings before a6.  The two chains share no buffer.
template <typename T>
h2_status factor_impl(h2_ctx* c, Factor<T>& F, int prec) {
  CKS(alloc_factor(c, F));
  const int L = c->L;
  cudaStream_t st = c->stream;
  if (!c->basis_stream) {
    // the highest priority: the other chain waits for each level's bases
    int least = 0, greatest = 0;
    CKC(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CKC(cudaStreamCreateWithPriority(&c->basis_stream, cudaStreamNonBlocking, greatest));
    CKC(cudaStreamCreateWithPriority(&c->coupling_stream, cudaStreamNonBlocking, greatest));
    CKC(cudaStreamCreateWithPriority(&c->product_stream, cudaStreamNonBlocking, least));
  }
  cudaStream_t sb = c->basis_stream, sc = c->coupling_stream, sp = c->product_stream;
  CKC(cudaMemsetAsync(c->status, 0, 4 * sizeof(int32_t), st));
  // timing marks: ev on the context's stream, evb on the basis stream
  std::vector<cudaEvent_t> ev, evb, sync;
  auto mark_on = [&](std::vector<cudaEvent_t>& v, cudaStream_t s) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    v.push_back(e);
  };
  auto mark = [&]() { mark_on(ev, st); };
  // s2 waits for everything issued so far on s1
  auto wait_for = [&](cudaStream_t s1, cudaStream_t s2) {
    cudaEvent_t e;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventRecord(e, s1);
    cudaStreamWaitEvent(s2, e, 0);
    sync.push_back(e);
  };
  auto release = [&]() {
    for (auto e : ev) cudaEventDestroy(e);
    for (auto e : evb) cudaEventDestroy(e);
    for (auto e : sync) cudaEventDestroy(e);
  };
  auto fail = [&](h2_status code, const std::string& msg) {
    c->err = msg;
    cudaStreamSynchronize(sb);
    cudaStreamSynchronize(sc);
    cudaStreamSynchronize(sp);
    cudaStreamSynchronize(st);
    release();
    return code;
  };
  mark();
  const int bf16 = (prec == H2_PREC_BF16) ? 1 : 0;
  F.bf16 = bf16;
  F.schur_tc = false;
  const bool mixed = !std::is_same<T, double>::value;
  // FP64 a3 for the FP16/BF16 factorizations: scratch for the largest level
  const bool lu64_mixed = mixed && c->rr_lu64;
  if (lu64_mixed && !F.rr_lu) {
    AllocSink sink(c, &F.allocs);
    size_t n = (size_t)c->lv[0].nb * c->lv[0].D * c->lv[0].D;
    for (int l = 1; l <= L; ++l) n = std::max(n, (size_t)c->lv[l].nb * c->lv[l].R * c->lv[l].R);
    CKC(dalloc(c, &F.rr_lu, n));
    CKC(dalloc(c, &F.rr_inv, n));
  }
  bool any_tc = false;
  for (int l = 1; l <= L; ++l) any_tc = any_tc || F.lv[l].tc || F.lv[l].tc_coup;
  if (mixed && any_tc) CKS(make_leaf_lowp(c, bf16));
  // the basis stream starts after earlier work on the context's stream (a
  // solve may still read U; the 16-bit couplings are made there)
  wait_for(st, sb);
  wait_for(st, sc);
  wait_for(st, sp);
  mark();
  const T* Aleaf = nullptr;
  if (!mixed) {
    Aleaf = reinterpret_cast<const T*>(c->A64);
  } else if (L == 0 || !F.lv[L].tc) {
    if (!c->A64) return fail(H2_ERR_STATE, "the leaf level needs the FP64 leaf blocks, which were released");
    launch_convert<double, T>(c->A64, F.lv[L].Ain, (int64_t)c->lv[L].NP * c->lv[L].D * c->lv[L].D, st);
    Aleaf = F.lv[L].Ain;
  }
  mark();

  // ---- basis stream: a1 (and the 16-bit copy of U), a2' per level
  std::string coup_err;
  for (int l = L; l >= 1; --l) {
    const DevLevel& d = c->lv[l];
    FacLevel<T>& f = F.lv[l];
    const int D = d.D, K = d.K, R = d.R;
    const int64_t DD = (int64_t)D * D;
    mark_on(evb, sb);
    // a1: complement bases.  X^orth = X (leaf) or blockdiag(T_2p, T_2p+1) X,
    // then Householder QR, the compact WY factor and U = P (I - V Tw V^T).
    {
      const int nb = d.nb;
      const int64_t DK = (int64_t)D * K, KK = (int64_t)K * K;
      // X in T, row-major D x K per box (the instance keeps FP64 and FP32 copies)
      const T* Xc = std::is_same<T, double>::value ? reinterpret_cast<const T*>(d.X) : reinterpret_cast<const T*>(d.X32);
      const T* Xin = Xc;
      if (l < L) {
        const int Kc = c->lv[l + 1].K;
        const T* Tc = F.lv[l + 1].Tm;
        const int64_t KcKc = (int64_t)Kc * Kc;
        gemm<T>(prec, Kc, K, Kc, Tc, 2 * KcKc, nullptr, Kc, false, Xc, DK, nullptr, K, false, f.Xo, DK, nullptr, K,
                T(1), T(0), nb, sb);
        gemm<T>(prec, Kc, K, Kc, Tc + KcKc, 2 * KcKc, nullptr, Kc, false, Xc + (int64_t)Kc * K, DK, nullptr, K,
                false, f.Xo + (int64_t)Kc * K, DK, nullptr, K, T(1), T(0), nb, sb);
        Xin = f.Xo;
      }
      // (the FP32 register form also forms the compact-WY factor Tw)
      const bool tw_done = launch_qr_panel<T>(nb, D, K, Xin, f.Vq, f.tau, f.Tm, f.Qs, sb, f.Tw);
      T* Sb = F.Wq;
      T* W1 = F.Wq + (int64_t)nb * KK;
      if (K > 0) {
        if (!tw_done) {
          gemm<T>(prec, K, K, D, f.Vq, DK, nullptr, D, false, f.Vq, DK, nullptr, D, true, Sb, KK, nullptr, K, T(1),
                  T(0), nb, sb);
          launch_wy_tfactor<T>(nb, K, Sb, f.tau, f.Tw, sb);
        }
        gemm<T>(prec, D, K, K, f.Vq, DK, nullptr, D, true, f.Tw, KK, nullptr, K, false, W1, DK, nullptr, K, T(1), T(0),
                nb, sb);
      }
      if constexpr (std::is_same<T, float>::value) {
        // one pass: U, its row-major copy and the 16-bit copy
        if (K > 0 && D % 4 == 0 && K % 4 == 0) {
          launch_form_u(nb, D, K, W1, f.Vq, f.U, f.Ur, f.tc ? f.U16 : nullptr, bf16, sb);
        } else {
          launch_perm_identity<T>(nb, D, K, f.U, sb);
          if (K > 0) {
            if (R > 0)
              gemm<T>(prec, R, D, K, f.Vq + K, DK, nullptr, D, true, W1, DK, nullptr, K, true, f.U, DD, nullptr, D,
                      T(-1), T(1), nb, sb);
            gemm<T>(prec, K, D, K, f.Vq, DK, nullptr, D, true, W1, DK, nullptr, K, true, f.U + (int64_t)R * D, DD,
                    nullptr, D, T(-1), T(1), nb, sb);
          }
          launch_transpose_blocks<T>(nb, D, f.U, f.Ur, sb);
          if (f.tc) launch_to_lowp<T>(bf16, f.U, f.U16, (int64_t)d.nb * DD, nullptr, sb);
        }
      } else {
        launch_perm_identity<T>(nb, D, K, f.U, sb);
        if (K > 0) {
          if (R > 0)
            gemm<T>(prec, R, D, K, f.Vq + K, DK, nullptr, D, true, W1, DK, nullptr, K, true, f.U, DD, nullptr, D,
                    T(-1), T(1), nb, sb);
          gemm<T>(prec, K, D, K, f.Vq, DK, nullptr, D, true, W1, DK, nullptr, K, true, f.U + (int64_t)R * D, DD,
                  nullptr, D, T(-1), T(1), nb, sb);
        }
        launch_transpose_blocks<T>(nb, D, f.U, f.Ur, sb);
        if (f.tc) launch_to_lowp<T>(bf16, f.U, f.U16, (int64_t)d.nb * DD, nullptr, sb);
      }
    }
    mark_on(evb, sb);
    // the couplings of level l follow its bases on the coupling stream
    CKC(cudaStreamWaitEvent(sc, evb.back(), 0));
    mark_on(evb, sc);
    // a2': couplings Shat_ij = T_i S_ij T_j^T
    if (d.FP > 0 && K > 0 && f.tc_coup) {
      // tensor cores: V^T = (S_s T_j,s^T)^T in 16 bits, then Shat = T_i,s V / (s_S s_T^2)
      const int64_t KK = (int64_t)K * K;
      unsigned int* am = F.amax + (L + 1) + l;
      CKC(cudaMemsetAsync(am, 0, sizeof(unsigned int), sc));
      launch_amax_blocks<T>(f.Tm, d.nb, KK, K, K, K, am, sc);
      launch_pow2_scale(am, std::sqrt(32768.0f / K), F.tscale + 2 * l, sc);
      launch_to_lowp<T>(bf16, f.Tm, f.T16, d.nb * KK, F.tscale + 2 * l, sc);
      launch_inv_scale_product(d.S16_scale[bf16], F.tscale + 2 * l, F.cscale + l, sc);
      bool ok = gemm_tc(bf16, K, K, K, d.S16[bf16], d.FP, K, K, nullptr, f.T16, d.nb, K, K, d.far_j, F.W16c, KK,
                        nullptr, K, 1, bf16, 1.0f, nullptr, d.FP, c->status + 2, sc, nullptr, -1, nullptr, nullptr,
                        nullptr, 0, 0) &&
                gemm_tc(bf16, K, K, K, f.T16, d.nb, K, K, d.far_i, F.W16c, d.FP, K, K, nullptr, f.Shat, KK, nullptr, K,
                        0, 0, 1.0f, F.cscale + l, d.FP, c->status + 2, sc, nullptr, -1, nullptr, nullptr, nullptr, 0,
                        0);
      if (!ok) {
        coup_err = "tensor-core coupling GEMM setup failed at level " + std::to_string(l);
        break;
      }
    } else if (d.FP > 0 && K > 0) {
      const int64_t KK = (int64_t)K * K;
      const T* Sc = std::is_same<T, double>::value ? reinterpret_cast<const T*>(d.S) : reinterpret_cast<const T*>(d.S32);
      gemm<T>(prec, K, K, K, Sc, KK, nullptr, K, false, f.Tm, KK, d.far_j, K, true, F.Wc, KK, nullptr, K, T(1),
              T(0), d.FP, sc);
      gemm<T>(prec, K, K, K, f.Tm, KK, d.far_i, K, false, F.Wc, KK, nullptr, K, false, f.Shat, KK, nullptr, K, T(1),
              T(0), d.FP, sc);
    }
    // max |Shat| for the 16-bit merge's scale, beside the main chain
    if (mixed && F.lv[l - 1].tc && std::is_same<T, float>::value) {
      unsigned int* am = F.amax + 2 * (L + 1) + l;
      CKC(cudaMemsetAsync(am, 0, sizeof(unsigned int), sc));
      launch_amax_blocks<float>(reinterpret_cast<const float*>(f.Shat), d.FP, (int64_t)K * K, K, K, K, am, sc);
    }
    mark_on(evb, sc);
  }
  if (!coup_err.empty()) return fail(H2_ERR_CUDA, coup_err);
  // evb holds four marks per level: [a1 start, a1 end = bases ready (basis
  // stream), a2' start, a2' end = couplings ready (coupling stream)]
  auto evb_at = [&](int l, int k) { return evb[(size_t)(L - l) * 4 + k]; };

  // levels whose projection covers the upper pairs only: symmetric near
  // lists on the tensor cores with the 16-bit substitution copy, R a
  // multiple of 32 (the transposed copy's tiles) and a parent merged in 16
  // bits (the merge reads the lower pairs' SS from their mirrors)
  for (int l = 0; l <= L; ++l) F.lv[l].proj_sym = false;
  for (int l = 2; l <= L; ++l) {
    const DevLevel& d = c->lv[l];
    F.lv[l].proj_sym = d.near_sym && F.lv[l].tc && F.lv[l - 1].tc && (bf16 || d.D <= 256) && d.R > 0 &&
                       d.R % 32 == 0 && d.K > 0;
  }
  // ---- the context's stream: a2, a3, a4/a5, a6 per level
  for (int l = L; l >= 1; --l) {
    const DevLevel& d = c->lv[l];
    FacLevel<T>& f = F.lv[l];
    const int D = d.D, K = d.K, R = d.R;
    const int64_t DD = (int64_t)D * D;
    mark();
    CKC(cudaStreamWaitEvent(st, evb_at(l, 1), 0));
    mark();
    // a2: Ahat_ij = U_i^T A_ij U_j
    if (f.tc) {
      // tensor cores: W^T = (s A_ij) U_j in 16 bits, then Ahat_ij = U_i^T W / s in FP32
      const void* A16 = (l == L) ? c->A16[bf16] : f.Ain16;
      const float* sc = (l == L) ? c->A16_scale[bf16] : F.scales + 2 * l;
      // The second GEMM also writes its raw accumulator s * Ahat in 16 bits
      // for the substitution.  |s Ahat_ij| <= ||s A_ij||_2 <= 128 D, inside
      // the FP16 range for D <= 256 (BF16 has the FP32 exponent range).
      const bool sub16 = bf16 || D <= 256;
      f.ahat_isc = sub16 ? sc + 1 : nullptr;
      f.err = c->status + 3;
      // tensor maps over the 16-bit copy for the TMA-fed substitution: the
      // quadrants must start on 16-byte columns and fit one pass of a CTA
      f.tma = false;
      if (sub16 && R > 0 && K > 0 && R % 8 == 0 && K % 8 == 0 && R <= 128 && K <= 128 &&
          (uint64_t)d.NP * D < (1ull << 31)) {
        const uint64_t rows = (uint64_t)d.NP * D;
        f.tma = make_tile_map(&f.tm_rr, f.Ahat16, bf16, rows, D, D, R, R) &&
                make_tile_map(&f.tm_sr, f.Ahat16, bf16, rows, D, D, K, R) &&
                make_tile_map(&f.tm_rs, f.Ahat16, bf16, rows, D, D, R, K);
      }
      // symmetric kernels: Ahat_ji = Ahat_ij^T, so only the upper pairs
      // (i <= j) are projected; the lower pairs' 16-bit blocks are their
      // mirrors transposed (beside the chain) and the merge reads their FP32
      // SS from the mirror (f.proj_sym, set before the loop).
      const int64_t np_proj = f.proj_sym ? d.n_up : d.NP;
      const int32_t* pq = f.proj_sym ? d.su_q : nullptr;
      const int32_t* pi = f.proj_sym ? d.su_i : d.near_i;
      const int32_t* pj = f.proj_sym ? d.su_j : d.near_j;
      // off-diagonal pairs keep only SS in FP32 (the merge's input); their
      // RR, RS and SR live in the 16-bit copy (the substitution's).  The
      // GEMM's epilogue also takes max |SS| of those pairs for the 16-bit
      // merge's scale.
      f.ahat_ss_only = sub16 && R % 16 == 0;
      unsigned int* am_ss = nullptr;
      if (f.ahat_ss_only && F.lv[l - 1].tc) {
        am_ss = F.amax + (l - 1);
        CKC(cudaMemsetAsync(am_ss, 0, sizeof(unsigned int), st));
      }
      bool ok = gemm_tc(bf16, D, D, D, A16, d.NP, D, D, pq, f.U16, d.nb, D, D, pj, F.W16, DD, nullptr, D, 1, bf16,
                        1.0f, nullptr, np_proj, c->status + 2, st) &&
                gemm_tc(bf16, D, D, D, f.U16, d.nb, D, D, pi, F.W16, np_proj, D, D, nullptr, f.Ahat, DD, pq, D, 0, 0,
                        1.0f, sc + 1, np_proj, c->status + 2, st, sub16 ? f.Ahat16 : nullptr, sub16 ? R : -1, pi,
                        pj, am_ss);
      if (ok && f.proj_sym && d.n_lw) {
        wait_for(st, sp);
        launch_transpose16_blocks(D, R, d.n_lw, d.lw_q, d.lw_m, f.Ahat16, sp);
      }
      if (!ok) return fail(H2_ERR_CUDA, "tensor-core GEMM setup failed at level " + std::to_string(l));
    } else if (!mixed && d.near_sym && d.n_lw > 0) {
      // FP64, symmetric near list: project the upper pairs i <= j, then
      // Ahat_ji = Ahat_ij^T for the lower ones (the kernels are symmetric)
      const T* Ain = (l == L) ? Aleaf : f.Ain;
      gemm<T>(prec, D, D, D, Ain, DD, d.su_q, D, false, f.U, DD, d.su_j, D, true, F.Wk, DD, nullptr, D, T(1), T(0),
              d.n_up, st);
      gemm<T>(prec, D, D, D, f.U, DD, d.su_i, D, false, F.Wk, DD, nullptr, D, false, f.Ahat, DD, d.su_q, D, T(1),
              T(0), d.n_up, st);
      launch_transpose_pairs<T>(D, d.n_lw, d.lw_q, d.lw_m, f.Ahat, st);
    } else {
      const T* Ain = (l == L) ? Aleaf : f.Ain;
      gemm<T>(prec, D, D, D, Ain, DD, nullptr, D, false, f.U, DD, d.near_j, D, true, F.Wk, DD, nullptr, D, T(1),
              T(0), d.NP, st);
      gemm<T>(prec, D, D, D, f.U, DD, d.near_i, D, false, F.Wk, DD, nullptr, D, false, f.Ahat, DD, nullptr, D, T(1),
              T(0), d.NP, st);
    }
    mark();
    // a3: LU of Ahat_ii^RR and its inverse (FP16/BF16 factorizations: in
    // FP64 from the FP32 blocks, or FP32 Gauss-Jordan)
    if (lu64_mixed)
      launch_lu_inverse_f64_for_f32(d.nb, D, R, reinterpret_cast<const float*>(f.Ahat), d.diag_pair, F.rr_lu,
                                    F.rr_inv, f.piv, reinterpret_cast<float*>(f.Ainv), c->status, l, st);
    else
      launch_lu_inverse<T>(d.nb, D, R, f.Ahat, d.diag_pair, f.lu, f.luT, f.piv, f.Ainv, c->status, l, st);
    mark();
    // the substitution's first product M1 = Ainv (U^R)^T, beside the chain
    // ((U^R)^T: the first R columns of the column-major U, as rows)
    if (R > 0) {
      wait_for(st, sp);
      gemm<T>(prec, R, D, R, f.Ainv, (int64_t)R * R, nullptr, R, false, f.U, DD, nullptr, D, false, f.M1,
              (int64_t)R * D, nullptr, D, T(1), T(0), d.nb, sp);
    }
    // a4 + a5: Z = Ainv Ahat_ii^RS; Ahat_ii^SS -= Ahat_ii^SR Z.  On the
    // tensor cores (16-bit operands, FP32 accumulation) where the level's
    // 16-bit copy s Ahat holds the diagonal blocks' SR quadrant: with the
    // symmetric Ahat_ii (Ahat_ii^RS = (Ahat_ii^SR)^T),
    //   Z^T = Ahat_ii^SR Ainv^T        (GEMM 1: A = s SR, B = s_i Ainv)
    //   SS -= Ahat_ii^SR (Z^T)^T       (GEMM 2: A = s SR, B = s_z Z^T)
    // with power-of-two scales s_i, s_z from max |Ainv|, max |Z^T|.
    const float* sc_l = (l == L) ? c->A16_scale[bf16] : F.scales + 2 * l;
    const bool schur_tc = mixed && f.tc && f.ahat_isc && d.near_sym && R > 0 && K > 0 && R % 64 == 0 &&
                          gemm_tc_supported(K, R, R, D, R, R) && gemm_tc_supported(K, K, R, D, R, D);
    if (schur_tc) {
      const int64_t nb = d.nb, RR = (int64_t)R * R, KR = (int64_t)K * R;
      float* Zt = reinterpret_cast<float*>(F.Wk);
      uint16_t* Ai16 = reinterpret_cast<uint16_t*>(F.W16);
      uint16_t* Z16 = Ai16 + nb * RR;
      CKC(cudaMemsetAsync(F.sch_amax, 0, 2 * sizeof(unsigned int), st));
      launch_amax_blocks<float>(reinterpret_cast<const float*>(f.Ainv), nb, RR, R, R, R, F.sch_amax, st);
      launch_pow2_scale(F.sch_amax, 16384.0f, F.sch, st);
      launch_to_lowp<float>(bf16, reinterpret_cast<const float*>(f.Ainv), Ai16, nb * RR, F.sch, st);
      launch_inv_scale_pair(sc_l, F.sch, F.sch + 4, st);
      const void* SR16 = static_cast<const uint16_t*>(f.Ahat16) + (int64_t)R * D;
      bool ok = gemm_tc(bf16, K, R, R, SR16, d.NP, D, D, d.diag_pair, Ai16, nb, R, R, nullptr, Zt, KR, nullptr, R, 0,
                        0, 1.0f, F.sch + 4, nb, c->status + 2, st, nullptr, -1, nullptr, nullptr, nullptr,
                        d.NP * (int64_t)D - R);
      if (ok) {
        launch_amax_blocks<float>(Zt, nb, KR, K, R, R, F.sch_amax + 1, st);
        launch_pow2_scale(F.sch_amax + 1, 16384.0f, F.sch + 2, st);
        launch_to_lowp<float>(bf16, Zt, Z16, nb * KR, F.sch + 2, st);
        launch_inv_scale_pair(sc_l, F.sch + 2, F.sch + 5, st);
        ok = gemm_tc(bf16, K, K, R, SR16, d.NP, D, D, d.diag_pair, Z16, nb, K, R, nullptr,
                     reinterpret_cast<float*>(f.Ahat) + (int64_t)R * D + R, DD, d.diag_pair, D, 3, 0, -1.0f,
                     F.sch + 5, nb, c->status + 2, st, nullptr, -1, nullptr, nullptr, nullptr, d.NP * (int64_t)D - R);
      }
      if (!ok) return fail(H2_ERR_CUDA, "tensor-core Schur update setup failed at level " + std::to_string(l));
      F.schur_tc = true;
    } else if (R > 0 && K > 0) {
      gemm<T>(prec, R, K, R, f.Ainv, (int64_t)R * R, nullptr, R, false, f.Ahat + R, DD, d.diag_pair, D, false, f.Z,
              (int64_t)R * K, nullptr, K, T(1), T(0), d.nb, st);
      gemm<T>(prec, K, K, R, f.Ahat + (int64_t)R * D, DD, d.diag_pair, D, false, f.Z, (int64_t)R * K, nullptr, K,
              false, f.Ahat + (int64_t)R * D + R, DD, d.diag_pair, D, T(-1), T(1), d.nb, st);
    }
    mark();
    CKC(cudaStreamWaitEvent(st, evb_at(l, 3), 0));
    mark();
    // a6: merge into the parent level's near blocks
    FacLevel<T>& pf = F.lv[l - 1];
    if (mixed && pf.tc) {
      // 16-bit parent blocks with a fresh power-of-two scale from max |SS|
      // (off-diagonal pairs: the projection's epilogue; diagonal pairs,
      // after their Schur update: here) and max |Shat| (coupling stream)
      unsigned int* am = F.amax + (l - 1);
      if (std::is_same<T, float>::value) {
        const float* Ah = reinterpret_cast<const float*>(f.Ahat);
        const float* Sh = reinterpret_cast<const float*>(f.Shat);
        if (f.tc && f.ahat_ss_only) {
          launch_amax_blocks<float>(Ah + (int64_t)R * D + R, d.nb, DD, K, K, D, am, st, d.diag_pair);
        } else {
          // (the lower pairs' SS are their mirrors' transposed: the upper
          // ones cover every value)
          CKC(cudaMemsetAsync(am, 0, sizeof(unsigned int), st));
          launch_amax_blocks<float>(Ah + (int64_t)R * D + R, f.proj_sym ? d.n_up : d.NP, DD, K, K, D, am, st,
                                    f.proj_sym ? d.su_q : nullptr);
        }
        launch_pow2_scale(am, 128.0f, F.scales + 2 * (l - 1), st, d.FP > 0 && K > 0 ? F.amax + 2 * (L + 1) + l : nullptr);
        // (pairs bound for a lower parent pair are skipped when the parent
        // projects its upper pairs only)
        launch_merge_lowp(D, K, d.NP, Ah, d.near_i, d.near_j, d.near_dst, d.FP, Sh, d.far_i, d.far_j, d.far_dst,
                          pf.Ain16, F.scales + 2 * (l - 1), bf16, st, f.proj_sym ? d.mirror : nullptr,
                          pf.proj_sym ? 1 : 0);
      }
    } else {
      launch_merge<T>(D, K, d.NP, f.Ahat, d.near_i, d.near_j, d.near_dst, d.FP, f.Shat, d.far_i, d.far_j, d.far_dst,
                      pf.Ain, st);
    }
    mark();
  }
  if (L >= 1) CKC(cudaStreamWaitEvent(st, evb.back(), 0));
  wait_for(sp, st);
  // a7: root
  const int D0 = c->lv[0].D;
  const T* Aroot = (L == 0) ? Aleaf : F.lv[0].Ain;
  const int nr = c->lv[0].nb;  // one root per system (the level-0 blocks are in box order)
  if (lu64_mixed)
    launch_lu_inverse_f64_for_f32(nr, D0, D0, reinterpret_cast<const float*>(Aroot), nullptr, F.rr_lu, F.rr_inv,
                                  F.root_piv, reinterpret_cast<float*>(F.root_inv), c->status, 0, st);
  else
    launch_lu_inverse<T>(nr, D0, D0, Aroot, nullptr, F.root_lu, F.root_luT, F.root_piv, F.root_inv, c->status, 0, st);
  mark();
  CKC(cudaGetLastError());
  CKC(cudaStreamSynchronize(st));
  // phase times
  PhaseTimes& t = c->times;
  t = PhaseTimes();
  auto el = [&](int a, int b) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ev[a], ev[b]);
    return (double)ms * 1e-3;
  };
  auto elb = [&](int a, int b) {
    float ms = 0;
    cudaEventElapsedTime(&ms, evb[a], evb[b]);
    return (double)ms * 1e-3;
  };
  // main-stream marks: [start, leaf copies, leaf conversion], then per level
  // [wait start, a2 start, a2 end, a3 end, a4/a5 end, a6 start, a6 end], then
  // the root.  The basis-stream phases (a1, a2') overlap the others; the
  // main stream's waits for them are wait_basis.
  t.a2_proj += el(1, 2);  // leaf conversion counted with the projection
  int k = 3;
  for (int l = L; l >= 1; --l) {
    const int kb = (L - l) * 4;
    t.a1_qr += elb(kb, kb + 1);
    t.a2c_coupling += elb(kb + 2, kb + 3);
    t.wait_basis += el(k, k + 1) + el(k + 4, k + 5);
    t.a2_proj += el(k + 1, k + 2);
    t.a3_lu += el(k + 2, k + 3);
    t.a5_schur += el(k + 3, k + 4);
    t.a6_merge += el(k + 5, k + 6);
    k += 7;
  }
  t.a7_root = el(k - 1, k);
  t.total_factor = el(1, k);
  release();
  int32_t stw[4];
  CKC(cudaMemcpy(stw, c->status, sizeof(stw), cudaMemcpyDeviceToHost));
  if (stw[2] != 0) {
    c->err = "a bounded wait in the tensor-core GEMM expired";
    return H2_ERR_TIMEOUT;
  }
  if (stw[0] != 0) {
    c->err = "zero pivot in the LU of level " + std::to_string(stw[0] - 1) + " box " + std::to_string(stw[1]);
    return H2_ERR_SINGULAR;
  }
  F.ready = true;
  c->used_tc = false;
  for (int l = 1; l <= L; ++l) c->used_tc = c->used_tc || F.lv[l].tc;
  return H2_OK;
}

// ---------------------------------------------------------------------------
// substitution (Eq. 24-31 and its mirror)
// ---------------------------------------------------------------------------
// One sweep: input in the leaf level's vin (root_vec when L = 0), output in
// the leaf level's xs (root_x when L = 0).
// Calls fn(Ahat, iscale) with the level's projected blocks in the type the
// substitution reads them in: the 16-bit copy s * Ahat with 1 / s where the
// factorization wrote one, else Ahat itself with no scale.
template <typename T, typename Fn>
void with_ahat(const FacLevel<T>& f, int bf16, Fn&& fn) {
  if constexpr (std::is_same<T, float>::value) {
    if (f.Ahat16 && f.ahat_isc) {
      if (bf16) fn(reinterpret_cast<const __nv_bfloat16*>(f.Ahat16), f.ahat_isc);
      else fn(reinterpret_cast<const __half*>(f.Ahat16), f.ahat_isc);
      return;
    }
  }
  fn(static_cast<const T*>(f.Ahat), static_cast<const float*>(nullptr));
}

template <typename T>
void ulv_sweep(h2_ctx* c, Factor<T>& F) {
  const int L = c->L;
  cudaStream_t st = c->stream;
  // the children's input of level l (below the leaf level: their SR sums)
  auto child_in = [&](int l) {
    ChildIn<T> ch;
    if (l < L) {
      const DevLevel& dc = c->lv[l + 1];
      const FacLevel<T>& fc = F.lv[l + 1];
      ch.c = fc.c;
      ch.part = fc.part;
      ch.ptr = dc.near_ptr;
      with_ahat(fc, F.bf16, [&](auto, const float* isc) { ch.iscale = isc; });
      ch.D = dc.D, ch.R = dc.R, ch.K = dc.K;
    }
    return ch;
  };
  auto fwd = [&](int l) {
    const DevLevel& d = c->lv[l];
    FacLevel<T>& f = F.lv[l];
    launch_fwd1<T>(d, f, child_in(l), st);
    with_ahat(f, F.bf16, [&](auto A, const float* isc) {
      using TS = std::remove_const_t<std::remove_pointer_t<decltype(A)>>;
      launch_fwd2<T, TS>(d, f, A, isc, st);
      launch_fwd3<T, TS>(d, f, A, isc, l == 1 ? F.root_vec : nullptr, st);
    });
  };
  auto bwd = [&](int l) {
    const DevLevel& d = c->lv[l];
    FacLevel<T>& f = F.lv[l];
    const T* px = (l > 1) ? F.lv[l - 1].xs : F.root_x;
    with_ahat(f, F.bf16, [&](auto A, const float* isc) {
      using TS = std::remove_const_t<std::remove_pointer_t<decltype(A)>>;
      launch_bwd1<T, TS>(d, f, A, isc, px, st);
      launch_bwd2<T, TS>(d, f, A, isc, px, st);
    });
  };
  for (int l = L; l >= 1; --l) fwd(l);
  launch_gemv_rows<T>(c->lv[0].nb, c->lv[0].D, F.root_inv, F.root_vec, F.root_x, st);
  for (int l = 1; l <= L; ++l) bwd(l);
}
template <typename T>
T* ulv_in(h2_ctx* c, Factor<T>& F) { return c->L >= 1 ? F.lv[c->L].vin : F.root_vec; }
template <typename T>
T* ulv_out(h2_ctx* c, Factor<T>& F) { return c->L >= 1 ? F.lv[c->L].xs : F.root_x; }

int64_t nslots(const h2_ctx* c) { return (int64_t)c->lv[c->L].nb * c->lv[c->L].D; }

// x += ULV^-1 r for FP64 tree vectors; the sweep runs in T on r / ||r||.
template <typename T>
void ulv_apply_impl(h2_ctx* c, Factor<T>& F, const double* r, double* x) {
  const int64_t n = nslots(c);
  launch_norm2<double>(r, n, c->red, c->stream);
  launch_scale_to<T>(r, c->red, ulv_in(c, F), n, c->stream);
  ulv_sweep<T>(c, F);
  launch_axpy_from<T>(ulv_out(c, F), c->red, x, n, c->stream);
}

// Capture fn's work on the context's stream into a CUDA graph (on a private
// capture stream); nullptr if the capture or instantiation fails, in which
// case the caller runs fn directly.
template <class Fn>
cudaGraphExec_t capture_graph(h2_ctx* c, long long& kernels, Fn fn) {
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaStream_t keep = c->stream;
  c->stream = c->cap_stream;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  const long long n0 = g_launches.load();
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    fn();
    if (cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && g) {
      if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    }
  }
  kernels = g_launches.load() - n0;
  g_launches -= kernels;  // counted again per replay
  if (g) cudaGraphDestroy(g);
  c->stream = keep;
  cudaGetLastError();
  return ex;
}

void drop_graphs(h2_ctx* c) {
  if (c->g_ulv) cudaGraphExecDestroy(c->g_ulv);
  c->g_ulv = nullptr;
}

// z = ULV^-1 v for FP32 tree vectors (mixed-precision factorization); the
// sweep (about a hundred dependent launches) replays as one CUDA graph.
void ulv_apply_f32(h2_ctx* c, const float* v, float* z) {
  const int64_t n = nslots(c);
  Factor<float>& F = c->f32;
  cudaMemcpyAsync(ulv_in(c, F), v, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  if (c->use_graphs && !c->g_ulv) c->g_ulv = capture_graph(c, c->g_ulv_kernels, [&] { ulv_sweep<float>(c, F); });
  if (c->use_graphs && c->g_ulv) {
    cudaGraphLaunch(c->g_ulv, c->stream);
    g_launches += c->g_ulv_kernels;
  } else {
    ulv_sweep<float>(c, F);
  }
  cudaMemcpyAsync(z, ulv_out(c, F), n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
}

// ---------------------------------------------------------------------------
// H^2 matvec over the FP64 instance (refinement residual) or its FP32 copy
// (inner solver of the mixed-precision refinement)
// ---------------------------------------------------------------------------
using EventPairs = std::vector<std::pair<cudaEvent_t, cudaEvent_t>>;

// y = A_H2 x; with leaf_ev set, the leaf-level kernel (near blocks plus the
// leaf basis) is bracketed by a pair of events appended there.
template <typename T>
void matvec_t(h2_ctx* c, const T* A, T* const* X, T* const* S, T* xh, T* yh, const T* x, T* y,
              EventPairs* leaf_ev = nullptr) {
  const int L = c->L;
  cudaStream_t st = c->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (leaf_ev) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  // leaf step: y = X_L yh_L + near-field; the FP32 copy may hold only the
  // i <= j halves of the symmetric near blocks
  auto leaf = [&](const T* XL, const T* yhL) {
    if constexpr (std::is_same<T, float>::value) {
      if (c->sym) {
        const DevLevel& lf = c->lv[L];
        if (leaf_ev) cudaEventRecord(e0, st);
        launch_matvec_sym_pairs(lf.D, c->npu, c->sym_i, c->sym_j, A, x, c->part32, false, st);
        if (leaf_ev) cudaEventRecord(e1, st), leaf_ev->push_back({e0, e1});
        launch_matvec_sym_sum<float>(lf.nb, lf.D, L ? lf.K : 0, c->sym_ptr, c->sym_ent, XL, yhL, c->part32, y, st);
        return;
      }
    }
    if (leaf_ev) cudaEventRecord(e0, st);
    launch_matvec_leaf<T>(c->lv[L], A, XL, x, yhL, y, st);
    if (leaf_ev) cudaEventRecord(e1, st), leaf_ev->push_back({e0, e1});
  };
  if (L == 0) {
    leaf(nullptr, nullptr);
    return;
  }
  const std::vector<int64_t>& off = c->hat_off;
  if constexpr (std::is_same<T, float>::value) {
    if (c->cb_ok && c->sym) {
      // the leaf near-field products need only x: they run on the leaf
      // stream beside the upward pass, the couplings (every level in one
      // launch) and the downward pass, which adds each level's coupling
      // sums as it goes; the per-box leaf sums follow the join
      if (!c->leaf_stream) {
        cudaStreamCreateWithFlags(&c->leaf_stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&c->mv_fork, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->mv_join, cudaEventDisableTiming);
      }
      cudaStream_t sl = c->leaf_stream;
      const DevLevel& lf = c->lv[L];
      cudaEventRecord(c->mv_fork, st);
      cudaStreamWaitEvent(sl, c->mv_fork, 0);
      if (leaf_ev) cudaEventRecord(e0, sl);
      launch_matvec_sym_pairs(lf.D, c->npu, c->sym_i, c->sym_j, A, x, c->part32, false, sl);
      if (leaf_ev) cudaEventRecord(e1, sl), leaf_ev->push_back({e0, e1});
      cudaEventRecord(c->mv_join, sl);
      launch_matvec_up<T>(c->lv[L], X[L], x, xh + off[L], st);
      for (int l = L - 1; l >= 1; --l) launch_matvec_up<T>(c->lv[l], X[l], xh + off[l + 1], xh + off[l], st);
      launch_matvec_sym_pairs(c->cb_K, c->cb_n, c->cb_i, c->cb_j, c->S32u_all, xh, c->part32c, true, st);
      const DevLevel& d1 = c->lv[1];
      if (d1.FP > 0 && d1.K > 0)
        launch_matvec_sym_sum<float>(d1.nb, d1.K, 0, d1.fs_ptr, d1.fs_ent, nullptr, nullptr,
                                     c->part32c + d1.fs_goff * 2 * d1.K, yh + off[1], st);
      else
        cudaMemsetAsync(yh + off[1], 0, sizeof(T) * (size_t)d1.nb * d1.K, st);
      for (int l = 1; l < L; ++l) {
        const DevLevel& dc = c->lv[l + 1];
        const bool has = dc.FP > 0 && dc.K > 0;
        launch_matvec_down_far<float>(c->lv[l], X[l], yh + off[l], yh + off[l + 1], has ? dc.fs_ptr : nullptr,
                                      has ? dc.fs_ent : nullptr, c->part32c + dc.fs_goff * 2 * dc.K, st);
      }
      cudaStreamWaitEvent(st, c->mv_join, 0);
      launch_matvec_sym_sum<float>(lf.nb, lf.D, lf.K, c->sym_ptr, c->sym_ent, X[L], yh + off[L], c->part32, y, st,
                                   false);
      return;
    }
  }
  launch_matvec_up<T>(c->lv[L], X[L], x, xh + off[L], st);
  for (int l = L - 1; l >= 1; --l) launch_matvec_up<T>(c->lv[l], X[l], xh + off[l + 1], xh + off[l], st);
  for (int l = 1; l <= L; ++l) {
    const DevLevel& d = c->lv[l];
    if constexpr (std::is_same<T, float>::value) {
      if (d.far_sym) {  // stored halves of the symmetric couplings
        launch_matvec_sym_pairs(d.K, d.fpu, d.fs_i, d.fs_j, d.S32u, xh + off[l], c->part32, true, st);
        launch_matvec_sym_sum<float>(d.nb, d.K, 0, d.fs_ptr, d.fs_ent, nullptr, nullptr, c->part32, yh + off[l], st);
        continue;
      }
    }
    launch_matvec_far<T>(d, S[l], xh + off[l], yh + off[l], st);
  }
  for (int l = 1; l < L; ++l) launch_matvec_down<T>(c->lv[l], X[l], yh + off[l], yh + off[l + 1], st);
  leaf(X[L], yh + off[L]);
}

void matvec_impl(h2_ctx* c, const double* x, double* y) {
  matvec_t<double>(c, c->A64, c->X64p.data(), c->S64p.data(), c->xhat, c->yhat, x, y);
}
// The same product with the couplings and the leaf step in FP32-pair
// arithmetic on the FP32 split of the FP64 matrix (about 2^-48 per entry);
// the upward and downward passes stay FP64.
void matvec_df(h2_ctx* c, const double* x, double* y) {
  const int L = c->L;
  cudaStream_t st = c->stream;
  const DevLevel& lf = c->lv[L];
  const std::vector<int64_t>& off = c->hat_off;
  launch_split_df(x, c->xdf_h, c->xdf_l, nslots(c), st);
  if (L >= 1) {
    // upward pass, couplings of all levels in one launch, downward pass
    launch_matvec_up_df(lf, c->X32p[L], c->Xlo[L], c->xdf_h, c->xdf_l, c->hdf_h + off[L], c->hdf_l + off[L], st);
    for (int l = L - 1; l >= 1; --l)
      launch_matvec_up_df(c->lv[l], c->X32p[l], c->Xlo[l], c->hdf_h + off[l + 1], c->hdf_l + off[l + 1],
                          c->hdf_h + off[l], c->hdf_l + off[l], st);
    // levels with the longest far lists first (their CTAs take longest)
    std::vector<int> order;
    for (int l = 1; l <= L; ++l) order.push_back(l);
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
      return c->lv[u].FP * (int64_t)c->lv[v].nb > c->lv[v].FP * (int64_t)c->lv[u].nb;
    });
    FarDfArgs fa{};
    int cta = 0;
    for (int l : order) {
      const DevLevel& d = c->lv[l];
      if (d.FP == 0 || d.K == 0) {
        // no couplings: yhat starts at zero
        cudaMemsetAsync(c->ydf_h + off[l], 0, sizeof(float) * d.nb * d.K, st);
        cudaMemsetAsync(c->ydf_l + off[l], 0, sizeof(float) * d.nb * d.K, st);
        continue;
      }
      if (fa.nlev == kMaxFarDfLevels) {
        launch_matvec_far_df_all(fa, st);
        fa = FarDfArgs{};
        cta = 0;
      }
      FarDfLevel& f = fa.lv[fa.nlev++];
      f = {d.far_ptr, d.far_j, c->S32p[l], c->Slo[l], c->hdf_h + off[l], c->hdf_l + off[l], c->ydf_h + off[l],
           c->ydf_l + off[l], d.nb, d.K, (d.K + 63) / 64, cta};
      cta += d.nb * f.nch;
    }
    launch_matvec_far_df_all(fa, st);
    for (int l = 1; l < L; ++l)
      launch_matvec_down_df(c->lv[l], c->X32p[l], c->Xlo[l], c->ydf_h + off[l], c->ydf_l + off[l],
                            c->ydf_h + off[l + 1], c->ydf_l + off[l + 1], st);
  }
  const float* yhh = L ? c->ydf_h + off[L] : nullptr;
  const float* yhl = L ? c->ydf_l + off[L] : nullptr;
  if (c->sym) {
    // the partial products as FP32 pairs in the space of the FP64 ones
    float* ph = reinterpret_cast<float*>(c->part64);
    float* pl = ph + c->npu * 2 * lf.D;
    launch_matvec_sym_pairs_df(lf.D, c->npu, c->sym_i, c->sym_j, c->A32, c->Alo, c->xdf_h, c->xdf_l, ph, pl, st);
    launch_matvec_sym_sum_df(lf.nb, lf.D, L ? lf.K : 0, c->sym_ptr, c->sym_ent, L ? c->X32p[L] : nullptr,
                             L ? c->Xlo[L] : nullptr, yhh, yhl, ph, pl, y, st);
  } else {
    launch_matvec_leaf_df(lf, c->A32, c->Alo, L ? c->X32p[L] : nullptr, L ? c->Xlo[L] : nullptr, c->xdf_h, c->xdf_l,
                          yhh, yhl, y, st);
  }
}
void matvec32(h2_ctx* c, const float* x, float* y, EventPairs* leaf_ev = nullptr) {
  matvec_t<float>(c, c->A32, c->X32p.data(), c->S32p.data(), c->xhat32, c->yhat32, x, y, leaf_ev);
}

// The substitution's TMA-fed kernels set status[3] when a bounded wait
// gives up: clear it before a solve, read it after.
h2_status subst_clear(h2_ctx* c) {
  CKC(cudaMemsetAsync(c->status + 3, 0, sizeof(int32_t), c->stream));
  return H2_OK;
}
h2_status subst_check(h2_ctx* c) {
  int32_t w = 0;
  CKC(cudaMemcpyAsync(&w, c->status + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CKC(cudaStreamSynchronize(c->stream));
  if (w != 0) {
    c->err = "a substitution kernel's wait for its tensor copies timed out";
    return H2_ERR_TIMEOUT;
  }
  return H2_OK;
}

// Fill the RR, RS and SR quadrants of the off-diagonal pairs of an exported
// mixed-precision Ahat (host, FP32) from the 16-bit copy.
h2_status export_ahat_quadrants(const h2_ctx* c, int level, float* out) {
  const FacLevel<float>& f = c->f32.lv[level];
  const DevLevel& d = c->lv[level];
  const size_t D = d.D, R = d.R, n = (size_t)d.NP * D * D;
  std::vector<uint16_t> h(n);
  float isc = 1.0f;
  if (cudaMemcpy(h.data(), f.Ahat16, n * 2, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&isc, f.ahat_isc, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return H2_ERR_CUDA;
  const bool bf = c->f32.bf16 == 1;
  // upper-pair projection: a lower pair's FP32 SS is its mirror's transposed
  if (f.proj_sym) {
    for (int64_t q = 0; q < d.NP; ++q) {
      if (d.h_near_i[q] <= d.h_near_j[q]) continue;
      const size_t m = (size_t)d.h_mirror[q];
      for (size_t r = R; r < D; ++r)
        for (size_t col = R; col < D; ++col) out[(size_t)q * D * D + r * D + col] = out[m * D * D + col * D + r];
    }
  }
  for (int64_t q = 0; q < d.NP; ++q) {
    if (d.h_near_i[q] == d.h_near_j[q]) continue;
    for (size_t r = 0; r < D; ++r)
      for (size_t col = 0; col < D; ++col) {
        if (r >= R && col >= R) continue;
        const size_t e = (size_t)q * D * D + r * D + col;
        float v;
        if (bf) {
          __nv_bfloat16_raw raw;
          raw.x = h[e];
          v = __bfloat162float(__nv_bfloat16(raw));
        } else {
          __half_raw raw;
          raw.x = h[e];
          v = __half2float(__half(raw));
        }
        out[e] = v * isc;
      }
  }
  return H2_OK;
}

bool factor_ready(const h2_ctx* c) {
  return (c->prec == H2_PREC_FP64 && c->f64.ready) || (c->prec > 0 && c->f32.ready);
}

void ulv_apply_any(h2_ctx* c, const double* r, double* x) {
  if (c->prec == H2_PREC_FP64) ulv_apply_impl<double>(c, c->f64, r, x);
  else ulv_apply_impl<float>(c, c->f32, r, x);
}

// CUDA-event timing of the substitution and matvec calls inside a solve
struct SolveTimer {
  using Pairs = EventPairs;
  Pairs sub, mv, mv32, leaf32;  // leaf32: the leaf kernel inside each FP32 matvec
  cudaStream_t st;
  explicit SolveTimer(cudaStream_t s) : st(s) {}
  template <class Fn>
  void run(Pairs& v, Fn fn) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    fn();
    cudaEventRecord(b, st);
    v.push_back({a, b});
  }
  static double total(Pairs& v) {
    double t = 0;
    for (auto& e : v) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e.first, e.second);
      t += ms * 1e-3;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    v.clear();
    return t;
  }
};

// copy an N-vector in (orig order, host or device) to the padded tree vector
h2_status vec_in(h2_ctx* c, const double* src, double* tree) {
  const double* dsrc = src;
  if (!is_device_ptr(src)) {
    CKC(cudaMemcpyAsync(c->io_a, src, c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    dsrc = c->io_a;
  }
  launch_gather(c->slot_pt, dsrc, tree, nslots(c), c->stream);
  return H2_OK;
}

h2_status vec_out(h2_ctx* c, const double* tree, double* dst) {
  bool dev = is_device_ptr(dst);
  double* ddst = dev ? dst : c->io_b;
  launch_scatter(c->slot_pt, tree, ddst, nslots(c), c->stream);
  if (!dev) {
    CKC(cudaMemcpyAsync(dst, ddst, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CKC(cudaStreamSynchronize(c->stream));
  }
  return H2_OK;
}

// ---------------------------------------------------------------------------
// One FGMRES cycle (right preconditioned, classical Gram-Schmidt applied
// twice, Givens rotations on the host) on vectors of type T.  r is the
// right-hand side with norm beta; the cycle stops after m steps or when the
// residual estimate falls to tol_abs.  On return W.y[0..k) hold the
// coefficients of the solution update sum_j y_j Z_j.
// ---------------------------------------------------------------------------
struct GmresWork {
  int m0 = 0;
  double *h1 = nullptr, *h2 = nullptr, *yv = nullptr, *part = nullptr, *nrm = nullptr;
  double* host = nullptr;  // pinned: h1, h2, ||w||^2 as laid out on the device
  std::vector<double> Hm, cs, sn, g, y;
};

template <typename T, class Prec, class Mv>
h2_status fgmres_cycle(h2_ctx* c, GmresWork& W, int m, double beta, const T* r, double tol_abs, T* V, T* Z, int& k,
                       int& its, Prec prec, Mv mv) {
  cudaStream_t st = c->stream;
  const int64_t n = nslots(c);
  const int m0 = W.m0;
  launch_norm2<T>(r, n, W.nrm, st);
  launch_scaled_copy<T, T>(r, W.nrm, true, V, n, st);
  std::fill(W.g.begin(), W.g.end(), 0.0);
  W.g[0] = beta;
  k = 0;
  for (int j = 0; j < m; ++j) {
    T* vj = V + (int64_t)j * n;
    T* zj = Z + (int64_t)j * n;
    T* w = V + (int64_t)(j + 1) * n;
    prec(vj, zj);
    mv(zj, w);
    launch_multi_dot<T>(V, n, j + 1, w, n, W.part, W.h1, false, st);
    launch_multi_axpy<T, T>(V, n, j + 1, W.h1, -1.0, w, n, st);
    launch_multi_dot<T>(V, n, j + 1, w, n, W.part, W.h2, false, st);
    launch_multi_axpy<T, T>(V, n, j + 1, W.h2, -1.0, w, n, st);
    launch_norm2<T>(w, n, W.nrm, st);
    // h1, h2 and ||w||^2 lie next to each other: one read
    CKC(cudaMemcpyAsync(W.host, W.h1, (2 * (size_t)(m0 + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    launch_scaled_copy<T, T>(w, W.nrm, true, w, n, st);
    CKC(cudaStreamSynchronize(st));
    const double* a1 = W.host;
    const double* a2 = W.host + (m0 + 2);
    const double nw2 = W.host[2 * (m0 + 2)];
    double* col = &W.Hm[(size_t)j * (m0 + 1)];
    for (int i = 0; i <= j; ++i) col[i] = a1[i] + a2[i];
    col[j + 1] = std::sqrt(nw2);
    for (int i = 0; i < j; ++i) {
      double t = W.cs[i] * col[i] + W.sn[i] * col[i + 1];
      col[i + 1] = -W.sn[i] * col[i] + W.cs[i] * col[i + 1];
      col[i] = t;
    }
    double d = std::hypot(col[j], col[j + 1]);
    W.cs[j] = d > 0 ? col[j] / d : 1.0;
    W.sn[j] = d > 0 ? col[j + 1] / d : 0.0;
    col[j] = d;
    col[j + 1] = 0.0;
    W.g[j + 1] = -W.sn[j] * W.g[j];
    W.g[j] = W.cs[j] * W.g[j];
    ++its;
    k = j + 1;
    if (!std::isfinite(W.g[j + 1])) break;
    if (tol_abs > 0 && std::fabs(W.g[j + 1]) <= tol_abs) break;
    if (nw2 == 0.0) break;  // invariant Krylov space: exact solution
  }
  for (int i = k - 1; i >= 0; --i) {
    double t = W.g[i];
    for (int q = i + 1; q < k; ++q) t -= W.Hm[(size_t)q * (m0 + 1) + i] * W.y[q];
    W.y[i] = t / W.Hm[(size_t)i * (m0 + 1) + i];
  }
  return H2_OK;
}

h2_status gmres_work(h2_ctx* c, GmresWork& W) {
  const int m0 = std::max(1, c->restart);
  const int64_t n = nslots(c);
  if (c->gm_cap < m0) {
    CKC(dalloc(c, &c->gm_V, (size_t)(m0 + 1) * n));
    CKC(dalloc(c, &c->gm_Z, (size_t)m0 * n));
    CKC(dalloc(c, &c->gm_V32, (size_t)(m0 + 1) * n));
    CKC(dalloc(c, &c->gm_Z32, (size_t)m0 * n));
    CKC(dalloc(c, &c->gm_r32, (size_t)n));
    CKC(dalloc(c, &c->gm_h, 3 * (size_t)(m0 + 2) + 257));
    if (c->gm_host) cudaFreeHost(c->gm_host);
    CKC(cudaMallocHost(&c->gm_host, (2 * (size_t)(m0 + 2) + 1) * sizeof(double)));
    CKC(dalloc(c, &c->gm_part, (size_t)(m0 + 1) * 128));
    c->gm_cap = m0;
  }
  W.m0 = m0;
  W.h1 = c->gm_h;
  W.h2 = c->gm_h + (m0 + 2);
  W.nrm = c->gm_h + 2 * (m0 + 2);  // 257 doubles: the norm kernels' slot
  W.yv = c->gm_h + 2 * (m0 + 2) + 257;
  W.host = c->gm_host;
  W.part = c->gm_part;
  W.Hm.assign((size_t)(m0 + 1) * m0, 0.0);
  W.cs.assign(m0, 0.0);
  W.sn.assign(m0, 0.0);
  W.g.assign(m0 + 1, 0.0);
  W.y.assign(m0, 0.0);
  return H2_OK;
}

// r = b - A_H2 x in FP64; returns ||r||
// r = b - A_H2 x in FP64 and its norm; pairs: the matvec in FP32-pair
// arithmetic (matvec_df) instead of FP64 instructions.
h2_status fp64_residual(h2_ctx* c, SolveTimer& tm, double& rnorm, bool pairs = false) {
  const int64_t n = nslots(c);
  cudaStream_t st = c->stream;
  tm.run(tm.mv, [&] {
    if (pairs) matvec_df(c, c->x64, c->y64);
    else matvec_impl(c, c->x64, c->y64);
  });
  launch_residual(c->b64, c->y64, c->r64, n, st);
  launch_norm2<double>(c->r64, n, c->red + 600, st);
  double rn2 = 0;
  CKC(cudaMemcpyAsync(&rn2, c->red + 600, sizeof(double), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  rnorm = std::sqrt(rn2);
  return H2_OK;
}

// FGMRES-based refinement in FP64 (restart cycles; true residual after each).
// On entry x64 = 0 and r64 = b64.  its counts preconditioner applications.
h2_status gmres_refine(h2_ctx* c, SolveTimer& tm, double bnorm, double target, int max_iters, int& its,
                       double& rel) {
  GmresWork W;
  CKS(gmres_work(c, W));
  const int64_t n = nslots(c);
  double beta = bnorm;
  rel = 1.0;
  auto prec = [&](const double* v, double* z) {
    tm.run(tm.sub, [&] {
      cudaMemsetAsync(z, 0, n * sizeof(double), c->stream);
      ulv_apply_any(c, v, z);
    });
  };
  auto mv = [&](const double* z, double* w) { tm.run(tm.mv, [&] { matvec_impl(c, z, w); }); };
  while (its < max_iters && (target <= 0 || beta > target * bnorm)) {
    int k = 0;
    CKS(fgmres_cycle<double>(c, W, std::min(W.m0, max_iters - its), beta, c->r64, target * bnorm, c->gm_V, c->gm_Z,
                             k, its, prec, mv));
    CKC(cudaMemcpyAsync(W.yv, W.y.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_multi_axpy<double, double>(c->gm_Z, n, k, W.yv, 1.0, c->x64, n, c->stream);
    CKS(fp64_residual(c, tm, beta));
    rel = beta / bnorm;
    c->times.history.push_back(rel);
    if (!std::isfinite(rel)) break;
  }
  return H2_OK;
}

// Mixed-precision refinement (for the FP32-storage factorizations): the
// residual r = b - A_H2 x and the update x += d in FP64; each correction d
// solves A d = r approximately by FGMRES in FP32, with the FP32 copy of
// A_H2 and the ULV preconditioner, to the relative accuracy
// max(inner_tol, target / (2 relres)).
h2_status nested_refine(h2_ctx* c, SolveTimer& tm, double bnorm, double target, int max_iters, int& its,
                        double& rel) {
  GmresWork W;
  CKS(gmres_work(c, W));
  const int64_t n = nslots(c);
  cudaStream_t st = c->stream;
  double beta = bnorm;
  rel = 1.0;
  auto prec = [&](const float* v, float* z) { tm.run(tm.sub, [&] { ulv_apply_f32(c, v, z); }); };
  auto mv = [&](const float* z, float* w) { tm.run(tm.mv32, [&] { matvec32(c, z, w, &tm.leaf32); }); };
  while (its < max_iters && (target <= 0 || beta > target * bnorm)) {
    launch_norm2<double>(c->r64, n, c->red, st);
    launch_scaled_copy<double, float>(c->r64, c->red, true, c->gm_r32, n, st);
    const double tol_in = std::max(c->inner_tol, target > 0 ? 0.5 * target * bnorm / beta : 0.0);
    int k = 0;
    CKS(fgmres_cycle<float>(c, W, std::min(W.m0, max_iters - its), 1.0, c->gm_r32, tol_in, c->gm_V32, c->gm_Z32, k,
                            its, prec, mv));
    for (int i = 0; i < k; ++i) W.y[i] *= beta;
    CKC(cudaMemcpyAsync(W.yv, W.y.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_multi_axpy<float, double>(c->gm_Z32, n, k, W.yv, 1.0, c->x64, n, st);
    CKS(fp64_residual(c, tm, beta, !c->resid64));
    rel = beta / bnorm;
    c->times.history.push_back(rel);
    if (!std::isfinite(rel)) break;
  }
  return H2_OK;
}

// ---------------------------------------------------------------------------
// device-memory estimates checked before allocating (h2_set_memory_limit)
// ---------------------------------------------------------------------------
uint64_t g_mem_limit = 0;  // process-wide cap on one context's device bytes (0: none)

// The instance's largest device arrays: the leaf near blocks (FP64, the FP32
// pair of the stored halves, the 16-bit copy), bases and couplings.
double instance_bytes(const HostH2& H) {
  const int L = H.L;
  const HostLevel& lf = H.lv[L];
  const double D = lf.D, NP = lf.near.size() / 2.0;
  double b = NP * D * D * (8.0 + 2.0) + (NP + lf.nb) / 2.0 * D * D * 8.0;
  for (int l = 1; l <= L; ++l) {
    const HostLevel& h = H.lv[l];
    b += (double)h.nb * h.D * h.K * 16.0 + (h.far.size() / 2.0) * h.K * h.K * 22.0;
  }
  return b + (double)lf.nb * D * 8.0 * 8.0;
}

// One factorization's largest arrays in storage type of size sz (8: FP64,
// 4: FP16/BF16 factorizations with FP32 storage).
double factor_bytes(const h2_ctx* c, int sz) {
  double b = 0, wk = 0;
  for (int l = 1; l <= c->L; ++l) {
    const DevLevel& d = c->lv[l];
    const double D = d.D, K = d.K, R = d.R, nb = d.nb, NP = (double)d.NP;
    b += NP * D * D * (sz + (sz == 4 ? 2.0 : 0.0));                  // Ahat (+ 16-bit copy)
    if (l < c->L) b += NP * D * D * (sz == 4 ? 2.0 : sz);            // the level's input blocks
    b += nb * (3 * D * D + 2 * D * K + 2 * K * K + R * K + 2 * R * R + R * D) * sz;
    b += (double)d.FP * K * K * sz;
    wk = std::max(wk, NP * D * D * sz);
  }
  return b + wk;
}

// H2_ERR_OOM when need exceeds the cap or the device's free memory; the cap
// is checked first, before any CUDA call.
h2_status check_fits(double need, const char* what, std::string& err) {
  char buf[256];
  if (g_mem_limit > 0 && need > (double)g_mem_limit) {
    std::snprintf(buf, sizeof buf, "%s needs about %.0f device bytes; the memory limit is %llu", what, need,
                  (unsigned long long)g_mem_limit);
    err = buf;
    return H2_ERR_OOM;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
    if (need > (double)fr) {
      std::snprintf(buf, sizeof buf, "%s needs about %.0f device bytes; %zu are free", what, need, fr);
      err = buf;
      return H2_ERR_OOM;
    }
  } else {
    cudaGetLastError();
  }
  return H2_OK;
}

// Free a factorization's arrays (its CUDA graphs first); the next
// h2_factor allocates them again.
template <typename T>
void release_factor(h2_ctx* c, Factor<T>& F) {
  if (F.allocs.empty() && F.lv.empty()) return;
  for (cudaStream_t s : {c->stream, c->basis_stream, c->coupling_stream, c->product_stream, c->leaf_stream,
                         c->cap_stream})
    if (s || s == c->stream) cudaStreamSynchronize(s);
  drop_graphs(c);
  for (void* q : F.allocs) cudaFree(q);
  F = Factor<T>();
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

h2_status h2_build(h2_ctx** out, const h2_params* p, const double* points, int64_t N) {
  g_last_error.clear();
  if (!out) { g_last_error = "out is NULL"; return H2_ERR_INVALID_ARG; }
  *out = nullptr;
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points) { g_last_error = "N < 1 or points NULL"; return H2_ERR_INVALID_ARG; }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  h2_ctx* c = new h2_ctx();
  c->params = *p;
  c->kfn = KernelFn{p->kernel, p->eps, p->ell, p->diag_shift};
  std::string e = build_host(*p, points, N, c->host);
  if (!e.empty()) {
    g_last_error = e;
    delete c;
    return H2_ERR_SINGULAR;
  }
  s = check_fits(instance_bytes(c->host), "the H^2 instance", g_last_error);
  if (s != H2_OK) {
    delete c;
    return s;
  }
  s = setup_device(c);
  if (s != H2_OK) {
    g_last_error = c->err;
    h2_destroy(c);
    return s;
  }
  *out = c;
  return H2_OK;
}

int32_t h2_tree_depth(int64_t N, int32_t leaf_size) {
  if (N < 1 || leaf_size < 1) return -1;
  return depth_of(N, leaf_size);
}

h2_status h2_build_forest(h2_ctx** out, const h2_params* p, const double* const* points, const int64_t* N,
                          int32_t count) {
  g_last_error.clear();
  if (!out) { g_last_error = "out is NULL"; return H2_ERR_INVALID_ARG; }
  *out = nullptr;
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (count < 1 || !points || !N) { g_last_error = "count < 1 or NULL arrays"; return H2_ERR_INVALID_ARG; }
  int depth = -1;
  for (int32_t k = 0; k < count; ++k) {
    if (N[k] < 1 || !points[k]) { g_last_error = "system " + std::to_string(k) + ": N < 1 or points NULL"; return H2_ERR_INVALID_ARG; }
    for (int64_t t = 0; t < 3 * N[k]; ++t)
      if (!std::isfinite(points[k][t])) {
        g_last_error = "system " + std::to_string(k) + ": non-finite coordinate";
        return H2_ERR_INVALID_ARG;
      }
    const int d = depth_of(N[k], p->leaf_size);
    if (d < 1 || (depth >= 0 && d != depth)) {
      g_last_error = "the systems of a forest need one common tree depth >= 1 (system " + std::to_string(k) +
                     " has " + std::to_string(d) + ")";
      return H2_ERR_INVALID_ARG;
    }
    depth = d;
  }
  // one rank per level for all systems (the constant-rank batches of Section
  // 4.1): each level takes its systems' largest tolerance rank, and the
  // systems below it are compressed again at that rank
  std::vector<HostH2> parts(count);
  for (int32_t k = 0; k < count; ++k) {
    std::string e = build_host(*p, points[k], N[k], parts[k]);
    if (!e.empty()) {
      g_last_error = "system " + std::to_string(k) + ": " + e;
      return H2_ERR_SINGULAR;
    }
  }
  // the shared rank: the largest, rounded up to a multiple of 64 (upper
  // boxes of dimension 2K then fit the tensor-core tiles), at most the
  // smallest box of the level (leaves: the fewest points of any leaf)
  std::vector<int> Kf(depth + 1, 0);
  int64_t leaf_min = INT64_MAX;
  for (const HostH2& P : parts)
    for (size_t i = 0; i + 1 < P.leaf_offsets.size(); ++i)
      leaf_min = std::min<int64_t>(leaf_min, P.leaf_offsets[i + 1] - P.leaf_offsets[i]);
  for (int l = depth; l >= 1; --l) {
    for (const HostH2& P : parts) Kf[l] = std::max(Kf[l], P.lv[l].K);
    const int64_t nmin = (l == depth) ? leaf_min : 2 * (int64_t)Kf[l + 1];
    Kf[l] = (int)std::min<int64_t>((Kf[l] + 63) / 64 * 64, nmin);
  }
  for (int32_t k = 0; k < count; ++k) {
    bool same = true;
    for (int l = 1; l <= depth; ++l) same = same && parts[k].lv[l].K == Kf[l];
    if (same) continue;
    parts[k] = HostH2();
    std::string e = build_host(*p, points[k], N[k], parts[k], nullptr, false, nullptr, &Kf);
    if (!e.empty()) {
      g_last_error = "system " + std::to_string(k) + ": " + e;
      return H2_ERR_SINGULAR;
    }
  }
  h2_ctx* c = new h2_ctx();
  c->params = *p;
  c->kfn = KernelFn{p->kernel, p->eps, p->ell, p->diag_shift};
  std::string e = combine_forest(parts, c->host);
  parts.clear();
  if (!e.empty()) {
    g_last_error = e;
    delete c;
    return H2_ERR_INVALID_ARG;
  }
  s = check_fits(instance_bytes(c->host), "the H^2 forest", g_last_error);
  if (s != H2_OK) {
    delete c;
    return s;
  }
  s = setup_device(c);
  if (s != H2_OK) {
    g_last_error = c->err;
    h2_destroy(c);
    return s;
  }
  *out = c;
  return H2_OK;
}

h2_status h2_plan(const h2_params* p, const double* points, int64_t N, char* json, size_t cap) {
  g_last_error.clear();
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points || !json) { g_last_error = "N < 1 or NULL pointer"; return H2_ERR_INVALID_ARG; }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  HostH2 H;
  std::string e = build_host(*p, points, N, H);
  if (!e.empty()) { g_last_error = e; return H2_ERR_SINGULAR; }
  std::ostringstream o;
  double bytes_build = 0, bytes_factor64 = 0;
  o << "{\"N\":" << N << ",\"L\":" << H.L << ",\"levels\":[";
  for (int l = 0; l <= H.L; ++l) {
    const HostLevel& h = H.lv[l];
    double D = h.D, K = l ? h.K : 0, R = D - K, NP = h.near.size() / 2, FP = h.far.size() / 2, nb = h.nb;
    if (l) o << ",";
    o << "{\"l\":" << l << ",\"nb\":" << h.nb << ",\"D\":" << h.D << ",\"K\":" << (l ? h.K : 0)
      << ",\"NP\":" << (int64_t)NP << ",\"FP\":" << (int64_t)FP;
    if (l == H.L && !H.ranks_leaf.empty())
      o << ",\"rank_max\":" << *std::max_element(H.ranks_leaf.begin(), H.ranks_leaf.end())
        << ",\"rank_min\":" << *std::min_element(H.ranks_leaf.begin(), H.ranks_leaf.end());
    o << "}";
    bytes_build += 8.0 * (nb * D * K + FP * K * K) + (l == H.L ? 8.0 * NP * D * D : 0.0);
    bytes_factor64 += 8.0 * (2 * NP * D * D + nb * (D * D + D * K + 2 * R * R + R * K) + FP * K * K);
  }
  o << "],\"device_bytes_build\":" << bytes_build << ",\"device_bytes_factor_fp64\":" << bytes_factor64
    << ",\"compress_s\":" << H.rec.compress_s << "}";
  std::string str = o.str();
  if (str.size() + 1 > cap) { g_last_error = "cap too small"; return H2_ERR_INVALID_ARG; }
  std::memcpy(json, str.c_str(), str.size() + 1);
  return H2_OK;
}

h2_status h2_import(h2_ctx** out, const h2_params* p, const h2_instance* in) {
  g_last_error.clear();
  if (!out || !in) { g_last_error = "NULL argument"; return H2_ERR_INVALID_ARG; }
  *out = nullptr;
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (in->N < 1 || in->L < 0 || in->L > 30 || !in->points || !in->perm || !in->leaf_offsets || !in->D || !in->K) {
    g_last_error = "inconsistent instance";
    return H2_ERR_INVALID_ARG;
  }
  h2_ctx* c = new h2_ctx();
  c->params = *p;
  c->kfn = KernelFn{p->kernel, p->eps, p->ell, p->diag_shift};
  HostH2& H = c->host;
  H.N = in->N;
  H.L = in->L;
  H.points.assign(in->points, in->points + 3 * in->N);
  H.perm.assign(in->perm, in->perm + in->N);
  H.leaf_offsets.assign(in->leaf_offsets, in->leaf_offsets + (1 << in->L) + 1);
  H.lv.assign(in->L + 1, HostLevel());
  std::string err;
  for (int l = 0; l <= in->L; ++l) {
    HostLevel& h = H.lv[l];
    h.nb = 1 << l;
    h.D = in->D[l];
    h.K = l ? in->K[l] : 0;
    if (h.D < 0 || h.K < 0 || h.K > h.D || (l < in->L && h.D != 2 * in->K[l + 1])) err = "bad D/K";
    h.near.assign(in->near[l], in->near[l] + 2 * in->n_near[l]);
    if (in->n_far[l] > 0) h.far.assign(in->far[l], in->far[l] + 2 * in->n_far[l]);
    for (int32_t v : h.near)
      if (v < 0 || v >= h.nb) err = "near pair index out of range";
    for (int32_t v : h.far)
      if (v < 0 || v >= h.nb) err = "far pair index out of range";
    if (l >= 1) {
      h.X.assign(in->X[l], in->X[l] + (size_t)h.nb * h.D * h.K);
      h.SK.assign(in->SK[l], in->SK[l] + (size_t)h.nb * h.K);
      for (int64_t v : h.SK)
        if (v < 0 || v >= in->N) err = "skeleton index out of range";
    }
  }
  for (int i = 0; i < (1 << in->L); ++i)
    if (H.leaf_offsets[i + 1] - H.leaf_offsets[i] > H.lv[in->L].D || H.leaf_offsets[i + 1] < H.leaf_offsets[i])
      err = "leaf larger than D_L";
  if (H.leaf_offsets[0] != 0 || H.leaf_offsets[1 << in->L] != in->N) err = "bad leaf offsets";
  for (int64_t t = 0; t < in->N; ++t)
    if (H.perm[t] < 0 || H.perm[t] >= in->N) err = "perm out of range";
  if (!err.empty()) {
    g_last_error = err;
    delete c;
    return H2_ERR_INVALID_ARG;
  }
  s = check_fits(instance_bytes(c->host), "the H^2 instance", g_last_error);
  if (s != H2_OK) {
    delete c;
    return s;
  }
  s = setup_device(c);
  if (s != H2_OK) {
    g_last_error = c->err;
    h2_destroy(c);
    return s;
  }
  *out = c;
  return H2_OK;
}

h2_status h2_factor(h2_ctx* c, int32_t prec) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (prec < H2_PREC_FP64 || prec > H2_PREC_BF16) {
    c->err = "unknown precision";
    return H2_ERR_INVALID_ARG;
  }
  if (!c->A64 && (prec == H2_PREC_FP64 || (prec == H2_PREC_BF16 && !c->A16[1]))) {
    c->err = "this factorization needs the FP64 leaf blocks, which were released (H2_OPT_FP64_LEAF)";
    return H2_ERR_STATE;
  }
  c->prec = -1;
  drop_graphs(c);
  const bool fresh = (prec == H2_PREC_FP64) ? c->f64.lv.empty() : c->f32.lv.empty();
  if (fresh) CKS(check_fits(factor_bytes(c, prec == H2_PREC_FP64 ? 8 : 4), "the factorization", c->err));
  h2_status s = (prec == H2_PREC_FP64) ? factor_impl<double>(c, c->f64, prec) : factor_impl<float>(c, c->f32, prec);
  if (s == H2_OK) c->prec = prec;
  return s;
}

h2_status h2_release_factorization(h2_ctx* c) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->err.clear();
  release_factor(c, c->f64);
  release_factor(c, c->f32);
  c->prec = -1;
  CKC(cudaGetLastError());
  return H2_OK;
}

h2_status h2_ulv_apply(h2_ctx* c, const double* b, double* x) {
  if (!c || !b || !x) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (!factor_ready(c)) { c->err = "no factorization"; return H2_ERR_STATE; }
  const DevLevel& lf = c->lv[c->L];
  const int64_t nslot = (int64_t)lf.nb * lf.D;
  CKS(vec_in(c, b, c->r64));
  CKC(cudaMemsetAsync(c->x64, 0, nslot * sizeof(double), c->stream));
  CKS(subst_clear(c));
  ulv_apply_any(c, c->r64, c->x64);
  CKC(cudaGetLastError());
  CKS(vec_out(c, c->x64, x));
  CKC(cudaStreamSynchronize(c->stream));
  return subst_check(c);
}

h2_status h2_matvec(h2_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (!c->A64) { c->err = "the FP64 leaf blocks were released (H2_OPT_FP64_LEAF)"; return H2_ERR_STATE; }
  CKS(vec_in(c, x, c->x64));
  matvec_impl(c, c->x64, c->y64);
  CKC(cudaGetLastError());
  CKS(vec_out(c, c->y64, y));
  CKC(cudaStreamSynchronize(c->stream));
  return H2_OK;
}

h2_status h2_solve_many(h2_ctx* c, const double* B, double* X, int32_t nrhs, double target, int32_t max_iters,
                        double* relres_out, int32_t* iters_out) {
  if (!c || !B || !X || nrhs < 0) return H2_ERR_INVALID_ARG;
  for (int32_t k = 0; k < nrhs; ++k) {
    double rel = 0;
    int32_t its = 0;
    const h2_status s = h2_solve(c, B + (int64_t)k * c->N, X + (int64_t)k * c->N, target, max_iters, &rel, &its);
    if (relres_out) relres_out[k] = rel;
    if (iters_out) iters_out[k] = its;
    if (s != H2_OK) {
      c->err = "right-hand side " + std::to_string(k) + ": " + c->err;
      return s;
    }
  }
  return H2_OK;
}

h2_status h2_matvec_many(h2_ctx* c, const double* X, double* Y, int32_t nrhs) {
  if (!c || !X || !Y || nrhs < 0) return H2_ERR_INVALID_ARG;
  for (int32_t k = 0; k < nrhs; ++k) CKS(h2_matvec(c, X + (int64_t)k * c->N, Y + (int64_t)k * c->N));
  return H2_OK;
}

h2_status h2_solve(h2_ctx* c, const double* b, double* x, double target, int32_t max_iters, double* relres_out,
                   int32_t* iters_out) {
  if (!c || !b || !x || max_iters < 0) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (!factor_ready(c)) { c->err = "no factorization"; return H2_ERR_STATE; }
  if (!c->A64 && c->resid64) {
    c->err = "the FP64 residual needs the FP64 leaf blocks, which were released (H2_OPT_FP64_LEAF)";
    return H2_ERR_STATE;
  }
  cudaStream_t st = c->stream;
  const DevLevel& lf = c->lv[c->L];
  const int64_t nslot = (int64_t)lf.nb * lf.D;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  CKS(vec_in(c, b, c->b64));
  launch_norm2<double>(c->b64, nslot, c->red + 300, st);  // ||b||^2 apart from the substitution scratch
  double bn2 = 0;
  CKC(cudaMemcpyAsync(&bn2, c->red + 300, sizeof(double), cudaMemcpyDeviceToHost, st));
  CKC(cudaMemsetAsync(c->x64, 0, nslot * sizeof(double), st));
  CKC(cudaMemcpyAsync(c->r64, c->b64, nslot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CKS(subst_clear(c));
  CKC(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bn2);
  double rel = bnorm > 0 ? 1.0 : 0.0;
  int it = 0;
  c->times.history.clear();
  SolveTimer timer(st);
  struct TimerGuard {
    SolveTimer* t;
    ~TimerGuard() {
      SolveTimer::total(t->sub);
      SolveTimer::total(t->mv);
      SolveTimer::total(t->mv32);
      SolveTimer::total(t->leaf32);
    }
  } guard{&timer};
  int method = c->refine_method;
  if (method == 3) method = (c->prec == H2_PREC_FP64) ? 1 : 2;
  if (method == 2 && c->prec == H2_PREC_FP64) method = 1;
  c->times.method = method;
  if (bnorm > 0 && method == 1) {
    CKS(gmres_refine(c, timer, bnorm, target, max_iters, it, rel));
  } else if (bnorm > 0 && method == 2) {
    CKS(nested_refine(c, timer, bnorm, target, max_iters, it, rel));
  } else {
    while (it < max_iters && (target <= 0 || rel > target) && bnorm > 0) {
      timer.run(timer.sub, [&] { ulv_apply_any(c, c->r64, c->x64); });
      double rn = 0;
      CKS(fp64_residual(c, timer, rn));
      rel = rn / bnorm;
      c->times.history.push_back(rel);
      ++it;
      if (!std::isfinite(rel)) break;
    }
  }
  CKC(cudaGetLastError());
  CKS(vec_out(c, c->x64, x));
  cudaEventRecord(e1, st);
  CKC(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->times.solve_total = ms * 1e-3;
  c->times.n_subst = (int)timer.sub.size();
  c->times.n_matvec = (int)timer.mv.size();
  c->times.n_matvec32 = (int)timer.mv32.size();
  c->times.n_leaf32 = (int)timer.leaf32.size();
  c->times.leaf32 = SolveTimer::total(timer.leaf32);
  c->times.subst = SolveTimer::total(timer.sub);
  c->times.matvec = SolveTimer::total(timer.mv);
  c->times.matvec32 = SolveTimer::total(timer.mv32);  // the guard then finds the lists empty
  c->times.iters = it;
  c->times.relres = rel;
  if (relres_out) *relres_out = rel;
  if (iters_out) *iters_out = it;
  CKS(subst_check(c));
  if (target > 0 && !(rel <= target)) {
    c->err = "refinement stopped at relative residual " + std::to_string(rel);
    return H2_ERR_NOT_CONVERGED;
  }
  return H2_OK;
}

h2_status h2_set_refinement(h2_ctx* c, int32_t method, int32_t restart) {
  if (!c || method < 0 || method > 3 || restart < 1 || restart > 1000) return H2_ERR_INVALID_ARG;
  c->refine_method = method;
  c->restart = restart;
  return H2_OK;
}

h2_status h2_set_option(h2_ctx* c, int32_t option, int64_t value) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if ((value != 0 && value != 1) && option != H2_OPT_TC_KERNEL && !(option == H2_OPT_BOX_STREAM && value == 2) &&
      option != H2_OPT_PAIR_CTAS && option != H2_OPT_BOX_CTAS) {
    c->err = "option value must be 0 or 1";
    return H2_ERR_INVALID_ARG;
  }
  switch (option) {
    case H2_OPT_RR_LU_FP64: c->rr_lu64 = value != 0; return H2_OK;
    case H2_OPT_RESIDUAL_FP64: c->resid64 = value != 0; return H2_OK;
    case H2_OPT_TC_KERNEL:
      if (value < 0 || value > 2) {
        c->err = "tensor-core kernel form outside 0..2";
        return H2_ERR_INVALID_ARG;
      }
      g_tc_kernel = (int)value;
      return H2_OK;
    case H2_OPT_GRAPHS:
      c->use_graphs = value != 0;
      drop_graphs(c);
      return H2_OK;
    case H2_OPT_PAIR_CTAS:
      if (value < 1 || value > 3) {
        c->err = "pair-kernel CTAs per SM outside 1..3";
        return H2_ERR_INVALID_ARG;
      }
      g_pair_ctas_per_sm = (int)value;
      drop_graphs(c);
      return H2_OK;
    case H2_OPT_BOX_CTAS:
      if (value < 1 || value > 8) {
        c->err = "per-box CTAs per SM outside 1..8";
        return H2_ERR_INVALID_ARG;
      }
      g_box_ctas_per_sm = (int)value;
      drop_graphs(c);
      return H2_OK;
    case H2_OPT_BOX_STREAM:
      g_box_stream = (int)value;
      drop_graphs(c);
      return H2_OK;
    case H2_OPT_FP64_LEAF:
      if (value == 1) {
        if (c->A64) return H2_OK;
        c->err = "the FP64 leaf blocks were released and cannot be restored";
        return H2_ERR_STATE;
      }
      if (!c->A64) return H2_OK;
      // the mixed-precision path keeps what it needs: the FP32 pair of the
      // leaf blocks (residual, inner matvec) and their FP16 copy (projection)
      if (!c->A32 || !c->Alo || !c->A16[0] || c->L < 1) {
        c->err = "the FP64 leaf blocks are still needed (no FP16 copy of the leaf blocks)";
        return H2_ERR_STATE;
      }
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return H2_ERR_CUDA;
      for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
        if (*it == (void*)c->A64) {
          c->allocs.erase(it);
          break;
        }
      cudaFree(c->A64);
      c->A64 = nullptr;
      return H2_OK;
    default: c->err = "unknown option"; return H2_ERR_INVALID_ARG;
  }
}

h2_status h2_matvec_arith(h2_ctx* c, const double* x, double* y, int32_t arith) {
  if (!c || !x || !y) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (arith < 0 || arith > 2) {
    c->err = "arith must be 0 (FP64), 1 (FP32) or 2 (FP32 pairs)";
    return H2_ERR_INVALID_ARG;
  }
  const int64_t n = nslots(c);
  CKS(vec_in(c, x, c->x64));
  if (arith == 0 && !c->A64) {
    c->err = "the FP64 leaf blocks were released (H2_OPT_FP64_LEAF)";
    return H2_ERR_STATE;
  }
  if (arith == 0) {
    matvec_impl(c, c->x64, c->y64);
  } else if (arith == 2) {
    matvec_df(c, c->x64, c->y64);
  } else {
    if (!c->mv32_x) {
      CKC(dalloc(c, &c->mv32_x, (size_t)n));
      CKC(dalloc(c, &c->mv32_y, (size_t)n));
    }
    launch_convert<double, float>(c->x64, c->mv32_x, n, c->stream);
    matvec32(c, c->mv32_x, c->mv32_y);
    launch_convert<float, double>(c->mv32_y, c->y64, n, c->stream);
  }
  CKC(cudaGetLastError());
  CKS(vec_out(c, c->y64, y));
  CKC(cudaStreamSynchronize(c->stream));
  return H2_OK;
}

h2_status h2_autotune(h2_ctx* c, int32_t prec, char* json, size_t cap) {
  if (!c || (prec != H2_PREC_FP16 && prec != H2_PREC_BF16)) return H2_ERR_INVALID_ARG;
  c->err.clear();
  std::ostringstream o;
  o.precision(6);
  // (1) the kernel form of the factorization's main-chain GEMMs: each form
  // factors twice (the first also allocates), the second is timed
  double tf[3] = {0, 0, 0};
  int best_form = 2;
  for (int form = 0; form < 3; ++form) {
    g_tc_kernel = form;
    for (int rep = 0; rep < 2; ++rep) CKS(h2_factor(c, prec));
    tf[form] = c->times.total_factor;
  }
  best_form = 0;
  for (int form = 1; form < 3; ++form)
    if (tf[form] < tf[best_form]) best_form = form;
  g_tc_kernel = best_form;
  CKS(h2_factor(c, prec));
  o << "{\"tc_kernel\":" << best_form << ",\"factor_s\":[" << tf[0] << "," << tf[1] << "," << tf[2] << "]";
  // (2) the substitution's launch shapes, timed on ULV applications
  const int64_t n = nslots(c);
  float *v = nullptr, *z = nullptr;
  if (cudaMalloc(&v, n * sizeof(float)) != cudaSuccess || cudaMalloc(&z, n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    if (v) cudaFree(v);
    c->err = "autotune: no room for two vectors";
    return H2_ERR_OOM;
  }
  cudaMemsetAsync(v, 0, n * sizeof(float), c->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  struct Shape {
    int pair, box, stream, graphs;
    float ms;
  };
  std::vector<Shape> tried;
  Shape best{g_pair_ctas_per_sm.load(), g_box_ctas_per_sm.load(), g_box_stream.load(), c->use_graphs ? 1 : 0, 1e30f};
  h2_status st = subst_clear(c);
  for (int pair : {2, 3})
    for (int box : {1, 2, 4})
      for (int stream : {0, 1})
        for (int graphs : {0, 1}) {
          if (st != H2_OK) break;
          g_pair_ctas_per_sm = pair;
          g_box_ctas_per_sm = box;
          g_box_stream = stream;
          c->use_graphs = graphs != 0;
          drop_graphs(c);
          for (int w = 0; w < 2; ++w) ulv_apply_f32(c, v, z);
          cudaEventRecord(e0, c->stream);
          for (int k = 0; k < 6; ++k) ulv_apply_f32(c, v, z);
          cudaEventRecord(e1, c->stream);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = H2_ERR_CUDA;
            break;
          }
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= 6;
          tried.push_back({pair, box, stream, graphs, ms});
          if (ms < best.ms) best = tried.back();
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(v);
  cudaFree(z);
  if (st == H2_OK) st = subst_check(c);
  g_pair_ctas_per_sm = best.pair;
  g_box_ctas_per_sm = best.box;
  g_box_stream = best.stream;
  c->use_graphs = best.graphs != 0;
  drop_graphs(c);
  if (st != H2_OK) {
    if (c->err.empty()) c->err = "autotune: a substitution run failed";
    return st;
  }
  o << ",\"pair_ctas_per_sm\":" << best.pair << ",\"box_ctas_per_sm\":" << best.box << ",\"box_stream\":" << best.stream
    << ",\"graphs\":" << best.graphs << ",\"subst_ms\":" << best.ms << ",\"tried\":[";
  for (size_t k = 0; k < tried.size(); ++k)
    o << (k ? "," : "") << "[" << tried[k].pair << "," << tried[k].box << "," << tried[k].stream << ","
      << tried[k].graphs << "," << tried[k].ms << "]";
  o << "]}";
  const std::string s = o.str();
  if (json) {
    if (s.size() + 1 > cap) return H2_ERR_INVALID_ARG;
    std::memcpy(json, s.c_str(), s.size() + 1);
  }
  return H2_OK;
}

h2_status h2_wait_selftest(h2_ctx* c, int64_t timeout_ns) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->err.clear();
  if (timeout_ns < 1 || timeout_ns > 10000000000ll) {
    c->err = "timeout_ns outside 1 .. 1e10";
    return H2_ERR_INVALID_ARG;
  }
  // the substitution kernels' status word: cleared, set by the waiting
  // kernel when it gives up, read back
  CKS(subst_clear(c));
  launch_wait_selftest((unsigned long long)timeout_ns, c->status + 3, c->stream);
  CKC(cudaGetLastError());
  const h2_status s = subst_check(c);
  if (s == H2_ERR_TIMEOUT) {
    c->err = "self-test: the bounded wait gave up after " + std::to_string(timeout_ns) + " ns as designed";
    CKS(subst_clear(c));
    CKC(cudaStreamSynchronize(c->stream));
  }
  return s;
}

h2_status h2_set_memory_limit(uint64_t bytes) {
  g_mem_limit = bytes;
  return H2_OK;
}

h2_status h2_rank_data(const h2_params* p, const double* points, int64_t N, float* feats, float* targets,
                       int32_t* levels, int64_t cap, int64_t* nbox) {
  g_last_error.clear();
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points || !nbox || cap < 0) { g_last_error = "N < 1 or NULL pointer"; return H2_ERR_INVALID_ARG; }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  HostH2 H;
  std::string e = build_host(*p, points, N, H);
  if (!e.empty()) { g_last_error = e; return H2_ERR_SINGULAR; }
  int64_t total = 0;
  for (int l = H.L; l >= 1; --l) total += H.lv[l].nb;
  *nbox = total;
  if (cap < total) { g_last_error = "cap too small"; return H2_ERR_INVALID_ARG; }
  if (total && (!feats || !targets || !levels)) { g_last_error = "NULL output array"; return H2_ERR_INVALID_ARG; }
  int64_t k = 0;
  for (int l = H.L; l >= 1; --l)
    for (int i = 0; i < H.lv[l].nb; ++i, ++k) {
      std::memcpy(feats + k * kRankFeatures, &H.rec.feats[l][(size_t)i * kRankFeatures], sizeof(float) * kRankFeatures);
      const int n = H.rec.dims[l][i];
      targets[k] = n > 0 ? (float)H.rec.ranks[l][i] / (float)n : 0.f;
      levels[k] = l;
    }
  return H2_OK;
}

namespace {
// the rank model as the construction calls it
struct ModelPredictor : RankPredictor {
  h2_rank_model* m;
  explicit ModelPredictor(h2_rank_model* mm) : m(mm) {}
  bool predict(const std::vector<float>& f, int nb, std::vector<float>& out) override {
    out.assign(nb, 0.f);
    return h2_rank_model_predict(m, f.data(), nb, out.data()) == H2_OK;
  }
};
}  // namespace

h2_status h2_plan_predicted(const h2_params* p, const double* points, int64_t N, h2_rank_model* model, char* json,
                            size_t cap) {
  g_last_error.clear();
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points || !json || !model) { g_last_error = "N < 1 or NULL pointer"; return H2_ERR_INVALID_ARG; }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  HostH2 H;
  ModelPredictor pred(model);
  std::string e = build_host(*p, points, N, H, &pred, true);
  if (!e.empty()) { g_last_error = e; return H2_ERR_CUDA; }
  std::ostringstream o;
  double bytes_build = 0;
  o << "{\"N\":" << N << ",\"L\":" << H.L << ",\"levels\":[";
  for (int l = 0; l <= H.L; ++l) {
    const HostLevel& h = H.lv[l];
    const double D = h.D, K = l ? h.K : 0, NP = h.near.size() / 2, FP = h.far.size() / 2, nb = h.nb;
    if (l) o << ",";
    o << "{\"l\":" << l << ",\"nb\":" << h.nb << ",\"D\":" << h.D << ",\"K\":" << (l ? h.K : 0)
      << ",\"NP\":" << (int64_t)NP << ",\"FP\":" << (int64_t)FP << "}";
    bytes_build += 8.0 * (nb * D * K + FP * K * K) + (l == H.L ? 8.0 * NP * D * D : 0.0);
  }
  o << "],\"device_bytes_build\":" << bytes_build << "}";
  std::string str = o.str();
  if (str.size() + 1 > cap) { g_last_error = "cap too small"; return H2_ERR_INVALID_ARG; }
  std::memcpy(json, str.c_str(), str.size() + 1);
  return H2_OK;
}

h2_status h2_build_predicted(h2_ctx** out, const h2_params* p, const double* points, int64_t N,
                             h2_rank_model* model) {
  g_last_error.clear();
  if (!out || !model) { g_last_error = "NULL argument"; return H2_ERR_INVALID_ARG; }
  *out = nullptr;
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points) { g_last_error = "N < 1 or points NULL"; return H2_ERR_INVALID_ARG; }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  h2_ctx* c = new h2_ctx();
  c->params = *p;
  c->kfn = KernelFn{p->kernel, p->eps, p->ell, p->diag_shift};
  ModelPredictor pred(model);
  std::string e = build_host(*p, points, N, c->host, &pred);
  if (!e.empty()) {
    g_last_error = e;
    delete c;
    return H2_ERR_SINGULAR;
  }
  s = check_fits(instance_bytes(c->host), "the H^2 instance", g_last_error);
  if (s != H2_OK) {
    delete c;
    return s;
  }
  s = setup_device(c);
  if (s != H2_OK) {
    g_last_error = c->err;
    h2_destroy(c);
    return s;
  }
  *out = c;
  return H2_OK;
}

h2_status h2_build_gpu(h2_ctx** out, const h2_params* p, const double* points, int64_t N, h2_rank_model* model,
                       int32_t gs_sweeps) {
  g_last_error.clear();
  if (!out) { g_last_error = "out is NULL"; return H2_ERR_INVALID_ARG; }
  *out = nullptr;
  h2_status s = check_params(p, g_last_error);
  if (s != H2_OK) return s;
  if (N < 1 || !points || gs_sweeps < 0 || gs_sweeps > 16) {
    g_last_error = "N < 1, points NULL or gs_sweeps outside 0..16";
    return H2_ERR_INVALID_ARG;
  }
  for (int64_t t = 0; t < 3 * N; ++t)
    if (!std::isfinite(points[t])) { g_last_error = "non-finite coordinate"; return H2_ERR_INVALID_ARG; }
  h2_ctx* c = new h2_ctx();
  c->params = *p;
  c->kfn = KernelFn{p->kernel, p->eps, p->ell, p->diag_shift};
  GpuCompressor* gpu = make_gpu_compressor(c->kfn, points, N, gs_sweeps);
  if (!gpu) {
    g_last_error = "GPU construction: device upload of the points failed";
    delete c;
    return H2_ERR_CUDA;
  }
  ModelPredictor pred(model);
  std::string e = build_host(*p, points, N, c->host, model ? &pred : nullptr, false, gpu);
  delete gpu;
  if (!e.empty()) {
    g_last_error = e;
    delete c;
    return e.rfind("GPU construction", 0) == 0 ? H2_ERR_CUDA : H2_ERR_SINGULAR;
  }
  s = check_fits(instance_bytes(c->host), "the H^2 instance", g_last_error);
  if (s != H2_OK) {
    delete c;
    return s;
  }
  s = setup_device(c);
  if (s != H2_OK) {
    g_last_error = c->err;
    h2_destroy(c);
    return s;
  }
  *out = c;
  return H2_OK;
}

h2_status h2_set_stream(h2_ctx* c, void* stream) {
  if (!c) return H2_ERR_INVALID_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return H2_OK;
}

h2_status h2_stats(const h2_ctx* c, char* json, size_t cap) {
  if (!c || !json) return H2_ERR_INVALID_ARG;
  std::ostringstream o;
  o.precision(9);
  const PhaseTimes& t = c->times;
  double fl_proj = 0, fl_lu = 0, fl_schur = 0, fl_coup = 0, fl_qr = 0, by_proj = 0;
  o << "{\"N\":" << c->N << ",\"L\":" << c->L << ",\"systems\":" << (c->lv.empty() ? 0 : c->lv[0].nb)
    << ",\"prec\":" << c->prec << ",\"levels\":[";
  // (per-level sizes; flop counts below use the actual ranks, not padded tiles)
  for (int l = 0; l <= c->L; ++l) {
    const DevLevel& d = c->lv[l];
    double D = d.D, K = d.K, R = d.R;
    if (l) o << ",";
    o << "{\"l\":" << l << ",\"nb\":" << d.nb << ",\"D\":" << d.D << ",\"K\":" << d.K << ",\"NP\":" << d.NP
      << ",\"FP\":" << d.FP << "}";
    if (l == 0) {
      fl_lu += d.nb * 2.0 * D * D * D;
      continue;
    }
    // the projection's flops: the pairs actually projected (symmetric near
    // lists: the upper pairs i <= j; the lower ones are their transposes)
    const bool up_only = (c->prec == H2_PREC_FP64) ? (d.near_sym && d.n_lw > 0)
                                                   : ((int)c->f32.lv.size() > l && c->f32.lv[l].proj_sym);
    const double npj = (double)(up_only ? d.n_up : d.NP);
    fl_proj += npj * 4.0 * D * D * D;
    // algorithmic bytes of the tensor-core projection: the 16-bit input
    // blocks and bases read once, the outputs written once (FP32 SS of the
    // off-diagonal pairs or whole FP32 blocks, and the 16-bit copy)
    if (c->prec != H2_PREC_FP64 && (int)c->f32.lv.size() > l && c->f32.lv[l].tc) {
      const FacLevel<float>& f = c->f32.lv[l];
      const double out32 = f.ahat_ss_only ? (npj - d.nb) * K * K + (double)d.nb * D * D : npj * D * D;
      by_proj += 2.0 * npj * D * D + 2.0 * d.nb * D * D + 4.0 * out32 + (f.ahat_isc ? 2.0 * npj * D * D : 0.0);
    }
    fl_lu += d.nb * 2.0 * R * R * R;
    fl_schur += d.nb * (2.0 * R * R * K + 2.0 * K * K * R);
    fl_coup += d.FP * 4.0 * K * K * K;
    fl_qr += d.nb * (4.0 * D * K * K + 4.0 * D * D * K);
  }
  // algorithmic traffic of one substitution (Eq. 31 form; storage width w)
  // and one FP64 matvec
  const double w = (c->prec == H2_PREC_FP64) ? 8.0 : 4.0;
  double by_sub = 0, by_mv = 0, fl_mv = 0;
  for (int l = 1; l <= c->L; ++l) {
    const DevLevel& d = c->lv[l];
    const double D = d.D, K = d.K, R = d.R;
    // Ahat read in 16 bits where the factorization kept a 16-bit copy
    const bool a16 = c->prec != H2_PREC_FP64 && (int)c->f32.lv.size() > l && c->f32.lv[l].ahat_isc;
    const double wa = a16 ? 2.0 : w;
    // per box: M1 and U^S (fwd1), U (bwd2) and three reads of the inverse
    by_sub += wa * ((double)(d.NP - d.nb) * R * R + (double)d.NP * 2.0 * R * K) + w * d.nb * (2.0 * D * D + 3.0 * R * R);
    by_mv += 8.0 * (2.0 * d.nb * D * K + (double)d.FP * K * K);
    fl_mv += 2.0 * (2.0 * d.nb * D * K + (double)d.FP * K * K);
  }
  double by_leaf32 = 0;
  {
    const DevLevel& lf = c->lv[c->L];
    // the mixed solve's matvecs read only the stored halves of symmetric
    // leaf blocks (the FP64 path reads all of them)
    const bool symm = c->sym && c->prec != H2_PREC_FP64;
    const double npl = symm ? (double)c->npu : (double)lf.NP;
    by_mv += 8.0 * npl * lf.D * lf.D;
    fl_mv += 2.0 * (double)lf.NP * lf.D * lf.D;
    // the FP32 matvec's leaf kernel: the near blocks read once, x read, y or
    // (symmetric storage) two partial products per stored pair written
    const double K = c->L ? lf.K : 0;
    by_leaf32 = symm ? 4.0 * ((double)c->npu * lf.D * lf.D + (double)lf.nb * lf.D + 2.0 * c->npu * lf.D)
                     : 4.0 * ((double)lf.NP * lf.D * lf.D + (double)lf.nb * lf.D * K + 2.0 * lf.nb * lf.D + lf.nb * K);
  }
  o << "],\"bytes_proj\":" << by_proj << ",\"bytes_subst\":" << by_sub << ",\"bytes_matvec\":" << by_mv << ",\"flops_matvec\":" << fl_mv
    << ",\"bytes_matvec32\":" << by_mv / 2 << ",\"bytes_matvec32_leaf\":" << by_leaf32 << ",\"leaf_kernel\":\""
    << ((c->sym && c->prec != H2_PREC_FP64) ? "mv_sym_pair_kernel<float>" : "mv_leaf_kernel<float>") << "\"";
  o << ",\"flops\":{\"a1_qr\":" << fl_qr << ",\"a2_proj\":" << fl_proj << ",\"a3_lu\":" << fl_lu
    << ",\"a45_schur\":" << fl_schur << ",\"a2c_coupling\":" << fl_coup << "}";
  o << ",\"times\":{\"a1_qr\":" << t.a1_qr << ",\"a2_proj\":" << t.a2_proj << ",\"a3_lu\":" << t.a3_lu
    << ",\"a45_schur\":" << t.a5_schur << ",\"a2c_coupling\":" << t.a2c_coupling << ",\"a6_merge\":" << t.a6_merge
    << ",\"a7_root\":" << t.a7_root << ",\"wait_basis\":" << t.wait_basis << ",\"factor\":" << t.total_factor << ",\"solve\":" << t.solve_total
    << ",\"solve_subst\":" << t.subst << ",\"solve_matvec\":" << t.matvec << ",\"solve_matvec32\":" << t.matvec32
    << ",\"matvec32_leaf\":" << t.leaf32
    << "},\"calls\":{\"subst\":" << t.n_subst << ",\"matvec\":" << t.n_matvec << ",\"matvec32\":" << t.n_matvec32 << ",\"matvec32_leaf\":" << t.n_leaf32
    << "},\"method\":" << t.method
    << ",\"iters\":" << t.iters << ",\"relres\":" << t.relres
    << ",\"kernel_launches\":" << g_launches.load() << ",\"refine_method\":" << c->refine_method
    << ",\"restart\":" << c->restart << ",\"tensor_cores\":" << (c->used_tc ? "true" : "false")
    << ",\"schur_tensor_cores\":" << ((c->prec > 0 && c->f32.schur_tc) ? "true" : "false")
    << ",\"rr_lu_fp64\":" << (c->rr_lu64 ? "true" : "false")
    << ",\"history\":[";
  for (size_t k = 0; k < t.history.size(); ++k) o << (k ? "," : "") << t.history[k];
  o << "]";
  // the construction's rank layout: the predictor's ranks (-1: not used),
  // the final ranks, the boxes and levels that fell back to the plain pass
  const RankRecord& rec = c->host.rec;
  o << ",\"construction\":{\"compress_s\":" << rec.compress_s << ",\"fallback_boxes\":" << rec.fallback_boxes
    << ",\"fallback_levels\":" << rec.fallback_levels << ",\"gpu_levels\":" << rec.gpu_levels
    << ",\"flops_prefactor\":" << rec.flops_prefactor << ",\"flops_far\":" << rec.flops_far << ",\"K_pred\":[";
  for (int l = 0; l <= c->L; ++l) o << (l ? "," : "") << (l < (int)rec.K_pred.size() ? rec.K_pred[l] : -1);
  o << "],\"K\":[";
  for (int l = 0; l <= c->L; ++l) o << (l ? "," : "") << c->lv[l].K;
  o << "]}}";
  std::string s = o.str();
  if (s.size() + 1 > cap) return H2_ERR_INVALID_ARG;
  std::memcpy(json, s.c_str(), s.size() + 1);
  return H2_OK;
}

h2_status h2_export(const h2_ctx* c, const char* name, int32_t level, void* dst, size_t cap_bytes, size_t* count,
                    int32_t* elem_size) {
  if (!c || !name || !count || !elem_size) return H2_ERR_INVALID_ARG;
  const std::string n(name);
  if (n == "perm") {
    *count = c->host.perm.size();
    *elem_size = 8;
    if (dst) {
      if (cap_bytes < *count * 8) return H2_ERR_INVALID_ARG;
      std::memcpy(dst, c->host.perm.data(), *count * 8);
    }
    return H2_OK;
  }
  if (level < 0 || level > c->L) return H2_ERR_INVALID_ARG;
  const DevLevel& d = c->lv[level];
  const void* src = nullptr;
  size_t cnt = 0;
  int es = 8;
  const bool f64 = c->prec == H2_PREC_FP64;
  const bool ready = factor_ready(c);
  auto pick = [&](const void* p64, const void* p32, size_t k, bool need_factor) -> h2_status {
    if (need_factor && !ready) return H2_ERR_STATE;
    src = f64 ? p64 : p32;
    es = f64 ? 8 : 4;
    cnt = k;
    return H2_OK;
  };
  h2_status s = H2_OK;
  const size_t nb = d.nb, D = d.D, K = d.K, R = d.R;
  if (n == "X") {
    if (level == 0) return H2_ERR_INVALID_ARG;
    src = d.X; cnt = nb * D * K; es = 8;
  } else if (n == "A") {
    if (level == c->L) {
      if (!c->A64) return H2_ERR_STATE;
      src = c->A64; cnt = (size_t)d.NP * D * D; es = 8;
    }
    else s = pick(c->f64.lv.empty() ? nullptr : c->f64.lv[level].Ain,
                  c->f32.lv.empty() ? nullptr : c->f32.lv[level].Ain, (size_t)d.NP * D * D, true);
  } else if (level >= 1 && (n == "U" || n == "T" || n == "Ahat" || n == "Ainv" || n == "Shat")) {
    const FacLevel<double>* a = c->f64.lv.empty() ? nullptr : &c->f64.lv[level];
    const FacLevel<float>* b = c->f32.lv.empty() ? nullptr : &c->f32.lv[level];
    if (!ready || (f64 && !a) || (!f64 && !b)) return H2_ERR_STATE;
    if (n == "U") s = pick(a ? a->U : nullptr, b ? b->U : nullptr, nb * D * D, true);
    if (n == "T") s = pick(a ? a->Tm : nullptr, b ? b->Tm : nullptr, nb * K * K, true);
    if (n == "Ahat") s = pick(a ? a->Ahat : nullptr, b ? b->Ahat : nullptr, (size_t)d.NP * D * D, true);
    if (n == "Ainv") s = pick(a ? a->Ainv : nullptr, b ? b->Ainv : nullptr, nb * R * R, true);
    if (n == "Shat") s = pick(a ? a->Shat : nullptr, b ? b->Shat : nullptr, (size_t)d.FP * K * K, true);
  } else if (level >= 1 && (n == "lu" || n == "piv")) {
    if (!ready) return H2_ERR_STATE;
    const bool p64 = f64;
    if (n == "lu" && !p64) return H2_ERR_INVALID_ARG;  // the mixed factorization keeps only the inverses
    src = (n == "lu") ? (const void*)(p64 ? c->f64.lv[level].lu : (const double*)(const void*)c->f32.lv[level].luT)
                      : (const void*)(p64 ? c->f64.lv[level].piv : c->f32.lv[level].piv);
    es = (n == "lu") ? (p64 ? 8 : 4) : 4;
    cnt = (n == "lu") ? nb * R * R : nb * R;
  } else if (n == "root" || n == "root_piv" || n == "root_inv") {
    if (!ready) return H2_ERR_STATE;
    const size_t D0 = c->lv[0].D, nr = c->lv[0].nb;  // nr roots (one per system of a forest)
    if (n == "root" && !f64) return H2_ERR_INVALID_ARG;  // as for "lu"
    if (n == "root") {
      src = f64 ? (const void*)c->f64.root_lu : (const void*)c->f32.root_luT;
      es = f64 ? 8 : 4;
      cnt = nr * D0 * D0;
    }
    if (n == "root_piv") {
      src = f64 ? (const void*)c->f64.root_piv : (const void*)c->f32.root_piv;
      es = 4;
      cnt = nr * D0;
    }
    if (n == "root_inv") s = pick(c->f64.root_inv, c->f32.root_inv, nr * D0 * D0, true);
  } else {
    return H2_ERR_INVALID_ARG;
  }
  if (s != H2_OK) return s;
  *count = cnt;
  *elem_size = es;
  if (dst) {
    if (!src) return H2_ERR_STATE;
    if (cap_bytes < cnt * es) return H2_ERR_INVALID_ARG;
    if (cudaMemcpy(dst, src, cnt * es, cudaMemcpyDeviceToHost) != cudaSuccess) return H2_ERR_CUDA;
    // mixed levels whose off-diagonal pairs keep only SS in FP32: the other
    // quadrants come from the 16-bit copy s * Ahat, times 1 / s
    if (n == "Ahat" && !f64 && c->f32.lv[level].ahat_ss_only) return export_ahat_quadrants(c, level, (float*)dst);
  }
  return H2_OK;
}

const char* h2_last_error(const h2_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

void h2_destroy(h2_ctx* c) {
  if (!c) return;
  if (c->mv_fork) cudaEventDestroy(c->mv_fork);
  if (c->mv_join) cudaEventDestroy(c->mv_join);
  drop_graphs(c);
  for (cudaStream_t s : {c->basis_stream, c->coupling_stream, c->product_stream, c->leaf_stream, c->cap_stream}) {
    if (!s) continue;
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->f64.allocs) cudaFree(p);
  for (void* p : c->f32.allocs) cudaFree(p);
  if (c->gm_host) cudaFreeHost(c->gm_host);
  delete c;
}

}  // extern "C"
