// lq_api.cpp -- host runtime behind the C ABI in include/lecqmc.h: lattices
// in checkerboard form, one device arena per simulation, chain descriptors,
// and the launches of the sm_103a kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/lecqmc.h"
#include "lq_device.h"
#include "lq_kernels.h"
#include "lq_lattice.h"
#include "lq_internal.h"

static thread_local std::string g_err;

static lq_status fail(lq_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
static lq_status cuda_fail(cudaError_t e, const char* where) {
  return fail(LQ_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

// ---------------------------------------------------------------------------
// lattices
// ---------------------------------------------------------------------------
struct lq_lattice {
  int N = 0;
  std::vector<int> bi, bj, sub, fam;
  std::vector<double> kb, eps;
  bool has_eps = false;
  int G = 0;
  // family-sorted copies (read by the allocation-free entry point)
  std::vector<int> fam_off, sorted_i, sorted_j;
  std::vector<double> sorted_k;
  // each site's distinct bond partners, ascending (nearest-neighbour swaps)
  std::vector<int> nb_off, nb_site;
  // K in compressed rows, bonds summed and the onsite term on the diagonal
  // (the exact kinetic propagator), and max_i sum_j |K_ij|
  std::vector<int> k_off, k_col;
  std::vector<double> k_val;
  double k_rownorm = 0.0;
};

// each bond, in order, goes to the lowest family where neither site is used
static void assign_families(lq_lattice* L) {
  std::vector<std::vector<char>> used;
  L->fam.assign(L->bi.size(), 0);
  L->G = 0;
  for (size_t b = 0; b < L->bi.size(); ++b) {
    int g = 0;
    for (;; ++g) {
      if (g == (int)used.size()) used.emplace_back(L->N, 0);
      if (!used[g][L->bi[b]] && !used[g][L->bj[b]]) break;
    }
    used[g][L->bi[b]] = used[g][L->bj[b]] = 1;
    L->fam[b] = g;
    L->G = std::max(L->G, g + 1);
  }
}

static lq_status make_lattice(int N, const std::vector<int>& bi, const std::vector<int>& bj,
                              const std::vector<double>& kb, const double* onsite, const int* sub, lq_lattice** out) {
  if (!out) return fail(LQ_EINVAL, "null output pointer");
  if (N < 1) return fail(LQ_EINVAL, "n_sites must be >= 1");
  for (size_t b = 0; b < bi.size(); ++b) {
    if (bi[b] < 0 || bi[b] >= N || bj[b] < 0 || bj[b] >= N || bi[b] == bj[b])
      return fail(LQ_EINVAL, "bond " + std::to_string(b) + " has a bad site index");
    if (!std::isfinite(kb[b])) return fail(LQ_EINVAL, "non-finite hopping");
  }
  lq_lattice* L = new (std::nothrow) lq_lattice();
  if (!L) return fail(LQ_ENOMEM, "host allocation");
  L->N = N;
  L->bi = bi; L->bj = bj; L->kb = kb;
  L->eps.assign(N, 0.0);
  L->sub.resize(N);
  for (int i = 0; i < N; ++i) {
    if (onsite) { L->eps[i] = onsite[i]; if (onsite[i] != 0.0) L->has_eps = true; }
    L->sub[i] = sub ? (sub[i] ? 1 : 0) : (i & 1);
  }
  assign_families(L);
  const int nb = (int)L->bi.size();
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return L->fam[a] < L->fam[b]; });
  L->fam_off.assign(L->G + 1, 0);
  for (int b = 0; b < nb; ++b) L->fam_off[L->fam[b] + 1]++;
  for (int g = 0; g < L->G; ++g) L->fam_off[g + 1] += L->fam_off[g];
  for (int t = 0; t < nb; ++t) {
    L->sorted_i.push_back(L->bi[order[t]]);
    L->sorted_j.push_back(L->bj[order[t]]);
    L->sorted_k.push_back(L->kb[order[t]]);
  }
  std::vector<std::vector<int>> adj(N);
  for (int b = 0; b < nb; ++b) {
    adj[L->bi[b]].push_back(L->bj[b]);
    adj[L->bj[b]].push_back(L->bi[b]);
  }
  L->nb_off.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
    L->nb_off[i + 1] = L->nb_off[i] + (int)adj[i].size();
    L->nb_site.insert(L->nb_site.end(), adj[i].begin(), adj[i].end());
  }
  {
    std::vector<std::map<int, double>> rows(N);
    for (int i = 0; i < N; ++i)
      if (L->eps[i] != 0.0) rows[i][i] += L->eps[i];
    for (int b = 0; b < nb; ++b) {
      rows[L->bi[b]][L->bj[b]] += L->kb[b];
      rows[L->bj[b]][L->bi[b]] += L->kb[b];
    }
    L->k_off.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) {
      double rs = 0.0;
      for (const auto& e : rows[i]) {
        L->k_col.push_back(e.first);
        L->k_val.push_back(e.second);
        rs += std::fabs(e.second);
      }
      L->k_off[i + 1] = (int)L->k_col.size();
      L->k_rownorm = std::max(L->k_rownorm, rs);
    }
  }
  *out = L;
  return LQ_OK;
}

lq_lattice_view lq_lattice_get_view(const lq_lattice* L) {
  lq_lattice_view v;
  v.N = L->N; v.nb = (int)L->bi.size(); v.G = L->G; v.has_eps = L->has_eps;
  v.fam_off = L->fam_off.data(); v.sorted_i = L->sorted_i.data(); v.sorted_j = L->sorted_j.data();
  v.sorted_k = L->sorted_k.data(); v.eps = L->eps.data(); v.sub = L->sub.data();
  v.nb_off = L->nb_off.data(); v.nb_site = L->nb_site.data();
  v.nnz = (int)L->k_col.size(); v.k_off = L->k_off.data(); v.k_col = L->k_col.data(); v.k_val = L->k_val.data();
  v.k_rownorm = L->k_rownorm;
  return v;
}

lq_status lq_internal_fail(lq_status s, const std::string& msg) { return fail(s, msg); }

extern "C" lq_status lq_lattice_from_bonds(int32_t n_sites, int32_t n_bonds, const int32_t* bi, const int32_t* bj,
                                           const double* kij, const double* onsite, const int32_t* sublattice,
                                           lq_lattice** out) {
  if (n_bonds < 0 || (n_bonds > 0 && (!bi || !bj || !kij))) return fail(LQ_EINVAL, "bad bond arrays");
  std::vector<int> vi(bi, bi + n_bonds), vj(bj, bj + n_bonds);
  std::vector<double> vk(kij, kij + n_bonds);
  return make_lattice(n_sites, vi, vj, vk, onsite, sublattice, out);
}

extern "C" lq_status lq_lattice_chain(int32_t n, double t, int32_t periodic, lq_lattice** out) {
  if (n < 1) return fail(LQ_EINVAL, "n_sites must be >= 1");
  std::vector<int> bi, bj;
  std::vector<double> kb;
  for (int parity = 0; parity < 2; ++parity) {
    for (int i = parity; i + 1 < n; i += 2) { bi.push_back(i); bj.push_back(i + 1); kb.push_back(-t); }
    if (periodic && n > 2 && (n - 1) % 2 == parity) { bi.push_back(n - 1); bj.push_back(0); kb.push_back(-t); }
  }
  return make_lattice(n, bi, bj, kb, nullptr, nullptr, out);
}

extern "C" lq_status lq_lattice_square(int32_t lx, int32_t ly, double t, int32_t periodic, lq_lattice** out) {
  if (lx < 1 || ly < 1) return fail(LQ_EINVAL, "lx, ly must be >= 1");
  std::vector<int> bi, bj, sub(lx * ly);
  std::vector<double> kb;
  auto idx = [lx](int x, int y) { return x + lx * y; };
  for (int parity = 0; parity < 2; ++parity)
    for (int y = 0; y < ly; ++y)
      for (int x = parity; x < lx; x += 2) {
        if (x + 1 < lx) { bi.push_back(idx(x, y)); bj.push_back(idx(x + 1, y)); kb.push_back(-t); }
        else if (periodic && lx > 2) { bi.push_back(idx(x, y)); bj.push_back(idx(0, y)); kb.push_back(-t); }
      }
  for (int parity = 0; parity < 2; ++parity)
    for (int y = parity; y < ly; y += 2)
      for (int x = 0; x < lx; ++x) {
        if (y + 1 < ly) { bi.push_back(idx(x, y)); bj.push_back(idx(x, y + 1)); kb.push_back(-t); }
        else if (periodic && ly > 2) { bi.push_back(idx(x, y)); bj.push_back(idx(x, 0)); kb.push_back(-t); }
      }
  for (int y = 0; y < ly; ++y)
    for (int x = 0; x < lx; ++x) sub[idx(x, y)] = (x + y) & 1;
  return make_lattice(lx * ly, bi, bj, kb, nullptr, sub.data(), out);
}

extern "C" lq_status lq_lattice_flatband(int32_t nc, double t1, double t2, double t3, double t4, int32_t periodic,
                                         lq_lattice** out) {
  if (nc < 1) return fail(LQ_EINVAL, "n_cells must be >= 1");
  const int N = 2 * nc;
  auto A1 = [nc](int R) { return 2 * (((R % nc) + nc) % nc); };
  auto A2 = [nc](int R) { return 2 * (((R % nc) + nc) % nc) + 1; };
  const bool wrap = periodic && nc > 2;
  const int nR = wrap ? nc : nc - 1;
  std::vector<int> bi, bj;
  std::vector<double> kb;
  auto add = [&](int i, int j, double k) { if (k != 0.0) { bi.push_back(i); bj.push_back(j); kb.push_back(k); } };
  for (int parity = 0; parity < 2; ++parity)
    for (int R = parity; R < nR; R += 2) add(A1(R), A1(R + 1), t1 * t2);
  for (int parity = 0; parity < 2; ++parity)
    for (int R = parity; R < nR; R += 2) add(A2(R), A2(R + 1), t3 * t4);
  for (int R = 0; R < nc; ++R) add(A1(R), A2(R), t1 * t3 + t2 * t4);
  for (int R = 0; R < nc; ++R)
    if (R + 1 < nc || wrap) add(A1(R), A2(R + 1), t1 * t4);
  for (int R = 0; R < nc; ++R)
    if (R - 1 >= 0 || wrap) add(A1(R), A2(R - 1), t2 * t3);
  std::vector<double> eps(N);
  for (int R = 0; R < nc; ++R) { eps[2 * R] = t1 * t1 + t2 * t2; eps[2 * R + 1] = t3 * t3 + t4 * t4; }
  return make_lattice(N, bi, bj, kb, eps.data(), nullptr, out);
}

extern "C" lq_status lq_lattice_cross_stitch(int32_t nc, double t_intra, double t_leg, double t_cross,
                                             int32_t periodic, lq_lattice** out) {
  if (nc < 1) return fail(LQ_EINVAL, "n_cells must be >= 1");
  auto a = [nc](int R) { return 2 * (R % nc); };
  auto b = [nc](int R) { return 2 * (R % nc) + 1; };
  const bool wrap = periodic && nc > 2;
  const int nR = wrap ? nc : nc - 1;
  std::vector<int> bi, bj;
  std::vector<double> kb;
  auto add = [&](int i, int j, double k) { bi.push_back(i); bj.push_back(j); kb.push_back(k); };
  for (int R = 0; R < nc; ++R) add(a(R), b(R), -t_intra);
  for (int leg = 0; leg < 2; ++leg)
    for (int parity = 0; parity < 2; ++parity)
      for (int R = parity; R < nR; R += 2) add(leg ? b(R) : a(R), leg ? b(R + 1) : a(R + 1), -t_leg);
  for (int parity = 0; parity < 2; ++parity)
    for (int R = parity; R < nR; R += 2) { add(a(R), b(R + 1), -t_cross); add(b(R), a(R + 1), -t_cross); }
  return make_lattice(2 * nc, bi, bj, kb, nullptr, nullptr, out);
}

extern "C" lq_status lq_lattice_info(const lq_lattice* L, int32_t* n_sites, int32_t* n_bonds, int32_t* n_fam) {
  if (!L) return fail(LQ_EINVAL, "null lattice");
  if (n_sites) *n_sites = L->N;
  if (n_bonds) *n_bonds = (int32_t)L->bi.size();
  if (n_fam) *n_fam = L->G;
  return LQ_OK;
}

extern "C" lq_status lq_lattice_bonds(const lq_lattice* L, int32_t* bi, int32_t* bj, double* kij, int32_t* fam) {
  if (!L) return fail(LQ_EINVAL, "null lattice");
  for (size_t b = 0; b < L->bi.size(); ++b) {
    if (bi) bi[b] = L->bi[b];
    if (bj) bj[b] = L->bj[b];
    if (kij) kij[b] = L->kb[b];
    if (fam) fam[b] = L->fam[b];
  }
  return LQ_OK;
}

extern "C" lq_status lq_lattice_destroy(lq_lattice* L) {
  delete L;
  return LQ_OK;
}

// ---------------------------------------------------------------------------
// simulations
// ---------------------------------------------------------------------------
struct ChainHost {
  int N, L, tw, n, ns[2];
  int G, nb, nnz;
  int exact, taylor_q;  // exact kinetic propagator and its Taylor degree
  double cost;
};

struct lq_sim {
  int n_chains = 0, prec = 0;
  cudaStream_t st = nullptr;
  lq_allocator alloc{};
  bool has_alloc = false;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<LqChainDev> h;     // host mirror of the descriptors
  std::vector<ChainHost> info;
  LqChainDev* d_chains = nullptr;
  int* d_order = nullptr;        // chains by decreasing cost
  int* d_single = nullptr;       // scratch list of one chain
  int* d_queue = nullptr;
  // with chains in both plan classes, the large class runs on a second stream
  // (its own chain queue) concurrently with the small one, joined by events
  int* d_queue2 = nullptr;
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int* d_all = nullptr;          // 0..n-1
  int M = 1, Nmax = 1, buf_bytes = 0, grid = 1;
  // sweeps run one launch per plan class: chains with at most LQ_NS_SMALL
  // particles per spin (shared-memory plan), then the larger ones (global
  // workspace); d_order holds the small class first, each by decreasing cost
  struct PlanClass {
    int n = 0, off = 0, M = 1, Nmax = 1, buf = 0, grid = 1, pcols = 1, threads = LQ_THREADS;
  } cls[2];
  char* ws = nullptr;            // global workspace of big plans (grid x per-CTA slab)
  size_t ws_bytes = 0;
  bool mirror_fresh = false;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static lq_status pull(lq_sim* S) {
  CK(cudaStreamSynchronize(S->st));
  if (!S->mirror_fresh) {
    CK(cudaMemcpy(S->h.data(), S->d_chains, sizeof(LqChainDev) * S->n_chains, cudaMemcpyDeviceToHost));
    S->mirror_fresh = true;
  }
  return LQ_OK;
}

static lq_status check_chain(const lq_sim* S, int c) {
  if (!S) return fail(LQ_EINVAL, "null simulation");
  if (c < 0 || c >= S->n_chains) return fail(LQ_EINVAL, "chain index out of range");
  return LQ_OK;
}

static size_t csr_bytes(int N, int nnz) {
  return al256((size_t)(N + 1) * 4) + al256((size_t)std::max(nnz, 1) * 4) + al256((size_t)std::max(nnz, 1) * 8) +
         al256((size_t)std::max(nnz, 1) * 4);
}

static size_t footprint_one(int N, int nb, int G, int L, int tw, const int ns[2], int prec, int max_records,
                            int exact) {
  const size_t PS = prec == LQ_FP64 ? sizeof(double) : sizeof(float);
  const int n = (L + tw - 1) / tw;
  size_t b = al256((G + 1) * 4) + 3 * al256(nb * 4) + 3 * al256(nb * 8) + 2 * al256(nb * 4) + 3 * al256(N * 8) +
             al256(N * 4) + al256(N * 4) + al256((size_t)(N + 1) * 4) + al256((size_t)std::max(2 * nb, 1) * 4) +
             al256((size_t)L * N) + csr_bytes(N, N + 2 * nb);
  for (int sg = 0; sg < 2; ++sg) {
    const size_t pn = (size_t)N * ns[sg], qn = (size_t)ns[sg] * ns[sg];
    b += al256(std::max(ns[sg], 1) * 4);
    b += 2 * al256((n + 1) * pn * PS) + 2 * al256((n + 1) * qn * 8);
    b += al256((n + 1) * pn * PS) + al256((n + 1) * qn * 8);
    b += al256(tw * pn * PS) + al256(pn * PS) + al256(pn * 8);
  }
  b += al256((size_t)2 * N * 8) + al256((size_t)n * LQ_NS_MAX * 2 * 8) + al256((size_t)max_records * LQ_NOBS * 8);
  const int M = std::max(std::max(ns[0], ns[1]), 1);
  b += al256(lq::workspace_bytes(M, N, lq::staging_bytes(M, N, exact ? 2 : 1)));  // one CTA's workspace (big plans)
  return b + al256(sizeof(LqChainDev)) + 4 * al256(sizeof(int) * 1026);
}

static lq_status create_impl(const lq_lattice* const* lats, const lq_params* params, int32_t n_chains,
                             const uint32_t* chain_ids, void* stream, const lq_allocator* alloc, bool build,
                             lq_sim** out);

extern "C" lq_status lq_sim_create(const lq_lattice* const* lats, const lq_params* params, int32_t n_chains,
                                   const uint32_t* chain_ids, void* stream, const lq_allocator* alloc, lq_sim** out) {
  return create_impl(lats, params, n_chains, chain_ids, stream, alloc, true, out);
}

lq_status lq_internal_sim_create_unbuilt(const lq_lattice* lat, const lq_params* params, uint32_t chain_id,
                                         void* stream, const lq_allocator* alloc, lq_sim** out) {
  return create_impl(&lat, params, 1, &chain_id, stream, alloc, false, out);
}

static lq_status create_impl(const lq_lattice* const* lats, const lq_params* params, int32_t n_chains,
                             const uint32_t* chain_ids, void* stream, const lq_allocator* alloc, bool build,
                             lq_sim** out) {
  if (!out || !lats || !params || n_chains < 1) return fail(LQ_EINVAL, "bad arguments to lq_sim_create");
  const int prec = params[0].precision;
  if (prec != LQ_FP64 && prec != LQ_MIXED && prec != LQ_MIXED_DW)
    return fail(LQ_EINVAL, "precision must be LQ_FP64, LQ_MIXED or LQ_MIXED_DW");
  std::vector<ChainHost> info(n_chains);
  int M = 1, Nmax = 1, any_exact = 0;
  for (int c = 0; c < n_chains; ++c) {
    const lq_lattice* Lt = lats[c];
    const lq_params& p = params[c];
    if (!Lt) return fail(LQ_EINVAL, "null lattice for chain " + std::to_string(c));
    if (p.precision != prec) return fail(LQ_EINVAL, "all chains must share one precision");
    if (!(p.beta > 0) || !(p.dtau > 0) || !std::isfinite(p.U)) return fail(LQ_EINVAL, "beta, dtau must be > 0");
    const double Lf = p.beta / p.dtau;
    const long Ll = std::lround(Lf);
    if (Ll < 1 || std::fabs(Lf - (double)Ll) > 1e-9 * std::max(1.0, Lf) || Ll > (1 << 24) - 1)
      return fail(LQ_EINVAL, "beta/dtau must be a positive integer");
    if (p.n_stab < 1) return fail(LQ_EINVAL, "n_stab must be >= 1");
    if (p.swap_mode != LQ_SWAP_UNIFORM && p.swap_mode != LQ_SWAP_NEIGHBOUR)
      return fail(LQ_EINVAL, "swap_mode must be LQ_SWAP_UNIFORM or LQ_SWAP_NEIGHBOUR");
    if (p.left_swaps != 0 && p.left_swaps != 1) return fail(LQ_EINVAL, "left_swaps must be 0 or 1");
    if (p.kinetic != LQ_CHECKERBOARD && p.kinetic != LQ_EXACT)
      return fail(LQ_EINVAL, "kinetic must be LQ_CHECKERBOARD or LQ_EXACT");
    if (p.kinetic == LQ_EXACT && p.dtau * Lt->k_rownorm > LQ_EXACT_THETA_MAX)
      return fail(LQ_EUNSUPPORTED, "LQ_EXACT needs dtau * max_i sum_j |K_ij| <= 2");
    if (p.n_up < 0 || p.n_dn < 0 || p.n_up > Lt->N || p.n_dn > Lt->N)
      return fail(LQ_EINVAL, "particle numbers must be in [0, N]");
    if (p.n_up > LQ_MAX_PARTICLES || p.n_dn > LQ_MAX_PARTICLES)
      return fail(LQ_EUNSUPPORTED, "at most LQ_MAX_PARTICLES particles per spin");
    ChainHost& ci = info[c];
    ci.N = Lt->N; ci.L = (int)Ll; ci.tw = p.n_stab; ci.n = (ci.L + ci.tw - 1) / ci.tw;
    ci.ns[0] = p.n_up; ci.ns[1] = p.n_dn; ci.G = Lt->G; ci.nb = (int)Lt->bi.size(); ci.nnz = (int)Lt->k_col.size();
    ci.exact = p.kinetic == LQ_EXACT;
    ci.taylor_q = ci.exact ? lq_taylor_degree(p.dtau * Lt->k_rownorm) : 0;
    ci.cost = (double)ci.L * ci.N * (ci.ns[0] * ci.ns[0] + ci.ns[1] * ci.ns[1] + (3.0 * ci.G + 1) * (ci.ns[0] + ci.ns[1]) + 1);
    M = std::max(M, std::max(ci.ns[0], ci.ns[1]));
    Nmax = std::max(Nmax, ci.N);
    any_exact |= ci.exact;
  }
  lq_sim* S = new (std::nothrow) lq_sim();
  if (!S) return fail(LQ_ENOMEM, "host allocation");
  S->n_chains = n_chains;
  S->prec = prec;
  S->st = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) { S->alloc = *alloc; S->has_alloc = true; }
  S->info = info;
  S->M = M;
  S->Nmax = Nmax;
  const size_t PS = prec == LQ_FP64 ? sizeof(double) : sizeof(float);
  // shared-memory staging buffer: at least one full column of the largest
  // panel, and room for a chunk of rows in the flip loop
  S->buf_bytes = lq::staging_bytes(M, Nmax, any_exact ? 2 : 1);
  {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = lq::smem_bytes(M, Nmax, S->buf_bytes);
    const int per_sm = lq::max_active_sweep_ctas(prec, M, smem);
    if (per_sm < 1) { delete S; return fail(LQ_EUNSUPPORTED, "shared-memory plan does not fit one CTA per SM"); }
    S->grid = std::min(n_chains, sms * per_sm);
    S->ws_bytes = (size_t)S->grid * lq::workspace_bytes(M, Nmax, S->buf_bytes);
  }
  // arena layout
  std::vector<size_t> off(n_chains);
  size_t tot = 0;
  auto lat_bytes = [&](int c) {
    const ChainHost& ci = info[c];
    return al256((ci.G + 1) * 4) + 3 * al256(ci.nb * 4) + 3 * al256(ci.nb * 8) + 2 * al256(ci.nb * 4) +
           3 * al256(ci.N * 8) + al256(ci.N * 4) + al256(ci.N * 4) + al256((size_t)(ci.N + 1) * 4) +
           al256((size_t)std::max(2 * ci.nb, 1) * 4) + csr_bytes(ci.N, ci.nnz);
  };
  const int max_records = 1 << 16;
  auto chain_bytes = [&](int c) {
    const ChainHost& ci = info[c];
    size_t b = lat_bytes(c) + al256((size_t)ci.L * ci.N);
    for (int sg = 0; sg < 2; ++sg) {
      const size_t pn = (size_t)ci.N * ci.ns[sg], qn = (size_t)ci.ns[sg] * ci.ns[sg];
      b += al256(std::max(ci.ns[sg], 1) * 4);
      b += 2 * al256((ci.n + 1) * pn * PS) + 2 * al256((ci.n + 1) * qn * 8);
      b += al256((ci.n + 1) * pn * PS) + al256((ci.n + 1) * qn * 8);
      b += al256(ci.tw * pn * PS) + al256(pn * PS) + al256(pn * 8);
    }
    b += al256((size_t)2 * ci.N * 8) + al256((size_t)ci.n * LQ_NS_MAX * 2 * 8);
    b += al256((size_t)max_records * LQ_NOBS * 8);
    return b;
  };
  for (int c = 0; c < n_chains; ++c) { off[c] = tot; tot += chain_bytes(c); }
  const size_t desc_off = tot;
  tot += al256(sizeof(LqChainDev) * n_chains) + 3 * al256(sizeof(int) * (n_chains + 1)) +
         al256(sizeof(int) * (n_chains + 1 + 1024)) + al256(sizeof(int) * (1 + 1024));
  const size_t ws_off = tot;
  tot += al256(S->ws_bytes);
  S->arena_bytes = tot;
  if (S->has_alloc) S->arena = (char*)S->alloc.alloc(S->alloc.ctx, tot, stream);
  else if (cudaMalloc((void**)&S->arena, tot) != cudaSuccess) S->arena = nullptr;
  if (!S->arena) { delete S; return fail(LQ_ENOMEM, "device arena of " + std::to_string(tot) + " bytes"); }
  cudaError_t e = cudaMemsetAsync(S->arena, 0, tot, S->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
  if (e != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(e, "arena memset"); }
  S->d_chains = (LqChainDev*)(S->arena + desc_off);
  size_t o2 = desc_off + al256(sizeof(LqChainDev) * n_chains);
  S->d_order = (int*)(S->arena + o2); o2 += al256(sizeof(int) * (n_chains + 1));
  S->d_single = (int*)(S->arena + o2); o2 += al256(sizeof(int) * (n_chains + 1));
  S->d_all = (int*)(S->arena + o2); o2 += al256(sizeof(int) * (n_chains + 1));
  S->d_queue = (int*)(S->arena + o2);  // [0]: chain queue, [1..1024]: per-SM CTA counters
  S->d_queue2 = (int*)(S->arena + o2 + al256(sizeof(int) * (n_chains + 1 + 1024)));
  S->ws = S->ws_bytes ? S->arena + ws_off : nullptr;
  // descriptors + host-side constant data (lattice tables, P = first sites)
  S->h.resize(n_chains);
  std::vector<char> stage;
  for (int c = 0; c < n_chains; ++c) {
    const lq_lattice* Lt = lats[c];
    const lq_params& p = params[c];
    const ChainHost& ci = info[c];
    LqChainDev& D = S->h[c];
    std::memset(&D, 0, sizeof(D));
    char* base = S->arena + off[c];
    size_t o = 0;
    auto take = [&](size_t bytes) { char* q = base + o; o += al256(bytes); return q; };
    // lattice, bonds sorted by family (stable)
    std::vector<int> order(ci.nb);
    for (int b = 0; b < ci.nb; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Lt->fam[a] < Lt->fam[b]; });
    std::vector<int> fo(ci.G + 1, 0), vi(ci.nb), vj(ci.nb);
    std::vector<double> vc(ci.nb), vs(ci.nb), vk(ci.nb), ce(ci.N), ep(ci.N);
    std::vector<float> vcf(ci.nb), vsf(ci.nb), cef(ci.N);
    for (int b = 0; b < ci.nb; ++b) fo[Lt->fam[b] + 1]++;
    for (int g = 0; g < ci.G; ++g) fo[g + 1] += fo[g];
    for (int t = 0; t < ci.nb; ++t) {
      const int b = order[t];
      vi[t] = Lt->bi[b]; vj[t] = Lt->bj[b]; vk[t] = Lt->kb[b];
      lq_bond_factors(p.dtau, Lt->kb[b], &vc[t], &vs[t]);
      vcf[t] = (float)vc[t]; vsf[t] = (float)vs[t];
    }
    for (int i = 0; i < ci.N; ++i) { ep[i] = Lt->eps[i]; ce[i] = lq_onsite_factor(p.dtau, Lt->eps[i]); cef[i] = (float)ce[i]; }
    // families whose bonds share one cosh and hold every site once take the
    // two-FMA form on FP64 panels: -tanh in the FP64 table, the cosh product
    // applied once per slice (FP32 panels keep the four-term form)
    double cprod = 1.0;
    const unsigned unif = lq_uniform_families(lq_lattice_get_view(Lt), p.dtau, &cprod);
    for (int g = 0; g < ci.G && g < 32; ++g)
      if ((unif >> g) & 1u)
        for (int t = fo[g]; t < fo[g + 1]; ++t) vs[t] = lq_bond_tanh(p.dtau, vk[t]);
    auto up = [&](void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S->st);
    };
    int* d_fo = (int*)take((ci.G + 1) * 4);
    int* d_bi = (int*)take(ci.nb * 4);
    int* d_bj = (int*)take(ci.nb * 4);
    (void)take(ci.nb * 4);
    double* d_bc = (double*)take(ci.nb * 8);
    double* d_bs = (double*)take(ci.nb * 8);
    double* d_bk = (double*)take(ci.nb * 8);
    float* d_bcf = (float*)take(ci.nb * 4);
    float* d_bsf = (float*)take(ci.nb * 4);
    double* d_ce = (double*)take(ci.N * 8);
    double* d_ep = (double*)take(ci.N * 8);
    (void)take(ci.N * 8);
    float* d_cef = (float*)take(ci.N * 4);
    int* d_sub = (int*)take(ci.N * 4);
    int* d_nbo = (int*)take((size_t)(ci.N + 1) * 4);
    int* d_nbs = (int*)take((size_t)std::max(2 * ci.nb, 1) * 4);
    int* d_ko = (int*)take((size_t)(ci.N + 1) * 4);
    int* d_kc = (int*)take((size_t)std::max(ci.nnz, 1) * 4);
    double* d_kv = (double*)take((size_t)std::max(ci.nnz, 1) * 8);
    float* d_kvf = (float*)take((size_t)std::max(ci.nnz, 1) * 4);
    std::vector<float> kvf(Lt->k_val.begin(), Lt->k_val.end());
    std::vector<cudaError_t> es;
    es.push_back(up(d_ko, Lt->k_off.data(), (size_t)(ci.N + 1) * 4));
    if (ci.nnz) {
      es.push_back(up(d_kc, Lt->k_col.data(), (size_t)ci.nnz * 4));
      es.push_back(up(d_kv, Lt->k_val.data(), (size_t)ci.nnz * 8));
      es.push_back(up(d_kvf, kvf.data(), (size_t)ci.nnz * 4));
    }
    es.push_back(up(d_fo, fo.data(), fo.size() * 4));
    if (ci.nb) {
      es.push_back(up(d_bi, vi.data(), ci.nb * 4)); es.push_back(up(d_bj, vj.data(), ci.nb * 4));
      es.push_back(up(d_bc, vc.data(), ci.nb * 8)); es.push_back(up(d_bs, vs.data(), ci.nb * 8));
      es.push_back(up(d_bk, vk.data(), ci.nb * 8));
      es.push_back(up(d_bcf, vcf.data(), ci.nb * 4)); es.push_back(up(d_bsf, vsf.data(), ci.nb * 4));
    }
    es.push_back(up(d_ce, ce.data(), ci.N * 8)); es.push_back(up(d_ep, ep.data(), ci.N * 8));
    es.push_back(up(d_cef, cef.data(), ci.N * 4)); es.push_back(up(d_sub, Lt->sub.data(), ci.N * 4));
    es.push_back(up(d_nbo, Lt->nb_off.data(), (size_t)(ci.N + 1) * 4));
    if (!Lt->nb_site.empty()) es.push_back(up(d_nbs, Lt->nb_site.data(), Lt->nb_site.size() * 4));
    // the staging vectors must outlive the async copies
    for (cudaError_t ee : es)
      if (ee != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(ee, "lattice upload"); }
    e = cudaStreamSynchronize(S->st);
    if (e != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(e, "lattice upload"); }
    D.lat.N = ci.N; D.lat.nb = ci.nb; D.lat.G = ci.G;
    D.lat.fam_off = d_fo; D.lat.bond_i = d_bi; D.lat.bond_j = d_bj;
    D.lat.bond_c = d_bc; D.lat.bond_s = d_bs; D.lat.bond_cf = d_bcf; D.lat.bond_sf = d_bsf; D.lat.bond_k = d_bk;
    D.lat.unif = unif; D.lat.cprod = cprod;
    D.lat.ceps = Lt->has_eps ? d_ce : nullptr;
    D.lat.cepsf = Lt->has_eps ? d_cef : nullptr;
    D.lat.eps = Lt->has_eps ? d_ep : nullptr;
    D.lat.sub = d_sub;
    D.lat.nb_off = d_nbo;
    D.lat.nb_site = d_nbs;
    D.lat.exact = ci.exact;
    D.lat.taylor_q = ci.taylor_q;
    D.lat.mdtau = -p.dtau;
    D.lat.k_off = d_ko;
    D.lat.k_col = d_kc;
    D.lat.k_val = d_kv;
    D.lat.k_valf = d_kvf;
    D.N = ci.N; D.L = ci.L; D.tw = ci.tw; D.n = ci.n; D.ns[0] = ci.ns[0]; D.ns[1] = ci.ns[1];
    D.charge = p.U < 0;
    D.prec = prec;
    D.swap_mode = p.swap_mode;
    D.left_swaps = p.left_swaps;
    D.lambda = std::acosh(std::exp(p.dtau * std::fabs(p.U) / 2.0));
    D.dfac_p = std::exp(D.lambda); D.dfac_m = std::exp(-D.lambda);
    D.delta_p = std::expm1(-2.0 * D.lambda); D.delta_m = std::expm1(2.0 * D.lambda);
    D.cfac_p = std::exp(2.0 * D.lambda); D.cfac_m = std::exp(-2.0 * D.lambda);
    D.opd_p = 1.0 + D.delta_p; D.opd_m = 1.0 + D.delta_m;
    lq_dw_split(D.delta_p, D.dw_delta_p); lq_dw_split(D.delta_m, D.dw_delta_m);
    lq_dw_split(D.cfac_p, D.dw_cfac_p); lq_dw_split(D.cfac_m, D.dw_cfac_m);
    D.key0 = (uint32_t)p.seed; D.key1 = (uint32_t)(p.seed >> 32);
    D.chain_id = chain_ids ? chain_ids[c] : (uint32_t)c;
    D.sweep = 0;
    D.s = (int8_t*)take((size_t)ci.L * ci.N);
    for (int sg = 0; sg < 2; ++sg) {
      const size_t pn = (size_t)ci.N * ci.ns[sg], qn = (size_t)ci.ns[sg] * ci.ns[sg];
      D.occ[sg] = (int*)take(std::max(ci.ns[sg], 1) * 4);
      D.QR[sg][0] = take((ci.n + 1) * pn * PS);
      D.QR[sg][1] = take((ci.n + 1) * pn * PS);
      D.VR[sg][0] = (double*)take((ci.n + 1) * qn * 8);
      D.VR[sg][1] = (double*)take((ci.n + 1) * qn * 8);
      D.QL[sg] = take((ci.n + 1) * pn * PS);
      D.VL[sg] = (double*)take((ci.n + 1) * qn * 8);
      D.stored[sg] = take(ci.tw * pn * PS);
      D.live[sg] = take(pn * PS);
      D.work[sg] = take(pn * 8);
      D.cur[sg] = 0;
    }
    D.vec = (double*)take((size_t)2 * ci.N * 8);
    D.rot = (double*)take((size_t)ci.n * LQ_NS_MAX * 2 * 8);
    D.records = (double*)take((size_t)max_records * LQ_NOBS * 8);
    D.max_records = max_records;
    D.sign = 1;
    // default state: all fields +1, the first N_sigma sites occupied
    std::vector<int8_t> s(ci.L * (size_t)ci.N, 1);
    e = cudaMemcpy(D.s, s.data(), s.size(), cudaMemcpyHostToDevice);
    for (int sg = 0; sg < 2 && e == cudaSuccess; ++sg) {
      std::vector<int> occ(std::max(ci.ns[sg], 1));
      for (int a = 0; a < ci.ns[sg]; ++a) occ[a] = a;
      e = cudaMemcpy(D.occ[sg], occ.data(), occ.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(e, "state upload"); }
  }
  // order: decreasing cost (longest chains first)
  std::vector<int> ord(n_chains), all(n_chains);
  for (int c = 0; c < n_chains; ++c) ord[c] = all[c] = c;
  auto big_of = [&](int c) { return std::max(info[c].ns[0], info[c].ns[1]) > LQ_NS_SMALL; };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (big_of(a) != big_of(b)) return !big_of(a);
    return info[a].cost > info[b].cost;
  });
  {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 2; ++k) {
      lq_sim::PlanClass& pc = S->cls[k];
      pc.off = k ? S->cls[0].n : 0;
      for (int c = 0; c < n_chains; ++c) {
        if (big_of(c) != (k == 1)) continue;
        pc.n++;
        pc.M = std::max(pc.M, std::max(info[c].ns[0], info[c].ns[1]));
        pc.Nmax = std::max(pc.Nmax, info[c].N);
        if (info[c].exact) pc.pcols = 2;
      }
      if (!pc.n) continue;
      pc.buf = lq::staging_bytes(pc.M, pc.Nmax, pc.pcols);
      const int per_sm = lq::max_active_sweep_ctas(prec, pc.M, lq::smem_bytes(pc.M, pc.Nmax, pc.buf));
      if (per_sm < 1) { lq_sim_destroy(S); return fail(LQ_EUNSUPPORTED, "shared-memory plan does not fit one CTA per SM"); }
      pc.grid = std::min(pc.n, sms * per_sm);
    }
  }
  if (S->cls[0].n && S->cls[1].n) {
    cudaError_t es = cudaStreamCreateWithFlags(&S->st2, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&S->ev_join, cudaEventDisableTiming);
    if (es != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(es, "second stream"); }
  }
  e = cudaMemcpy(S->d_chains, S->h.data(), sizeof(LqChainDev) * n_chains, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(S->d_order, ord.data(), sizeof(int) * n_chains, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(S->d_all, all.data(), sizeof(int) * n_chains, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(e, "descriptor upload"); }
  if (build) {
    // build the chains for the default state
    S->mirror_fresh = false;
    e = lq::launch_build(prec, S->d_chains, S->d_all, n_chains, S->M, S->Nmax, S->buf_bytes, S->grid, S->st, S->ws, S->ws_bytes);
    if (e != cudaSuccess) { lq_sim_destroy(S); return cuda_fail(e, "initial chain build"); }
  } else {
    S->mirror_fresh = true;  // the host descriptors were just uploaded
  }
  *out = S;
  return LQ_OK;
}

static lq_status rebuild(lq_sim* S, const int* d_list, int n) {
  S->mirror_fresh = false;
  cudaError_t e = lq::launch_build(S->prec, S->d_chains, d_list, n, S->M, S->Nmax, S->buf_bytes,
                                   std::min(n, S->grid), S->st, S->ws, S->ws_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "chain build");
  return LQ_OK;
}

static lq_status rebuild_one(lq_sim* S, int c) {
  CK(cudaMemcpyAsync(S->d_single, &c, sizeof(int), cudaMemcpyHostToDevice, S->st));
  CK(cudaStreamSynchronize(S->st));
  return rebuild(S, S->d_single, 1);
}

extern "C" lq_status lq_sim_init(lq_sim* S) {
  if (!S) return fail(LQ_EINVAL, "null simulation");
  S->mirror_fresh = false;
  cudaError_t e = lq::launch_init(S->d_chains, S->d_all, S->n_chains, std::min(S->n_chains, 1024), S->st);
  if (e != cudaSuccess) return cuda_fail(e, "init");
  return rebuild(S, S->d_all, S->n_chains);
}

extern "C" lq_status lq_sim_set_fields(lq_sim* S, int32_t c, const int8_t* hs) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if (!hs) return fail(LQ_EINVAL, "null field array");
  if ((st = pull(S)) != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  for (size_t k = 0; k < (size_t)ci.L * ci.N; ++k)
    if (hs[k] != 1 && hs[k] != -1) return fail(LQ_EINVAL, "fields must be +-1");
  CK(cudaMemcpy(S->h[c].s, hs, (size_t)ci.L * ci.N, cudaMemcpyHostToDevice));
  return rebuild_one(S, c);
}

extern "C" lq_status lq_sim_get_fields(lq_sim* S, int32_t c, int8_t* hs) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  CK(cudaMemcpy(hs, S->h[c].s, (size_t)S->info[c].L * S->info[c].N, cudaMemcpyDeviceToHost));
  return LQ_OK;
}

extern "C" lq_status lq_sim_set_fock(lq_sim* S, int32_t c, const int32_t* up, const int32_t* dn) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  const int32_t* in[2] = {up, dn};
  for (int sg = 0; sg < 2; ++sg) {
    if (ci.ns[sg] && !in[sg]) return fail(LQ_EINVAL, "null occupation array");
    std::vector<char> seen(ci.N, 0);
    for (int a = 0; a < ci.ns[sg]; ++a) {
      const int i = in[sg][a];
      if (i < 0 || i >= ci.N || seen[i]) return fail(LQ_EINVAL, "occupations must be distinct sites in [0, N)");
      seen[i] = 1;
    }
  }
  for (int sg = 0; sg < 2; ++sg)
    if (ci.ns[sg]) CK(cudaMemcpy(S->h[c].occ[sg], in[sg], ci.ns[sg] * 4, cudaMemcpyHostToDevice));
  return rebuild_one(S, c);
}

extern "C" lq_status lq_sim_get_fock(lq_sim* S, int32_t c, int32_t* up, int32_t* dn) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  int32_t* outp[2] = {up, dn};
  for (int sg = 0; sg < 2; ++sg)
    if (ci.ns[sg] && outp[sg]) CK(cudaMemcpy(outp[sg], S->h[c].occ[sg], ci.ns[sg] * 4, cudaMemcpyDeviceToHost));
  return LQ_OK;
}

extern "C" lq_status lq_sim_set_sweep_index(lq_sim* S, uint32_t sweep) {
  if (!S) return fail(LQ_EINVAL, "null simulation");
  lq_status st = pull(S);
  if (st != LQ_OK) return st;
  for (auto& D : S->h) D.sweep = sweep;
  CK(cudaMemcpy(S->d_chains, S->h.data(), sizeof(LqChainDev) * S->n_chains, cudaMemcpyHostToDevice));
  return LQ_OK;
}

extern "C" lq_status lq_sim_sweep(lq_sim* S, int32_t n_sweeps, int32_t measure) {
  if (!S || n_sweeps < 0) return fail(LQ_EINVAL, "bad arguments to lq_sim_sweep");
  if (n_sweeps == 0) return LQ_OK;
  S->mirror_fresh = false;
  cudaError_t e = cudaSuccess;
  const lq_sim::PlanClass& small = S->cls[0];
  const lq_sim::PlanClass& large = S->cls[1];
  if (small.n && large.n && S->st2) {
    // the large class first, on the second stream, so that its long chains
    // start at once; the small class fills the other SMs meanwhile
    e = cudaEventRecord(S->ev_fork, S->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->st2, S->ev_fork, 0);
    const bool forked = e == cudaSuccess;
    if (e == cudaSuccess)
      e = lq::launch_sweep(S->prec, S->d_chains, S->d_order + large.off, large.n, S->d_queue2, n_sweeps, measure,
                           large.M, large.Nmax, large.buf, large.grid, S->st2, S->ws, S->ws_bytes, nullptr, 0,
                           large.threads);
    if (e == cudaSuccess)
      e = lq::launch_sweep(S->prec, S->d_chains, S->d_order + small.off, small.n, S->d_queue, n_sweeps, measure,
                           small.M, small.Nmax, small.buf, small.grid, S->st, nullptr, 0, nullptr, 0, small.threads);
    if (forked) {
      // join even after a failed launch, so that nothing later on the
      // caller's stream overtakes the second stream's work
      cudaError_t ej = cudaEventRecord(S->ev_join, S->st2);
      if (ej == cudaSuccess) ej = cudaStreamWaitEvent(S->st, S->ev_join, 0);
      if (ej != cudaSuccess) cudaStreamSynchronize(S->st2);
      if (e == cudaSuccess) e = ej;
    }
  } else {
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      const lq_sim::PlanClass& pc = S->cls[k];
      if (pc.n)
        e = lq::launch_sweep(S->prec, S->d_chains, S->d_order + pc.off, pc.n, S->d_queue, n_sweeps, measure, pc.M,
                             pc.Nmax, pc.buf, pc.grid, S->st, S->ws, S->ws_bytes, nullptr, 0,
                             pc.threads);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
  return LQ_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the batched launch: per plan class, the shared-memory staging
// buffer (it sets the propagation's column chunks, the flip loop's chunk of
// sites, and through the shared memory per CTA the CTAs per SM).  Candidates
// are timed on real sweeps of that class (without measurement), and the
// choice is cached per (precision, class, N_sigma, N, chain-count bucket).
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune_cache;  // -> (staging bytes, threads)
int chain_bucket(int n) {
  int b = 0;
  while ((1 << b) < n) ++b;
  return b;
}
}  // namespace

extern "C" lq_status lq_sim_autotune(lq_sim* S, int32_t sweeps_per_candidate, int32_t* host_buf2) {
  if (!S || sweeps_per_candidate < 0) return fail(LQ_EINVAL, "bad arguments to lq_sim_autotune");
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  S->mirror_fresh = false;
  for (int k = 0; k < 2; ++k) {
    lq_sim::PlanClass& pc = S->cls[k];
    if (host_buf2) host_buf2[k] = pc.n ? pc.buf : 0;
    if (!pc.n) continue;
    const auto key = std::make_tuple(S->prec, k, pc.M, pc.Nmax, chain_bucket(pc.n));
    const int need = lq::staging_min_bytes(pc.M, pc.Nmax, pc.pcols);
    // a feasible (grid, fits) for a candidate (staging buffer, threads per CTA)
    auto feasible = [&](int buf, int threads, int* grid) {
      if (buf < need) return false;
      const size_t smem = lq::smem_bytes(pc.M, pc.Nmax, buf);
      if (smem > 227 * 1024) return false;
      const int per_sm = lq::max_active_sweep_ctas(S->prec, pc.M, smem, threads);
      if (per_sm < 1) return false;
      *grid = std::min(pc.n, sms * per_sm);
      return (size_t)(*grid) * lq::workspace_bytes(pc.M, pc.Nmax, buf) <= S->ws_bytes;
    };
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      auto it = g_tune_cache.find(key);
      int grid = 0;
      if (it != g_tune_cache.end() && feasible(it->second.first, it->second.second, &grid)) {
        pc.buf = it->second.first;
        pc.threads = it->second.second;
        pc.grid = grid;
        if (host_buf2) host_buf2[k] = pc.buf;
        continue;
      }
    }
    if (sweeps_per_candidate == 0) continue;
    std::vector<int> cand = {pc.buf, 24 * 1024, 32 * 1024, 40 * 1024, 48 * 1024, 64 * 1024, 96 * 1024, 128 * 1024,
                             160 * 1024, 200 * 1024};
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    // half-size CTAs (more chains per SM) for plans of at most LQ_NS_SMALL particles per spin
    std::vector<int> tcand = {LQ_THREADS};
    if (!(pc.M > LQ_NS_SMALL)) tcand.push_back(LQ_THREADS / 2);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 0.f;
    int best_buf = pc.buf, best_grid = pc.grid, best_threads = pc.threads;
    bool have = false;
    for (int threads : tcand) {
      int last_grid = -1;
      for (int buf : cand) {
        int grid = 0;
        if (!feasible(buf, threads, &grid)) continue;
        // with half-size CTAs only the staging sizes that change the CTAs per SM are worth a sweep
        if (threads != LQ_THREADS && grid == last_grid) continue;
        last_grid = grid;
        cudaError_t e = cudaEventRecord(e0, S->st);
        if (e == cudaSuccess)
          e = lq::launch_sweep(S->prec, S->d_chains, S->d_order + pc.off, pc.n, S->d_queue, sweeps_per_candidate, 0,
                               pc.M, pc.Nmax, buf, grid, S->st, S->ws, S->ws_bytes, nullptr, 0, threads);
        if (e == cudaSuccess) e = cudaEventRecord(e1, S->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return cuda_fail(e, "autotune sweep");
        }
        if (!have || ms < best_ms) {
          best_ms = ms;
          best_buf = buf;
          best_grid = grid;
          best_threads = threads;
          have = true;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pc.buf = best_buf;
    pc.grid = best_grid;
    pc.threads = best_threads;
    if (host_buf2) host_buf2[k] = pc.buf;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = std::make_pair(pc.buf, pc.threads);
  }
  return LQ_OK;
}

extern "C" lq_status lq_sim_run_host(lq_sim* S, const int8_t* hf, const int32_t* ho, int32_t n_sweeps,
                                     int32_t measure, int8_t* hf_out, int32_t* ho_out, double* hrec) {
  if (!S || !hf || !ho || n_sweeps < 0) return fail(LQ_EINVAL, "bad arguments to lq_sim_run_host");
  lq_status st = pull(S);
  if (st != LQ_OK) return st;
  size_t fo = 0, oo = 0;
  for (int c = 0; c < S->n_chains; ++c) {
    const ChainHost& ci = S->info[c];
    const LqChainDev& D = S->h[c];
    const size_t nf = (size_t)ci.L * ci.N;
    CK(cudaMemcpyAsync(D.s, hf + fo, nf, cudaMemcpyHostToDevice, S->st));
    for (int sg = 0; sg < 2; ++sg) {
      if (ci.ns[sg]) CK(cudaMemcpyAsync(D.occ[sg], ho + oo, ci.ns[sg] * 4, cudaMemcpyHostToDevice, S->st));
      oo += ci.ns[sg];
    }
    fo += nf;
  }
  cudaError_t e = lq::launch_clear_records(S->d_chains, S->n_chains, S->st);
  if (e != cudaSuccess) return cuda_fail(e, "clear records");
  if ((st = rebuild(S, S->d_all, S->n_chains)) != LQ_OK) return st;
  if ((st = lq_sim_sweep(S, n_sweeps, measure)) != LQ_OK) return st;
  S->mirror_fresh = false;
  if ((st = pull(S)) != LQ_OK) return st;
  for (int c = 0; c < S->n_chains; ++c)
    if (S->h[c].err & LQ_ERR_BADINPUT) return fail(LQ_EINVAL, "chain " + std::to_string(c) + ": fields must be +-1 and occupied sites distinct in [0, N)");
  fo = 0;
  oo = 0;
  for (int c = 0; c < S->n_chains; ++c) {
    const ChainHost& ci = S->info[c];
    const LqChainDev& D = S->h[c];
    const size_t nf = (size_t)ci.L * ci.N;
    if (hf_out) CK(cudaMemcpyAsync(hf_out + fo, D.s, nf, cudaMemcpyDeviceToHost, S->st));
    for (int sg = 0; sg < 2; ++sg) {
      if (ho_out && ci.ns[sg]) CK(cudaMemcpyAsync(ho_out + oo, D.occ[sg], ci.ns[sg] * 4, cudaMemcpyDeviceToHost, S->st));
      oo += ci.ns[sg];
    }
    if (hrec && measure)
      CK(cudaMemcpyAsync(hrec + (size_t)c * n_sweeps * LQ_NOBS, D.records, sizeof(double) * n_sweeps * LQ_NOBS,
                         cudaMemcpyDeviceToHost, S->st));
    fo += nf;
  }
  CK(cudaStreamSynchronize(S->st));
  return LQ_OK;
}

extern "C" lq_status lq_sim_set_launch_config(lq_sim* S, int32_t plan_class, int32_t staging_bytes,
                                             int32_t threads) {
  if (!S || plan_class < 0 || plan_class > 1) return fail(LQ_EINVAL, "bad arguments to lq_sim_set_launch_config");
  lq_sim::PlanClass& pc = S->cls[plan_class];
  if (!pc.n) return fail(LQ_EINVAL, "the plan class has no chains");
  if (threads != LQ_THREADS && !(threads == LQ_THREADS / 2 && pc.M <= LQ_NS_SMALL))
    return fail(LQ_EINVAL, "threads must be 256 (or 128 for the class of at most 32 particles per spin)");
  if (staging_bytes < lq::staging_min_bytes(pc.M, pc.Nmax, pc.pcols))
    return fail(LQ_EINVAL, "staging buffer below the plan's minimum");
  const size_t smem = lq::smem_bytes(pc.M, pc.Nmax, staging_bytes);
  const int per_sm = smem > 227 * 1024 ? 0 : lq::max_active_sweep_ctas(S->prec, pc.M, smem, threads);
  if (per_sm < 1) return fail(LQ_EUNSUPPORTED, "the launch does not fit one CTA per SM");
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(pc.n, sms * per_sm);
  if ((size_t)grid * lq::workspace_bytes(pc.M, pc.Nmax, staging_bytes) > S->ws_bytes)
    return fail(LQ_EUNSUPPORTED, "the launch needs more workspace than the simulation holds");
  pc.buf = staging_bytes;
  pc.threads = threads;
  pc.grid = grid;
  return LQ_OK;
}

extern "C" lq_status lq_sim_launch_config(const lq_sim* S, int32_t* host_cfg8) {
  if (!S || !host_cfg8) return fail(LQ_EINVAL, "bad arguments to lq_sim_launch_config");
  for (int k = 0; k < 2; ++k) {
    const lq_sim::PlanClass& pc = S->cls[k];
    host_cfg8[4 * k + 0] = pc.n;
    host_cfg8[4 * k + 1] = pc.n ? pc.buf : 0;
    host_cfg8[4 * k + 2] = pc.n ? pc.threads : 0;
    host_cfg8[4 * k + 3] = pc.n ? pc.grid : 0;
  }
  return LQ_OK;
}

extern "C" lq_status lq_sim_sync(lq_sim* S) {
  if (!S) return fail(LQ_EINVAL, "null simulation");
  S->mirror_fresh = false;
  lq_status st = pull(S);
  if (st != LQ_OK) return st;
  for (int c = 0; c < S->n_chains; ++c)
    if (S->h[c].err & LQ_ERR_BADINPUT)
      return fail(LQ_EINVAL, "chain " + std::to_string(c) + " was given invalid fields or occupations");
  for (int c = 0; c < S->n_chains; ++c)
    if (S->h[c].err)
      return fail(LQ_ENUMERIC, "chain " + std::to_string(c) + " reported numerical error flags " +
                                   std::to_string(S->h[c].err));
  return LQ_OK;
}

extern "C" lq_status lq_sim_log_weight(lq_sim* S, int32_t c, double* la, int32_t* sg) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = rebuild_one(S, c)) != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  if (la) *la = S->h[c].hook[6];
  if (sg) *sg = (int32_t)S->h[c].hook[7];
  return LQ_OK;
}

extern "C" lq_status lq_sim_tracked_weight(lq_sim* S, int32_t c, double* la, int32_t* sg) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  if (la) *la = S->h[c].logw;
  if (sg) *sg = S->h[c].sign;
  return LQ_OK;
}

// Numeric health check: rebuild every chain's QR chains from its fields and
// Fock state (the state is fully reconstructible from them), compare the fresh
// log|W| and sign with the tracked ones, and keep the rebuilt chains.
extern "C" lq_status lq_sim_check_drift(lq_sim* S, double tol, double* host_max_rel, int32_t* host_n_bad) {
  if (!S || !(tol >= 0.0)) return fail(LQ_EINVAL, "bad arguments to lq_sim_check_drift");
  lq_status st = pull(S);
  if (st != LQ_OK) return st;
  std::vector<double> lw(S->n_chains);
  std::vector<int> sg(S->n_chains);
  for (int c = 0; c < S->n_chains; ++c) { lw[c] = S->h[c].logw; sg[c] = S->h[c].sign; }
  if ((st = rebuild(S, S->d_all, S->n_chains)) != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  double worst = 0.0;
  int bad = 0;
  for (int c = 0; c < S->n_chains; ++c) {
    const double fresh = S->h[c].logw;
    const double rel = std::fabs(fresh - lw[c]) / std::max(1.0, std::fabs(fresh));
    const bool off = !(rel <= tol) || S->h[c].sign != sg[c];
    worst = std::max(worst, std::isfinite(rel) ? rel : INFINITY);
    bad += off;
  }
  if (host_max_rel) *host_max_rel = worst;
  if (host_n_bad) *host_n_bad = bad;
  if (bad)
    return fail(LQ_ENUMERIC, std::to_string(bad) + " chain(s) drifted beyond the tolerance (largest relative drift " +
                                 std::to_string(worst) + "); their chains were rebuilt from fields and Fock states");
  return lq_sim_sync(S);
}

extern "C" lq_status lq_sim_field_ratio(lq_sim* S, int32_t c, int32_t l, int32_t i, double* r) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if (l < 0 || l >= S->info[c].L || i < 0 || i >= S->info[c].N) return fail(LQ_EINVAL, "slice or site out of range");
  if ((st = rebuild_one(S, c)) != LQ_OK) return st;
  S->mirror_fresh = false;
  cudaError_t e = lq::launch_field_ratio(S->prec, S->d_chains, c, l, i, S->M, S->Nmax, S->buf_bytes, S->st, S->ws, S->ws_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "field ratio");
  if ((st = pull(S)) != LQ_OK) return st;
  if (r) *r = S->h[c].hook[0];
  return LQ_OK;
}

extern "C" lq_status lq_sim_swap_ratio(lq_sim* S, int32_t c, int32_t sg, int32_t k, int32_t j, double* r,
                                       double* parts) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  if (sg < 0 || sg > 1 || k < 0 || k >= ci.ns[sg] || j < 0 || j >= ci.N) return fail(LQ_EINVAL, "bad swap indices");
  if ((st = pull(S)) != LQ_OK) return st;
  std::vector<int> occ(ci.ns[sg]);
  CK(cudaMemcpy(occ.data(), S->h[c].occ[sg], ci.ns[sg] * 4, cudaMemcpyDeviceToHost));
  for (int a = 0; a < ci.ns[sg]; ++a)
    if (occ[a] == j) return fail(LQ_EINVAL, "target site is occupied");
  if ((st = rebuild_one(S, c)) != LQ_OK) return st;
  S->mirror_fresh = false;
  cudaError_t e = lq::launch_swap_ratio(S->prec, S->d_chains, c, sg, k, j, S->M, S->Nmax, S->buf_bytes, S->st, S->ws, S->ws_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "swap ratio");
  if ((st = pull(S)) != LQ_OK) return st;
  const double* h = S->h[c].hook;
  if (r) *r = h[1] * std::exp(h[0]);
  if (parts) for (int q = 0; q < 6; ++q) parts[q] = h[q];
  return LQ_OK;
}

extern "C" lq_status lq_sim_records(lq_sim* S, int32_t c, int32_t max_rows, int32_t* n, double* out) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  const int k = std::min(S->h[c].nrec, std::max(max_rows, 0));
  if (n) *n = S->h[c].nrec;
  if (k > 0 && out) CK(cudaMemcpy(out, S->h[c].records, sizeof(double) * k * LQ_NOBS, cudaMemcpyDeviceToHost));
  return LQ_OK;
}

extern "C" lq_status lq_sim_clear_records(lq_sim* S) {
  if (!S) return fail(LQ_EINVAL, "null simulation");
  lq_status st = pull(S);
  if (st != LQ_OK) return st;
  for (auto& D : S->h) D.nrec = 0;
  CK(cudaMemcpy(S->d_chains, S->h.data(), sizeof(LqChainDev) * S->n_chains, cudaMemcpyHostToDevice));
  return LQ_OK;
}

extern "C" lq_status lq_sim_stats(lq_sim* S, int32_t c, int64_t* out) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if ((st = pull(S)) != LQ_OK) return st;
  for (int k = 0; k < 4; ++k) out[k] = S->h[c].cnt[k];
  return LQ_OK;
}

extern "C" lq_status lq_sim_profile(lq_sim* S, int32_t c, int64_t* out) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if (!out) return fail(LQ_EINVAL, "null output");
  if ((st = pull(S)) != LQ_OK) return st;
  for (int k = 0; k < 12; ++k) out[k] = S->h[c].prof[k];
  return LQ_OK;
}

extern "C" lq_status lq_sim_chain_panel(lq_sim* S, int32_t c, int32_t side, int32_t sg, int32_t j, double* Q,
                                        double* V) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  if (sg < 0 || sg > 1 || j < 0 || j > ci.n || side < 0 || side > 1) return fail(LQ_EINVAL, "bad panel index");
  if ((st = pull(S)) != LQ_OK) return st;
  const LqChainDev& D = S->h[c];
  const size_t pn = (size_t)ci.N * ci.ns[sg], qn = (size_t)ci.ns[sg] * ci.ns[sg];
  const size_t PS = S->prec == LQ_FP64 ? 8 : 4;
  const char* qsrc = (const char*)(side ? D.QL[sg] : D.QR[sg][D.cur[sg]]) + j * pn * PS;
  if (Q && pn) {
    if (PS == 8) CK(cudaMemcpy(Q, qsrc, pn * 8, cudaMemcpyDeviceToHost));
    else {
      std::vector<float> tmp(pn);
      CK(cudaMemcpy(tmp.data(), qsrc, pn * 4, cudaMemcpyDeviceToHost));
      for (size_t k = 0; k < pn; ++k) Q[k] = tmp[k];
    }
  }
  if (V && qn) {
    const double* vsrc = (side ? D.VL[sg] : D.VR[sg][D.cur[sg]]) + j * qn;
    CK(cudaMemcpy(V, vsrc, qn * 8, cudaMemcpyDeviceToHost));
  }
  return LQ_OK;
}

extern "C" lq_status lq_sim_chain_info(const lq_sim* S, int32_t c, int32_t* info6) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  const ChainHost& ci = S->info[c];
  info6[0] = ci.N; info6[1] = ci.L; info6[2] = ci.tw; info6[3] = ci.n; info6[4] = ci.ns[0]; info6[5] = ci.ns[1];
  return LQ_OK;
}

extern "C" lq_status lq_sim_device_bytes(const lq_sim* S, size_t* bytes) {
  if (!S || !bytes) return fail(LQ_EINVAL, "null argument");
  *bytes = S->arena_bytes;
  return LQ_OK;
}

extern "C" lq_status lq_sim_destroy(lq_sim* S) {
  if (!S) return LQ_OK;
  if (S->st2) {
    cudaStreamSynchronize(S->st2);
    cudaStreamDestroy(S->st2);
  }
  if (S->ev_fork) cudaEventDestroy(S->ev_fork);
  if (S->ev_join) cudaEventDestroy(S->ev_join);
  if (S->arena) {
    cudaStreamSynchronize(S->st);
    if (S->has_alloc) S->alloc.free(S->alloc.ctx, S->arena, S->arena_bytes, S->st);
    else cudaFree(S->arena);
  }
  delete S;
  return LQ_OK;
}

extern "C" const char* lq_last_error(void) { return g_err.c_str(); }
extern "C" const char* lq_version(void) { return "lecqmc-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// internal hooks (serving loop) and observable statistics
// ---------------------------------------------------------------------------
lq_sim_launch_info lq_internal_sim_info(const lq_sim* S) {
  lq_sim_launch_info i;
  i.d_chains = S->d_chains; i.n_chains = S->n_chains; i.prec = S->prec; i.M = S->M; i.Nmax = S->Nmax;
  i.buf_bytes = S->buf_bytes; i.arena_bytes = S->arena_bytes;
  i.cost = S->n_chains > 0 ? S->info[0].cost : 0.0;
  return i;
}

void lq_internal_sim_invalidate(lq_sim* S) { S->mirror_fresh = false; }

const LqChainDev* lq_internal_sim_host_desc(const lq_sim* S) { return S->h.data(); }

size_t lq_internal_footprint(const lq_lattice* L, const lq_params* p) {
  const long Ll = std::lround(p->beta / p->dtau);
  const int ns[2] = {p->n_up, p->n_dn};
  return footprint_one(L->N, (int)L->bi.size(), L->G, (int)Ll, std::max(p->n_stab, 1), ns, p->precision, 1 << 16,
                       p->kinetic == LQ_EXACT);
}

extern "C" lq_status lq_request_footprint(const lq_lattice* L, const lq_params* p, size_t* bytes) {
  if (!L || !p || !bytes) return fail(LQ_EINVAL, "bad arguments to lq_request_footprint");
  if (!(p->beta > 0) || !(p->dtau > 0) || p->n_stab < 1 || p->n_up < 0 || p->n_dn < 0 || p->n_up > L->N ||
      p->n_dn > L->N)
    return fail(LQ_EINVAL, "parameters out of range");
  *bytes = lq_internal_footprint(L, p);
  return LQ_OK;
}

void lq_internal_obs_stats(const double* rec, int n, int nbins, double* mean, double* err) {
  for (int k = 0; k < LQ_NOBS; ++k) { mean[k] = NAN; err[k] = NAN; }
  if (n <= 0) return;
  double tot[LQ_NOBS] = {0};
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < LQ_NOBS; ++k) tot[k] += rec[(size_t)r * LQ_NOBS + k];
  mean[0] = tot[0] / n;
  for (int k = 1; k < LQ_NOBS; ++k) mean[k] = tot[k] / tot[0];
  err[0] = 0.0;
  nbins = std::min(nbins, n);
  if (nbins < 2) return;
  const int per = n / nbins;
  std::vector<double> bsum((size_t)nbins * LQ_NOBS, 0.0);
  for (int b = 0; b < nbins; ++b)
    for (int r = b * per; r < (b + 1) * per; ++r)
      for (int k = 0; k < LQ_NOBS; ++k) bsum[(size_t)b * LQ_NOBS + k] += rec[(size_t)r * LQ_NOBS + k];
  double used[LQ_NOBS] = {0};
  for (int b = 0; b < nbins; ++b)
    for (int k = 0; k < LQ_NOBS; ++k) used[k] += bsum[(size_t)b * LQ_NOBS + k];
  for (int k = 0; k < LQ_NOBS; ++k) {
    double jm = 0.0, j2 = 0.0;
    for (int b = 0; b < nbins; ++b) {
      const double num = used[k] - bsum[(size_t)b * LQ_NOBS + k];
      const double den = (k == 0) ? (double)(nbins - 1) * per : used[0] - bsum[(size_t)b * LQ_NOBS];
      const double v = num / den;
      jm += v;
      j2 += v * v;
    }
    jm /= nbins;
    const double var = (double)(nbins - 1) / nbins * std::max(0.0, j2 - nbins * jm * jm);
    err[k] = std::sqrt(var);
  }
}

extern "C" lq_status lq_sim_measure(lq_sim* S, int32_t c, int32_t n_bins, double* mean, double* err) {
  lq_status st = check_chain(S, c);
  if (st != LQ_OK) return st;
  if (!mean || !err || n_bins < 2) return fail(LQ_EINVAL, "need mean/err outputs and n_bins >= 2");
  if ((st = pull(S)) != LQ_OK) return st;
  const int n = S->h[c].nrec;
  std::vector<double> rec((size_t)std::max(n, 1) * LQ_NOBS);
  if (n > 0) CK(cudaMemcpy(rec.data(), S->h[c].records, sizeof(double) * n * LQ_NOBS, cudaMemcpyDeviceToHost));
  lq_internal_obs_stats(rec.data(), n, n_bins, mean, err);
  return LQ_OK;
}
