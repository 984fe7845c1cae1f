// lq_cp.cu -- constrained-path inner loop of LEC-QMC on the GPU (SM Sec. VI).
//
// For a fixed Fock state eta (the columns of P) a population of walkers
// samples the Hubbard-Stratonovich fields slice by slice against the trial
// Psi_l^T = P^T e^{-(beta - tau_l) H_0}: everything that still acts on the
// walker after the fields of slice l, with the fields off.  A walker is an
// N x N_sigma panel Phi per spin, starting at P.  At site i of slice l the
// overlap ratio of the field value s is, by the matrix-determinant lemma,
//   r(s) = prod_sigma [1 + Delta_sigma(s) g_sigma],   g_sigma = Phi_i T Psi_i^T,
// T = (Psi_l^T Phi)^{-1} (times e^{-lambda s} in the charge channel); s is
// drawn with probability proportional to (1/2) max(0, r(s)), the weight
// takes the factor (1/2) sum_s max(0, r(s)) (a walker at factor 0 has crossed
// the trial's node and is dropped), row i of Phi takes e^{sigma' lambda s}
// and T its Sherman-Morrison update.  After the slice's sites Phi <- B_K Phi
// and Phi is re-orthonormalized (CholeskyQR2; a right factor of Phi cancels
// in every ratio), and T is rebuilt from the next trial panel.
//
// Without truncation the mean weight is R(eta) = sum_s 2^{-LN}
// <eta|U(s)|eta> / <eta|e^{-beta H_0}|eta>.  A branching population combs
// (systematic resampling) every few slices; its estimate is the product of
// the population's mean weights.  The random numbers are Philox4x32-10 with
// the counters of the oracle: (walker, sweep word, 7<<24 | slice, site) for
// independent walkers, (slot, run, 8<<24 | slice, site) for the fields of a
// population and (run, 0xFFFFFFFD, 9<<24 | slice, 0) for its comb.
//
// One CTA per walker: warp sigma computes spin sigma's row products (a lane
// per column), thread 0 takes the two-valued heat-bath decision.
#include "lq_sweep.cuh"

#include <cmath>
#include <string>
#include <vector>

#include "lq_internal.h"
#include "lq_lattice.h"

namespace lq {

// Trial panels Psi_l = (B_K^T)^{L-l} P, l = L-1 .. 0, orthonormalized
// (CholeskyQR2): CTA sigma builds spin sigma's L panels (N x m each).
__global__ void __launch_bounds__(LQ_THREADS, 1)
    cp_trial_kernel(const LqChainDev* base, double* psi0, double* psi1, double* vscr, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  load_chain(const_cast<LqChainDev*>(base), sm);
  LqChainDev& C = *sm.C;
  const int sg = blockIdx.x, m = C.ns[sg], N = C.N;
  if (m == 0) return;
  double* psi = sg ? psi1 : psi0;
  const size_t pn = (size_t)N * m;
  double* X = psi + (size_t)(C.L - 1) * pn;
  fill_P<double>(C, sg, X);
  for (int l = C.L - 1; l >= 0; --l) {
    double* dst = psi + (size_t)l * pn;
    const double* src = (l == C.L - 1) ? X : psi + (size_t)(l + 1) * pn;
    prop<double, double>(C, sg, dst, src, m, m, -1, 2, -1, sm);
    chol_qr2<double>(C, dst, m, vscr + (size_t)sg * m * m, sm);
  }
}

// Walkers through slices [l0, l1).  phi: each walker's two panels (spin 0
// then spin 1, N x m each); logw[w] += log of the walker's factors; alive[w]
// cleared when a factor is 0.  c0 of walker w is w, c1 the sweep or run word.
__global__ void __launch_bounds__(LQ_THREADS, 1)
    cp_walk_kernel(const LqChainDev* base, const double* psi0, const double* psi1, double* phi, double* logw,
                   int* alive, int n_walkers, int l0, int l1, uint32_t c1, uint32_t tag, double* vscr, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  __shared__ double sh_g[2], sh_c[2], sh_f[2];
  __shared__ int sh_dead;
  load_chain(const_cast<LqChainDev*>(base), sm);
  LqChainDev& C = *sm.C;
  const int N = C.N, MP = sm.MP, m0 = C.ns[0], m1 = C.ns[1];
  const size_t pn0 = (size_t)N * m0, pn1 = (size_t)N * m1;
  const int warp = TID >> 5, lane = TID & 31;
  double* xv = sm.vec;            // x = Phi_i T, per spin (M each)
  double* yv = sm.vec + 2 * sm.M; // y = T Psi_i^T, per spin
  for (int w = blockIdx.x; w < n_walkers; w += gridDim.x) {
    if (!alive[w]) continue;
    double* ph[2] = {phi + (size_t)w * (pn0 + pn1), phi + (size_t)w * (pn0 + pn1) + pn0};
    const double* ps[2] = {psi0, psi1};
    double lw = 0.0;  // thread 0
    if (TID == 0) sh_dead = 0;
    __syncthreads();
    for (int l = l0; l < l1 && !sh_dead; ++l) {
      // T = (Psi_l^T Phi)^{-1} per spin
      for (int sg = 0; sg < 2; ++sg) {
        const int m = sg ? m1 : m0;
        if (m == 0) continue;
        gram<double>(ps[sg] + (size_t)l * N * m, m, m, ph[sg], m, m, N, sm.W, MP);
        double la;
        int s1;
        inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
      }
      for (int i = 0; i < N; ++i) {
        // g_sigma = Phi_i T Psi_i^T with x = Phi_i T and y = T Psi_i^T
        if (warp < 2) {
          const int sg = warp, m = sg ? m1 : m0;
          const double* Tm = sm.T[sg];
          const double* pr = ph[sg] + (size_t)i * m;
          const double* qr = ps[sg] + ((size_t)l * N + i) * m;
          double part = 0.0;
          for (int b = lane; b < m; b += 32) {
            double x = 0.0, y = 0.0;
            for (int a = 0; a < m; ++a) {
              x = fma(pr[a], Tm[a * MP + b], x);
              y = fma(Tm[b * MP + a], qr[a], y);
            }
            xv[sg * sm.M + b] = x;
            yv[sg * sm.M + b] = y;
            part = fma(x, qr[b], part);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
          if (lane == 0) sh_g[sg] = m > 0 ? part : 0.0;
        }
        __syncthreads();
        if (TID == 0) {
          double a[2];
          for (int t = 0; t < 2; ++t) {
            const int s = t ? -1 : 1;
            double r = C.charge ? (s > 0 ? C.dfac_m : C.dfac_p) : 1.0;  // e^{-lambda s}
            for (int sg = 0; sg < 2; ++sg)
              if ((sg ? m1 : m0) > 0) r *= 1.0 + (dfac(C, sg, s) - 1.0) * sh_g[sg];
            a[t] = 0.5 * (r > 0.0 ? r : 0.0);
          }
          const double tot = a[0] + a[1];
          if (!(tot > 0.0)) {
            sh_dead = 1;
          } else {
            lw += log(tot);
            uint32_t rw[4];
            philox((uint32_t)w, c1, (tag << 24) | (uint32_t)l, (uint32_t)i, C.key0, C.key1, rw);
            const int s = (u53(rw[0], rw[1]) * tot < a[0]) ? 1 : -1;
            for (int sg = 0; sg < 2; ++sg) {
              const double f = dfac(C, sg, s), d = f - 1.0;
              sh_f[sg] = f;
              sh_c[sg] = d / (1.0 + d * sh_g[sg]);
            }
          }
        }
        __syncthreads();
        if (sh_dead) break;
        // Phi_i <- f Phi_i and T <- T - c y x (Sherman-Morrison), per spin
        for (int sg = 0; sg < 2; ++sg) {
          const int m = sg ? m1 : m0;
          const double c = sh_c[sg];
          double* Tm = sm.T[sg];
          for (int idx = TID; idx < m * m; idx += LQ_THREADS) {
            const int r = idx / m, b = idx - r * m;
            Tm[r * MP + b] = fma(-c * yv[sg * sm.M + r], xv[sg * sm.M + b], Tm[r * MP + b]);
          }
          for (int a = TID; a < m; a += LQ_THREADS) ph[sg][(size_t)i * m + a] *= sh_f[sg];
        }
        __syncthreads();
      }
      if (sh_dead) break;
      // Phi <- B_K Phi, re-orthonormalized
      for (int sg = 0; sg < 2; ++sg) {
        const int m = sg ? m1 : m0;
        prop<double, double>(C, sg, ph[sg], ph[sg], m, m, -1, 1, -1, sm);
        chol_qr2<double>(C, ph[sg], m, vscr + (size_t)blockIdx.x * 2 * sm.M * sm.M + (size_t)sg * sm.M * sm.M, sm);
      }
    }
    if (TID == 0) {
      if (sh_dead) alive[w] = 0;
      else logw[w] += lw;
    }
    __syncthreads();
  }
}

// New walker k <- old walker src[k] (both spins' panels).
__global__ void cp_gather_kernel(const double* phi, double* phi_new, const int* src, int n_walkers, size_t per) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)n_walkers * per;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t k = idx / per, e = idx - k * per;
    phi_new[idx] = phi[(size_t)src[k] * per + e];
  }
}

__global__ void cp_fill_kernel(const LqChainDev* base, double* phi, int n_walkers) {
  const LqChainDev& C = *base;
  const int N = C.N, m0 = C.ns[0], m1 = C.ns[1];
  const size_t pn0 = (size_t)N * m0, per = pn0 + (size_t)N * m1;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)n_walkers * per;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = idx % per;
    const int sg = e >= pn0, m = sg ? m1 : m0;
    const size_t f = sg ? e - pn0 : e;
    const int i = (int)(f / m), a = (int)(f - (size_t)i * m);
    phi[idx] = (C.occ[sg][a] == i) ? 1.0 : 0.0;
  }
}

}  // namespace lq

namespace {

// Philox4x32-10 on the host (Salmon, Moraes, Dror, Shaw, SC'11): the comb's
// uniform, the same generator and counter layout as the kernels'.
void host_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, uint32_t out[4]) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
double host_u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// Systematic (comb) resampling, Kitagawa (1996): new walker k copies the
// first old walker whose cumulative weight exceeds (k + u)/n of the total.
void comb(const std::vector<double>& w, double u, std::vector<int>& src) {
  const int n = (int)w.size();
  double tot = 0.0;
  for (double x : w) tot += x;
  double cum = w[0];
  for (int k = 0, j = 0; k < n; ++k) {
    const double pos = (k + u) / n * tot;
    while (j < n - 1 && cum <= pos) cum += w[++j];
    src[k] = j;
  }
}

lq_status cp_fail(lq_status s, const std::string& m) { return lq_internal_fail(s, m); }

// Device state of one constrained-path run: a one-chain simulation carries
// the lattice tables and HS constants; the trial panels, walkers and scratch
// are allocated here.
struct CpRun {
  lq_sim* sim = nullptr;
  LqChainDev desc;
  LqChainDev* d_desc = nullptr;
  double *psi0 = nullptr, *psi1 = nullptr, *phi = nullptr, *phi2 = nullptr, *logw = nullptr, *vscr = nullptr;
  int* alive = nullptr;
  int* src = nullptr;
  char* ws = nullptr;
  lq::SmemPlan plan;
  int grid = 1, n = 0;
  size_t per = 0;
  ~CpRun() {
    cudaFree(psi0); cudaFree(psi1); cudaFree(phi); cudaFree(phi2); cudaFree(logw); cudaFree(vscr);
    cudaFree(alive); cudaFree(src); cudaFree(ws);
    if (sim) lq_sim_destroy(sim);
  }
};

lq_status cp_setup(CpRun& R, const lq_lattice* lat, const lq_params* p, const int32_t* up, const int32_t* dn,
                   int n_walkers) {
  if (!lat || !p || n_walkers < 1) return cp_fail(LQ_EINVAL, "bad arguments to the constrained-path call");
  if (p->precision != LQ_FP64) return cp_fail(LQ_EUNSUPPORTED, "the constrained-path walkers run in LQ_FP64");
  lq_status st = lq_internal_sim_create_unbuilt(lat, p, 0u, nullptr, nullptr, &R.sim);
  if (st != LQ_OK) return st;
  // the Fock state eta: distinct sites in range
  const lq_lattice_view v = lq_lattice_get_view(lat);
  const int32_t* in[2] = {up, dn};
  const int ns[2] = {p->n_up, p->n_dn};
  for (int sg = 0; sg < 2; ++sg) {
    if (ns[sg] && !in[sg]) return cp_fail(LQ_EINVAL, "null occupation array");
    std::vector<char> seen(v.N, 0);
    for (int a = 0; a < ns[sg]; ++a) {
      const int i = in[sg][a];
      if (i < 0 || i >= v.N || seen[i]) return cp_fail(LQ_EINVAL, "occupations must be distinct sites in [0, N)");
      seen[i] = 1;
    }
  }
  R.desc = *lq_internal_sim_host_desc(R.sim);
  const lq_sim_launch_info inf = lq_internal_sim_info(R.sim);
  R.d_desc = inf.d_chains;
  cudaError_t e = cudaSuccess;
  for (int sg = 0; sg < 2 && e == cudaSuccess; ++sg)
    if (ns[sg]) e = cudaMemcpy(R.desc.occ[sg], in[sg], sizeof(int) * ns[sg], cudaMemcpyHostToDevice);
  const int N = v.N, L = R.desc.L, M = std::max(std::max(ns[0], ns[1]), 1);
  R.n = n_walkers;
  R.per = (size_t)N * (ns[0] + ns[1]);
  R.plan = lq::plan_smem(M, N, inf.buf_bytes);
  int dev = 0, sms = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  R.grid = std::min(n_walkers, sms);
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes ? bytes : 8);
  };
  alloc((void**)&R.psi0, sizeof(double) * (size_t)L * N * ns[0]);
  alloc((void**)&R.psi1, sizeof(double) * (size_t)L * N * ns[1]);
  alloc((void**)&R.phi, sizeof(double) * n_walkers * R.per);
  alloc((void**)&R.phi2, sizeof(double) * n_walkers * R.per);
  alloc((void**)&R.logw, sizeof(double) * n_walkers);
  alloc((void**)&R.alive, sizeof(int) * n_walkers);
  alloc((void**)&R.src, sizeof(int) * n_walkers);
  alloc((void**)&R.vscr, sizeof(double) * (size_t)std::max(R.grid, 2) * 2 * M * M);
  const size_t ws_bytes = (size_t)std::max(R.grid, 2) * R.plan.ws_cta;
  if (R.plan.big) alloc((void**)&R.ws, ws_bytes);
  R.plan.ws = R.ws;
  if (e == cudaSuccess) e = cudaMemset(R.logw, 0, sizeof(double) * n_walkers);
  if (e == cudaSuccess) {
    std::vector<int> ones(n_walkers, 1);
    e = cudaMemcpy(R.alive, ones.data(), sizeof(int) * n_walkers, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)lq::cp_trial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)R.plan.total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)lq::cp_walk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)R.plan.total);
  if (e == cudaSuccess) {
    lq::cp_trial_kernel<<<2, LQ_THREADS, R.plan.total>>>(R.d_desc, R.psi0, R.psi1, R.vscr, R.plan);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    lq::cp_fill_kernel<<<256, 256>>>(R.d_desc, R.phi, n_walkers);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cp_fail(LQ_ECUDA, std::string("constrained-path set-up: ") + cudaGetErrorString(e));
  return LQ_OK;
}

cudaError_t cp_run_slices(CpRun& R, int l0, int l1, uint32_t c1, uint32_t tag) {
  lq::cp_walk_kernel<<<R.grid, LQ_THREADS, R.plan.total>>>(R.d_desc, R.psi0, R.psi1, R.phi, R.logw, R.alive, R.n, l0,
                                                           l1, c1, tag, R.vscr, R.plan);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

}  // namespace

extern "C" lq_status lq_cp_walk(const lq_lattice* lattice, const lq_params* params, const int32_t* host_occ_up,
                                const int32_t* host_occ_dn, int32_t n_walkers, uint32_t sweep_word,
                                double* host_log_weights, int32_t* host_dropped) {
  if (!host_log_weights) return cp_fail(LQ_EINVAL, "null output");
  CpRun R;
  lq_status st = cp_setup(R, lattice, params, host_occ_up, host_occ_dn, n_walkers);
  if (st != LQ_OK) return st;
  cudaError_t e = cp_run_slices(R, 0, R.desc.L, sweep_word, 7u);
  std::vector<double> lw(n_walkers);
  std::vector<int> alive(n_walkers);
  if (e == cudaSuccess) e = cudaMemcpy(lw.data(), R.logw, sizeof(double) * n_walkers, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(alive.data(), R.alive, sizeof(int) * n_walkers, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cp_fail(LQ_ECUDA, std::string("lq_cp_walk: ") + cudaGetErrorString(e));
  int dropped = 0;
  for (int k = 0; k < n_walkers; ++k) {
    host_log_weights[k] = alive[k] ? lw[k] : -INFINITY;
    dropped += !alive[k];
  }
  if (host_dropped) *host_dropped = dropped;
  return LQ_OK;
}

extern "C" lq_status lq_cp_population(const lq_lattice* lattice, const lq_params* params, const int32_t* host_occ_up,
                                      const int32_t* host_occ_dn, int32_t n_walkers, int32_t comb_every, uint32_t run,
                                      double* host_log_estimate) {
  if (!host_log_estimate || comb_every < 0) return cp_fail(LQ_EINVAL, "bad arguments to lq_cp_population");
  CpRun R;
  lq_status st = cp_setup(R, lattice, params, host_occ_up, host_occ_dn, n_walkers);
  if (st != LQ_OK) return st;
  const int L = R.desc.L;
  double log_est = 0.0;
  std::vector<double> lw(n_walkers), w(n_walkers);
  std::vector<int> alive(n_walkers), src(n_walkers);
  const std::vector<int> ones(n_walkers, 1);
  int l0 = 0;
  cudaError_t e = cudaSuccess;
  while (l0 < L && e == cudaSuccess) {
    int l1 = L;
    if (comb_every > 0) l1 = std::min(L, (l0 / comb_every + 1) * comb_every);
    e = cp_run_slices(R, l0, l1, run, 8u);
    if (e == cudaSuccess) e = cudaMemcpy(lw.data(), R.logw, sizeof(double) * n_walkers, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(alive.data(), R.alive, sizeof(int) * n_walkers, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    double tot = 0.0;
    for (int k = 0; k < n_walkers; ++k) {
      w[k] = alive[k] ? std::exp(lw[k]) : 0.0;
      tot += w[k];
    }
    if (!(tot > 0.0)) { log_est = -INFINITY; break; }
    log_est += std::log(tot / n_walkers);
    if (l1 == L) break;
    uint32_t rw[4];
    host_philox(run, 0xFFFFFFFDu, (9u << 24) | (uint32_t)(l1 - 1), 0u, R.desc.key0, R.desc.key1, rw);
    comb(w, host_u53(rw[0], rw[1]), src);
    e = cudaMemcpy(R.src, src.data(), sizeof(int) * n_walkers, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      lq::cp_gather_kernel<<<256, 256>>>(R.phi, R.phi2, R.src, n_walkers, R.per);
      e = cudaGetLastError();
    }
    std::swap(R.phi, R.phi2);
    if (e == cudaSuccess) e = cudaMemset(R.logw, 0, sizeof(double) * n_walkers);
    if (e == cudaSuccess) e = cudaMemcpy(R.alive, ones.data(), sizeof(int) * n_walkers, cudaMemcpyHostToDevice);
    l0 = l1;
  }
  if (e != cudaSuccess) return cp_fail(LQ_ECUDA, std::string("lq_cp_population: ") + cudaGetErrorString(e));
  *host_log_estimate = log_est;
  return LQ_OK;
}
