// lq_noalloc.cu -- a single-chain sweep entry point that allocates no device
// memory.
//
// Some callers cannot allocate device memory themselves: code running under
// an allocator-free plug-in contract, processes whose memory is reserved up
// front by a host framework, or callers inside code that may not call
// cudaMalloc for latency or determinism reasons.  lq_sweep_noalloc serves
// them: the caller owns the inputs and outputs (fields, occupations,
// records), and every scratch buffer the sweep needs (QR chains, stored and
// live panels, lattice tables, the chain descriptor) lives in one file-scope
// __device__ array of fixed size.  Each GPU that loads the library holds that
// array until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/lecqmc.h"
#include "lq_device.h"
#include "lq_kernels.h"
#include "lq_lattice.h"

// The one scratch array; all calls on a device share it.
static __device__ __align__(256) unsigned char g_lq_scratch[LQ_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Upload the dtau-dependent lattice factors.  They are computed on the host
// with the same expressions as the regular entry point's tables
// (lq_bond_factors, lq_onsite_factor), a chunk at a time through a small
// stack buffer: a copy from pageable host memory has taken its source by the
// time cudaMemcpyAsync returns, so the buffer can be refilled at once.
cudaError_t upload_factors(const lq_lattice_view& v, double dtau, unsigned char* base, size_t o_bc, size_t o_bs,
                           size_t o_bcf, size_t o_bsf, size_t o_ce, size_t o_cef, cudaStream_t st) {
  constexpr int CH = 256;
  double c[CH], s[CH];
  float cf[CH], sf[CH];
  cudaError_t e = cudaSuccess;
  double cprod;
  const unsigned unif = lq_uniform_families(v, dtau, &cprod);
  int g = 0;
  for (int b0 = 0; b0 < v.nb && e == cudaSuccess; b0 += CH) {
    const int n = std::min(CH, v.nb - b0);
    for (int t = 0; t < n; ++t) {
      lq_bond_factors(dtau, v.sorted_k[b0 + t], &c[t], &s[t]);
      cf[t] = (float)c[t];
      sf[t] = (float)s[t];
      while (g + 1 < v.G && b0 + t >= v.fam_off[g + 1]) ++g;
      if (g < 32 && ((unif >> g) & 1u)) s[t] = lq_bond_tanh(dtau, v.sorted_k[b0 + t]);
    }
    e = cudaMemcpyAsync(base + o_bc + (size_t)b0 * 8, c, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bs + (size_t)b0 * 8, s, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bcf + (size_t)b0 * 4, cf, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bsf + (size_t)b0 * 4, sf, (size_t)n * 4, cudaMemcpyHostToDevice, st);
  }
  for (int i0 = 0; i0 < v.N && e == cudaSuccess; i0 += CH) {
    const int n = std::min(CH, v.N - i0);
    for (int t = 0; t < n; ++t) {
      c[t] = lq_onsite_factor(dtau, v.eps[i0 + t]);
      cf[t] = (float)c[t];
    }
    e = cudaMemcpyAsync(base + o_ce + (size_t)i0 * 8, c, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_cef + (size_t)i0 * 4, cf, (size_t)n * 4, cudaMemcpyHostToDevice, st);
  }
  return e;
}

// FP32 copies of n doubles, converted through the same small stack buffer.
cudaError_t upload_floats(const double* src, int n, unsigned char* dst, cudaStream_t st) {
  constexpr int CH = 256;
  float f[CH];
  cudaError_t e = cudaSuccess;
  for (int i0 = 0; i0 < n && e == cudaSuccess; i0 += CH) {
    const int k = std::min(CH, n - i0);
    for (int t = 0; t < k; ++t) f[t] = (float)src[i0 + t];
    e = cudaMemcpyAsync(dst + (size_t)i0 * 4, f, (size_t)k * 4, cudaMemcpyHostToDevice, st);
  }
  return e;
}

}  // namespace

extern "C" lq_status lq_sweep_noalloc(const lq_lattice* lat, const lq_params* p, uint32_t chain_id,
                                      uint32_t sweep_index, int8_t* dev_fields, int32_t* dev_occ, int32_t n_sweeps,
                                      double* dev_records, void* cuda_stream, double* host_log_weight,
                                      int32_t* host_sign, int64_t* host_counts4) {
  if (!lat || !p || !dev_fields || !dev_occ || n_sweeps < 0) return lq_internal_fail(LQ_EINVAL, "bad arguments to lq_sweep_noalloc");
  const lq_lattice_view v = lq_lattice_get_view(lat);
  if (p->precision != LQ_FP64 && p->precision != LQ_MIXED && p->precision != LQ_MIXED_DW)
    return lq_internal_fail(LQ_EINVAL, "bad precision");
  if (!(p->beta > 0) || !(p->dtau > 0) || !std::isfinite(p->U)) return lq_internal_fail(LQ_EINVAL, "beta, dtau must be > 0");
  const double Lf = p->beta / p->dtau;
  const long Ll = std::lround(Lf);
  if (Ll < 1 || std::fabs(Lf - (double)Ll) > 1e-9 * std::max(1.0, Lf) || Ll > (1 << 24) - 1)
    return lq_internal_fail(LQ_EINVAL, "beta/dtau must be a positive integer");
  if (p->n_stab < 1 || p->n_up < 0 || p->n_dn < 0 || p->n_up > v.N || p->n_dn > v.N)
    return lq_internal_fail(LQ_EINVAL, "n_stab must be >= 1 and particle numbers in [0, N]");
  if (p->swap_mode != LQ_SWAP_UNIFORM && p->swap_mode != LQ_SWAP_NEIGHBOUR)
    return lq_internal_fail(LQ_EINVAL, "swap_mode must be LQ_SWAP_UNIFORM or LQ_SWAP_NEIGHBOUR");
  if (p->left_swaps != 0 && p->left_swaps != 1) return lq_internal_fail(LQ_EINVAL, "left_swaps must be 0 or 1");
  if (p->kinetic != LQ_CHECKERBOARD && p->kinetic != LQ_EXACT)
    return lq_internal_fail(LQ_EINVAL, "kinetic must be LQ_CHECKERBOARD or LQ_EXACT");
  const int exact = p->kinetic == LQ_EXACT;
  if (exact && p->dtau * v.k_rownorm > LQ_EXACT_THETA_MAX)
    return lq_internal_fail(LQ_EUNSUPPORTED, "LQ_EXACT needs dtau * max_i sum_j |K_ij| <= 2");
  if (p->n_up > LQ_MAX_PARTICLES || p->n_dn > LQ_MAX_PARTICLES)
    return lq_internal_fail(LQ_EUNSUPPORTED, "at most LQ_MAX_PARTICLES particles per spin");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return lq_internal_fail(LQ_ECUDA, "no current CUDA device");
  // set-up, once per device, with that device current
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_lq_scratch);
    if (e != cudaSuccess || !ptr)
      return lq_internal_fail(LQ_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  unsigned char* base = g_scratch_addr[dev];
  // carve the scratch: descriptor, order/queue words, lattice tables, chain state
  const int N = v.N, nb = v.nb, G = v.G, L = (int)Ll, tw = p->n_stab, n = (L + tw - 1) / tw;
  const int ns[2] = {p->n_up, p->n_dn};
  const size_t PS = p->precision == LQ_FP64 ? sizeof(double) : sizeof(float);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
  const size_t o_desc = take(sizeof(LqChainDev));
  const size_t o_order = take(sizeof(int));
  const size_t o_queue = take(sizeof(int) * (1 + 1024));
  const size_t o_fo = take((G + 1) * 4), o_bi = take(nb * 4), o_bj = take(nb * 4), o_bk = take(nb * 8);
  const size_t o_bc = take(nb * 8), o_bs = take(nb * 8), o_bcf = take(nb * 4), o_bsf = take(nb * 4);
  const size_t o_eps = take(N * 8), o_ce = take(N * 8), o_cef = take(N * 4), o_sub = take(N * 4);
  const size_t o_nbo = take((size_t)(N + 1) * 4), o_nbs = take((size_t)std::max(2 * nb, 1) * 4);
  const size_t o_ko = take((size_t)(N + 1) * 4), o_kc = take((size_t)std::max(v.nnz, 1) * 4);
  const size_t o_kv = take((size_t)std::max(v.nnz, 1) * 8), o_kvf = take((size_t)std::max(v.nnz, 1) * 4);
  size_t o_QR[2][2], o_VR[2][2], o_QL[2], o_VL[2], o_st[2], o_live[2], o_work[2];
  for (int sg = 0; sg < 2; ++sg) {
    const size_t pn = (size_t)N * ns[sg], qn = (size_t)ns[sg] * ns[sg];
    o_QR[sg][0] = take((n + 1) * pn * PS); o_QR[sg][1] = take((n + 1) * pn * PS);
    o_VR[sg][0] = take((n + 1) * qn * 8); o_VR[sg][1] = take((n + 1) * qn * 8);
    o_QL[sg] = take((n + 1) * pn * PS); o_VL[sg] = take((n + 1) * qn * 8);
    o_st[sg] = take(tw * pn * PS); o_live[sg] = take(pn * PS); o_work[sg] = take(pn * 8);
  }
  const size_t o_vec = take((size_t)2 * N * 8), o_rot = take((size_t)n * LQ_NS_MAX * 2 * 8);
  const int M = std::max(std::max(ns[0], ns[1]), 1);
  const int buf_bytes = lq::staging_bytes(M, N, exact ? 2 : 1);
  const size_t ws_bytes = lq::workspace_bytes(M, N, buf_bytes);  // one CTA's slab (big plans only)
  const size_t o_ws = take(ws_bytes);
  if (o > (size_t)LQ_NOALLOC_SCRATCH_BYTES)
    return lq_internal_fail(LQ_EUNSUPPORTED, "lq_sweep_noalloc: this chain needs " + std::to_string(o) +
                                                 " scratch bytes, more than LQ_NOALLOC_SCRATCH_BYTES (" +
                                                 std::to_string((size_t)LQ_NOALLOC_SCRATCH_BYTES) + ")");
  // the shared-memory plan must fit one CTA per SM, as lq_sim_create requires
  if (lq::max_active_sweep_ctas(p->precision, M, lq::smem_bytes(M, N, buf_bytes)) < 1)
    return lq_internal_fail(LQ_EUNSUPPORTED, "shared-memory plan does not fit one CTA per SM");
  // lattice tables (host vectors owned by the lattice) and zeroed counters
  auto up = [&](size_t at, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(base + at, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  e = up(o_fo, v.fam_off, (G + 1) * 4);
  if (e == cudaSuccess) e = up(o_bi, v.sorted_i, nb * 4);
  if (e == cudaSuccess) e = up(o_bj, v.sorted_j, nb * 4);
  if (e == cudaSuccess) e = up(o_bk, v.sorted_k, nb * 8);
  if (e == cudaSuccess) e = up(o_eps, v.eps, N * 8);
  if (e == cudaSuccess) e = up(o_sub, v.sub, N * 4);
  if (e == cudaSuccess) e = up(o_nbo, v.nb_off, (size_t)(N + 1) * 4);
  if (e == cudaSuccess) e = up(o_nbs, v.nb_site, (size_t)v.nb_off[N] * 4);
  if (e == cudaSuccess) e = up(o_ko, v.k_off, (size_t)(N + 1) * 4);
  if (e == cudaSuccess) e = up(o_kc, v.k_col, (size_t)v.nnz * 4);
  if (e == cudaSuccess) e = up(o_kv, v.k_val, (size_t)v.nnz * 8);
  if (e == cudaSuccess) e = upload_floats(v.k_val, v.nnz, base + o_kvf, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_order, 0, sizeof(int), st);
  if (e != cudaSuccess) return lq_internal_fail(LQ_ECUDA, std::string("lq_sweep_noalloc upload: ") + cudaGetErrorString(e));
  if (e == cudaSuccess) e = upload_factors(v, p->dtau, base, o_bc, o_bs, o_bcf, o_bsf, o_ce, o_cef, st);
  if (e != cudaSuccess) return lq_internal_fail(LQ_ECUDA, std::string("lq_sweep_noalloc upload: ") + cudaGetErrorString(e));
  // descriptor
  LqChainDev D;
  std::memset(&D, 0, sizeof(D));
  D.lat.N = N; D.lat.nb = nb; D.lat.G = G;
  D.lat.fam_off = (const int*)(base + o_fo);
  D.lat.bond_i = (const int*)(base + o_bi);
  D.lat.bond_j = (const int*)(base + o_bj);
  D.lat.bond_c = (const double*)(base + o_bc);
  D.lat.bond_s = (const double*)(base + o_bs);
  D.lat.cprod = 1.0;
  D.lat.unif = lq_uniform_families(v, p->dtau, &D.lat.cprod);
  D.lat.bond_cf = (const float*)(base + o_bcf);
  D.lat.bond_sf = (const float*)(base + o_bsf);
  D.lat.bond_k = (const double*)(base + o_bk);
  D.lat.ceps = v.has_eps ? (const double*)(base + o_ce) : nullptr;
  D.lat.cepsf = v.has_eps ? (const float*)(base + o_cef) : nullptr;
  D.lat.eps = v.has_eps ? (const double*)(base + o_eps) : nullptr;
  D.lat.sub = (const int*)(base + o_sub);
  D.lat.nb_off = (const int*)(base + o_nbo);
  D.lat.nb_site = (const int*)(base + o_nbs);
  D.lat.exact = exact;
  D.lat.taylor_q = exact ? lq_taylor_degree(p->dtau * v.k_rownorm) : 0;
  D.lat.mdtau = -p->dtau;
  D.lat.k_off = (const int*)(base + o_ko);
  D.lat.k_col = (const int*)(base + o_kc);
  D.lat.k_val = (const double*)(base + o_kv);
  D.lat.k_valf = (const float*)(base + o_kvf);
  D.N = N; D.L = L; D.tw = tw; D.n = n; D.ns[0] = ns[0]; D.ns[1] = ns[1];
  D.charge = p->U < 0;
  D.prec = p->precision;
  D.swap_mode = p->swap_mode;
  D.left_swaps = p->left_swaps;
  D.lambda = std::acosh(std::exp(p->dtau * std::fabs(p->U) / 2.0));
  D.dfac_p = std::exp(D.lambda); D.dfac_m = std::exp(-D.lambda);
  D.delta_p = std::expm1(-2.0 * D.lambda); D.delta_m = std::expm1(2.0 * D.lambda);
  D.cfac_p = std::exp(2.0 * D.lambda); D.cfac_m = std::exp(-2.0 * D.lambda);
  D.opd_p = 1.0 + D.delta_p; D.opd_m = 1.0 + D.delta_m;
  lq_dw_split(D.delta_p, D.dw_delta_p); lq_dw_split(D.delta_m, D.dw_delta_m);
  lq_dw_split(D.cfac_p, D.dw_cfac_p); lq_dw_split(D.cfac_m, D.dw_cfac_m);
  D.key0 = (uint32_t)p->seed; D.key1 = (uint32_t)(p->seed >> 32);
  D.chain_id = chain_id;
  D.sweep = sweep_index;
  D.s = dev_fields;
  D.occ[0] = dev_occ;
  D.occ[1] = dev_occ + ns[0];
  for (int sg = 0; sg < 2; ++sg) {
    D.QR[sg][0] = base + o_QR[sg][0]; D.QR[sg][1] = base + o_QR[sg][1];
    D.VR[sg][0] = (double*)(base + o_VR[sg][0]); D.VR[sg][1] = (double*)(base + o_VR[sg][1]);
    D.QL[sg] = base + o_QL[sg]; D.VL[sg] = (double*)(base + o_VL[sg]);
    D.stored[sg] = base + o_st[sg]; D.live[sg] = base + o_live[sg]; D.work[sg] = (double*)(base + o_work[sg]);
    D.cur[sg] = 0;
  }
  D.vec = (double*)(base + o_vec);
  D.rot = (double*)(base + o_rot);
  D.records = dev_records;
  D.max_records = dev_records ? n_sweeps : 0;
  D.sign = 1;
  e = cudaMemcpyAsync(base + o_desc, &D, sizeof(D), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return lq_internal_fail(LQ_ECUDA, std::string("descriptor upload: ") + cudaGetErrorString(e));
  LqChainDev* dchain = (LqChainDev*)(base + o_desc);
  const int* dorder = (const int*)(base + o_order);
  int* dqueue = (int*)(base + o_queue);
  void* ws = ws_bytes ? (void*)(base + o_ws) : nullptr;
  e = lq::launch_build(p->precision, dchain, dorder, 1, M, N, buf_bytes, 1, st, ws, ws_bytes);
  if (e == cudaSuccess && n_sweeps > 0)
    e = lq::launch_sweep(p->precision, dchain, dorder, 1, dqueue, n_sweeps, dev_records ? 1 : 0, M, N, buf_bytes, 1, st,
                         ws, ws_bytes);
  if (e != cudaSuccess) return lq_internal_fail(LQ_ECUDA, std::string("lq_sweep_noalloc launch: ") + cudaGetErrorString(e));
  if (host_log_weight || host_sign || host_counts4) {
    LqChainDev out;
    e = cudaMemcpyAsync(&out, dchain, sizeof(out), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return lq_internal_fail(LQ_ECUDA, std::string("lq_sweep_noalloc readback: ") + cudaGetErrorString(e));
    if (out.err & LQ_ERR_BADINPUT) return lq_internal_fail(LQ_EINVAL, "fields must be +-1 and occupied sites distinct in [0, N)");
    if (out.err) return lq_internal_fail(LQ_ENUMERIC, "numerical error flags " + std::to_string(out.err));
    if (host_log_weight) *host_log_weight = out.logw;
    if (host_sign) *host_sign = out.sign;
    if (host_counts4) for (int k = 0; k < 4; ++k) host_counts4[k] = out.cnt[k];
  }
  return LQ_OK;
}
