// lq_sweep.cuh -- device code of the canonical-ensemble DQMC sweep with the
// stabilized QR update (LEC-QMC, arXiv 2601.08552), included by the
// translation units that instantiate the kernels (one sweep-kernel instance
// per unit, so that they compile in parallel).
//
// One CTA owns one Markov chain for a whole sweep (persistent over a queue of
// chains, longest first).  Inside a CTA:
//   * slice propagation (B_l = e^{-dtau K} e^{-dtau V(s_l)}, Eq. 1 and the
//     Trotter form of SM Sec. VI) streams column chunks of an N x N_sigma panel
//     through shared memory and applies the checkerboard families there;
//   * restabilization every tau_w slices (B_i Q_{i-1} = Q_i V_i, SM Sec. I.A)
//     is CholeskyQR2 with FP64 Gram matrices and a positive diagonal;
//   * field flips (the Sherman-Morrison ratio of SM Sec. VI) run as a
//     submatrix update over windows of K sites: the window's dense products
//     are batched, and the serial chain of a site is its diagonal block
//     element, the ratio and a K x K rank-1 update.  Up to 32 particles per
//     spin one leader warp runs the chain of both spins (K = 4, one block
//     element per lane, the spins' factors exchanged by one shuffle) and
//     forms the next window's block from three K x K blocks, while the other
//     warps run the window's dense work one window behind it (named
//     barriers); above 32 a four-warp group per spin (K = 8) shares the dense
//     work and the m x m matrices sit in a global workspace per CTA;
//   * particle-hole swaps: removal by permutation + Givens retriangulation
//     (Eqs. S9-S12), addition by propagating one vector and orthogonalising
//     it twice against each Q_i (Eqs. S1-S8, Eq. 4); the target is uniform
//     over the empty sites or over the empty nearest neighbours (with the
//     Metropolis-Hastings factor);
//   * equal-time measurements at the block boundaries of the down pass.
// Panels are FP64 (LQ_FP64) or FP32 (LQ_MIXED, LQ_MIXED_DW); QR, log-det
// factors and inverses stay FP64 in all modes, and the flip algebra is FP64
// except in LQ_MIXED_DW (double-word FP32).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/lecqmc.h"
#include "lq_device.h"
#include "lq_kernels.h"

namespace lq {

// ---------------------------------------------------------------------------
// shared-memory plan (same arithmetic on host and device)
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct SmemPlan {
  int M, MP, Nmax, buf_bytes, big, s_global, win_global, vec_global;
  // offsets of T0, T1 and W are in shared memory for small plans and in the
  // CTA's slab of the global workspace for big ones (M > LQ_NS_SMALL); the
  // four scratch matrices S, the field-flip window and the scratch vectors
  // stay in shared memory while they fit there, in that order of priority
  size_t off_T0, off_T1, off_W, off_S, off_vec, off_red, off_obs, off_gx, off_ip, off_occ, off_bits, off_chain, off_win,
      off_buf, total;
  size_t ws_cta;  // global workspace bytes per CTA (0 for small plans)
  char* ws;       // the launch's workspace, grid x ws_cta bytes (set by the launcher)
};

// largest dynamic shared memory a plan may take (the opt-in limit is 227 KB)
#define LQ_SMEM_CAP (220 * 1024)

__host__ __device__ inline SmemPlan plan_smem(int M, int Nmax, int buf_bytes) {
  SmemPlan p;
  p.M = M < 1 ? 1 : M;
  p.MP = p.M | 1;
  p.Nmax = Nmax;
  p.buf_bytes = buf_bytes;
  p.big = p.M > LQ_NS_SMALL;
  p.ws = nullptr;
  const size_t mat = (size_t)p.M * p.MP * 8;
  const size_t vec_b = al16((size_t)10 * p.M * 8), win_b = al16((size_t)2 * LQ_WIN_ELEMS(p.MP) * 8);
  const size_t s_b = al16(4 * mat);
  size_t o = 0, g = 0;
  p.off_red = o; o = al16(o + 64 * 8);
  p.off_obs = o; o = al16(o + 16 * 8);
  p.off_gx = o; o = al16(o + 8 * 8);
  p.off_ip = o; o = al16(o + 32 * 4);
  p.off_occ = o; o = al16(o + (size_t)2 * p.M * 4);
  p.off_bits = o; o = al16(o + (size_t)(Nmax / 32 + 2) * 4);
  p.off_chain = o; o = al16(o + sizeof(LqChainDev));
  p.off_buf = o; o = al16(o + (size_t)buf_bytes);
  // big plans move the scratch matrices, then the window, then the vectors
  // to the global workspace until the rest fits
  p.s_global = p.big && o + vec_b + win_b + s_b > LQ_SMEM_CAP;
  p.win_global = p.big && o + vec_b + win_b + (p.s_global ? 0 : s_b) > LQ_SMEM_CAP;
  p.vec_global = p.big && o + vec_b + (p.win_global ? 0 : win_b) + (p.s_global ? 0 : s_b) > LQ_SMEM_CAP;
  size_t& om = p.big ? g : o;  // where T and the Gauss-Jordan workspace go
  p.off_T0 = om; om = al16(om + mat);
  p.off_T1 = om; om = al16(om + mat);
  p.off_W = om; om = al16(om + (size_t)p.M * 2 * p.MP * 8);  // Gauss-Jordan / Gram workspace
  size_t& os = p.s_global ? g : o;
  p.off_S = os; os = al16(os + s_b);
  size_t& ow = p.win_global ? g : o;
  p.off_win = ow; ow = al16(ow + win_b);
  size_t& ov = p.vec_global ? g : o;
  p.off_vec = ov; ov = al16(ov + vec_b);
  p.ws_cta = p.big ? ((g + 255) & ~(size_t)255) : 0;
  p.total = o;
  return p;
}

struct Smem {
  double* T[2];
  double* W;     // M x 2MP
  double* S;     // 6 x (M x MP)
  double* vec;   // 10 x M
  double* red;
  double* obs;
  double* gx;
  int* ip;
  int* occ2;     // 2 x M ints
  unsigned* bits;
  LqChainDev* C;
  void* win;     // field-flip window (X, Y, G, c) per spin
  void* buf;
  int buf_bytes, M, MP;
};

// The dynamic shared memory as an array.  A pointer rebased on it is known
// to the compiler to point into shared memory, so accesses through it are
// shared loads and stores rather than generic ones (which cost a generic
// address resolution each).  Only for buffers that the plan keeps in shared
// memory: every buffer of a small plan (BIG = false).
extern __shared__ __align__(16) char lq_dyn_smem[];
template <class T> __device__ __forceinline__ T* sh_rebase(T* p) {
  return (T*)(lq_dyn_smem + ((size_t)__cvta_generic_to_shared(p) - (size_t)__cvta_generic_to_shared(lq_dyn_smem)));
}
template <bool BIG, class T> __device__ __forceinline__ T* plan_ptr(T* p) {
  if (BIG) return p;
  return sh_rebase(p);
}

__device__ inline Smem carve(const SmemPlan& p, char* base) {
  Smem s;
  char* mb = p.big ? p.ws + (size_t)blockIdx.x * p.ws_cta : base;
  s.T[0] = (double*)(mb + p.off_T0);
  s.T[1] = (double*)(mb + p.off_T1);
  s.W = (double*)(mb + p.off_W);
  s.S = (double*)((p.s_global ? mb : base) + p.off_S);
  s.vec = (double*)((p.vec_global ? mb : base) + p.off_vec);
  s.red = (double*)(base + p.off_red);
  s.obs = (double*)(base + p.off_obs);
  s.gx = (double*)(base + p.off_gx);
  s.ip = (int*)(base + p.off_ip);
  s.occ2 = (int*)(base + p.off_occ);
  s.bits = (unsigned*)(base + p.off_bits);
  s.C = (LqChainDev*)(base + p.off_chain);
  s.win = (void*)((p.win_global ? mb : base) + p.off_win);
  s.buf = (void*)(base + p.off_buf);
  s.buf_bytes = p.buf_bytes;
  s.M = p.M;
  s.MP = p.MP;
  return s;
}

#define TID ((int)threadIdx.x)
// threads of the running CTA: LQ_THREADS (256), or 128 for sweep launches of
// plans with at most LQ_NS_SMALL particles per spin that the autotuner runs
// four CTAs per SM
#define NTHR ((int)blockDim.x)
#define FULL 0xffffffffu

// Device global timer in nanoseconds.
__device__ __forceinline__ long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// Per-phase cycle counters of a chain (thread 0, clock64), for profiling.
enum { PH_FLIP = 0, PH_PROP = 1, PH_QR = 2, PH_BLOCKINV = 3, PH_SWAP = 4, PH_MEAS = 5 };
// Only the outermost timer of a nest records, so the phases add up.
struct ProfShared {
  LqChainDev* C;
  int depth;
};
static __device__ ProfShared* prof_shared() {
  __shared__ ProfShared ps;
  return &ps;
}
struct PhaseTimer {
  int ph, outer;
  long long t0;
  __device__ explicit PhaseTimer(int p) : ph(p), outer(0), t0(0) {
    if (threadIdx.x == 0) {
      ProfShared* ps = prof_shared();
      outer = (ps->depth++ == 0);
      t0 = clock64();
    }
  }
  __device__ ~PhaseTimer() {
    if (threadIdx.x == 0) {
      ProfShared* ps = prof_shared();
      --ps->depth;
      if (outer && ps->C) ps->C->prof[ph] += clock64() - t0;
    }
  }
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and 53-bit uniforms
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double dfac(const LqChainDev& C, int sigma, int s) {
  int sp = C.charge ? 1 : (sigma == 0 ? 1 : -1);
  return (sp * s > 0) ? C.dfac_p : C.dfac_m;
}
__device__ __forceinline__ double delta_of(const LqChainDev& C, int sigma, int s) {
  int sp = C.charge ? 1 : (sigma == 0 ? 1 : -1);
  return (sp * s > 0) ? C.delta_p : C.delta_m;
}

__device__ __forceinline__ double opd_of(const LqChainDev& C, int sigma, int s) {
  int sp = C.charge ? 1 : (sigma == 0 ? 1 : -1);
  return (sp * s > 0) ? C.opd_p : C.opd_m;
}

template <class R> __device__ __forceinline__ const R* bc_ptr(const LqLatticeDev& L);
template <> __device__ __forceinline__ const double* bc_ptr<double>(const LqLatticeDev& L) { return L.bond_c; }
template <> __device__ __forceinline__ const float* bc_ptr<float>(const LqLatticeDev& L) { return L.bond_cf; }
template <class R> __device__ __forceinline__ const R* bs_ptr(const LqLatticeDev& L);
template <> __device__ __forceinline__ const double* bs_ptr<double>(const LqLatticeDev& L) { return L.bond_s; }
template <> __device__ __forceinline__ const float* bs_ptr<float>(const LqLatticeDev& L) { return L.bond_sf; }
template <class R> __device__ __forceinline__ const R* ceps_ptr(const LqLatticeDev& L);
template <> __device__ __forceinline__ const double* ceps_ptr<double>(const LqLatticeDev& L) { return L.ceps; }
template <> __device__ __forceinline__ const float* ceps_ptr<float>(const LqLatticeDev& L) { return L.cepsf; }

__device__ __forceinline__ void bar_pair() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// CTA-wide sum in a fixed order (deterministic).
static __device__ double cta_sum(double v, Smem& sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();
  if ((TID & 31) == 0) sm.red[TID >> 5] = v;
  __syncthreads();
  if (TID < 32) {
    double t = (TID < NTHR / 32) ? sm.red[TID] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (TID == 0) sm.red[40] = t;
  }
  __syncthreads();
  return sm.red[40];
}


// ---------------------------------------------------------------------------
// Double-word arithmetic on FP32 pairs (value = h + l, |l| <= ulp(h)/2):
// Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based TwoProd error-free
// transformations, combined into sum and product as in Joldes, Muller and
// Popescu (ACM TOMS 2017).  Relative error about 2^-46 per operation.  The
// _rn intrinsics keep the compiler from contracting or reassociating.
// ---------------------------------------------------------------------------
struct dw {
  float h, l;
};
__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw dw_add(dw a, dw b) {
  const dw s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dw dw_neg(dw a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dw dw_mul(dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dw dw_mulf(dw a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return fast_two_sum(p, e);
}
// acc += a * t (a FP32, t double-word), unnormalized accumulator
__device__ __forceinline__ void dw_acc(dw& acc, float a, dw t) {
  const float ph = __fmul_rn(a, t.h);
  float pl = __fmaf_rn(a, t.h, -ph);
  pl = __fmaf_rn(a, t.l, pl);
  const dw s = two_sum(acc.h, ph);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(pl, s.l));
}
// a / b: a fast FP32 quotient estimate, then one correction with the
// double-word remainder a - b q1 (the estimate's few-ulp error is removed by
// the second term, whose own relative error is FP32 level)
__device__ __forceinline__ dw dw_div(dw a, dw b) {
  const float q1 = __fdividef(a.h, b.h);
  const dw r = dw_add(a, dw_neg(dw_mulf(b, q1)));
  return fast_two_sum(q1, __fdividef(r.h, b.h));
}
__device__ __forceinline__ dw dw_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ dw dw_shfl_xor(dw a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
__device__ __forceinline__ dw dw_shfl(dw a, int src) {
  return {__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
}
// a > b for normalized double-words
__device__ __forceinline__ bool dw_gt(dw a, dw b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// ---------------------------------------------------------------------------
// Propagation: dst <- D_post * Op * D_pre * src for an N x m panel.
// op: 0 none, 1 B_K = E_{G-1}..E_0 C_eps, 2 B_K^T = C_eps E_0..E_{G-1}.
// Columns are independent, so the panel goes through shared memory in column
// chunks; each family is one parallel pass of 2x2 rotations there.
// ---------------------------------------------------------------------------
template <class R> __device__ __forceinline__ const R* kval_ptr(const LqLatticeDev& L);
template <> __device__ __forceinline__ const double* kval_ptr<double>(const LqLatticeDev& L) { return L.k_val; }
template <> __device__ __forceinline__ const float* kval_ptr<float>(const LqLatticeDev& L) { return L.k_valf; }

// Exact kinetic propagator: dst <- D_post e^{-dtau K} D_pre src.  K is
// symmetric, so B_K and B_K^T are the same operator.  For each column chunk,
// Horner's rule y <- x + (-dtau/k) K y, k = q .. 1, starting from y = x,
// evaluates sum_{j <= q} (-dtau K)^j x / j! with two buffers in shared
// memory; x = D_pre src is re-read from src at each step (src is written, in
// place, only after the last step).
template <class R, class S>
__device__ void prop_exact(const LqChainDev& C, int sigma, R* dst, const S* src, int m, int ld, int preD, int postD,
                           Smem& sm) {
  const int N = C.N;
  const LqLatticeDev& lat = C.lat;
  R* buf = (R*)sm.buf;
  int cmax = sm.buf_bytes / (int)(2 * sizeof(R) * N);
  if (cmax > m) cmax = m;
  if (cmax < 1) cmax = 1;  // the staging plan holds at least two columns for exact chains
  const int8_t* spre = preD >= 0 ? C.s + (size_t)preD * N : nullptr;
  const int8_t* spost = postD >= 0 ? C.s + (size_t)postD * N : nullptr;
  const R* kv = kval_ptr<R>(lat);
  const int* ko = lat.k_off;
  const int* kc = lat.k_col;
  for (int c0 = 0; c0 < m; c0 += cmax) {
    const int cw = min(cmax, m - c0);
    const int tot = N * cw;
    R* y0 = buf;
    R* y1 = buf + tot;
    for (int idx = TID; idx < tot; idx += NTHR) {
      const int i = idx / cw, a = idx - i * cw;
      R v = (R)src[(size_t)i * ld + c0 + a];
      if (spre) v *= (R)dfac(C, sigma, spre[i]);
      y0[idx] = v;
    }
    __syncthreads();
    for (int k = lat.taylor_q; k >= 1; --k) {
      const R ck = (R)(lat.mdtau / (double)k);
      for (int idx = TID; idx < tot; idx += NTHR) {
        const int i = idx / cw, a = idx - i * cw;
        R acc = (R)0;
        for (int p = ko[i]; p < ko[i + 1]; ++p) acc += kv[p] * y0[kc[p] * cw + a];
        R x = (R)src[(size_t)i * ld + c0 + a];
        if (spre) x *= (R)dfac(C, sigma, spre[i]);
        y1[idx] = x + ck * acc;
      }
      __syncthreads();
      R* t = y0; y0 = y1; y1 = t;
    }
    for (int idx = TID; idx < tot; idx += NTHR) {
      const int i = idx / cw, a = idx - i * cw;
      R v = y0[idx];
      if (spost) v *= (R)dfac(C, sigma, spost[i]);
      dst[(size_t)i * ld + c0 + a] = v;
    }
    __syncthreads();
  }
}

template <class R, class S>
__device__ void prop(const LqChainDev& C, int sigma, R* dst, const S* src, int m, int ld, int preD, int op, int postD,
                     Smem& sm) {
  PhaseTimer pt_(1);
  if (m == 0) return;
  if (op != 0 && C.lat.exact) {
    prop_exact<R, S>(C, sigma, dst, src, m, ld, preD, postD, sm);
    return;
  }
  const int N = C.N;
  const LqLatticeDev& lat = C.lat;
  R* buf = sh_rebase((R*)sm.buf);  // the staging buffer is in shared memory in every plan
  int cmax = sm.buf_bytes / (int)(sizeof(R) * N);
  if (cmax > m) cmax = m;
  const int8_t* spre = preD >= 0 ? C.s + (size_t)preD * N : nullptr;
  const int8_t* spost = postD >= 0 ? C.s + (size_t)postD * N : nullptr;
  const R* ceps = ceps_ptr<R>(lat);
  const R* bcv = bc_ptr<R>(lat);
  const R* bsv = bs_ptr<R>(lat);
  for (int c0 = 0; c0 < m; c0 += cmax) {
    const int cw = min(cmax, m - c0);
    const int tot = N * cw;
    // four elements' loads in flight per thread before their stores
    int idx = TID;
    for (; idx + 3 * NTHR < tot; idx += 4 * NTHR) {
      R v4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = (idx + q * NTHR) / cw, a = idx + q * NTHR - i * cw;
        v4[q] = (R)src[(size_t)i * ld + c0 + a];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = (idx + q * NTHR) / cw;
        R v = v4[q];
        if (spre) v *= (R)dfac(C, sigma, spre[i]);
        if (op == 1 && ceps) v *= ceps[i];
        buf[idx + q * NTHR] = v;
      }
    }
    for (; idx < tot; idx += NTHR) {
      int i = idx / cw, a = idx - i * cw;
      R v = (R)src[(size_t)i * ld + c0 + a];
      if (spre) v *= (R)dfac(C, sigma, spre[i]);
      if (op == 1 && ceps) v *= ceps[i];
      buf[idx] = v;
    }
    __syncthreads();
    if (op != 0) {
      for (int gg = 0; gg < lat.G; ++gg) {
        const int g = (op == 1) ? gg : lat.G - 1 - gg;
        const int b0 = lat.fam_off[g], work = (lat.fam_off[g + 1] - b0) * cw;
        if (sizeof(R) == 8 && g < 32 && ((lat.unif >> g) & 1u)) {
          // FP64 panels: c_g [[1, t], [t, 1]] with the scalar c_g deferred to the store
          for (int idx = TID; idx < work; idx += NTHR) {
            int bb = idx / cw, a = idx - bb * cw;
            int b = b0 + bb;
            int i = lat.bond_i[b], j = lat.bond_j[b];
            R t = bsv[b];
            R xi = buf[i * cw + a], xj = buf[j * cw + a];
            buf[i * cw + a] = xi + t * xj;
            buf[j * cw + a] = xj + t * xi;
          }
        } else {
          for (int idx = TID; idx < work; idx += NTHR) {
            int bb = idx / cw, a = idx - bb * cw;
            int b = b0 + bb;
            int i = lat.bond_i[b], j = lat.bond_j[b];
            R c = bcv[b], s = bsv[b];
            R xi = buf[i * cw + a], xj = buf[j * cw + a];
            buf[i * cw + a] = c * xi + s * xj;
            buf[j * cw + a] = s * xi + c * xj;
          }
        }
        __syncthreads();
      }
    }
    const bool scale = sizeof(R) == 8 && op != 0 && lat.unif != 0u;
    const R cpr = (R)lat.cprod;
    for (int idx = TID; idx < tot; idx += NTHR) {
      int i = idx / cw, a = idx - i * cw;
      R v = buf[idx];
      if (scale) v *= cpr;
      if (op == 2 && ceps) v *= ceps[i];
      if (spost) v *= (R)dfac(C, sigma, spost[i]);
      dst[(size_t)i * ld + c0 + a] = v;
    }
    __syncthreads();
  }
}

// W[a*ldw + b] = sum_i A[i*lda + a] * B[i*ldb + b], a < ma, b < mb (rows with
// sub[i] == mval only, when sub is given).  Accumulates in Acc.
template <class Acc, class RA, class RB>
__device__ void gram(const RA* A, int lda, int ma, const RB* B, int ldb, int mb, int N, double* W, int ldw,
                     const int* sub = nullptr, int mval = 0) {
  const int nout = ma * mb;
  if (nout > 0) {
    int tpo = NTHR / nout;
    if (tpo > 32) tpo = 32;
    if (tpo < 1) tpo = 1;
    while (tpo & (tpo - 1)) tpo &= tpo - 1;  // power of two
    const int per = NTHR / tpo;
    for (int o0 = 0; o0 < nout; o0 += per) {
      const int o = o0 + TID / tpo, part = TID % tpo;
      Acc acc = 0;
      int a = 0, b = 0;
      if (o < nout) {
        a = o / mb;
        b = o - a * mb;
        int i = part;
        // four rows' operands in flight before their FMAs (same summation order)
        for (; i + 3 * tpo < N; i += 4 * tpo) {
          Acc a4[4], b4[4];
          bool k4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const size_t r = (size_t)(i + q * tpo);
            a4[q] = (Acc)A[r * lda + a];
            b4[q] = (Acc)B[r * ldb + b];
            k4[q] = !sub || sub[r] == mval;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (k4[q]) acc += a4[q] * b4[q];
        }
        for (; i < N; i += tpo)
          if (!sub || sub[i] == mval) acc += (Acc)A[(size_t)i * lda + a] * (Acc)B[(size_t)i * ldb + b];
      }
      for (int off = tpo >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off, tpo);
      if (part == 0 && o < nout) W[a * ldw + b] = (double)acc;
    }
  }
  __syncthreads();
}

// Gauss-Jordan inverse with partial pivoting of W (m x m, destroyed) into T.
// Returns log|det W| and its sign; a zero pivot sets LQ_ERR_SINGULAR.
static __device__ void inverse(double* W, int ldw, double* T, int ldt, int m, Smem& sm, double* logabs, int* sgn) {
  double* fac = sm.vec + 9 * sm.M;
  for (int idx = TID; idx < m * m; idx += NTHR) {
    int r = idx / m, c = idx - r * m;
    T[r * ldt + c] = (r == c) ? 1.0 : 0.0;
  }
  if (TID == 0) { sm.red[41] = 0.0; sm.ip[0] = 1; sm.ip[1] = 0; }
  __syncthreads();
  for (int col = 0; col < m; ++col) {
    if (TID < 32) {
      double best = -1.0;
      int bi = col;
      for (int r = col + TID; r < m; r += 32) {
        double v = fabs(W[r * ldw + col]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        double ob = __shfl_xor_sync(FULL, best, off);
        int oi = __shfl_xor_sync(FULL, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (TID == 0) { sm.ip[2] = bi; if (!(best > 0.0)) sm.ip[1] = 1; }
    }
    __syncthreads();
    if (sm.ip[1]) break;
    const int p = sm.ip[2];
    if (p != col) {
      for (int c = TID; c < m; c += NTHR) {
        double t = W[col * ldw + c]; W[col * ldw + c] = W[p * ldw + c]; W[p * ldw + c] = t;
        t = T[col * ldt + c]; T[col * ldt + c] = T[p * ldt + c]; T[p * ldt + c] = t;
      }
    }
    __syncthreads();
    const double d = W[col * ldw + col];
    if (TID == 0) {
      if (p != col) sm.ip[0] = -sm.ip[0];
      if (d < 0) sm.ip[0] = -sm.ip[0];
      sm.red[41] += log(fabs(d));
    }
    for (int r = TID; r < m; r += NTHR) fac[r] = (r == col) ? 0.0 : W[r * ldw + col] / d;
    __syncthreads();
    for (int idx = TID; idx < m * m; idx += NTHR) {
      int r = idx / m, c = idx - r * m;
      if (r != col) {
        T[r * ldt + c] -= fac[r] * T[col * ldt + c];
        if (c > col) W[r * ldw + c] -= fac[r] * W[col * ldw + c];
      }
    }
    __syncthreads();
    for (int c = TID; c < m; c += NTHR) {
      T[col * ldt + c] /= d;
      if (c > col) W[col * ldw + c] /= d;
    }
    __syncthreads();
  }
  if (sm.ip[1]) {
    for (int idx = TID; idx < m * m; idx += NTHR) T[(idx / m) * ldt + idx % m] = NAN;
    if (TID == 0) { sm.C->err |= LQ_ERR_SINGULAR; sm.red[41] = -INFINITY; sm.ip[0] = 0; }
  }
  __syncthreads();
  *logabs = sm.red[41];
  *sgn = sm.ip[0];
  __syncthreads();
}

// In-place Cholesky of the upper triangle of W (m x m, ld): W = R^T R.
static __device__ void cholesky(double* W, int ld, int m, Smem& sm) {
  for (int k = 0; k < m; ++k) {
    if (TID == 0) {
      double d = W[k * ld + k];
      if (!(d > 0.0)) { sm.C->err |= LQ_ERR_CHOLESKY; d = 1e-300; }
      W[k * ld + k] = sqrt(d);
    }
    __syncthreads();
    for (int j = k + 1 + TID; j < m; j += NTHR) W[k * ld + j] /= W[k * ld + k];
    __syncthreads();
    const int rem = m - k - 1;
    for (int idx = TID; idx < rem * rem; idx += NTHR) {
      int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j >= i) W[i * ld + j] -= W[k * ld + i] * W[k * ld + j];
    }
    __syncthreads();
  }
}

// X (N x m) <- Q with X = Q V, V upper triangular with a positive diagonal
// (CholeskyQR2, FP64 Gram and factors).  V goes to Vout (m x m, row-major).
template <class R>
__device__ void chol_qr2(const LqChainDev& C, R* X, int m, double* Vout, Smem& sm) {
  PhaseTimer pt_(2);
  if (m == 0) return;
  const int N = C.N, MP = sm.MP;
  double* Rk[2] = {sm.S, sm.S + sm.M * MP};
  for (int pass = 0; pass < 2; ++pass) {
    double* W = Rk[pass];
    gram<double>(X, m, m, X, m, m, N, W, MP);
    cholesky(W, MP, m, sm);
    double* rdiag = sm.vec + 8 * sm.M;
    for (int j = TID; j < m; j += NTHR) rdiag[j] = 1.0 / W[j * MP + j];
    __syncthreads();
    if (m <= LQ_NS_SMALL) {
      // X <- X R^{-1}, row by row (forward substitution on the row vector)
      for (int i = TID; i < N; i += NTHR) {
        R* row = X + (size_t)i * m;
        double y[LQ_NS_SMALL];
#pragma unroll 1
        for (int j = 0; j < m; ++j) {
          double acc = (double)row[j];
          for (int a = 0; a < j; ++a) acc -= y[a] * W[a * MP + j];
          y[j] = acc * rdiag[j];
        }
        for (int j = 0; j < m; ++j) row[j] = (R)y[j];
      }
    } else {
      // R^{-1} (upper triangular) by back substitution, one column per
      // thread; then X <- X R^{-1} with one warp per row, the row staged in
      // shared memory
      double* Ri = sm.S + 2 * sm.M * MP;
      for (int j = TID; j < m; j += NTHR) {
        Ri[j * MP + j] = rdiag[j];
        for (int i = j - 1; i >= 0; --i) {
          double acc = 0.0;
          for (int k = i + 1; k <= j; ++k) acc += W[i * MP + k] * Ri[k * MP + j];
          Ri[i * MP + j] = -acc * rdiag[i];
        }
      }
      __syncthreads();
      const int warp = TID >> 5, lane = TID & 31;
      double* rowbuf = (double*)sm.buf + (size_t)warp * m;
      for (int i = warp; i < N; i += NTHR / 32) {
        R* row = X + (size_t)i * m;
        for (int a = lane; a < m; a += 32) rowbuf[a] = (double)row[a];
        __syncwarp();
        for (int j = lane; j < m; j += 32) {
          double acc = 0.0;
          for (int a = 0; a <= j; ++a) acc = fma(rowbuf[a], Ri[a * MP + j], acc);
          row[j] = (R)acc;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int idx = TID; idx < m * m; idx += NTHR) {
    int a = idx / m, b = idx - a * m;
    double acc = 0.0;
    if (b >= a)
      for (int k = a; k <= b; ++k) acc += Rk[1][a * MP + k] * Rk[0][k * MP + b];
    Vout[idx] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Arithmetic policies of the field-flip loop: native FP64 (OpsF64) or
// double-word FP32 (OpsDW).  Row is the type of the panel rows staged in
// shared memory; T lives in shared memory as double (FP64) or as two float
// planes (double-word).
// ---------------------------------------------------------------------------
template <class RowT> struct OpsF64 {
  typedef double V;
  typedef RowT Row;
  typedef double U;
  struct TRef {
    double* t;
    __device__ V ld(int i) const { return t[i]; }
    __device__ void st(int i, V v) const { t[i] = v; }
  };
  __device__ static TRef tref(Smem& sm, int sg) { return TRef{sm.T[sg]}; }
  __device__ static TRef tref_at(double* Tsg, const Smem&) { return TRef{Tsg}; }
  __device__ static V zero() { return 0.0; }
  __device__ static void acc(V& s, Row a, V t) { s = fma((double)a, t, s); }
  __device__ static void accT(V& s, V t, Row a) { s = fma(t, (double)a, s); }
  __device__ static V finish(V s) { return s; }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V mulr(V a, Row b) { return a * (double)b; }
  __device__ static V fnma(V a, V b, V c) { return fma(-a, b, c); }  // c - a b
  __device__ static V xor_(V a, int o) { return __shfl_xor_sync(FULL, a, o); }
  __device__ static V from_lane(V a, int src) { return __shfl_sync(FULL, a, src); }
  __device__ static V one_plus(V d, V g) { return fma(d, g, 1.0); }
  // d / r without the IEEE division sequence: the hardware reciprocal seed
  // x0 (rcp.approx.ftz.f64) refined by one third-order step of the
  // Newton-Raphson family for 1/r.  With e = 1 - r x0 exact to rounding,
  // 1/r = x0 / (1 - e) = x0 (1 + e + e^2 + ...), so d x0 (1 + e + e^2) leaves
  // a truncation error e^3 (below 2^-60 for a seed good to 2^-20) and a few
  // roundings: at most 4 ulp from the correctly rounded quotient for normal
  // operands (tested against the IEEE quotient on the device).  Four FP64
  // instructions after the seed, against six for two second-order steps.
  __device__ static V div(V d, V r) {
    double x0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x0) : "d"(r));
    const double e = fma(-r, x0, 1.0);
    const double p = fma(e, e, e);
    const double y0 = d * x0;
    return fma(y0, p, y0);
  }
  // 1 / r by the same seed and third-order step: x0 (1 + e + e^2), three FP64
  // instructions after the seed
  __device__ static V rcp(V r) {
    double x0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x0) : "d"(r));
    const double e = fma(-r, x0, 1.0);
    const double p = fma(e, e, e);
    return fma(x0, p, x0);
  }
  __device__ static V of(double x) { return x; }
  __device__ static double pack(V v) { return v; }
  __device__ static V unpack(double v) { return v; }
  __device__ static U make_u(double u) { return u; }
  __device__ static V delta(const LqChainDev& C, bool pos) { return pos ? C.delta_p : C.delta_m; }
  __device__ static V cfac(const LqChainDev& C, bool pos) { return pos ? C.cfac_p : C.cfac_m; }
  // |r| > u, sign and non-finite flags, on the IEEE bit patterns
  __device__ static bool accept(V r, U u, bool* neg, bool* bad) {
    const long long rb = __double_as_longlong(r) & 0x7fffffffffffffffLL;
    *neg = __double_as_longlong(r) < 0;
    *bad = rb >= 0x7ff0000000000000LL;
    return !(*bad) && rb > __double_as_longlong(u);
  }
  // running product of accepted |r| as a mantissa in [0.5, 1) and an exponent
  struct Prod {
    double m;
    long long e;
    __device__ void init() { m = 1.0; e = 0; }
    __device__ void mul_pos(double x) {
      m *= x;
      const long long bits = __double_as_longlong(m);
      e += ((bits >> 52) & 0x7ff) - 1022;
      m = __longlong_as_double((bits & ~(0x7ffLL << 52)) | (1022LL << 52));
    }
    __device__ void mul(V r) { mul_pos(fabs(r)); }
    // multiply by the product held by lane (lane ^ o)
    __device__ void combine_xor(int o) {
      const double om = __shfl_xor_sync(FULL, m, o);
      const long long oe = __shfl_xor_sync(FULL, e, o);
      mul_pos(om);
      e += oe;
    }
    __device__ double log_value() const { return log(m) + (double)e * 0.69314718055994530942; }
  };
};

struct OpsDW {
  typedef dw V;
  typedef float Row;
  typedef dw U;
  struct TRef {
    float* h;
    float* l;
    __device__ V ld(int i) const { return dw{h[i], l[i]}; }
    __device__ void st(int i, V v) const { h[i] = v.h; l[i] = v.l; }
  };
  __device__ static TRef tref(Smem& sm, int sg) {
    float* h = (float*)sm.T[sg];
    return TRef{h, h + (size_t)sm.M * sm.MP};
  }
  __device__ static TRef tref_at(double* Tsg, const Smem& sm) {
    float* h = (float*)Tsg;
    return TRef{h, h + (size_t)sm.M * sm.MP};
  }
  __device__ static V zero() { return dw{0.f, 0.f}; }
  __device__ static void acc(V& s, Row a, V t) { dw_acc(s, a, t); }
  __device__ static void accT(V& s, V t, Row a) { dw_acc(s, a, t); }
  __device__ static V finish(V s) { return fast_two_sum(s.h, s.l); }
  __device__ static V add(V a, V b) { return dw_add(a, b); }
  __device__ static V mul(V a, V b) { return dw_mul(a, b); }
  __device__ static V mulr(V a, Row b) { return dw_mulf(a, b); }
  __device__ static V fnma(V a, V b, V c) { return dw_add(c, dw_neg(dw_mul(a, b))); }
  __device__ static V xor_(V a, int o) { return dw_shfl_xor(a, o); }
  __device__ static V from_lane(V a, int src) { return dw_shfl(a, src); }
  __device__ static V one_plus(V d, V g) { return dw_add(dw{1.f, 0.f}, dw_mul(d, g)); }
  __device__ static V div(V d, V r) { return dw_div(d, r); }
  __device__ static V rcp(V r) { return dw_div(dw{1.f, 0.f}, r); }
  __device__ static V of(double x) { return dw_from(x); }
  __device__ static double pack(V v) {
    return __longlong_as_double(((long long)__float_as_int(v.l) << 32) | (unsigned)__float_as_int(v.h));
  }
  __device__ static V unpack(double x) {
    const long long b = __double_as_longlong(x);
    return dw{__int_as_float((int)(b & 0xffffffff)), __int_as_float((int)(b >> 32))};
  }
  __device__ static U make_u(double u) { return dw_from(u); }
  __device__ static V delta(const LqChainDev& C, bool pos) {
    return pos ? dw{C.dw_delta_p[0], C.dw_delta_p[1]} : dw{C.dw_delta_m[0], C.dw_delta_m[1]};
  }
  __device__ static V cfac(const LqChainDev& C, bool pos) {
    return pos ? dw{C.dw_cfac_p[0], C.dw_cfac_p[1]} : dw{C.dw_cfac_m[0], C.dw_cfac_m[1]};
  }
  __device__ static bool accept(V r, U u, bool* neg, bool* bad) {
    *neg = r.h < 0.f;
    *bad = !(fabsf(r.h) <= 3.4e38f);
    const dw ra = *neg ? dw_neg(r) : r;
    return !(*bad) && dw_gt(ra, u);
  }
  struct Prod {
    dw m;
    long long e;
    __device__ void init() { m = dw{1.f, 0.f}; e = 0; }
    __device__ void mul_pos(dw x) {
      m = dw_mul(m, x);
      // exact rescale by a power of two: keep m.h in [0.5, 1)
      const int ex = ((__float_as_int(m.h) >> 23) & 0xff) - 126;
      const float sc = __int_as_float((127 - ex) << 23);
      m.h *= sc;
      m.l *= sc;
      e += ex;
    }
    __device__ void mul(V r) { mul_pos(r.h < 0.f ? dw_neg(r) : r); }
    __device__ void combine_xor(int o) {
      const dw om = dw_shfl_xor(m, o);
      const long long oe = __shfl_xor_sync(FULL, e, o);
      mul_pos(om);
      e += oe;
    }
    __device__ double log_value() const { return log((double)m.h + (double)m.l) + (double)e * 0.69314718055994530942; }
  };
};

// ---------------------------------------------------------------------------
// Field flips over all sites of slice l (ascending) by the submatrix update:
// windows of K consecutive sites.  With X = R~_W T (rows x_t), Y = T L~_W
// (columns y_t) and the window Green's block G = X L~_W (K x K), a flip at
// window site t has ratio factor 1 + Delta G[t][t] and, by Sherman-Morrison,
//   T' = T - c y_t x_t^T,   c = Delta / (1 + Delta G[t][t]),
// which changes the rest of the window as
//   G[u][v] -= c G[u][t] G[t][v],  x_j -= c G[j][t] x_t,  y_j -= c G[t][j] y_t  (u, v, j > t).
// So the serial chain of a site is G[t][t], the ratio, the exchange of the
// two spins' factors and one K x K rank-1 update; the m-length dot products
// are batched per window, the x/y recurrences run after the window's sites,
// and T takes the window's rank-1 terms at its end.
//
// For m <= 32 particles per spin the window is K = 4 sites and the serial
// chain of BOTH spins runs on one leader warp (lanes 0-15 spin up, 16-31 spin
// down, one block element per lane).  The other warps (the workers) run one
// window behind it, so that the leader never waits for the dense work:
//   leader, window w:  the chain of w's sites on its block G_w (in registers),
//                      then the c-scaled factors CG_w (CG[j][t] = c_t G[j][t],
//                      CG[t][j] = c_t G[t][j], j > t) for the workers, then
//                      the next window's block from three K x K blocks that
//                      the workers formed against T_w (the T before window w):
//                        A1 = Z L~_{w+1} ... rows of w+1, columns of w,
//                        A2 = X_w L~_{w+1},  B = Z L~_{w+1} (rows and columns of w+1),
//                      Z = R~_{w+1} T_w.  Window w's flips act on them by the
//                      same recurrences as on x and y,
//                        A1[u][j] -= CG[t][j] A1[u][t],  A2[j][v] -= CG[j][t] A2[t][v]  (j > t),
//                      and G_{w+1} = B - sum_t c_t A1[u][t] A2[t][v]: eleven
//                      FP64 instructions on the leader instead of the window
//                      products, the recurrences and the T update.
//   workers, window w: (with CG_{w-1}) the x/y recurrences of window w-1 and
//                      T_w = T_{w-1} - sum_t (c_t y_t) x_t^T, then x_t, y_t
//                      of window w, z of window w+1 and the three blocks.
// They meet at named barriers: the leader arrives at P once CG_w is stored
// and the workers wait there before window w-1's update; the workers arrive
// at Q once the blocks of window w+1 are stored and the leader waits there.
// Each alternates between two barrier ids and two buffers by window parity,
// so neither side can arrive twice at one barrier before the other has
// passed it.  Each chunk of staged sites starts with the whole CTA forming
// x, y and the block of its window 0 and the three blocks of its window 1.
// On GB300 an FP64 warp instruction occupies its sub-partition for tens of
// cycles whatever the number of active lanes, so the leader's chain is the
// count of dependent FP64 instructions on one warp: this path keeps it at the
// ratio, the quotient, the product and one update per site for both spins at
// once, and moves every m-length product off it.
// ---------------------------------------------------------------------------
// Named barriers with compile-time ids (so the kernel reserves only the ids it
// names).  Ids of the pipelined pair path: 1 and 2 (P: a window's CG stored;
// the leader arrives, the workers wait), 3 and 4 (Q: the next window's blocks
// stored; the workers arrive, the leader waits), 5 (the workers among
// themselves).  The m > 32 path uses 1-3 in another phase of the sweep, in
// which every instance completes before it returns.
template <int ID> __device__ __forceinline__ void nbar_sync(int n) {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(n) : "memory");
}
template <int ID> __device__ __forceinline__ void nbar_arrive(int n) {
  asm volatile("bar.arrive %0, %1;" ::"n"(ID), "r"(n) : "memory");
}
#define LQ_BAR_P 1
#define LQ_BAR_Q 3
#define LQ_BAR_W 5
// the barrier of parity p (0 or 1) of a pair of ids (warp-uniform branch)
#define LQ_NBAR_SYNC(B, p, n) ((p) ? nbar_sync<(B) + 1>(n) : nbar_sync<(B)>(n))
#define LQ_NBAR_ARRIVE(B, p, n) ((p) ? nbar_arrive<(B) + 1>(n) : nbar_arrive<(B)>(n))

template <class R, class Ops, int MT, bool BIG>
__device__ void flip_slice_pair(LqChainDev& C, int l, R* Rp0, R* Rp1, const R* Lp0, const R* Lp1, uint32_t tag,
                                Smem& sm) {
  PhaseTimer pt_(PH_FLIP);
  typedef typename Ops::V V;
  typedef typename Ops::Row Row;
  typedef typename Ops::U U;
  constexpr int K = 4, KK = K * K;
  constexpr int NT = 2 * MT * MT;  // T elements of both spins
  // one accumulator per m-long product: on GB300 a dependent FP64 FMA costs
  // its sub-partition the same 64 cycles as an independent one, so partial
  // sums would only add instructions
  const int N = C.N, MP = sm.MP;
  const int m0 = C.ns[0], m1 = C.ns[1];
  const size_t per_site = (size_t)4 * MP * sizeof(Row) + 8 + sizeof(U) + 4 + 4;
  int cs = (int)(sm.buf_bytes / per_site);
  if (cs > 512) cs = 512;
  Row* rrow = plan_ptr<BIG>((Row*)sm.buf);
  Row* lrow = rrow + (size_t)2 * cs * MP;
  double* racc = (double*)(lrow + (size_t)2 * cs * MP);  // accepted ratios (packed), multiplied per chunk
  U* uni = (U*)(racc + cs);
  int* sf = (int*)(uni + cs);
  int* af = sf + cs;
  const Row opf_p = (Row)C.opd_p, opf_m = (Row)C.opd_m;
  // The ratio of a flip at site t is dd(s) (1/Delta_up + G_up[t][t]) (1/Delta_dn + G_dn[t][t]) with
  // dd(s) = Delta_up Delta_dn (times the charge channel's constant), and c = Delta/(1 + Delta G[t][t])
  // = 1/(1/Delta + G[t][t]).  So the chain forms 1/Delta + G[t][t] (one add), its reciprocal and the
  // product of the two spins' factors; |dd(s)| moves into the Metropolis threshold (u/|dd(s)|, formed
  // at staging), its sign into the sign bit and its magnitude into the chunk's weight product.  Without
  // an interaction (lambda = 0) 1/Delta and dd are replaced by 1 and the window block by 0, so that
  // every ratio is exactly 1.
  const bool lam0 = C.lambda == 0.0;
  // dd(s) for s > 0 (dd_p) and s < 0 (dd_m)
  const double dd_p = lam0 ? 1.0 : C.charge ? C.delta_p * C.delta_p * C.cfac_p : C.delta_p * C.delta_m;
  const double dd_m = lam0 ? 1.0 : C.charge ? C.delta_m * C.delta_m * C.cfac_m : C.delta_p * C.delta_m;
  const double thr_p = 1.0 / fabs(dd_p), thr_m = 1.0 / fabs(dd_m);
  const int ddn = (dd_p < 0.0 ? 1 : 0) | (dd_m < 0.0 ? 2 : 0);
  // 1/Delta for s sp > 0 and < 0, formed once per slice (an IEEE division is a dozen FP64 instructions)
  const V id_p = Ops::of(lam0 ? 1.0 : 1.0 / C.delta_p), id_m = Ops::of(lam0 ? 1.0 : 1.0 / C.delta_m);
  const int warp = TID >> 5, lane = TID & 31;
  const int lw = sm.ip[14], mate = sm.ip[15];
  const bool leader = warp == lw;
  // workers: the other warps (NWK threads, all in the workers' barriers).  The FP64 work goes to the
  // warps of fmask, renumbered 0 .. NFW/32 - 1; the others' indexes start beyond every element count
  // (no element, no recurrence task).  For up to 8 particles per spin (one round of window products
  // on four warps) these are the warps on the two sub-partitions that neither resident CTA leads
  // from (sm.ip[13]), so that FP64 bursts of the workers never queue ahead of a leader's chain;
  // otherwise every worker but the leader's mate.
  unsigned fmask = ((1u << (NTHR >> 5)) - 1u) & ~(1u << lw);
  if (mate >= 0) fmask &= ~(1u << mate);
  if (MT <= 8 && __popc((unsigned)sm.ip[13]) == 4) fmask = (unsigned)sm.ip[13];
  const int NWK = NTHR - 32, NFW = 32 * __popc(fmask);
  const bool fwk = (fmask >> warp) & 1u;
  const int fw = fwk ? __popc(fmask & ((1u << warp) - 1u)) : NFW / 32;
  const int wt = fwk ? fw * 32 + lane : (1 << 30);
  V* const win0 = plan_ptr<BIG>((V*)sm.win);
  double* const T0s = plan_ptr<BIG>(sm.T[0]);
  double* const T1s = plan_ptr<BIG>(sm.T[1]);
  // window buffers of spin sg: X, Y, Z (K x MP each), then by window parity p the blocks A1, A2, B
  // (K x K each), the c-scaled factors CG (K x K) and c (K)
  auto Xb = [&](int sg) { return win0 + (size_t)sg * LQ_WIN_ELEMS(MP); };
  auto Yb = [&](int sg) { return Xb(sg) + K * MP; };
  auto Zb = [&](int sg) { return Yb(sg) + K * MP; };
  auto BLb = [&](int sg, int p, int kind) { return Zb(sg) + K * MP + (p * 3 + kind) * KK; };
  auto CGb = [&](int sg, int p) { return Zb(sg) + K * MP + 6 * KK + p * KK; };
  auto cb = [&](int sg, int p) { return Zb(sg) + K * MP + 8 * KK + p * K; };

  // x_t = R~_t T and y_t = T L~_t of the window at t0 (kw sites), z_t = R~_t T of the window at t0 + K
  // (kz sites); element (sg, kind, t, b), kind 0 x, 1 y, 2 z
  auto products = [&](int t0, int kw, int kz, int tid, int nth) {
    constexpr int NE = 2 * 3 * K * MT;
#pragma unroll 1
    for (int e = tid; e < NE; e += nth) {
      const int b = e % MT, t = (e / MT) % K, kind = (e / (MT * K)) % 3, sg = e / (3 * MT * K);
      const int m = sg ? m1 : m0;
      if (t < (kind == 2 ? kz : kw) && b < m) {
        const typename Ops::TRef T = Ops::tref_at(sg ? T1s : T0s, sm);
        const Row* row = (kind == 1 ? lrow : rrow) + ((size_t)sg * cs + t0 + (kind == 2 ? K : 0) + t) * MP;
        // operands of CH terms loaded ahead of their FMAs, so that the
        // loads overlap and the dependent FMA chain does not wait on each
        constexpr int CH = MT < 8 ? MT : 8;
        V acc = Ops::zero();
#pragma unroll
        for (int a0 = 0; a0 < MT; a0 += CH) {
          V tv[CH];
          Row rv[CH];
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            const int a = a0 + q;
            tv[q] = a < m ? T.ld(kind == 1 ? b * MP + a : a * MP + b) : Ops::zero();
            rv[q] = a < m ? row[a] : (Row)0;
          }
#pragma unroll
          for (int q = 0; q < CH; ++q)
            if (a0 + q < m) {
              if (kind == 1) Ops::accT(acc, tv[q], rv[q]);
              else Ops::acc(acc, rv[q], tv[q]);
            }
        }
        (kind == 0 ? Xb(sg) : kind == 1 ? Yb(sg) : Zb(sg))[t * MP + b] = Ops::finish(acc);
      }
    }
  };
  // K x K blocks (m-long dots of a window vector with a staged L~ row): kind 0 A1 = Z L~_{t0+K},
  // 1 A2 = X L~_{t0+K}, 2 B = Z L~_{t0+K}... rows of Z or X, columns at t0 (A1) or t0 + K (A2, B),
  // into parity p; kind 3 (with g0) the window's own block X L~_{t0} into the B slot of parity 0.
  // Entries outside the windows are zero.
  auto blocks = [&](int t0, int kw, int kz, int p, bool g0, int tid, int nth) {
    const int nk = g0 ? 4 : 3;
#pragma unroll 1
    for (int e = tid; e < 2 * nk * KK; e += nth) {
      const int v = e % K, u = (e / K) % K, kind = (e / KK) % nk, sg = e / (nk * KK);
      const int m = sg ? m1 : m0;
      const bool rz = kind == 0 || kind == 2, cz = kind == 1 || kind == 2;
      V acc = Ops::zero();
      if (u < (rz ? kz : kw) && v < (cz ? kz : kw)) {
        const V* xr = (rz ? Zb(sg) : Xb(sg)) + u * MP;
        const Row* lr = lrow + ((size_t)sg * cs + t0 + (cz ? K : 0) + v) * MP;
        constexpr int CH = MT < 8 ? MT : 8;
#pragma unroll
        for (int b0 = 0; b0 < MT; b0 += CH) {
          V xv[CH];
          Row lv[CH];
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            xv[q] = b0 + q < m ? xr[b0 + q] : Ops::zero();
            lv[q] = b0 + q < m ? lr[b0 + q] : (Row)0;
          }
#pragma unroll
          for (int q = 0; q < CH; ++q)
            if (b0 + q < m) Ops::accT(acc, xv[q], lv[q]);
        }
        acc = Ops::finish(acc);
      }
      (kind == 3 ? BLb(sg, 0, 2) : BLb(sg, p, kind))[u * K + v] = acc;
    }
  };
  // the x (xy = 0) or y (xy = 1) recurrences of spin sg over a window of kw sites with the factors
  // of parity p: x_j -= CG[j][t] x_t, y_j -= CG[t][j] y_t (j > t, t ascending), then y_t <- c_t y_t;
  // one warp, element (j, b)
  auto recur = [&](int kw, int p, int sg, int xy) {
    const int m = sg ? m1 : m0;
    V* Wm = xy ? Yb(sg) : Xb(sg);
    const V* CG = CGb(sg, p);
    constexpr int RE = (K * MT + 31) / 32;
    for (int t = 0; t + 1 < kw; ++t) {
#pragma unroll
      for (int it = 0; it < RE; ++it) {
        const int e = lane + 32 * it, j = e / MT, b = e % MT;
        if (e < K * MT && j > t && j < kw && b < m)
          Wm[j * MP + b] = Ops::fnma(xy ? CG[t * K + j] : CG[j * K + t], Wm[t * MP + b], Wm[j * MP + b]);
      }
      __syncwarp();
    }
    if (xy) {
      const V* cw = cb(sg, p);
#pragma unroll
      for (int it = 0; it < RE; ++it) {
        const int e = lane + 32 * it, j = e / MT, b = e % MT;
        if (e < K * MT && j < kw && b < m) Wm[j * MP + b] = Ops::mul(cw[j], Wm[j * MP + b]);
      }
    }
  };
  // T <- T - sum_t (c_t y_t) x_t^T over a window of kw sites, element (sg, a, b)
  auto tupdate = [&](int kw, int tid, int nth) {
#pragma unroll 1
    for (int e = tid; e < NT; e += nth) {
      const int b = e % MT, a = (e / MT) % MT, sg = e / (MT * MT);
      const int m = sg ? m1 : m0;
      if (a < m && b < m) {
        const typename Ops::TRef T = Ops::tref_at(sg ? T1s : T0s, sm);
        const V* Xs = Xb(sg);
        const V* Ys = Yb(sg);
        V ys[K], xs[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
          ys[t] = t < kw ? Ys[t * MP + a] : Ops::zero();
          xs[t] = t < kw ? Xs[t * MP + b] : Ops::zero();
        }
        V tv = T.ld(a * MP + b);
#pragma unroll
        for (int t = 0; t < K; ++t)
          if (t < kw) tv = Ops::fnma(ys[t], xs[t], tv);
        T.st(a * MP + b, tv);
      }
    }
  };
  // the x/y recurrences (four warp tasks: spin x {x, y}) and the T update of a finished window
  auto window_update = [&](int kw, int p) {
    for (int d = fw; d < 4 && fw < NFW / 32; d += NFW / 32) recur(kw, p, d >> 1, d & 1);
    nbar_sync<LQ_BAR_W>(NWK);
    tupdate(kw, wt, NFW);
  };

  // sub-phase cycles: staging and write-back, the chunk's first window products, the leader's chains
  // (its own clock) and the rest of the window loop (thread 0's clock, less the chains)
  __shared__ long long tsub, tchain;
  if (TID == 0) tsub = clock64();
  auto lap = [&](int k) {
    if (TID == 0) {
      const long long t = clock64();
      C.prof[k] += t - tsub;
      tsub = t;
    }
  };
  for (int i0 = 0; i0 < N; i0 += cs) {
    const int cn = min(cs, N - i0);
    for (int sg = 0; sg < 2; ++sg) {
      const int m = sg ? m1 : m0;
      const R* rp = sg ? Rp1 : Rp0;
      const R* lp = sg ? Lp1 : Lp0;
      Row* rr = rrow + (size_t)sg * cs * MP;
      Row* ll = lrow + (size_t)sg * cs * MP;
      // four rows' loads in flight per thread before their stores
      const int a = TID % MT, step = NTHR / MT;
      int ii = TID / MT;
      for (; ii + 3 * step < cn; ii += 4 * step) {
        R r4[4], l4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const size_t g = (size_t)(i0 + ii + q * step) * m + a;
          r4[q] = a < m ? rp[g] : (R)0;
          l4[q] = a < m ? lp[g] : (R)0;
        }
        if (a < m) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            rr[(size_t)(ii + q * step) * MP + a] = (Row)r4[q];
            ll[(size_t)(ii + q * step) * MP + a] = (Row)l4[q];
          }
        }
      }
      for (; ii < cn; ii += step) {
        if (a < m) {
          rr[(size_t)ii * MP + a] = (Row)rp[(size_t)(i0 + ii) * m + a];
          ll[(size_t)ii * MP + a] = (Row)lp[(size_t)(i0 + ii) * m + a];
        }
      }
    }
    for (int ii = TID; ii < cn; ii += NTHR) {
      uint32_t w[4];
      philox(C.chain_id, C.sweep, (tag << 24) | (uint32_t)l, (uint32_t)(i0 + ii), C.key0, C.key1, w);
      const int s = C.s[(size_t)l * N + i0 + ii];
      uni[ii] = Ops::make_u(u53(w[0], w[1]) * (s > 0 ? thr_p : thr_m));
      sf[ii] = s;
    }
    if (TID == 0) tchain = 0;
    __syncthreads();
    lap(8);
    const int nw = (cn + K - 1) / K;
    // the chunk's first window: x, y of window 0 and z of window 1, then window 0's block and the
    // blocks of window 1, by the whole CTA
    {
      const int kw = min(K, cn), kz = nw > 1 ? min(K, cn - K) : 0;
      products(0, kw, kz, TID, NTHR);
      __syncthreads();
      blocks(0, kw, kz, 1, true, TID, NTHR);
      __syncthreads();
    }
    lap(9);
    if (leader) {
      int wsign = 1, nacc = 0, nbad = 0;  // kept by lane 0
      // lane 16 h + 4 u + v holds G[u][v] of spin h in a register for the
      // whole window: every read of the serial chain is a shuffle
      const int h = lane >> 4, hl = lane & 15;
      const int m = h ? m1 : m0;
      const int u = hl >> 2, v = hl & 3, hb = lane & 16;
      const bool upd = m > 0 && !lam0;
      const int sp = C.charge ? 1 : (h == 0 ? 1 : -1);
      V G = upd ? BLb(h, 0, 2)[u * K + v] : Ops::zero();
      long long tch = 0;
      for (int w = 0; w < nw; ++w) {
        const int t0 = w * K, kw = min(K, cn - t0);
        const long long tl0 = clock64();
        int sacc = 0, sbad = 0, sneg = 0;
        // the window's fields and uniforms, loaded before the chain starts
        int sw[K];
        U uw[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
          sw[t] = t < kw ? sf[t0 + t] : 1;
          uw[t] = uni[t0 + (t < kw ? t : 0)];
        }
        // c of site v (cv) and of site u (cu) of this half's spin, 0 when not flipped
        V cv = Ops::zero(), cu = Ops::zero();
#pragma unroll
        for (int t = 0; t < K; ++t) {
          if (t < kw) {
            const int ii = t0 + t;
            const int s = sw[t];
            const U uu = uw[t];
            const V idd = (sp * s > 0) ? id_p : id_m;
            // G[u][t] and G[t][v] are final for this step (rows and columns
            // below t only change at later steps)
            const V gut = Ops::from_lane(G, hb + 4 * u + t);
            const V gtv = Ops::from_lane(G, hb + 4 * t + v);
            // every lane takes part in every shuffle (the halves' spins may differ
            // in m; an empty spin's block is zero)
            const V g = Ops::from_lane(G, hb + 5 * t);
            const V wp = Ops::mul(gut, gtv);  // G[u][t] G[t][v], independent of this site's decision
            const V rs = Ops::add(idd, g);     // 1/Delta_sigma + G_tt of this half's spin
            const V c = Ops::rcp(rs);          // Delta/(1 + Delta G_tt), used if accepted
            const V ro = Ops::xor_(rs, 16);    // the other spin's factor
            const V rup = h ? ro : rs, rdn = h ? rs : ro;
            const V r = Ops::mul(rup, rdn);    // ratio / dd(s), the same in both halves
            bool neg, bad;
            const bool acc = Ops::accept(r, uu, &neg, &bad);
            neg ^= (ddn >> (s > 0 ? 0 : 1)) & 1;
            const bool flip = acc && upd;
            if (flip && u > t && v > t) G = Ops::fnma(c, wp, G);
            const V cf = flip ? c : Ops::zero();
            if (v == t) cv = cf;
            if (u == t) cu = cf;
            sacc |= acc << t;
            sneg |= neg << t;
            sbad |= bad << t;
            if (lane == t) racc[ii] = Ops::pack(r);
          }
        }
        if (lane < kw) af[t0 + lane] = (sacc >> lane) & 1;
        if (lane == 0) {
          nacc += __popc(sacc);
          nbad += __popc(sbad);
          if (__popc(sacc & sneg) & 1) wsign = -wsign;
        }
        // c-scaled factors of the recurrences: CG[j][t] = c_t G[j][t] (lane (j, t), j > t) and
        // CG[t][j] = c_t G[t][j] (lane (t, j)), for the workers and the next block
        const V cg = (u < kw && v < kw && u != v) ? Ops::mul(u > v ? cv : cu, G) : Ops::zero();
        CGb(h, w & 1)[u * K + v] = cg;
        if (u == 0) cb(h, w & 1)[v] = cv;
        __syncwarp();
        LQ_NBAR_ARRIVE(LQ_BAR_P, w & 1, NTHR);
        tch += clock64() - tl0;
        if (w + 1 < nw) {
          // the next window's block: the three blocks against T_w, taken through this window's flips
          const int p = (w + 1) & 1;
          if (w >= 1) LQ_NBAR_SYNC(LQ_BAR_Q, p, NTHR);  // window 1's blocks came with window 0's
          V a1 = BLb(h, p, 0)[u * K + v], a2 = BLb(h, p, 1)[u * K + v];
          const V bb = BLb(h, p, 2)[u * K + v];
#pragma unroll
          for (int t = 0; t + 1 < K; ++t) {
            if (t + 1 < kw) {
              const V cgtv = Ops::from_lane(cg, hb + 4 * t + v);  // CG[t][v]
              const V cgut = Ops::from_lane(cg, hb + 4 * u + t);  // CG[u][t]
              const V a1ut = Ops::from_lane(a1, hb + 4 * u + t);
              const V a2tv = Ops::from_lane(a2, hb + 4 * t + v);
              if (v > t) a1 = Ops::fnma(cgtv, a1ut, a1);
              if (u > t) a2 = Ops::fnma(cgut, a2tv, a2);
            }
          }
          a1 = Ops::mul(cv, a1);  // c_t A1[u][t] (t = v)
          V gn = bb;
#pragma unroll
          for (int t = 0; t < K; ++t)
            if (t < kw) gn = Ops::fnma(Ops::from_lane(a1, hb + 4 * u + t), Ops::from_lane(a2, hb + 4 * t + v), gn);
          G = upd ? gn : Ops::zero();
        }
      }
      if (lane == 0) tchain = tch;
      // product of the chunk's accepted ratios, lane-parallel
      typename Ops::Prod wpr;
      wpr.init();
      const V add_p = Ops::of(fabs(dd_p)), add_m = Ops::of(fabs(dd_m));
      for (int ii = lane; ii < cn; ii += 32)
        if (af[ii]) wpr.mul(Ops::mul(Ops::unpack(racc[ii]), sf[ii] > 0 ? add_p : add_m));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wpr.combine_xor(o);
      if (lane == 0) {
        C.cnt[0] += cn;
        C.cnt[1] += nacc;
        C.logw += wpr.log_value();
        if (wsign < 0) C.sign = -C.sign;
        if (nbad) C.err |= LQ_ERR_NONFINITE;
      }
    } else {
      for (int w = 1; w < nw; ++w) {
        const int t0 = w * K, kw = min(K, cn - t0), kz = w + 1 < nw ? min(K, cn - t0 - K) : 0;
        LQ_NBAR_SYNC(LQ_BAR_P, (w - 1) & 1, NTHR);  // CG of window w - 1
        window_update(K, (w - 1) & 1);
        nbar_sync<LQ_BAR_W>(NWK);
        products(t0, kw, kz, wt, NFW);
        if (w + 1 < nw) {
          nbar_sync<LQ_BAR_W>(NWK);
          blocks(t0, kw, kz, (w + 1) & 1, false, wt, NFW);
          LQ_NBAR_ARRIVE(LQ_BAR_Q, (w + 1) & 1, NTHR);
        }
      }
      LQ_NBAR_SYNC(LQ_BAR_P, (nw - 1) & 1, NTHR);
      window_update(cn - (nw - 1) * K, (nw - 1) & 1);
    }
    __syncthreads();
    if (TID == 0) {
      const long long t = clock64();
      C.prof[10] += tchain;
      C.prof[11] += (t - tsub) - tchain;
      tsub = t;
    }
    // rows back to the panel; accepted sites scale their row by 1 + Delta_sigma
    for (int sg = 0; sg < 2; ++sg) {
      const int m = sg ? m1 : m0;
      const int sp = C.charge ? 1 : (sg == 0 ? 1 : -1);
      R* rp = sg ? Rp1 : Rp0;
      const Row* rr = rrow + (size_t)sg * cs * MP;
      for (int ii = TID / MT; ii < cn; ii += NTHR / MT) {
        const int a = TID % MT;
        if (a < m) {
          Row v = rr[(size_t)ii * MP + a];
          if (af[ii]) v *= (sp * sf[ii] > 0) ? opf_p : opf_m;
          rp[(size_t)(i0 + ii) * m + a] = (R)v;
        }
      }
    }
    for (int ii = TID; ii < cn; ii += NTHR)
      if (af[ii]) C.s[(size_t)l * N + i0 + ii] = (int8_t)(-sf[ii]);
    __syncthreads();
    lap(8);
  }
}

__device__ __forceinline__ void bar_group(int sg) { asm volatile("bar.sync %0, 128;" ::"r"(2 + sg) : "memory"); }

// ---------------------------------------------------------------------------
// Field flips for m > 32: the same submatrix update with each spin on a group
// of four warps (spin = warp / 4).  The window's dense parts run over the
// group's 128 threads, each owning whole columns:
//   X = R~_W T  (thread owns column b of X: T column b, coalesced),
//   Y = T L~_W  (thread owns row b of T),
//   the x/y recurrences (thread owns column b of X and of Y: no barrier),
//   T -= sum_t (c_t y_t) x_t^T  (thread owns column b of T);
// the serial per-site chain (ratio, the two spins' exchange, the K x K
// block's rank-1 updates) runs on the group's first warp, as in the small path.
// ---------------------------------------------------------------------------
// x_t = R_t T and y_t = T L_t for the KT window sites tlo.. (KT a compile-time
// count, so no FP64 instruction issues for a site the thread does not own):
// the calling thread owns column b of X (T column b) and row b of T.
template <class Ops, int KT>
__device__ __forceinline__ void window_xy(const typename Ops::TRef& T, const typename Ops::Row* rbase,
                                          const typename Ops::Row* lbase, typename Ops::V* Xw, typename Ops::V* Yw,
                                          int t0, int tlo, int kw, int m, int MP, int b0, int bstep) {
  typedef typename Ops::V V;
  const int nt = min(KT, kw - tlo);
  if (nt <= 0) return;
  for (int b = b0; b < m; b += bstep) {
    V xa[KT], ya[KT];
#pragma unroll
    for (int t = 0; t < KT; ++t) { xa[t] = Ops::zero(); ya[t] = Ops::zero(); }
    if (nt == KT) {
      for (int a = 0; a < m; ++a) {
        const V tc = T.ld(a * MP + b), tr = T.ld(b * MP + a);
#pragma unroll
        for (int t = 0; t < KT; ++t) {
          Ops::acc(xa[t], rbase[(size_t)(t0 + tlo + t) * MP + a], tc);
          Ops::accT(ya[t], tr, lbase[(size_t)(t0 + tlo + t) * MP + a]);
        }
      }
    } else {  // ragged last window of a chunk
      for (int a = 0; a < m; ++a) {
        const V tc = T.ld(a * MP + b), tr = T.ld(b * MP + a);
        for (int t = 0; t < nt; ++t) {
          Ops::acc(xa[t], rbase[(size_t)(t0 + tlo + t) * MP + a], tc);
          Ops::accT(ya[t], tr, lbase[(size_t)(t0 + tlo + t) * MP + a]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KT; ++t)
      if (t < nt) {
        Xw[(tlo + t) * MP + b] = Ops::finish(xa[t]);
        Yw[(tlo + t) * MP + b] = Ops::finish(ya[t]);
      }
  }
}

template <class R, class Ops>
__device__ void flip_slice_big(LqChainDev& C, int l, R* Rp0, R* Rp1, const R* Lp0, const R* Lp1, uint32_t tag,
                               Smem& sm) {
  PhaseTimer pt_(PH_FLIP);
  typedef typename Ops::V V;
  typedef typename Ops::Row Row;
  typedef typename Ops::U U;
  constexpr int K = LQ_WIN, KP = LQ_WIN + 1;
  constexpr int GE = (K * K) / 32;
  const int N = C.N, MP = sm.MP;
  const int m0 = C.ns[0], m1 = C.ns[1];
  const size_t per_site = (size_t)4 * MP * sizeof(Row) + 8 + sizeof(U) + 4 + 4;
  int cs = (int)(sm.buf_bytes / per_site);
  if (cs > 512) cs = 512;
  Row* rrow = (Row*)sm.buf;
  Row* lrow = rrow + (size_t)2 * cs * MP;
  double* racc = (double*)(lrow + (size_t)2 * cs * MP);
  U* uni = (U*)(racc + cs);
  int* sf = (int*)(uni + cs);
  int* af = sf + cs;
  const Row opf_p = (Row)C.opd_p, opf_m = (Row)C.opd_m;
  const int warp = TID >> 5, lane = TID & 31;
  const int sg = warp >> 2, gt = TID & 127;
  const bool leader = (warp & 3) == 0;
  for (int i0 = 0; i0 < N; i0 += cs) {
    const int cn = min(cs, N - i0);
    for (int s2 = 0; s2 < 2; ++s2) {
      const int m = s2 ? m1 : m0;
      const R* rp = s2 ? Rp1 : Rp0;
      const R* lp = s2 ? Lp1 : Lp0;
      Row* rr = rrow + (size_t)s2 * cs * MP;
      Row* ll = lrow + (size_t)s2 * cs * MP;
      for (int idx = TID; idx < cn * m; idx += NTHR) {
        const int ii = idx / m, a = idx - ii * m;
        rr[(size_t)ii * MP + a] = (Row)rp[(size_t)(i0 + ii) * m + a];
        ll[(size_t)ii * MP + a] = (Row)lp[(size_t)(i0 + ii) * m + a];
      }
    }
    for (int ii = TID; ii < cn; ii += NTHR) {
      uint32_t w[4];
      philox(C.chain_id, C.sweep, (tag << 24) | (uint32_t)l, (uint32_t)(i0 + ii), C.key0, C.key1, w);
      uni[ii] = Ops::make_u(u53(w[0], w[1]));
      sf[ii] = C.s[(size_t)l * N + i0 + ii];
    }
    __syncthreads();
    {
      const int m = sg ? m1 : m0;
      const typename Ops::TRef T = Ops::tref(sm, sg);
      const bool upd = m > 0 && C.lambda != 0.0;
      const int sp = C.charge ? 1 : (sg == 0 ? 1 : -1);
      const V d_p = Ops::delta(C, true), d_m = Ops::delta(C, false);
      const V cf_p = Ops::cfac(C, true), cf_m = Ops::cfac(C, false);
      V* Xw = (V*)sm.win + (size_t)sg * LQ_WIN_ELEMS(MP);
      V* Yw = Xw + K * MP;
      V* Gw = Yw + K * MP;
      V* cw = Gw + K * KP;
      const Row* rbase = rrow + (size_t)sg * cs * MP;
      const Row* lbase = lrow + (size_t)sg * cs * MP;
      int wsign = 1, nacc = 0, nbad = 0;
      for (int t0 = 0; t0 < cn; t0 += K) {
        const int kw = min(K, cn - t0);
        // x_t = R_t T (thread owns column b) and y_t = T L_t (thread owns row b
        // of T).  With m <= 64 the group's two halves take the window's first
        // and last K/2 sites, so every thread works.
        const int TG = m <= 64 ? 2 : 1, KT = K / TG;
        const int bstep = 128 / TG, tg = gt / bstep, tlo = tg * KT;
        if (TG == 2)
          window_xy<Ops, K / 2>(T, rbase, lbase, Xw, Yw, t0, tlo, kw, m, MP, gt % bstep, bstep);
        else
          window_xy<Ops, K>(T, rbase, lbase, Xw, Yw, t0, tlo, kw, m, MP, gt % bstep, bstep);
        bar_group(sg);
        // G[u][v] = x_u . L_v (four partial sums: the m-long chain is latency bound)
        if (gt < K * K) {
          const int u = gt / K, v = gt % K;
          if (u < kw && v < kw) {
            const Row* lr = lbase + (size_t)(t0 + v) * MP;
            const V* xr = Xw + u * MP;
            V g0 = Ops::zero(), g1 = Ops::zero(), g2 = Ops::zero(), g3 = Ops::zero();
            int b = 0;
            for (; b + 3 < m; b += 4) {
              Ops::accT(g0, xr[b], lr[b]);
              Ops::accT(g1, xr[b + 1], lr[b + 1]);
              Ops::accT(g2, xr[b + 2], lr[b + 2]);
              Ops::accT(g3, xr[b + 3], lr[b + 3]);
            }
            for (; b < m; ++b) Ops::accT(g0, xr[b], lr[b]);
            Gw[u * KP + v] = Ops::add(Ops::add(Ops::finish(g0), Ops::finish(g1)),
                                      Ops::add(Ops::finish(g2), Ops::finish(g3)));
          }
        }
        bar_group(sg);
        if (leader) {
          for (int t = 0; t < kw; ++t) {
            const int ii = t0 + t;
            const int s = sf[ii];
            const bool pos = sp * s > 0;
            const V d = pos ? d_p : d_m;
            const V g = m > 0 ? Gw[t * KP + t] : Ops::zero();
            const V rs = Ops::one_plus(d, g);  // 1 + Delta_sigma G_tt
            const V c = Ops::div(d, rs);       // used if accepted
            const int par = (i0 + ii) & 1;
            if (lane == 0) sm.gx[par * 2 + sg] = Ops::pack(rs);
            bar_pair();
            V r = Ops::mul(Ops::unpack(sm.gx[par * 2]), Ops::unpack(sm.gx[par * 2 + 1]));
            if (C.charge) r = Ops::mul(r, s > 0 ? cf_p : cf_m);
            bool neg, bad;
            const bool acc = Ops::accept(r, uni[ii], &neg, &bad);
            const bool flip = acc && upd;
            if (lane == 0) cw[t] = flip ? c : Ops::zero();
            if (flip) {
#pragma unroll
              for (int it = 0; it < GE; ++it) {
                const int e = lane + 32 * it, u = e / K, v = e % K;
                if (u > t && v > t && u < kw && v < kw)
                  Gw[u * KP + v] = Ops::fnma(Ops::mul(c, Gw[u * KP + t]), Gw[t * KP + v], Gw[u * KP + v]);
              }
            }
            if (sg == 0) {
              if (lane == 0) {
                af[ii] = acc ? 1 : 0;
                racc[ii] = Ops::pack(r);
              }
              nbad += bad;
              if (acc) {
                wsign = neg ? -wsign : wsign;
                ++nacc;
              }
            }
            __syncwarp();
          }
        }
        bar_group(sg);
        // x_j, y_j at their flip times (column t and row t of G are frozen
        // once site t is done); y is stored scaled by c_j for the T update.
        // A thread owns column b of X and of Y (with m <= 64 one half of the
        // group takes X, the other Y).
        for (int b = gt % bstep; b < m; b += bstep) {
#pragma unroll
          for (int xy = 0; xy < 2; ++xy) {
            if (TG == 2 && xy != tg) continue;
            V* Wm = xy ? Yw : Xw;
            V v[K];
#pragma unroll
            for (int t = 0; t < K; ++t)
              if (t < kw) v[t] = Wm[t * MP + b];
#pragma unroll
            for (int t = 0; t < K - 1; ++t) {
              if (t + 1 < kw) {
                const V ct = cw[t];
#pragma unroll
                for (int j = t + 1; j < K; ++j)
                  if (j < kw) v[j] = Ops::fnma(Ops::mul(ct, xy ? Gw[t * KP + j] : Gw[j * KP + t]), v[t], v[j]);
              }
            }
#pragma unroll
            for (int t = 0; t < K; ++t)
              if (t < kw) Wm[t * MP + b] = xy ? Ops::mul(cw[t], v[t]) : v[t];
          }
        }
        bar_group(sg);
        // T <- T - sum_t (c_t y_t) x_t^T: thread owns column b (with m <= 64,
        // one half of the rows each)
        {
          const int ah = (m + TG - 1) / TG, alo = tg * ah, ahi = min(m, alo + ah);
          for (int b = gt % bstep; b < m; b += bstep) {
            V xb[K];
#pragma unroll
            for (int t = 0; t < K; ++t) xb[t] = (t < kw) ? Xw[t * MP + b] : Ops::zero();
            for (int a = alo; a < ahi; ++a) {
              V tv = T.ld(a * MP + b);
#pragma unroll
              for (int t = 0; t < K; ++t)
                if (t < kw) tv = Ops::fnma(Yw[t * MP + a], xb[t], tv);
              T.st(a * MP + b, tv);
            }
          }
        }
        bar_group(sg);
      }
      if (sg == 0 && leader) {
        typename Ops::Prod wp;
        wp.init();
        for (int ii = lane; ii < cn; ii += 32)
          if (af[ii]) wp.mul(Ops::unpack(racc[ii]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wp.combine_xor(o);
        if (lane == 0) {
          C.cnt[0] += cn;
          C.cnt[1] += nacc;
          C.logw += wp.log_value();
          if (wsign < 0) C.sign = -C.sign;
          if (nbad) C.err |= LQ_ERR_NONFINITE;
        }
      }
    }
    __syncthreads();
    // rows back to the panel; accepted sites scale their row by 1 + Delta_sigma
    for (int s2 = 0; s2 < 2; ++s2) {
      const int m = s2 ? m1 : m0;
      const int sp2 = C.charge ? 1 : (s2 == 0 ? 1 : -1);
      R* rp = s2 ? Rp1 : Rp0;
      const Row* rr = rrow + (size_t)s2 * cs * MP;
      for (int idx = TID; idx < cn * m; idx += NTHR) {
        const int ii = idx / m, a = idx - ii * m;
        Row v = rr[(size_t)ii * MP + a];
        if (af[ii]) v *= (sp2 * sf[ii] > 0) ? opf_p : opf_m;
        rp[(size_t)(i0 + ii) * m + a] = (R)v;
      }
    }
    for (int ii = TID; ii < cn; ii += NTHR)
      if (af[ii]) C.s[(size_t)l * N + i0 + ii] = (int8_t)(-sf[ii]);
    __syncthreads();
  }
}

// the smallest compile-time column bound that holds both spins' particle
// numbers; kernels built for big plans (BIG) also take the m > 32 path
template <class R, class Ops, bool BIG>
__device__ void flip_slice_any(LqChainDev& C, int l, R* a, R* b, const R* c, const R* d, uint32_t tag, Smem& sm) {
  const int m = max(C.ns[0], C.ns[1]);
  if (BIG && m > LQ_NS_SMALL) flip_slice_big<R, Ops>(C, l, a, b, c, d, tag, sm);
  else if (m <= 4) flip_slice_pair<R, Ops, 4, BIG>(C, l, a, b, c, d, tag, sm);
  else if (m <= 8) flip_slice_pair<R, Ops, 8, BIG>(C, l, a, b, c, d, tag, sm);
  else if (m <= 16) flip_slice_pair<R, Ops, 16, BIG>(C, l, a, b, c, d, tag, sm);
  else flip_slice_pair<R, Ops, 32, BIG>(C, l, a, b, c, d, tag, sm);
}

// T (FP64, ld MP) -> double-word halves in place of T[sg]
static __device__ void t_to_dw(Smem& sm, int sg, int m) {
  double* T = sm.T[sg];
  const int MP = sm.MP;
  __syncthreads();
  double* tmp = sm.W;  // staging copy
  for (int idx = TID; idx < m * MP; idx += NTHR) tmp[idx] = T[idx];
  __syncthreads();
  float* Th = (float*)T;
  float* Tl = Th + (size_t)sm.M * MP;
  for (int idx = TID; idx < m * MP; idx += NTHR) {
    const dw v = dw_from(tmp[idx]);
    Th[idx] = v.h;
    Tl[idx] = v.l;
  }
  __syncthreads();
}

template <class R, bool BIG> struct FlipDispatch {
  __device__ static void run(LqChainDev& C, int l, R* a, R* b, const R* c, const R* d, uint32_t tag, Smem& sm) {
    flip_slice_any<R, OpsF64<R>, BIG>(C, l, a, b, c, d, tag, sm);
  }
};
template <bool BIG> struct FlipDispatch<float, BIG> {
  __device__ static void run(LqChainDev& C, int l, float* a, float* b, const float* c, const float* d, uint32_t tag,
                             Smem& sm) {
    // FP64 algebra on FP32 panels: the rows are widened once as they are
    // staged, so the flip loop itself converts nothing
    if (C.prec == 2) flip_slice_any<float, OpsDW, BIG>(C, l, a, b, c, d, tag, sm);
    else flip_slice_any<float, OpsF64<double>, BIG>(C, l, a, b, c, d, tag, sm);
  }
};
// ---------------------------------------------------------------------------
// helpers on the chain layout
// ---------------------------------------------------------------------------
template <class R> __device__ __forceinline__ R* qr_panel(const LqChainDev& C, int sg, int buf, int j) {
  return (R*)C.QR[sg][buf] + (size_t)j * C.N * C.ns[sg];
}
template <class R> __device__ __forceinline__ R* ql_panel(const LqChainDev& C, int sg, int j) {
  return (R*)C.QL[sg] + (size_t)j * C.N * C.ns[sg];
}
__device__ __forceinline__ double* vr_mat(const LqChainDev& C, int sg, int buf, int j) {
  return C.VR[sg][buf] + (size_t)j * C.ns[sg] * C.ns[sg];
}
__device__ __forceinline__ int bnd(const LqChainDev& C, int j) { return min(j * C.tw, C.L); }

template <class R> __device__ void fill_P(const LqChainDev& C, int sg, R* P) {
  const int m = C.ns[sg];
  for (int idx = TID; idx < C.N * m; idx += NTHR) P[idx] = (R)0;
  __syncthreads();
  for (int a = TID; a < m; a += NTHR) P[(size_t)C.occ[sg][a] * m + a] = (R)1;
  __syncthreads();
}

// Right chain Q^R_0 = P, B_j Q^R_{j-1} = Q^R_j V^R_j (current buffer).
template <class R> __device__ void build_right(LqChainDev& C, int sg, Smem& sm) {
  const int m = C.ns[sg], cb = C.cur[sg];
  fill_P<R>(C, sg, qr_panel<R>(C, sg, cb, 0));
  for (int j = 1; j <= C.n; ++j) {
    R* X = qr_panel<R>(C, sg, cb, j);
    const int lo = bnd(C, j - 1), hi = bnd(C, j);
    prop<R, R>(C, sg, X, qr_panel<R>(C, sg, cb, j - 1), m, m, lo, 1, -1, sm);
    for (int l = lo + 1; l < hi; ++l) prop<R, R>(C, sg, X, X, m, m, l, 1, -1, sm);
    chol_qr2<R>(C, X, m, vr_mat(C, sg, cb, j), sm);
  }
}

// Left chain Q^L_n = P, B_j^T Q^L_j = Q^L_{j-1} V^L_{j-1}.
template <class R> __device__ void build_left(LqChainDev& C, int sg, Smem& sm) {
  const int m = C.ns[sg];
  fill_P<R>(C, sg, ql_panel<R>(C, sg, C.n));
  for (int j = C.n; j >= 1; --j) {
    R* Z = ql_panel<R>(C, sg, j - 1);
    const int lo = bnd(C, j - 1), hi = bnd(C, j);
    prop<R, R>(C, sg, Z, ql_panel<R>(C, sg, j), m, m, -1, 2, hi - 1, sm);
    for (int l = hi - 2; l >= lo; --l) prop<R, R>(C, sg, Z, Z, m, m, -1, 2, l, sm);
    chol_qr2<R>(C, Z, m, C.VL[sg] + (size_t)(j - 1) * m * m, sm);
  }
}

// log|W| and sign from the current right chain.
template <class R> __device__ void log_weight(LqChainDev& C, Smem& sm, double* out_log, int* out_sign) {
  double lw = 0.0;
  int sgn = 1;
  for (int sg = 0; sg < 2; ++sg) {
    const int m = C.ns[sg], cb = C.cur[sg], MP = sm.MP;
    double part = 0.0;
    for (int idx = TID; idx < C.n * m; idx += NTHR) {
      int j = 1 + idx / m, a = idx % m;
      part += log(vr_mat(C, sg, cb, j)[a * m + a]);
    }
    lw += cta_sum(part, sm);
    const R* Qn = qr_panel<R>(C, sg, cb, C.n);
    for (int idx = TID; idx < m * m; idx += NTHR) {
      int a = idx / m, b = idx - a * m;
      sm.W[a * MP + b] = (double)Qn[(size_t)C.occ[sg][a] * m + b];
    }
    __syncthreads();
    double la;
    int s1;
    inverse(sm.W, MP, sm.S, MP, m, sm, &la, &s1);
    lw += la;
    sgn *= s1;
  }
  if (C.charge) {
    double part = 0.0;
    for (int idx = TID; idx < C.L * C.N; idx += NTHR) part += (double)C.s[idx];
    lw += -C.lambda * cta_sum(part, sm);
  }
  *out_log = lw;
  *out_sign = sgn;
}

// ---------------------------------------------------------------------------
// Up pass: stored left panels per block, live right panel, QR at block tops.
// ---------------------------------------------------------------------------
template <class R, bool BIG> __device__ void up_pass(LqChainDev& C, Smem& sm) {
  const int N = C.N, MP = sm.MP;
  for (int j = 1; j <= C.n; ++j) {
    const int lo = bnd(C, j - 1), hi = bnd(C, j), nl = hi - lo;
    for (int sg = 0; sg < 2; ++sg) {
      const int m = C.ns[sg];
      const size_t pn = (size_t)N * m;
      R* St = (R*)C.stored[sg];
      prop<R, R>(C, sg, St + (nl - 1) * pn, ql_panel<R>(C, sg, j), m, m, -1, 2, -1, sm);
      for (int l = hi - 2; l >= lo; --l) prop<R, R>(C, sg, St + (l - lo) * pn, St + (l + 1 - lo) * pn, m, m, l + 1, 2, -1, sm);
      prop<R, R>(C, sg, (R*)C.live[sg], qr_panel<R>(C, sg, C.cur[sg], j - 1), m, m, lo, 0, -1, sm);
      PhaseTimer pt_(PH_BLOCKINV);
      gram<double>((const R*)St, m, m, (const R*)C.live[sg], m, m, N, sm.W, MP);
      double la;
      int s1;
      inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
      if (C.prec == 2) t_to_dw(sm, sg, m);
    }
    for (int l = lo; l < hi; ++l) {
      const size_t o0 = (size_t)(l - lo) * N * C.ns[0], o1 = (size_t)(l - lo) * N * C.ns[1];
      FlipDispatch<R, BIG>::run(C, l, (R*)C.live[0], (R*)C.live[1], (const R*)C.stored[0] + o0, (const R*)C.stored[1] + o1, 1u, sm);
      for (int sg = 0; sg < 2; ++sg) {
        const int m = C.ns[sg];
        if (l + 1 < hi) {
          prop<R, R>(C, sg, (R*)C.live[sg], (const R*)C.live[sg], m, m, -1, 1, l + 1, sm);
        } else {
          R* X = qr_panel<R>(C, sg, C.cur[sg], j);
          prop<R, R>(C, sg, X, (const R*)C.live[sg], m, m, -1, 1, -1, sm);
          chol_qr2<R>(C, X, m, vr_mat(C, sg, C.cur[sg], j), sm);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Measurement at block boundary jb from Q^L_jb and Q^R_jb.
// ---------------------------------------------------------------------------
template <class R> __device__ void measure(LqChainDev& C, int jb, Smem& sm) {
  PhaseTimer pt_(5);
  const int N = C.N, MP = sm.MP, M = sm.M;
  const LqLatticeDev& lat = C.lat;
  const R* QLb[2];
  const R* QRb[2];
  double* A[2];
  int sgn = 1;
  double* Ms = sm.S;  // Ms + k*M*MP, k = 0..3
  for (int sg = 0; sg < 2; ++sg) {
    const int m = C.ns[sg];
    QLb[sg] = ql_panel<R>(C, sg, jb);
    QRb[sg] = qr_panel<R>(C, sg, C.cur[sg], jb);
    A[sg] = (double*)C.work[sg];
    gram<double>(QLb[sg], m, m, QRb[sg], m, m, N, sm.W, MP);
    double la;
    int s1;
    inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
    sgn *= s1;
    const double* Tm = sm.T[sg];
    for (int idx = TID; idx < N * m; idx += NTHR) {
      int i = idx / m, b = idx - i * m;
      double acc = 0.0;
      for (int a = 0; a < m; ++a) acc += (double)QRb[sg][(size_t)i * m + a] * Tm[a * MP + b];
      A[sg][idx] = acc;
    }
    __syncthreads();
  }
  const int m0 = C.ns[0], m1 = C.ns[1];
  // densities, double occupancy, onsite energy, sublattice densities
  double nu = 0, nd = 0, docc = 0, eon = 0, na[2][2] = {{0, 0}, {0, 0}};
  for (int i = TID; i < N; i += NTHR) {
    double du = 0, dd = 0;
    for (int b = 0; b < m0; ++b) du += A[0][(size_t)i * m0 + b] * (double)QLb[0][(size_t)i * m0 + b];
    for (int b = 0; b < m1; ++b) dd += A[1][(size_t)i * m1 + b] * (double)QLb[1][(size_t)i * m1 + b];
    nu += du; nd += dd; docc += du * dd;
    if (lat.eps) eon += lat.eps[i] * (du + dd);
    int a = lat.sub[i];
    na[0][a] += du; na[1][a] += dd;
  }
  double ekin = 0.0;
  for (int b = TID; b < lat.nb; b += NTHR) {
    int i = lat.bond_i[b], j = lat.bond_j[b];
    double t = 0.0;
    for (int sg = 0; sg < 2; ++sg) {
      const int m = C.ns[sg];
      for (int q = 0; q < m; ++q)
        t += (double)QLb[sg][(size_t)i * m + q] * A[sg][(size_t)j * m + q] +
             (double)QLb[sg][(size_t)j * m + q] * A[sg][(size_t)i * m + q];
    }
    ekin += lat.bond_k[b] * t;
  }
  nu = cta_sum(nu, sm); nd = cta_sum(nd, sm); docc = cta_sum(docc, sm);
  ekin = cta_sum(ekin + eon, sm);
  double Na[2][2];
  for (int sg = 0; sg < 2; ++sg)
    for (int a = 0; a < 2; ++a) Na[sg][a] = cta_sum(na[sg][a], sm);
  // tr(M^s_a M^s_b), M^s_a = sum_{i in a} A[i,:]^T Q^L[i,:]
  double trMM[2][2][2];
  for (int sg = 0; sg < 2; ++sg) {
    const int m = C.ns[sg];
    for (int a = 0; a < 2; ++a) gram<double>(A[sg], m, m, QLb[sg], m, m, N, Ms + a * M * MP, MP, lat.sub, a);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double part = 0.0;
        for (int idx = TID; idx < m * m; idx += NTHR) {
          int p = idx / m, q = idx - p * m;
          part += Ms[a * M * MP + p * MP + q] * Ms[b * M * MP + q * MP + p];
        }
        trMM[sg][a][b] = cta_sum(part, sm);
      }
  }
  // tr(rho_up rho_dn) = sum_pq X[p][q] Y[q][p], X = A_dn^T Q^L_up, Y = A_up^T Q^L_dn
  gram<double>(A[1], m1, m1, QLb[0], m0, m0, N, Ms + 2 * M * MP, MP);
  gram<double>(A[0], m0, m0, QLb[1], m1, m1, N, Ms + 3 * M * MP, MP);
  double part = 0.0;
  for (int idx = TID; idx < m1 * m0; idx += NTHR) {
    int p = idx / m0, q = idx - p * m0;
    part += Ms[2 * M * MP + p * MP + q] * Ms[3 * M * MP + q * MP + p];
  }
  const double trud = cta_sum(part, sm);
  if (TID == 0) {
    double szz[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double t = 0.0;
        for (int sg = 0; sg < 2; ++sg) t += Na[sg][a] * Na[sg][b] + (a == b ? Na[sg][a] : 0.0) - trMM[sg][a][b];
        t -= Na[0][a] * Na[1][b] + Na[1][a] * Na[0][b];
        szz[a][b] = 0.25 * t;
      }
    const double ncell = N / 2.0, s = (double)sgn;
    sm.obs[0] += s;
    sm.obs[1] += s * nu;
    sm.obs[2] += s * nd;
    sm.obs[3] += s * docc / N;
    sm.obs[4] += s * ekin / N;
    sm.obs[5] += s * szz[0][0] / ncell;
    sm.obs[6] += s * szz[1][1] / ncell;
    sm.obs[7] += s * szz[0][1] / ncell;
    sm.obs[8] += s * 0.5 * (nu + nd - 2.0 * trud) / ncell;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Down pass: stored right panels per block, live left panel, QR at block
// bottoms, measurement at each boundary below a finished block.
// ---------------------------------------------------------------------------
template <class R, bool BIG> __device__ void down_pass(LqChainDev& C, int do_measure, Smem& sm) {
  const int N = C.N, MP = sm.MP;
  for (int sg = 0; sg < 2; ++sg) fill_P<R>(C, sg, ql_panel<R>(C, sg, C.n));
  if (TID < LQ_NOBS) sm.obs[TID] = 0.0;
  __syncthreads();
  for (int j = C.n; j >= 1; --j) {
    const int lo = bnd(C, j - 1), hi = bnd(C, j), nl = hi - lo;
    for (int sg = 0; sg < 2; ++sg) {
      const int m = C.ns[sg];
      const size_t pn = (size_t)N * m;
      R* St = (R*)C.stored[sg];
      prop<R, R>(C, sg, St, qr_panel<R>(C, sg, C.cur[sg], j - 1), m, m, lo, 0, -1, sm);
      for (int l = lo + 1; l < hi; ++l) prop<R, R>(C, sg, St + (l - lo) * pn, St + (l - 1 - lo) * pn, m, m, -1, 1, l, sm);
      prop<R, R>(C, sg, (R*)C.live[sg], ql_panel<R>(C, sg, j), m, m, -1, 2, -1, sm);
      PhaseTimer pt_(PH_BLOCKINV);
      gram<double>((const R*)C.live[sg], m, m, (const R*)(St + (nl - 1) * pn), m, m, N, sm.W, MP);
      double la;
      int s1;
      inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
      if (C.prec == 2) t_to_dw(sm, sg, m);
    }
    for (int l = hi - 1; l >= lo; --l) {
      const size_t o0 = (size_t)(l - lo) * N * C.ns[0], o1 = (size_t)(l - lo) * N * C.ns[1];
      FlipDispatch<R, BIG>::run(C, l, (R*)C.stored[0] + o0, (R*)C.stored[1] + o1, (const R*)C.live[0], (const R*)C.live[1], 2u, sm);
      for (int sg = 0; sg < 2; ++sg) {
        const int m = C.ns[sg];
        if (l > lo) {
          prop<R, R>(C, sg, (R*)C.live[sg], (const R*)C.live[sg], m, m, l, 2, -1, sm);
        } else {
          R* Z = ql_panel<R>(C, sg, j - 1);
          prop<R, R>(C, sg, Z, (const R*)C.live[sg], m, m, l, 0, -1, sm);
          chol_qr2<R>(C, Z, m, C.VL[sg] + (size_t)(j - 1) * m * m, sm);
        }
      }
    }
    if (do_measure) measure<R>(C, j - 1, sm);
  }
  if (do_measure && TID == 0 && C.nrec < C.max_records) {
    for (int k = 0; k < LQ_NOBS; ++k) C.records[(size_t)C.nrec * LQ_NOBS + k] = sm.obs[k] / C.n;
    C.nrec++;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Particle-hole swap for spin sg: remove column k (Givens, Eqs. S9-S12), add
// site j (Gram-Schmidt twice, Eqs. S1-S8).  T0 = (P^T Q_end)^{-1} lives in
// sm.T[sg].  commit: 1 Metropolis with uniform u, 0 only report (hook).
//
// left = 0 walks the right chain at tau = beta: block i = Q^R_i, V^R_i of the
// current buffer, propagator B_i; the trial goes to the other buffer, which
// becomes current on acceptance.  left = 1 walks the left chain at tau = 0,
// read from beta down to 0: it is the right chain of B(beta,0)^T, block i =
// Q^L_{n-i}, V^L_{n-i}, propagator B_{n-i+1}^T.  Its trial goes, in the left
// chain's own indexing, to the spare right-chain buffer (the right chain is
// not needed between the down pass and the next up pass, which rebuilds it
// from P), and acceptance exchanges the two buffers' pointers.
// ---------------------------------------------------------------------------
template <class R>
__device__ void swap_attempt(LqChainDev& C, int sg, int k, int j, double u, int commit, Smem& sm,
                             double log_hastings = 0.0, int left = 0) {
  const int N = C.N, m = C.ns[sg], n = C.n, MP = sm.MP, M = sm.M;
  const int cb = C.cur[sg], tb = cb ^ 1;
  // storage index of walked block i, and the source / trial chains
  auto six = [&](int i) { return left ? n - i : i; };
  const R* qsrc = left ? (const R*)C.QL[sg] : (const R*)C.QR[sg][cb];
  const double* vsrc = left ? C.VL[sg] : C.VR[sg][cb];
  R* qtrial = (R*)C.QR[sg][tb];
  double* vtrial = C.VR[sg][tb];
  const size_t pn = (size_t)N * m;
  const int nrot = m - 1 - k, mr = m - 1;
  const int warp = TID >> 5, lane = TID & 31;
  double* Am = sm.S;                 // working V
  double* Mi = sm.S + M * MP;        // M^{-1}
  double* Tp = sm.S + 2 * M * MP;    // downdated inverse
  double* rc = sm.vec;               // rotations of the current block
  double* rs = sm.vec + M;
  double* v1 = sm.vec + 2 * M;
  double* v2 = sm.vec + 3 * M;
  double* av = sm.vec + 4 * M;
  double* bv = sm.vec + 5 * M;
  int* occr = sm.occ2;               // reduced column order (sites), then the new order
  const int* occ = C.occ[sg];
  double* rot = C.rot;
  // sub-phase cycles of the swap (thread 0): removal into prof[6], addition into prof[7]
  long long tsub = (TID == 0) ? clock64() : 0;
  // --- removal: retriangulate V_i U (i = 1) and V_i G_{i-1}^T (i > 1) -----
  if (warp == 0) {
    double logrN = 0.0;
    int sgnrN = 1;
    for (int i = 1; i <= n; ++i) {
      const double* Vi = vsrc + (size_t)six(i) * m * m;
      for (int cc = lane; cc < m; cc += 32) {
        const int src_col = (cc < k) ? cc : (cc < m - 1 ? cc + 1 : k);
        for (int r = 0; r < m; ++r) Am[r * MP + cc] = Vi[r * m + (i == 1 ? src_col : cc)];
      }
      __syncwarp();
      if (i > 1) {
        for (int rr = lane; rr < m; rr += 32) {
          for (int t = 0; t < nrot; ++t) {
            const int q = k + t;
            const double c = rc[t], s = rs[t];
            const double x = Am[rr * MP + q], y = Am[rr * MP + q + 1];
            Am[rr * MP + q] = c * x + s * y;
            Am[rr * MP + q + 1] = -s * x + c * y;
          }
        }
      }
      __syncwarp();
      for (int t = 0; t < nrot; ++t) {
        const int q = k + t;
        const double a = Am[q * MP + q], b = Am[(q + 1) * MP + q];
        const double r = hypot(a, b);
        const double c = (r != 0.0) ? a / r : 1.0, s = (r != 0.0) ? b / r : 0.0;
        __syncwarp();
        for (int cc = lane; cc < m; cc += 32) {
          const double x = Am[q * MP + cc], y = Am[(q + 1) * MP + cc];
          Am[q * MP + cc] = c * x + s * y;
          Am[(q + 1) * MP + cc] = -s * x + c * y;
        }
        __syncwarp();
        if (lane == 0) {
          Am[q * MP + q] = r;
          Am[(q + 1) * MP + q] = 0.0;
          rc[t] = c;
          rs[t] = s;
          rot[((size_t)(i - 1) * LQ_NS_MAX + t) * 2] = c;
          rot[((size_t)(i - 1) * LQ_NS_MAX + t) * 2 + 1] = s;
        }
        __syncwarp();
      }
      double* Vt = vtrial + (size_t)six(i) * m * m;
      for (int cc = lane; cc < m; cc += 32)
        for (int r = 0; r < m; ++r) Vt[r * m + cc] = Am[r * MP + cc];
      const double dN = Am[(m - 1) * MP + (m - 1)];
      logrN += log(fabs(dN));
      if (dN < 0) sgnrN = -sgnrN;
      __syncwarp();
    }
    // M^{-1} = G_n T0 U, then the downdate of Eq. S12
    const double* T0 = sm.T[sg];
    for (int cc = lane; cc < m; cc += 32) {
      const int src_col = (cc < k) ? cc : (cc < m - 1 ? cc + 1 : k);
      for (int r = 0; r < m; ++r) Mi[r * MP + cc] = T0[r * MP + src_col];
    }
    __syncwarp();
    for (int t = 0; t < nrot; ++t) {
      const int q = k + t;
      const double c = rc[t], s = rs[t];
      for (int cc = lane; cc < m; cc += 32) {
        const double x = Mi[q * MP + cc], y = Mi[(q + 1) * MP + cc];
        Mi[q * MP + cc] = c * x + s * y;
        Mi[(q + 1) * MP + cc] = -s * x + c * y;
      }
      __syncwarp();
    }
    const double mNN = Mi[(m - 1) * MP + (m - 1)];
    for (int rr = lane; rr < mr; rr += 32)
      for (int b = 0; b < mr; ++b) Tp[rr * MP + b] = Mi[rr * MP + b] - Mi[rr * MP + (m - 1)] * Mi[(m - 1) * MP + b] / mNN;
    for (int rr = lane; rr < mr; rr += 32) occr[rr] = occ[(rr < k) ? rr : rr + 1];
    if (lane == 0) {
      sm.ip[11] = occ[k];
      sm.red[48] = log(fabs(mNN)) - logrN;
      sm.ip[8] = ((mNN < 0) ? -1 : 1) * sgnrN;
      sm.ip[9] = (mNN != 0.0) ? 1 : 0;
    }
  }
  __syncthreads();
  // Q_i' = Q_i G_i^T for all blocks, streamed row by row
  {
    for (size_t idx = TID; idx < (size_t)n * N; idx += NTHR) {
      const int i = 1 + (int)(idx / N), row = (int)(idx % N);
      const R* src = qsrc + (size_t)six(i) * pn + (size_t)row * m;
      R* dst = qtrial + (size_t)six(i) * pn + (size_t)row * m;
      for (int a = 0; a < k; ++a) dst[a] = src[a];
      double x = (double)src[k];
      const double* rr = rot + (size_t)(i - 1) * LQ_NS_MAX * 2;
      for (int t = 0; t < nrot; ++t) {
        const double c = rr[2 * t], s = rr[2 * t + 1];
        const double y = (double)src[k + t + 1];
        dst[k + t] = (R)(c * x + s * y);
        x = -s * x + c * y;
      }
      dst[m - 1] = (R)x;
    }
  }
  __syncthreads();
  if (TID == 0) {
    const long long t1 = clock64();
    C.prof[6] += t1 - tsub;
    tsub = t1;
  }
  // --- addition of site j on the reduced chain ------------------------------
  double* q = C.vec;
  double* w = C.vec + N;
  for (int i = TID; i < N; i += NTHR) q[i] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  double logrho = 0.0;
  int valid = sm.ip[9];
  for (int i = 1; i <= n && valid; ++i) {
    if (!left) {
      const int lo = bnd(C, i - 1), hi = bnd(C, i);
      prop<double, double>(C, sg, w, q, 1, 1, lo, 1, -1, sm);
      for (int l = lo + 1; l < hi; ++l) prop<double, double>(C, sg, w, w, 1, 1, l, 1, -1, sm);
    } else {
      // B_{jl}^T with jl = n - i + 1: B_K^T then D_l, l from the block's top down
      const int lo = bnd(C, n - i), hi = bnd(C, n - i + 1);
      prop<double, double>(C, sg, w, q, 1, 1, -1, 2, hi - 1, sm);
      for (int l = hi - 2; l >= lo; --l) prop<double, double>(C, sg, w, w, 1, 1, -1, 2, l, sm);
    }
    R* Qi = qtrial + (size_t)six(i) * pn;
    for (int pass = 0; pass < 2; ++pass) {
      double* vv = pass ? v2 : v1;
      gram<double>(Qi, m, mr, w, 1, 1, N, vv, 1);
      for (int r = TID; r < N; r += NTHR) {
        double acc = 0.0;
        for (int a = 0; a < mr; ++a) acc += (double)Qi[(size_t)r * m + a] * vv[a];
        w[r] -= acc;
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int r = TID; r < N; r += NTHR) part += w[r] * w[r];
    const double rho = sqrt(cta_sum(part, sm));
    if (!(rho > 0.0)) { valid = 0; break; }
    for (int r = TID; r < N; r += NTHR) {
      const double qq = w[r] / rho;
      q[r] = qq;
      Qi[(size_t)r * m + (m - 1)] = (R)qq;
    }
    double* Vt = vtrial + (size_t)six(i) * m * m;
    for (int a = TID; a < mr; a += NTHR) {
      Vt[a * m + (m - 1)] = v1[a] + v2[a];
      Vt[(m - 1) * m + a] = 0.0;
    }
    if (TID == 0) Vt[(m - 1) * m + (m - 1)] = rho;
    logrho += log(rho);
    __syncthreads();
  }
  if (TID == 0) C.prof[7] += clock64() - tsub;
  // --- Schur complement s (Eq. S7), ratio, Metropolis, commit ---------------
  if (warp == 0) {
    const R* Qn = qtrial + (size_t)six(n) * pn;
    double s_add = 0.0;
    if (valid) {
      for (int rr = lane; rr < mr; rr += 32) {
        double acc = 0.0;
        for (int b = 0; b < mr; ++b) acc += Tp[rr * MP + b] * q[occr[b]];
        av[rr] = acc;
        double acc2 = 0.0;
        for (int a = 0; a < mr; ++a) acc2 += (double)Qn[(size_t)j * m + a] * Tp[a * MP + rr];
        bv[rr] = acc2;
      }
      __syncwarp();
      s_add = q[j];
      for (int a = 0; a < mr; ++a) s_add -= (double)Qn[(size_t)j * m + a] * av[a];
      if (s_add == 0.0) valid = 0;
    }
    const double log_rem = sm.red[48];
    const int sgn_rem = sm.ip[8];
    const double log_add = log(fabs(s_add)) + logrho;
    const int sgn_add = (s_add < 0) ? -1 : 1;
    const double logabs = valid ? log_rem + log_add : -INFINITY;
    const int sgn = sgn_rem * sgn_add;
    const double lacc = logabs + log_hastings;  // Metropolis-Hastings: weight ratio times the proposal ratio
    const int accept = commit && valid && (lacc >= 0.0 || u < exp(lacc));
    if (lane == 0) {
      C.hook[0] = logabs; C.hook[1] = sgn; C.hook[2] = log_rem; C.hook[3] = sgn_rem;
      C.hook[4] = log_add; C.hook[5] = sgn_add;
      sm.ip[10] = accept;
      if (commit) C.cnt[2]++;
    }
    __syncwarp();
    if (accept) {
      double* T0 = sm.T[sg];
      for (int rr = lane; rr < mr; rr += 32) {
        for (int b = 0; b < mr; ++b) T0[rr * MP + b] = Tp[rr * MP + b] + av[rr] * bv[b] / s_add;
        T0[rr * MP + (m - 1)] = -av[rr] / s_add;
        T0[(m - 1) * MP + rr] = -bv[rr] / s_add;
      }
      if (lane == 0) {
        T0[(m - 1) * MP + (m - 1)] = 1.0 / s_add;
        occr[m - 1] = j;
        C.logw += logabs;
        C.sign *= sgn;
        if (!isfinite(logabs)) C.err |= LQ_ERR_NONFINITE;
        C.cnt[3]++;
      }
    }
  }
  __syncthreads();
  if (sm.ip[10]) {
    const int removed = sm.ip[11];
    for (int a = TID; a < m; a += NTHR) C.occ[sg][a] = occr[a];
    R* P = qtrial + (size_t)six(0) * pn;
    for (size_t idx = TID; idx < pn; idx += NTHR) P[idx] = (R)0;
    __syncthreads();
    for (int a = TID; a < m; a += NTHR) P[(size_t)occr[a] * m + a] = (R)1;
    if (TID == 0) {
      sm.bits[removed >> 5] &= ~(1u << (removed & 31));
      sm.bits[j >> 5] |= 1u << (j & 31);
      if (!left) {
        C.cur[sg] = tb;
      } else {
        void* qt = C.QL[sg];
        C.QL[sg] = C.QR[sg][tb];
        C.QR[sg][tb] = qt;
        double* vt = C.VL[sg];
        C.VL[sg] = C.VR[sg][tb];
        C.VR[sg][tb] = vt;
      }
    }
  }
  __syncthreads();
}

// Occupancy bitmap of spin sg, and T0 = (P^T Q^R_n)^{-1} (left = 0) or
// (P^T Q^L_0)^{-1} (left = 1) into sm.T[sg].
template <class R> __device__ void swap_setup(LqChainDev& C, int sg, Smem& sm, int left = 0) {
  const int N = C.N, m = C.ns[sg], MP = sm.MP;
  for (int w = TID; w < N / 32 + 1; w += NTHR) sm.bits[w] = 0u;
  __syncthreads();
  if (TID == 0)
    for (int a = 0; a < m; ++a) sm.bits[C.occ[sg][a] >> 5] |= 1u << (C.occ[sg][a] & 31);
  const R* Qn = left ? ql_panel<R>(C, sg, 0) : qr_panel<R>(C, sg, C.cur[sg], C.n);
  for (int idx = TID; idx < m * m; idx += NTHR) {
    int a = idx / m, b = idx - a * m;
    sm.W[a * MP + b] = (double)Qn[(size_t)C.occ[sg][a] * m + b];
  }
  __syncthreads();
  double la;
  int s1;
  inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
}

// site index of the jidx-th empty site (ascending)
static __device__ int jth_empty(const Smem& sm, int N, int jidx) {
  int t = 0;
  for (int w = 0; w * 32 < N; ++w) {
    unsigned occw = sm.bits[w];
    int nbits = min(32, N - w * 32);
    unsigned valid = (nbits == 32) ? 0xffffffffu : ((1u << nbits) - 1u);
    unsigned emp = ~occw & valid;
    int c = __popc(emp);
    if (t + c > jidx) {
      int need = jidx - t;
      for (int b = 0; b < 32; ++b)
        if (emp & (1u << b)) {
          if (need == 0) return w * 32 + b;
          --need;
        }
    }
    t += c;
  }
  return -1;
}

// N_up then N_dn swap attempts: left = 0 at tau = beta on the right chain
// after the up pass (random-number tag 3), left = 1 at tau = 0 on the left
// chain after the down pass (tag 6).
template <class R> __device__ void swap_phase(LqChainDev& C, Smem& sm, int left = 0) {
  PhaseTimer pt_(4);
  const uint32_t tag = left ? 6u : 3u;
  for (int sg = 0; sg < 2; ++sg) {
    const int m = C.ns[sg];
    if (m == 0 || m == C.N) continue;
    swap_setup<R>(C, sg, sm, left);
    for (int att = 0; att < m; ++att) {
      if (TID == 0) {
        uint32_t w[4], w2[4];
        const uint32_t c2 = (tag << 24) | ((uint32_t)sg << 16) | (uint32_t)att;
        philox(C.chain_id, C.sweep, c2, 0u, C.key0, C.key1, w);
        philox(C.chain_id, C.sweep, c2, 1u, C.key0, C.key1, w2);
        const int k = (int)(u53(w[0], w[1]) * (double)m);
        double lh = 0.0;
        int j;
        if (C.swap_mode == LQ_SWAP_NEIGHBOUR) {
          // target uniform among the empty neighbours E(i) of i = occ[k];
          // the reverse move draws i among the empty neighbours E'(j) of j
          // after the move, so the proposal ratio is |E(i)| / |E'(j)|
          const int i = C.occ[sg][k];
          const int* nbs = C.lat.nb_site;
          const int t0 = C.lat.nb_off[i], t1 = C.lat.nb_off[i + 1];
          int ne = 0;
          for (int t = t0; t < t1; ++t) ne += !((sm.bits[nbs[t] >> 5] >> (nbs[t] & 31)) & 1u);
          j = -2;  // no empty neighbour: no move
          if (ne > 0) {
            const int jidx = (int)(u53(w[2], w[3]) * (double)ne);
            for (int t = t0, c = 0; t < t1; ++t)
              if (!((sm.bits[nbs[t] >> 5] >> (nbs[t] & 31)) & 1u)) {
                if (c == jidx) { j = nbs[t]; break; }
                ++c;
              }
            int ne2 = 0;
            for (int t = C.lat.nb_off[j]; t < C.lat.nb_off[j + 1]; ++t) {
              const int o = nbs[t];
              ne2 += (o == i) || !((sm.bits[o >> 5] >> (o & 31)) & 1u);
            }
            lh = log((double)ne) - log((double)ne2);
          }
        } else {
          const int jidx = (int)(u53(w[2], w[3]) * (double)(C.N - m));
          j = jth_empty(sm, C.N, jidx);
        }
        sm.ip[4] = k;
        sm.ip[5] = j;
        sm.red[50] = u53(w2[0], w2[1]);
        sm.red[51] = lh;
      }
      __syncthreads();
      if (sm.ip[5] == -2) {  // nearest-neighbour proposal with no empty neighbour: a rejected attempt
        if (TID == 0) C.cnt[2]++;
        __syncthreads();
        continue;
      }
      if (sm.ip[5] < 0) {  // cannot happen for jidx < N - m; never index with it
        if (TID == 0) sm.C->err |= LQ_ERR_NONFINITE;
        __syncthreads();
        continue;
      }
      swap_attempt<R>(C, sg, sm.ip[4], sm.ip[5], sm.red[50], 1, sm, sm.red[51], left);
    }
    // the next up pass starts the right chain from Q^R_0 = P
    if (left) fill_P<R>(C, sg, qr_panel<R>(C, sg, C.cur[sg], 0));
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ inline void load_chain(LqChainDev* g, Smem& sm) {
  if (TID == 0) { prof_shared()->C = sm.C; prof_shared()->depth = 0; }
  const int words = (int)(sizeof(LqChainDev) / 4);
  for (int w = TID; w < words; w += NTHR) ((int*)sm.C)[w] = ((const int*)g)[w];
  __syncthreads();
}
__device__ inline void store_chain(LqChainDev* g, Smem& sm) {
  __syncthreads();
  const int words = (int)(sizeof(LqChainDev) / 4);
  for (int w = TID; w < words; w += NTHR) ((int*)g)[w] = ((const int*)sm.C)[w];
  __syncthreads();
}

// The leader warp of the field-flip loop (m <= 32) is picked on a sub-partition
// that the other resident CTA of this SM does not lead from: the first CTA on
// an SM takes sub-partition 0, the second 2 (sub-partition = hardware warp
// slot mod 4).  FP64 issue on GB300 is per sub-partition, so this keeps the two
// leaders' serial chains on different FP64 pipes.  In a 256-thread CTA the
// other warp on the leader's sub-partition (its mate, sm.ip[15]) takes no
// FP64 work of the flip loop, so that the chain shares its pipe with fewer
// warps; sm.ip[13] lists the warps on sub-partitions 1 and 3, which no CTA
// leads from.  Any mapping is correct; only speed depends on it.
static __device__ void pick_flip_warps(int* sm_ctr, Smem& sm) {
  __shared__ int wsub[LQ_THREADS / 32];
  __shared__ int pair;
  if (TID == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    pair = sm_ctr ? (atomicAdd(&sm_ctr[smid & 1023], 1) & 1) : 0;
  }
  if ((TID & 31) == 0) {
    unsigned wid;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    wsub[TID >> 5] = (int)(wid & 3u);
  }
  __syncthreads();
  if (TID == 0) {
    int f0 = -1, mate = -1;
    for (int w = 0; w < NTHR / 32; ++w)
      if (f0 < 0 && wsub[w] == 2 * pair) f0 = w;
    if (f0 < 0) f0 = 0;
    unsigned odd = 0u;  // warps on sub-partitions 1 and 3
    if (NTHR == LQ_THREADS)
      for (int w = 0; w < NTHR / 32; ++w) {
        if (mate < 0 && w != f0 && wsub[w] == wsub[f0]) mate = w;
        if ((wsub[w] & 1) && w != f0) odd |= 1u << w;
      }
    sm.ip[13] = (int)odd;
    sm.ip[14] = f0;
    sm.ip[15] = mate;
  }
  __syncthreads();
}

template <class R, bool BIG>
__global__ void __launch_bounds__(LQ_THREADS, BIG ? 1 : 2)
    sweep_kernel(LqChainDev* chains, const int* order, int n_order, int* queue, int n_sweeps, const int* caps,
                 long long budget_ns, int do_measure, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  pick_flip_warps(queue + 1, sm);
  __shared__ int next, stop;
  for (;;) {
    if (TID == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int q = next;
    __syncthreads();
    if (q >= n_order) break;
    LqChainDev* g = chains + order[q];
    load_chain(g, sm);
    LqChainDev& C = *sh_rebase(sm.C);  // the descriptor copy is in shared memory in every plan
    // a chain runs caps[q] sweeps (n_sweeps without caps); with a budget it
    // starts no further sweep that, judged by the one just done, would end
    // more than budget_ns after the chain was taken
    const int cap = caps ? caps[q] : n_sweeps;
    const long long t_take = global_ns();
    long long t_prev = t_take;
    for (int t = 0; t < cap; ++t) {
      up_pass<R, BIG>(C, sm);
      swap_phase<R>(C, sm);
      down_pass<R, BIG>(C, do_measure, sm);
      if (C.left_swaps) swap_phase<R>(C, sm, 1);
      if (TID == 0) {
        const long long t_now = global_ns();
        C.sweep_ns_ring[C.sweep % LQ_SWEEP_RING] = t_now - t_prev;
        C.sweep++;
        C.sweep_ns_last = t_now - t_prev;
        C.sweep_ns_sum += t_now - t_prev;
        t_prev = t_now;
        stop = budget_ns > 0 && (t_now - t_take) + C.sweep_ns_last > budget_ns;
      }
      __syncthreads();
      if (stop) break;
    }
    store_chain(g, sm);
  }
}

template <class R>
__global__ void __launch_bounds__(LQ_THREADS, 2)
    build_kernel(LqChainDev* chains, const int* order, int n_order, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  for (int q = blockIdx.x; q < n_order; q += gridDim.x) {
    LqChainDev* g = chains + order[q];
    load_chain(g, sm);
    LqChainDev& C = *sm.C;
    // input check: fields +-1, occupied sites distinct and in range
    if (TID == 0) sm.ip[12] = 0;
    __syncthreads();
    for (int idx = TID; idx < C.L * C.N; idx += NTHR)
      if (C.s[idx] != 1 && C.s[idx] != -1) sm.ip[12] = 1;
    for (int sg = 0; sg < 2; ++sg) {
      for (int w = TID; w < C.N / 32 + 1; w += NTHR) sm.bits[w] = 0u;
      __syncthreads();
      if (TID == 0)
        for (int a = 0; a < C.ns[sg]; ++a) {
          const int i = C.occ[sg][a];
          if (i < 0 || i >= C.N || (sm.bits[i >> 5] >> (i & 31)) & 1u) { sm.ip[12] = 1; break; }
          sm.bits[i >> 5] |= 1u << (i & 31);
        }
      __syncthreads();
    }
    if (sm.ip[12]) {
      if (TID == 0) C.err |= LQ_ERR_BADINPUT;
      store_chain(g, sm);
      continue;
    }
    for (int sg = 0; sg < 2; ++sg) { build_right<R>(C, sg, sm); build_left<R>(C, sg, sm); }
    double lw;
    int s1;
    log_weight<R>(C, sm, &lw, &s1);
    if (TID == 0) { C.logw = lw; C.sign = s1; C.hook[6] = lw; C.hook[7] = s1; }
    store_chain(g, sm);
  }
}

}  // namespace lq

// A translation unit that defines one instance of the sweep kernel exposes it
// through two host functions: its address (attributes, occupancy) and a launch.
#define LQ_SWEEP_INSTANCE_DECL(NAME)                                                                              \
  const void* sweep_fn_##NAME();                                                                                \
  cudaError_t sweep_launch_##NAME(int grid, int threads, cudaStream_t st, LqChainDev* chains, const int* order,  \
                                  int n_order, int* queue, int n_sweeps, const int* caps, long long budget_ns,    \
                                  int do_measure, SmemPlan plan);
#define LQ_SWEEP_INSTANCE(R, BIG, NAME)                                                                           \
  namespace lq {                                                                                                \
  const void* sweep_fn_##NAME() { return (const void*)sweep_kernel<R, BIG>; }                                   \
  cudaError_t sweep_launch_##NAME(int grid, int threads, cudaStream_t st, LqChainDev* chains, const int* order,  \
                                  int n_order, int* queue, int n_sweeps, const int* caps, long long budget_ns,    \
                                  int do_measure, SmemPlan plan) {                                              \
    sweep_kernel<R, BIG><<<grid, threads, plan.total, st>>>(chains, order, n_order, queue, n_sweeps, caps,      \
                                                           budget_ns, do_measure, plan);                       \
    return cudaGetLastError();                                                                                  \
  }                                                                                                             \
  }
