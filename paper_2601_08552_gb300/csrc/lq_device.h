// Device-side descriptors shared by the host runtime (lq_api.cpp) and the
// CUDA kernels (lq_kernels.cu).  Plain structs of pointers and sizes; one
// LqChainDev per Markov chain lives in device memory and is updated in place
// by the sweep kernel.
#pragma once
#include <stdint.h>

// x = h + l as two FP32 values (host side; the double-word algebra of LQ_MIXED_DW)
static inline void lq_dw_split(double x, float out[2]) {
  out[0] = (float)x;
  out[1] = (float)(x - (double)out[0]);
}

#define LQ_NOBS 9          // sign, n_up, n_dn, docc, ekin, szz_00, szz_11, szz_01, s_par
#define LQ_NS_MAX 512      // particles per spin (the C ABI's LQ_MAX_PARTICLES)
#define LQ_NS_SMALL 32     // up to this many per spin, one leader warp runs both spins' flip chains and the
                           // m x m matrices live in shared memory; above it, a four-warp group per spin
                           // flips and those matrices live in a global workspace per CTA
#define LQ_THREADS 256     // threads per CTA (one CTA per chain)
#define LQ_WIN 8           // sites per field-flip window of the four-warp path (the pair path uses 4)
#define LQ_SWEEP_RING 32   // per-sweep wall times a chain descriptor keeps
// 8-byte elements of one spin's window: x rows, y rows (K x MP each), G (K x (K+1)), c (K),
// c-scaled G factors of the x/y recurrences (K x K)
#define LQ_WIN_ELEMS(MP) (2 * LQ_WIN * (MP) + LQ_WIN * (LQ_WIN + 1) + LQ_WIN + LQ_WIN * LQ_WIN)

// Error bits a kernel may set in LqChainDev::err.
#define LQ_ERR_SINGULAR 1  // a Gram / overlap matrix had a zero pivot
#define LQ_ERR_CHOLESKY 2  // CholeskyQR2 broke down (non-positive pivot)
#define LQ_ERR_NONFINITE 4 // a ratio or a log-weight became NaN / Inf
#define LQ_ERR_BADINPUT 8  // a field != +-1 or a repeated / out-of-range occupied site

// Lattice in checkerboard form: bonds sorted by family (stable in the bond
// order the lattice was built with); family g owns bonds [fam_off[g], fam_off[g+1]).
struct LqLatticeDev {
  int N, nb, G;
  const int* fam_off;       // G + 1
  const int* bond_i;        // nb
  const int* bond_j;        // nb
  const double* bond_c;     // cosh(dtau k_b)
  const double* bond_s;     // -sinh(dtau k_b); -tanh(dtau k_b) in the families of `unif`
  const float* bond_cf;     // cosh and -sinh in FP32 (FP32 panels, always the four-term form)
  const float* bond_sf;
  // bit g: every bond of family g has the same cosh c_g and the family holds
  // every site exactly once, so on FP64 panels its factor is applied as
  // [[1, t], [t, 1]] blocks (t = -tanh(dtau k_b)) and the scalar c_g waits
  // until the end of the slice; cprod is the product of those c_g
  unsigned unif;
  double cprod;
  const double* bond_k;     // k_b (kinetic-energy measurement)
  const double* ceps;       // exp(-dtau eps_i), or nullptr when eps == 0
  const float* cepsf;
  const double* eps;        // onsite eps_i, or nullptr
  const int* sub;           // sublattice label 0/1
  const int* nb_off;        // N + 1 offsets into nb_site
  const int* nb_site;       // each site's distinct bond partners, ascending
  // exact kinetic propagator e^{-dtau K} (LQ_EXACT): K in compressed rows
  // (the onsite term on the diagonal), applied as a Taylor polynomial of
  // degree taylor_q in -dtau K evaluated by Horner's rule
  int exact, taylor_q;
  double mdtau;             // -dtau
  const int* k_off;         // N + 1 row offsets
  const int* k_col;         // column of each entry, ascending within a row
  const double* k_val;      // K_ij
  const float* k_valf;      // the same in FP32 (FP32 panels)
};

struct LqChainDev {
  LqLatticeDev lat;
  int N, L, tw, n;          // sites, slices, slices per block, blocks
  int ns[2];                // particles per spin
  int charge;               // 1: U < 0 (charge channel)
  int prec;                 // 0: FP64 panels, 1: FP32 panels (mixed), 2: FP32 panels + double-word flips
  double lambda;
  double dfac_p, dfac_m;    // e^{+lambda}, e^{-lambda}
  double delta_p, delta_m;  // e^{-2 lambda} - 1, e^{+2 lambda} - 1
  double cfac_p, cfac_m;    // e^{+2 lambda}, e^{-2 lambda} (charge-channel scalar ratio)
  double opd_p, opd_m;      // 1 + delta_p, 1 + delta_m (row factor of an accepted flip)
  float dw_delta_p[2], dw_delta_m[2], dw_cfac_p[2], dw_cfac_m[2];  // double-word forms (LQ_MIXED_DW)
  uint32_t key0, key1, chain_id, sweep;
  int swap_mode;            // LQ_SWAP_UNIFORM or LQ_SWAP_NEIGHBOUR
  int left_swaps;           // 1: a second swap phase at tau = 0 on the left chain after the down pass
  // configuration
  int8_t* s;                // L x N fields, row = slice
  int* occ[2];              // ordered occupied sites (columns of P)
  // chains: panels are N x ns row-major, of the panel type (double or float)
  void* QR[2][2];           // right chain Q^R_0..Q^R_n, two buffers per spin
  double* VR[2][2];         // V^R_1..V^R_n (index 0 unused), two buffers per spin
  int cur[2];               // current buffer of the right chain
  void* QL[2];              // left chain Q^L_0..Q^L_n
  double* VL[2];            // V^L_0..V^L_{n-1}
  void* stored[2];          // tau_w panels of the block being updated
  void* live[2];            // the propagated panel of the block
  void* work[2];            // one scratch panel (measurement)
  double* vec;              // 2 x N scratch vectors (particle addition)
  double* rot;              // n x LQ_NS_MAX x 2 Givens coefficients (row stride LQ_NS_MAX x 2)
  double* records;          // max_records x LQ_NOBS
  int max_records, nrec;
  double logw;              // tracked log|W|
  int sign;                 // tracked sign
  int err;
  long long cnt[4];         // field attempts, field accepts, swap attempts, swap accepts
  double hook[8];           // test-hook outputs
  long long prof[12];       // cycles per phase: flips, propagation, QR, block inverse, swaps, measurement;
                            // then two parts of the swaps: removal (with Q streaming), addition; then
                            // four parts of the flips (chains of up to 32 particles per spin): row staging and
                            // write-back, each chunk's first window products and blocks, the leader's serial
                            // chains, the rest of the window loop (next block, waits)
  long long sweep_ns_last;  // wall time of the chain's most recent sweep (device global timer)
  long long sweep_ns_sum;   // summed wall time of its sweeps (the caller may reset it)
  long long sweep_ns_ring[LQ_SWEEP_RING];  // wall time of sweep k at [k % LQ_SWEEP_RING]
};
