/*
 * lq_oracle.c -- plain, slow, single-threaded FP64 CPU implementation of the
 * canonical-ensemble DQMC sweep with the stabilized QR update (LEC-QMC,
 * arXiv 2601.08552).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header or table with the CUDA library.
 *
 * Every step follows the paper's order and notation:
 *   - canonical weight det[P^T B_s(beta,0) P], Eq. (1);
 *   - B(beta,0) = prod_l B_l with B_l = e^{-dtau K} e^{-dtau V(s_l)}, the Trotter
 *     form of the propagator written in the constrained-path section
 *     (U(s) = prod e^{-dtau H0} e^{-dtau H_I}, SM Sec. VI);
 *   - stabilized QR chain B_i Q_{i-1} = Q_i V_i every tau_w slices (SM Sec. I.A,
 *     the "subsequent stabilization steps"), B_i the product of the tau_w
 *     slices of block i;
 *   - field flips with the Sherman-Morrison update of (L R)^{-1}: the ratio
 *     det(U_L^T (1+Delta_i) U_R) / det(U_L^T U_R) of SM Sec. VI;
 *   - particle removal: permutation U, Givens retriangulation G_i of V_i U
 *     (i = 1) and V_i G_{i-1}^T (i > 1), Q_i' = Q_i G_i^T, ratio 1/(s r_Ne)
 *     with 1/s = [M^{-1}]_{Ne,Ne}, M^{-1} = G_n (P^T Q)^{-1} U (Eq. S10) and
 *     the downdate of Eq. S12;
 *   - particle addition: w_i = B_i q_{i-1}, v_i = Q_i^T w_i,
 *     q_i = (w_i - Q_i v_i)/||.||, ratio s r_{Ne+1} (Eqs. S2-S4, S7, Eq. 4),
 *     bordered inverse of Eq. S8;
 *   - particle-hole swap = removal followed by addition, Metropolis on the
 *     product ratio (main text, "Canonical sampling").
 *
 * Readings where the paper is silent:
 *   - B_i is the product of the slices of block i only (the text's
 *     "B_s(i tau_w, 0)" contradicts B_i Q_{i-1} = Q_i V_i);
 *   - Hirsch discrete HS: U > 0 spin channel, cosh(lambda) = e^{dtau U/2},
 *     V_sigma = diag(e^{sigma lambda s}); U < 0 charge channel, same lambda
 *     with |U|, diag(e^{lambda s}) for both spins and a scalar e^{-lambda s};
 *   - checkerboard e^{-dtau K}: B_K = E_{G-1} ... E_1 E_0 C_eps, families
 *     assigned greedily in bond order, E_g the exact product of 2x2 bond
 *     exponentials, C_eps = diag(e^{-dtau eps_i});
 *   - QR with non-negative diagonal (unique Q); Gram-Schmidt applied twice;
 *   - sweep = up field pass, N_up then N_dn swap attempts, down field pass;
 *     sites ascending within a slice; measurement at the block boundaries of
 *     the down pass;
 *   - swap proposal: column k uniform among occupied columns, target uniform
 *     among empty sites; accept iff u < |r| (ties reject); the added particle
 *     is appended as the last column.  Alternative (swap_mode 1): target
 *     uniform among the empty nearest neighbours E(i) of the removed site i,
 *     accepted with the Metropolis-Hastings factor |E(i)| / |E'(j)|;
 *   - optional second swap phase (left_swaps): after the down pass, N_up then
 *     N_dn attempts at tau = 0 that walk the left chain from tau = beta down
 *     to 0.  det[P^T B(beta,0) P] = det[P^T B(beta,0)^T P], and the left chain
 *     is the right chain of B(beta,0)^T = B_1^T ... B_n^T, so the removal and
 *     addition steps above apply unchanged with B_i -> B_{n-i+1}^T;
 *   - constrained-path inner loop (SM Sec. VI; orc_cp_walk, not on the CUDA
 *     path): for a fixed Fock state, independent walkers sample each site's
 *     field with probability proportional to (1/2) max(0, r(s)), r the
 *     overlap ratio with the trial P^T e^{-(beta - tau_l) H_0}, carry the
 *     weight (1/2) sum_s max(0, r(s)) and are dropped at 0; orc_cp_population
 *     adds branching by systematic (comb) resampling every few slices, the
 *     estimate being the product of the population's mean weights.  The paper
 *     fixes neither the field-sampling law nor population control; these are
 *     the plainest choices whose estimate has the unconstrained R(eta) as its
 *     mean whenever nothing is truncated;
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (chain, sweep, tag<<24 | slice-or-attempt, site-or-sub);
 *     tags 1/2 up/down field passes, 3 swaps at tau = beta, 4/5 the initial
 *     fields and Fock states, 6 swaps at tau = 0, 7 constrained-path fields
 *     (counter word 0 = walker), 8 and 9 the fields and the comb of a
 *     branching population.
 *
 * Pins (tests/test_oracle_pins.py): Philox known answers, closed-form
 * spectra and the exact flat band, B_K against a matrix exponential,
 * log-weights against dense determinants and 60-digit arithmetic, field and
 * swap ratios against brute-force determinant ratios, QR-chain invariants,
 * tracked against fresh weights after sweeps, measurements against dense Wick
 * estimators, exhaustive enumeration against the Trotterized ED, and Monte
 * Carlo against that ED (both swap proposals, with and without the swaps at
 * tau = 0); the constrained-path walk against the exact R(eta) of the
 * Trotterized ED where no walker can be truncated (tests/test_oracle_cp.py).
 * Parity unpinned: the average sign at the benchmark sizes, where no exact
 * value exists beyond ED sizes, and the constrained-path estimate where the
 * constraint acts (an approximation with no exact value).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NOBS 9

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of the two-multiplier S-box with a    */
/* Weyl-sequence key schedule.                                               */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0,1) from two 32-bit words. */
static double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* lattice: hopping matrix K as bonds (i, j, kappa) plus onsite eps */
  int N, nb;
  int *bi, *bj;
  double *kb, *eps;
  int *sub;                 /* sublattice label 0/1 per site */
  int G;                    /* number of checkerboard families */
  int *fam_of;              /* family of each bond */
  double *bc, *bs;          /* cosh(dtau k), -sinh(dtau k) per bond */
  double *ceps;             /* exp(-dtau eps_i) */
  /* model / path-integral parameters */
  double U, beta, dtau, lambda;
  int charge;               /* 1: U < 0 charge channel */
  int L, tw, n;             /* slices, slices per block, blocks */
  int *bnd;                 /* block boundaries b_0 = 0 .. b_n = L */
  int ns[2];                /* N_up, N_dn */
  double dfac_p, dfac_m;    /* e^{+lambda}, e^{-lambda} */
  double delta_p, delta_m;  /* e^{-2 lambda} - 1, e^{+2 lambda} - 1 */
  uint32_t key[2], chain, sweep;
  /* configuration */
  int8_t* s;                /* fields, L x N, row = slice */
  int* occ[2];              /* ordered occupied sites = columns of P */
  /* stabilized chains, panels N x ns row-major */
  double *QR[2], *VR[2];    /* right chain Q^R_0..Q^R_n, V^R_1..V^R_n */
  double *QL[2], *VL[2];    /* left chain  Q^L_0..Q^L_n, V^L_0..V^L_{n-1} */
  /* bookkeeping */
  double logw;              /* tracked log|W| (init + sum of accepted log|r|) */
  int sign;
  long long cnt[4];         /* field attempts, field accepts, swap attempts, swap accepts */
  int max_records, nrec;
  double* records;          /* per sweep: mean over the measurements of sign*O */
  int want_corr;
  double *corr_nn, *corr_ss;
  long long ncorr;
  /* Fock-swap proposal: 0 uniform over empty sites, 1 empty nearest neighbour
   * of the removed particle's site (neighbours = distinct bond partners,
   * ascending, in nb_off / nb_site), 2 as 1 without the Hastings factor (a
   * deliberately wrong sampler for the tests) */
  int swap_mode;
  int *nb_off, *nb_site;
  int left_swaps;           /* 1: a second swap phase at tau = 0 after the down pass */
  double* BKd;              /* exact kinetic mode: the dense N x N e^{-dtau K}, else NULL */
} orc_sim;

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra (Golub & Van Loan, Matrix Computations).        */
/* ------------------------------------------------------------------------ */

/* Householder thin QR of A (N x m, row-major, N >= m).  On return A holds Q
 * (N x m, orthonormal columns) and R (m x m, row-major) is upper triangular
 * with a non-negative diagonal. */
static void qr_pos(double* A, int N, int m, double* R) {
  if (m == 0) return;
  double* W = dalloc((size_t)N * m);
  double* V = dalloc((size_t)N * m);   /* Householder vectors, column c in V[:, c] */
  double* beta = dalloc(m);
  memcpy(W, A, sizeof(double) * (size_t)N * m);
  for (int c = 0; c < m; ++c) {
    double nrm = 0.0;
    for (int r = c; r < N; ++r) nrm += W[r * m + c] * W[r * m + c];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { beta[c] = 0.0; continue; }
    double alpha = (W[c * m + c] > 0.0) ? -nrm : nrm;
    double vn = 0.0;
    for (int r = c; r < N; ++r) {
      double v = (r == c) ? W[c * m + c] - alpha : W[r * m + c];
      V[r * m + c] = v;
      vn += v * v;
    }
    beta[c] = 2.0 / vn;
    for (int cc = c; cc < m; ++cc) {
      double d = 0.0;
      for (int r = c; r < N; ++r) d += V[r * m + c] * W[r * m + cc];
      d *= beta[c];
      for (int r = c; r < N; ++r) W[r * m + cc] -= d * V[r * m + c];
    }
  }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) R[a * m + b] = (b >= a) ? W[a * m + b] : 0.0;
  /* Q = H_0 H_1 ... H_{m-1} [I; 0] */
  memset(A, 0, sizeof(double) * (size_t)N * m);
  for (int a = 0; a < m; ++a) A[a * m + a] = 1.0;
  for (int c = m - 1; c >= 0; --c) {
    if (beta[c] == 0.0) continue;
    for (int cc = 0; cc < m; ++cc) {
      double d = 0.0;
      for (int r = c; r < N; ++r) d += V[r * m + c] * A[r * m + cc];
      d *= beta[c];
      for (int r = c; r < N; ++r) A[r * m + cc] -= d * V[r * m + c];
    }
  }
  /* make diag(R) >= 0: flip row c of R and column c of Q together */
  for (int c = 0; c < m; ++c) {
    if (R[c * m + c] < 0.0) {
      for (int b = 0; b < m; ++b) R[c * m + b] = -R[c * m + b];
      for (int r = 0; r < N; ++r) A[r * m + c] = -A[r * m + c];
    }
  }
  free(W); free(V); free(beta);
}

/* Inverse of A (m x m) by LU with partial pivoting; returns log|det A| and
 * its sign.  A singular matrix gives logabs = -inf, sign = 0. */
static void inv_lu(const double* A, int m, double* Ainv, double* logabs, int* sign) {
  *logabs = 0.0; *sign = 1;
  if (m == 0) return;
  double* M = dalloc((size_t)m * m);
  int* piv = (int*)calloc(m, sizeof(int));
  memcpy(M, A, sizeof(double) * (size_t)m * m);
  for (int i = 0; i < m; ++i) piv[i] = i;
  for (int c = 0; c < m; ++c) {
    int p = c; double best = fabs(M[c * m + c]);
    for (int r = c + 1; r < m; ++r) if (fabs(M[r * m + c]) > best) { best = fabs(M[r * m + c]); p = r; }
    if (best == 0.0) { *logabs = -INFINITY; *sign = 0; free(M); free(piv); for (int i = 0; i < m * m; ++i) Ainv[i] = NAN; return; }
    if (p != c) {
      for (int b = 0; b < m; ++b) { double t = M[c * m + b]; M[c * m + b] = M[p * m + b]; M[p * m + b] = t; }
      int t = piv[c]; piv[c] = piv[p]; piv[p] = t;
      *sign = -*sign;
    }
    double d = M[c * m + c];
    if (d < 0) *sign = -*sign;
    *logabs += log(fabs(d));
    for (int r = c + 1; r < m; ++r) {
      double f = M[r * m + c] / d;
      M[r * m + c] = f;
      for (int b = c + 1; b < m; ++b) M[r * m + b] -= f * M[c * m + b];
    }
  }
  /* solve L U X = P I column by column */
  for (int col = 0; col < m; ++col) {
    double* x = dalloc(m);
    for (int r = 0; r < m; ++r) x[r] = (piv[r] == col) ? 1.0 : 0.0;
    for (int r = 0; r < m; ++r) for (int b = 0; b < r; ++b) x[r] -= M[r * m + b] * x[b];
    for (int r = m - 1; r >= 0; --r) {
      for (int b = r + 1; b < m; ++b) x[r] -= M[r * m + b] * x[b];
      x[r] /= M[r * m + r];
    }
    for (int r = 0; r < m; ++r) Ainv[r * m + col] = x[r];
    free(x);
  }
  free(M); free(piv);
}

/* C = A^T B for A (N x p), B (N x q), C (p x q). */
static void gram(const double* A, const double* B, int N, int p, int q, double* C) {
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < q; ++b) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) acc += A[i * p + a] * B[i * q + b];
      C[a * q + b] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Propagators                                                               */
/* ------------------------------------------------------------------------ */

/* Exact kinetic mode: X (N x m) <- B X or B^T X for the dense B = e^{-dtau K}
 * given by the caller (a plain matrix product through a copy of X). */
static void apply_dense(const orc_sim* S, double* X, int m, int transpose) {
  const int N = S->N;
  double* Y = dalloc((size_t)N * m);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      const double b = transpose ? S->BKd[(size_t)j * N + i] : S->BKd[(size_t)i * N + j];
      if (b == 0.0) continue;
      for (int a = 0; a < m; ++a) Y[(size_t)i * m + a] += b * X[(size_t)j * m + a];
    }
  memcpy(X, Y, sizeof(double) * (size_t)N * m);
  free(Y);
}

/* X (N x m) <- B_K X with B_K = E_{G-1} ... E_0 C_eps (checkerboard), or with
 * the dense e^{-dtau K} in the exact kinetic mode. */
static void apply_BK(const orc_sim* S, double* X, int m) {
  if (S->BKd) { apply_dense(S, X, m, 0); return; }
  for (int i = 0; i < S->N; ++i)
    for (int a = 0; a < m; ++a) X[i * m + a] *= S->ceps[i];
  for (int g = 0; g < S->G; ++g)
    for (int b = 0; b < S->nb; ++b) {
      if (S->fam_of[b] != g) continue;
      int i = S->bi[b], j = S->bj[b];
      double c = S->bc[b], s = S->bs[b];
      for (int a = 0; a < m; ++a) {
        double xi = X[i * m + a], xj = X[j * m + a];
        X[i * m + a] = c * xi + s * xj;
        X[j * m + a] = s * xi + c * xj;
      }
    }
}

/* X <- B_K^T X = C_eps E_0 ... E_{G-1} X (or the dense transpose). */
static void apply_BKT(const orc_sim* S, double* X, int m) {
  if (S->BKd) { apply_dense(S, X, m, 1); return; }
  for (int g = S->G - 1; g >= 0; --g)
    for (int b = 0; b < S->nb; ++b) {
      if (S->fam_of[b] != g) continue;
      int i = S->bi[b], j = S->bj[b];
      double c = S->bc[b], s = S->bs[b];
      for (int a = 0; a < m; ++a) {
        double xi = X[i * m + a], xj = X[j * m + a];
        X[i * m + a] = c * xi + s * xj;
        X[j * m + a] = s * xi + c * xj;
      }
    }
  for (int i = 0; i < S->N; ++i)
    for (int a = 0; a < m; ++a) X[i * m + a] *= S->ceps[i];
}

/* diagonal of e^{-dtau V_sigma(s_l)} at site i */
static double dfac(const orc_sim* S, int sigma, int8_t s) {
  int sp = S->charge ? 1 : (sigma == 0 ? 1 : -1);
  return (sp * s > 0) ? S->dfac_p : S->dfac_m;
}

static void apply_D(const orc_sim* S, double* X, int m, int l, int sigma) {
  const int8_t* sl = S->s + (size_t)l * S->N;
  for (int i = 0; i < S->N; ++i) {
    double f = dfac(S, sigma, sl[i]);
    for (int a = 0; a < m; ++a) X[i * m + a] *= f;
  }
}

/* ------------------------------------------------------------------------ */
/* Lattice setup                                                             */
/* ------------------------------------------------------------------------ */

/* Families: each bond, in the given order, goes to the lowest family in which
 * neither of its sites is used yet. */
static void assign_families(orc_sim* S) {
  int N = S->N, nb = S->nb;
  int cap = 4;
  unsigned char* used = (unsigned char*)calloc((size_t)N * cap, 1);
  S->G = 0;
  for (int b = 0; b < nb; ++b) {
    int g = 0;
    for (;; ++g) {
      if (g >= cap) {
        int ncap = cap * 2;
        unsigned char* nu = (unsigned char*)calloc((size_t)N * ncap, 1);
        memcpy(nu, used, (size_t)N * cap);
        free(used); used = nu; cap = ncap;
      }
      if (!used[(size_t)g * N + S->bi[b]] && !used[(size_t)g * N + S->bj[b]]) break;
    }
    used[(size_t)g * N + S->bi[b]] = 1;
    used[(size_t)g * N + S->bj[b]] = 1;
    S->fam_of[b] = g;
    if (g + 1 > S->G) S->G = g + 1;
  }
  free(used);
}

static size_t panel(const orc_sim* S, int sigma) { return (size_t)S->N * S->ns[sigma]; }
static size_t sq(const orc_sim* S, int sigma) { return (size_t)S->ns[sigma] * S->ns[sigma]; }

orc_sim* orc_create(int N, int nb, const int* bi, const int* bj, const double* kb, const double* eps,
                    const int* sub, double U, double beta, double dtau, int n_up, int n_dn, int tw,
                    uint64_t seed, uint32_t chain, int max_records, int want_corr) {
  if (N <= 0 || nb < 0 || n_up < 0 || n_dn < 0 || n_up > N || n_dn > N || tw <= 0 || dtau <= 0 || beta <= 0)
    return NULL;
  double Lf = beta / dtau;
  int L = (int)llround(Lf);
  if (L < 1 || fabs(Lf - L) > 1e-9 * (Lf > 1 ? Lf : 1)) return NULL;
  orc_sim* S = (orc_sim*)calloc(1, sizeof(orc_sim));
  S->N = N; S->nb = nb;
  S->bi = (int*)calloc(nb ? nb : 1, sizeof(int));
  S->bj = (int*)calloc(nb ? nb : 1, sizeof(int));
  S->kb = dalloc(nb); S->eps = dalloc(N); S->sub = (int*)calloc(N, sizeof(int));
  S->fam_of = (int*)calloc(nb ? nb : 1, sizeof(int));
  S->bc = dalloc(nb); S->bs = dalloc(nb); S->ceps = dalloc(N);
  for (int b = 0; b < nb; ++b) {
    S->bi[b] = bi[b]; S->bj[b] = bj[b]; S->kb[b] = kb[b];
    S->bc[b] = cosh(dtau * kb[b]);
    S->bs[b] = -sinh(dtau * kb[b]);
  }
  for (int i = 0; i < N; ++i) {
    S->eps[i] = eps ? eps[i] : 0.0;
    S->sub[i] = sub ? sub[i] : (i & 1);
    S->ceps[i] = exp(-dtau * S->eps[i]);
  }
  assign_families(S);
  S->U = U; S->beta = beta; S->dtau = dtau;
  S->charge = (U < 0);
  S->lambda = acosh(exp(dtau * fabs(U) / 2.0));
  S->dfac_p = exp(S->lambda); S->dfac_m = exp(-S->lambda);
  S->delta_p = expm1(-2.0 * S->lambda); S->delta_m = expm1(2.0 * S->lambda);
  S->L = L; S->tw = tw; S->n = (L + tw - 1) / tw;
  S->bnd = (int*)calloc(S->n + 1, sizeof(int));
  for (int j = 0; j <= S->n; ++j) S->bnd[j] = (j * tw < L) ? j * tw : L;
  S->ns[0] = n_up; S->ns[1] = n_dn;
  S->key[0] = (uint32_t)seed; S->key[1] = (uint32_t)(seed >> 32);
  S->chain = chain; S->sweep = 0;
  S->s = (int8_t*)calloc((size_t)L * N, 1);
  for (size_t k = 0; k < (size_t)L * N; ++k) S->s[k] = 1;
  for (int sg = 0; sg < 2; ++sg) {
    S->occ[sg] = (int*)calloc(S->ns[sg] ? S->ns[sg] : 1, sizeof(int));
    for (int a = 0; a < S->ns[sg]; ++a) S->occ[sg][a] = a;
    S->QR[sg] = dalloc((S->n + 1) * panel(S, sg));
    S->VR[sg] = dalloc((S->n + 1) * sq(S, sg));
    S->QL[sg] = dalloc((S->n + 1) * panel(S, sg));
    S->VL[sg] = dalloc((S->n + 1) * sq(S, sg));
  }
  /* neighbour lists: each site's distinct bond partners, ascending */
  S->nb_off = (int*)calloc(N + 1, sizeof(int));
  S->nb_site = (int*)calloc(2 * (size_t)(nb ? nb : 1), sizeof(int));
  {
    char* seen = (char*)calloc(N, 1);
    for (int i = 0; i < N; ++i) {
      S->nb_off[i + 1] = S->nb_off[i];
      for (int b = 0; b < nb; ++b) {
        int o = bi[b] == i ? bj[b] : (bj[b] == i ? bi[b] : -1);
        if (o >= 0 && o != i) seen[o] = 1;
      }
      for (int o = 0; o < N; ++o)
        if (seen[o]) { S->nb_site[S->nb_off[i + 1]++] = o; seen[o] = 0; }
    }
    free(seen);
  }
  S->max_records = max_records;
  S->records = dalloc((size_t)(max_records > 0 ? max_records : 1) * NOBS);
  S->want_corr = want_corr;
  if (want_corr) { S->corr_nn = dalloc((size_t)N * N); S->corr_ss = dalloc((size_t)N * N); }
  return S;
}

/* Exact kinetic mode (Eq. 1 with B_l = e^{-dtau K} e^{-dtau V(s_l)} and no
 * checkerboard splitting): B is the dense N x N matrix e^{-dtau K}, row-major,
 * computed by the caller; NULL returns to the checkerboard.  The caller
 * rebuilds the chains afterwards. */
void orc_set_dense_BK(orc_sim* S, const double* B) {
  free(S->BKd);
  S->BKd = NULL;
  if (!B) return;
  S->BKd = dalloc((size_t)S->N * S->N);
  memcpy(S->BKd, B, sizeof(double) * (size_t)S->N * S->N);
}

void orc_destroy(orc_sim* S) {
  if (!S) return;
  free(S->BKd);
  free(S->bi); free(S->bj); free(S->kb); free(S->eps); free(S->sub); free(S->fam_of);
  free(S->nb_off); free(S->nb_site);
  free(S->bc); free(S->bs); free(S->ceps); free(S->bnd); free(S->s);
  for (int sg = 0; sg < 2; ++sg) { free(S->occ[sg]); free(S->QR[sg]); free(S->VR[sg]); free(S->QL[sg]); free(S->VL[sg]); }
  free(S->records); free(S->corr_nn); free(S->corr_ss);
  free(S);
}

/* ------------------------------------------------------------------------ */
/* Chains and weights                                                        */
/* ------------------------------------------------------------------------ */

static void fill_P(const orc_sim* S, int sigma, double* P) {
  int m = S->ns[sigma];
  memset(P, 0, sizeof(double) * panel(S, sigma));
  for (int a = 0; a < m; ++a) P[(size_t)S->occ[sigma][a] * m + a] = 1.0;
}

/* Right chain: Q^R_0 = P, B_j Q^R_{j-1} = Q^R_j V^R_j. */
static void build_right(orc_sim* S, int sigma) {
  int m = S->ns[sigma];
  size_t pn = panel(S, sigma), qn = sq(S, sigma);
  fill_P(S, sigma, S->QR[sigma]);
  for (int j = 1; j <= S->n; ++j) {
    double* X = S->QR[sigma] + j * pn;
    memcpy(X, S->QR[sigma] + (j - 1) * pn, sizeof(double) * pn);
    for (int l = S->bnd[j - 1]; l < S->bnd[j]; ++l) { apply_D(S, X, m, l, sigma); apply_BK(S, X, m); }
    qr_pos(X, S->N, m, S->VR[sigma] + j * qn);
  }
}

/* Left chain: Q^L_n = P, (B_j)^T Q^L_j = Q^L_{j-1} V^L_{j-1}. */
static void build_left(orc_sim* S, int sigma) {
  int m = S->ns[sigma];
  size_t pn = panel(S, sigma), qn = sq(S, sigma);
  fill_P(S, sigma, S->QL[sigma] + S->n * pn);
  for (int j = S->n; j >= 1; --j) {
    double* Z = S->QL[sigma] + (j - 1) * pn;
    memcpy(Z, S->QL[sigma] + j * pn, sizeof(double) * pn);
    for (int l = S->bnd[j] - 1; l >= S->bnd[j - 1]; --l) { apply_BKT(S, Z, m); apply_D(S, Z, m, l, sigma); }
    qr_pos(Z, S->N, m, S->VL[sigma] + (j - 1) * qn);
  }
}

static double charge_log_factor(const orc_sim* S) {
  if (!S->charge) return 0.0;
  long long tot = 0;
  for (size_t k = 0; k < (size_t)S->L * S->N; ++k) tot += S->s[k];
  return -S->lambda * (double)tot;
}

/* log|W| and sign from the right chain: sum log diag V^R + log|det(P^T Q^R_n)|. */
void orc_log_weight(const orc_sim* S, double* logabs, int* sign) {
  double lw = charge_log_factor(S);
  int sg_tot = 1;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    size_t pn = panel(S, sg), qn = sq(S, sg);
    for (int j = 1; j <= S->n; ++j)
      for (int a = 0; a < m; ++a) lw += log(S->VR[sg][j * qn + a * m + a]);
    double* W = dalloc(qn); double* Wi = dalloc(qn);
    const double* Qn = S->QR[sg] + S->n * pn;
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) W[a * m + b] = Qn[(size_t)S->occ[sg][a] * m + b];
    double la; int s1;
    inv_lu(W, m, Wi, &la, &s1);
    lw += la; sg_tot *= s1;
    free(W); free(Wi);
  }
  *logabs = lw; *sign = sg_tot;
}

/* The same weight from the left chain: sum log diag V^L + log|det(Q^L_0^T P)|. */
void orc_log_weight_left(const orc_sim* S, double* logabs, int* sign) {
  double lw = charge_log_factor(S);
  int sg_tot = 1;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    size_t qn = sq(S, sg);
    for (int j = 0; j < S->n; ++j)
      for (int a = 0; a < m; ++a) lw += log(S->VL[sg][j * qn + a * m + a]);
    double* W = dalloc(qn); double* Wi = dalloc(qn);
    const double* Q0 = S->QL[sg];
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) W[a * m + b] = Q0[(size_t)S->occ[sg][b] * m + a];
    double la; int s1;
    inv_lu(W, m, Wi, &la, &s1);
    lw += la; sg_tot *= s1;
    free(W); free(Wi);
  }
  *logabs = lw; *sign = sg_tot;
}

int orc_build_chains(orc_sim* S) {
  for (int sg = 0; sg < 2; ++sg) { build_right(S, sg); build_left(S, sg); }
  orc_log_weight(S, &S->logw, &S->sign);
  return 0;
}

void orc_tracked(const orc_sim* S, double* logabs, int* sign) { *logabs = S->logw; *sign = S->sign; }

/* ------------------------------------------------------------------------ */
/* Configuration setters / initialisation                                   */
/* ------------------------------------------------------------------------ */

int orc_set_fields(orc_sim* S, const int8_t* s) {
  for (size_t k = 0; k < (size_t)S->L * S->N; ++k) {
    if (s[k] != 1 && s[k] != -1) return -1;
    S->s[k] = s[k];
  }
  return orc_build_chains(S);
}

int orc_set_fock(orc_sim* S, const int* up, const int* dn) {
  const int* in[2] = {up, dn};
  for (int sg = 0; sg < 2; ++sg) {
    char* seen = (char*)calloc(S->N, 1);
    for (int a = 0; a < S->ns[sg]; ++a) {
      int i = in[sg][a];
      if (i < 0 || i >= S->N || seen[i]) { free(seen); return -1; }
      seen[i] = 1;
    }
    free(seen);
  }
  for (int sg = 0; sg < 2; ++sg)
    for (int a = 0; a < S->ns[sg]; ++a) S->occ[sg][a] = in[sg][a];
  return orc_build_chains(S);
}

void orc_get_fields(const orc_sim* S, int8_t* s) { memcpy(s, S->s, (size_t)S->L * S->N); }
void orc_get_fock(const orc_sim* S, int* up, int* dn) {
  memcpy(up, S->occ[0], sizeof(int) * S->ns[0]);
  memcpy(dn, S->occ[1], sizeof(int) * S->ns[1]);
}

/* Fields uniform +-1 and occupations by a Fisher-Yates draw, both from Philox
 * with sweep word 0xFFFFFFFF (tags 4 and 5). */
int orc_init_from_seed(orc_sim* S) {
  uint32_t ctr[4], w[4];
  for (int l = 0; l < S->L; ++l)
    for (int i = 0; i < S->N; ++i) {
      ctr[0] = S->chain; ctr[1] = 0xFFFFFFFFu; ctr[2] = (4u << 24) | (uint32_t)l; ctr[3] = (uint32_t)i;
      orc_philox(ctr, S->key, w);
      S->s[(size_t)l * S->N + i] = (w[0] & 1u) ? 1 : -1;
    }
  int* perm = (int*)calloc(S->N, sizeof(int));
  for (int sg = 0; sg < 2; ++sg) {
    for (int i = 0; i < S->N; ++i) perm[i] = i;
    for (int t = 0; t < S->ns[sg]; ++t) {
      ctr[0] = S->chain; ctr[1] = 0xFFFFFFFFu; ctr[2] = (5u << 24) | (uint32_t)sg; ctr[3] = (uint32_t)t;
      orc_philox(ctr, S->key, w);
      int r = t + (int)(u53(w[0], w[1]) * (double)(S->N - t));
      int tmp = perm[t]; perm[t] = perm[r]; perm[r] = tmp;
    }
    /* ascending order of the chosen sites */
    for (int a = 0; a < S->ns[sg]; ++a) S->occ[sg][a] = perm[a];
    for (int a = 1; a < S->ns[sg]; ++a) {
      int v = S->occ[sg][a], b = a - 1;
      while (b >= 0 && S->occ[sg][b] > v) { S->occ[sg][b + 1] = S->occ[sg][b]; --b; }
      S->occ[sg][b + 1] = v;
    }
  }
  free(perm);
  return orc_build_chains(S);
}

/* ------------------------------------------------------------------------ */
/* Field flip at (slice l, site i)                                           */
/* ------------------------------------------------------------------------ */

/* Delta_sigma for flipping s at this site: the new/old ratio of the diagonal
 * factor minus one. */
static double delta_of(const orc_sim* S, int sigma, int8_t s) {
  int sp = S->charge ? 1 : (sigma == 0 ? 1 : -1);
  return (sp * s > 0) ? S->delta_p : S->delta_m;
}

/* g = R_i T L_i^T, the quantity whose 1 - g is G_ii. */
static double g_of(const double* Rrow, const double* T, const double* Lrow, int m) {
  double g = 0.0;
  for (int b = 0; b < m; ++b) {
    double x = 0.0;
    for (int a = 0; a < m; ++a) x += Rrow[a] * T[a * m + b];
    g += x * Lrow[b];
  }
  return g;
}

/* One Metropolis attempt.  Rrow[sigma] is row i of the right panel (scaled on
 * accept), Lrow[sigma] row i of the left panel (L~ transposed), T[sigma] the
 * current (L~ R~)^{-1}. */
static void flip_site(orc_sim* S, int l, int i, double* Rrow[2], const double* Lrow[2], double* T[2], uint32_t tag) {
  int8_t s = S->s[(size_t)l * S->N + i];
  double g[2], d[2], r = 1.0;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    g[sg] = g_of(Rrow[sg], T[sg], Lrow[sg], m);
    d[sg] = delta_of(S, sg, s);
    r *= 1.0 + d[sg] * g[sg];
  }
  if (S->charge) r *= (s > 0) ? exp(2.0 * S->lambda) : exp(-2.0 * S->lambda);
  uint32_t ctr[4] = {S->chain, S->sweep, (tag << 24) | (uint32_t)l, (uint32_t)i}, w[4];
  orc_philox(ctr, S->key, w);
  double u = u53(w[0], w[1]);
  S->cnt[0]++;
  if (!(u < fabs(r))) return;
  S->cnt[1]++;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    if (m == 0 || d[sg] == 0.0) continue;
    double* x = dalloc(m); double* y = dalloc(m);
    for (int b = 0; b < m; ++b) { double acc = 0.0; for (int a = 0; a < m; ++a) acc += Rrow[sg][a] * T[sg][a * m + b]; x[b] = acc; }
    for (int a = 0; a < m; ++a) { double acc = 0.0; for (int b = 0; b < m; ++b) acc += T[sg][a * m + b] * Lrow[sg][b]; y[a] = acc; }
    double c = d[sg] / (1.0 + d[sg] * g[sg]);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) T[sg][a * m + b] -= c * y[a] * x[b];
    for (int a = 0; a < m; ++a) Rrow[sg][a] *= 1.0 + d[sg];
    free(x); free(y);
  }
  S->s[(size_t)l * S->N + i] = (int8_t)(-s);
  S->logw += log(fabs(r));
  if (r < 0) S->sign = -S->sign;
}

/* T = (A^T B)^{-1} for two N x m panels. */
static void block_inverse(const orc_sim* S, const double* A, const double* B, int m, double* T) {
  double* W = dalloc((size_t)m * m);
  gram(A, B, S->N, m, m, W);
  double la; int sg;
  inv_lu(W, m, T, &la, &sg);
  free(W);
}

/* ------------------------------------------------------------------------ */
/* Up pass: stored left panels, live right panel, QR at each block top.      */
/* ------------------------------------------------------------------------ */
static void up_pass(orc_sim* S) {
  int N = S->N;
  for (int j = 1; j <= S->n; ++j) {
    int lo = S->bnd[j - 1], hi = S->bnd[j], nl = hi - lo;
    double *Lp[2], *X[2], *T[2];
    for (int sg = 0; sg < 2; ++sg) {
      int m = S->ns[sg];
      size_t pn = panel(S, sg);
      Lp[sg] = dalloc((size_t)nl * pn);
      /* L~_{hi-1}^T = B_K^T Q^L_j ; L~_l^T = B_K^T D_{l+1} L~_{l+1}^T */
      memcpy(Lp[sg] + (nl - 1) * pn, S->QL[sg] + j * pn, sizeof(double) * pn);
      apply_BKT(S, Lp[sg] + (nl - 1) * pn, m);
      for (int l = hi - 2; l >= lo; --l) {
        double* dst = Lp[sg] + (l - lo) * pn;
        memcpy(dst, Lp[sg] + (l + 1 - lo) * pn, sizeof(double) * pn);
        apply_D(S, dst, m, l + 1, sg);
        apply_BKT(S, dst, m);
      }
      X[sg] = dalloc(pn);
      memcpy(X[sg], S->QR[sg] + (j - 1) * pn, sizeof(double) * pn);
      T[sg] = dalloc(sq(S, sg));
    }
    for (int l = lo; l < hi; ++l) {
      for (int sg = 0; sg < 2; ++sg) apply_D(S, X[sg], S->ns[sg], l, sg);
      if (l == lo)
        for (int sg = 0; sg < 2; ++sg) block_inverse(S, Lp[sg], X[sg], S->ns[sg], T[sg]);
      for (int i = 0; i < N; ++i) {
        double* Rrow[2]; const double* Lrow[2];
        for (int sg = 0; sg < 2; ++sg) {
          int m = S->ns[sg];
          Rrow[sg] = X[sg] + (size_t)i * m;
          Lrow[sg] = Lp[sg] + (l - lo) * panel(S, sg) + (size_t)i * m;
        }
        flip_site(S, l, i, Rrow, Lrow, T, 1u);
      }
      for (int sg = 0; sg < 2; ++sg) apply_BK(S, X[sg], S->ns[sg]);
    }
    for (int sg = 0; sg < 2; ++sg) {
      size_t pn = panel(S, sg);
      memcpy(S->QR[sg] + j * pn, X[sg], sizeof(double) * pn);
      qr_pos(S->QR[sg] + j * pn, N, S->ns[sg], S->VR[sg] + j * sq(S, sg));
      free(Lp[sg]); free(X[sg]); free(T[sg]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Measurement at block boundary jb from Q^L_jb and Q^R_jb                   */
/* ------------------------------------------------------------------------ */

/* obs[0] = sign, obs[1..] = sign * O.  nn, ss (N x N, may be NULL) receive
 * sign * <n_i n_j> and sign * <S_i . S_j>. */
static void measure_boundary(const orc_sim* S, int jb, double* obs, double* nn, double* ss) {
  int N = S->N;
  double *A[2], *QLb[2], *rho[2] = {NULL, NULL};
  double* dens[2];
  int sgn = 1;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    size_t pn = panel(S, sg);
    const double* QRb = S->QR[sg] + jb * pn;
    QLb[sg] = S->QL[sg] + jb * pn;
    double* W = dalloc(sq(S, sg)); double* Tm = dalloc(sq(S, sg));
    gram(QLb[sg], QRb, N, m, m, W);
    double la; int s1;
    inv_lu(W, m, Tm, &la, &s1);
    sgn *= s1;
    A[sg] = dalloc(pn);
    for (int i = 0; i < N; ++i)
      for (int b = 0; b < m; ++b) {
        double acc = 0.0;
        for (int a = 0; a < m; ++a) acc += QRb[(size_t)i * m + a] * Tm[a * m + b];
        A[sg][(size_t)i * m + b] = acc;
      }
    dens[sg] = dalloc(N);
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int b = 0; b < m; ++b) acc += A[sg][(size_t)i * m + b] * QLb[sg][(size_t)i * m + b];
      dens[sg][i] = acc;
    }
    free(W); free(Tm);
  }
  /* rho_ij = <c_i^dag c_j> = sum_b Q^L[i,b] A[j,b] */
#define RHO(sg, i, j) rho_ij(A[sg], QLb[sg], S->ns[sg], i, j)
  double nup = 0, ndn = 0, docc = 0, ekin = 0;
  for (int i = 0; i < N; ++i) { nup += dens[0][i]; ndn += dens[1][i]; docc += dens[0][i] * dens[1][i]; }
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    for (int b = 0; b < S->nb; ++b) {
      int i = S->bi[b], j = S->bj[b];
      double rij = 0, rji = 0;
      for (int q = 0; q < m; ++q) {
        rij += QLb[sg][(size_t)i * m + q] * A[sg][(size_t)j * m + q];
        rji += QLb[sg][(size_t)j * m + q] * A[sg][(size_t)i * m + q];
      }
      ekin += S->kb[b] * (rij + rji);
    }
    for (int i = 0; i < N; ++i) ekin += S->eps[i] * dens[sg][i];
  }
  /* sublattice sums: N^sigma_a and M^sigma_a = sum_{i in a} A[i,:]^T Q^L[i,:] */
  double Na[2][2] = {{0, 0}, {0, 0}};
  double trMM[2][2][2];
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    double* M[2] = {dalloc(sq(S, sg)), dalloc(sq(S, sg))};
    for (int i = 0; i < N; ++i) {
      int a = S->sub[i];
      Na[sg][a] += dens[sg][i];
      for (int p = 0; p < m; ++p)
        for (int q = 0; q < m; ++q) M[a][p * m + q] += A[sg][(size_t)i * m + p] * QLb[sg][(size_t)i * m + q];
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double t = 0.0;
        for (int p = 0; p < m; ++p)
          for (int q = 0; q < m; ++q) t += M[a][p * m + q] * M[b][q * m + p];
        trMM[sg][a][b] = t;
      }
    free(M[0]); free(M[1]);
  }
  double szz[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double t = 0.0;
      for (int sg = 0; sg < 2; ++sg) t += Na[sg][a] * Na[sg][b] + (a == b ? Na[sg][a] : 0.0) - trMM[sg][a][b];
      t -= Na[0][a] * Na[1][b] + Na[1][a] * Na[0][b];
      szz[a][b] = 0.25 * t;
    }
  /* tr(rho_up rho_dn) = sum_{pq} X[p][q] Y[q][p], X = A_dn^T Q^L_up, Y = A_up^T Q^L_dn */
  double trud = 0.0;
  {
    int mu = S->ns[0], md = S->ns[1];
    for (int p = 0; p < md; ++p)
      for (int q = 0; q < mu; ++q) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < N; ++i) {
          x += A[1][(size_t)i * md + p] * QLb[0][(size_t)i * mu + q];
          y += A[0][(size_t)i * mu + q] * QLb[1][(size_t)i * md + p];
        }
        trud += x * y;
      }
  }
  double ncell = N / 2.0;
  double sg = (double)sgn;
  obs[0] = sg;
  obs[1] = sg * nup;
  obs[2] = sg * ndn;
  obs[3] = sg * docc / N;
  obs[4] = sg * ekin / N;
  obs[5] = sg * szz[0][0] / ncell;
  obs[6] = sg * szz[1][1] / ncell;
  obs[7] = sg * szz[0][1] / ncell;
  obs[8] = sg * 0.5 * (nup + ndn - 2.0 * trud) / ncell;
  if (nn || ss) {
    for (int s2 = 0; s2 < 2; ++s2) {
      int m = S->ns[s2];
      rho[s2] = dalloc((size_t)N * N);
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          double acc = 0.0;
          for (int q = 0; q < m; ++q) acc += QLb[s2][(size_t)i * m + q] * A[s2][(size_t)j * m + q];
          rho[s2][(size_t)i * N + j] = acc;
        }
    }
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double d = (i == j) ? 1.0 : 0.0;
        double same[2];
        for (int s2 = 0; s2 < 2; ++s2)
          same[s2] = dens[s2][i] * dens[s2][j] + rho[s2][(size_t)i * N + j] * (d - rho[s2][(size_t)j * N + i]);
        double cross = dens[0][i] * dens[1][j] + dens[1][i] * dens[0][j];
        double nnij = same[0] + same[1] + cross;
        double zz = 0.25 * (same[0] + same[1] - cross);
        double pm = rho[0][(size_t)i * N + j] * (d - rho[1][(size_t)j * N + i]);
        double mp = rho[1][(size_t)i * N + j] * (d - rho[0][(size_t)j * N + i]);
        if (nn) nn[(size_t)i * N + j] = sg * nnij;
        if (ss) ss[(size_t)i * N + j] = sg * (zz + 0.5 * (pm + mp));
      }
    free(rho[0]); free(rho[1]);
  }
#undef RHO
  for (int s2 = 0; s2 < 2; ++s2) { free(A[s2]); free(dens[s2]); }
}

/* ------------------------------------------------------------------------ */
/* Down pass: stored right panels, live left panel, QR at each block bottom, */
/* measurement at each block boundary below a finished block.                */
/* ------------------------------------------------------------------------ */
static void down_pass(orc_sim* S, int measure) {
  int N = S->N;
  double acc[NOBS] = {0};
  int nmeas = 0;
  double *nn = NULL, *ss = NULL;
  if (measure && S->want_corr) { nn = dalloc((size_t)N * N); ss = dalloc((size_t)N * N); }
  /* the swaps changed P: the left chain restarts from Q^L_n = P */
  for (int sg = 0; sg < 2; ++sg) fill_P(S, sg, S->QL[sg] + S->n * panel(S, sg));
  for (int j = S->n; j >= 1; --j) {
    int lo = S->bnd[j - 1], hi = S->bnd[j], nl = hi - lo;
    double *Rp[2], *Z[2], *T[2];
    for (int sg = 0; sg < 2; ++sg) {
      int m = S->ns[sg];
      size_t pn = panel(S, sg);
      Rp[sg] = dalloc((size_t)nl * pn);
      /* R~_lo = D_lo Q^R_{j-1} ; R~_l = D_l B_K R~_{l-1} */
      memcpy(Rp[sg], S->QR[sg] + (j - 1) * pn, sizeof(double) * pn);
      apply_D(S, Rp[sg], m, lo, sg);
      for (int l = lo + 1; l < hi; ++l) {
        double* dst = Rp[sg] + (l - lo) * pn;
        memcpy(dst, Rp[sg] + (l - 1 - lo) * pn, sizeof(double) * pn);
        apply_BK(S, dst, m);
        apply_D(S, dst, m, l, sg);
      }
      Z[sg] = dalloc(pn);
      memcpy(Z[sg], S->QL[sg] + j * pn, sizeof(double) * pn);
      T[sg] = dalloc(sq(S, sg));
    }
    for (int l = hi - 1; l >= lo; --l) {
      for (int sg = 0; sg < 2; ++sg) apply_BKT(S, Z[sg], S->ns[sg]);
      if (l == hi - 1)
        for (int sg = 0; sg < 2; ++sg) block_inverse(S, Z[sg], Rp[sg] + (l - lo) * panel(S, sg), S->ns[sg], T[sg]);
      for (int i = 0; i < N; ++i) {
        double* Rrow[2]; const double* Lrow[2];
        for (int sg = 0; sg < 2; ++sg) {
          int m = S->ns[sg];
          Rrow[sg] = Rp[sg] + (l - lo) * panel(S, sg) + (size_t)i * m;
          Lrow[sg] = Z[sg] + (size_t)i * m;
        }
        flip_site(S, l, i, Rrow, Lrow, T, 2u);
      }
      for (int sg = 0; sg < 2; ++sg) apply_D(S, Z[sg], S->ns[sg], l, sg);
    }
    for (int sg = 0; sg < 2; ++sg) {
      size_t pn = panel(S, sg);
      memcpy(S->QL[sg] + (j - 1) * pn, Z[sg], sizeof(double) * pn);
      qr_pos(S->QL[sg] + (j - 1) * pn, N, S->ns[sg], S->VL[sg] + (j - 1) * sq(S, sg));
      free(Rp[sg]); free(Z[sg]); free(T[sg]);
    }
    if (measure) {
      double obs[NOBS];
      measure_boundary(S, j - 1, obs, nn, ss);
      for (int k = 0; k < NOBS; ++k) acc[k] += obs[k];
      if (nn) {
        for (size_t k = 0; k < (size_t)N * N; ++k) { S->corr_nn[k] += nn[k]; S->corr_ss[k] += ss[k]; }
        S->ncorr++;
      }
      nmeas++;
    }
  }
  if (measure && nmeas > 0 && S->nrec < S->max_records) {
    for (int k = 0; k < NOBS; ++k) S->records[(size_t)S->nrec * NOBS + k] = acc[k] / nmeas;
    S->nrec++;
  }
  free(nn); free(ss);
}

/* ------------------------------------------------------------------------ */
/* Particle-hole swap: removal (Givens) then addition (Gram-Schmidt)         */
/* ------------------------------------------------------------------------ */

typedef struct {
  double logabs; int sign;   /* the swap ratio r = r_rem * r_add */
  double log_rem; int sign_rem;
  double log_add; int sign_add;
  double *Q, *V;             /* trial chain, in the walked chain's storage order */
  double* Tnew;              /* (P''^T Q''_n)^{-1} */
  int* occ_new;
  int valid;
} swap_trial;

/* Removal of column k followed by addition of site j for spin sigma, on the
 * current right chain and T0 = (P^T Q^R_n)^{-1}.  Nothing is committed. */
/* A swap walks one chain from its P end to the far end.  side 0: the right
 * chain, blocks i = 1..n at Q^R_i, V^R_i, propagator B_i.  side 1: the left
 * chain read from tau = beta down to 0, which is the right chain of the
 * transposed propagator B(beta,0)^T = B_1^T ... B_n^T (the weight
 * det[P^T B(beta,0) P] equals det[P^T B(beta,0)^T P]): its block i is
 * Q^L_{n-i}, V^L_{n-i}, with propagator B_{n-i+1}^T. */
static int chain_ix(const orc_sim* S, int side, int i) { return side ? S->n - i : i; }

static void chain_prop(const orc_sim* S, int side, int sigma, int i, double* x) {
  if (!side) {
    for (int l = S->bnd[i - 1]; l < S->bnd[i]; ++l) { apply_D(S, x, 1, l, sigma); apply_BK(S, x, 1); }
  } else {
    int jl = S->n - i + 1;
    for (int l = S->bnd[jl] - 1; l >= S->bnd[jl - 1]; --l) { apply_BKT(S, x, 1); apply_D(S, x, 1, l, sigma); }
  }
}

static void swap_core(const orc_sim* S, int side, int sigma, int k, int j, const double* T0, swap_trial* tr) {
  int N = S->N, m = S->ns[sigma], n = S->n;
  size_t pn = panel(S, sigma), qn = sq(S, sigma);
  tr->Q = dalloc((n + 1) * pn);
  tr->V = dalloc((n + 1) * qn);
  tr->Tnew = dalloc(qn);
  tr->occ_new = (int*)calloc(m, sizeof(int));
  tr->valid = 1;
  memcpy(tr->Q, side ? S->QL[sigma] : S->QR[sigma], sizeof(double) * (n + 1) * pn);
  memcpy(tr->V, side ? S->VL[sigma] : S->VR[sigma], sizeof(double) * (n + 1) * qn);
  /* column order after the permutation U: k moves to the last position */
  int* ord = (int*)calloc(m, sizeof(int));
  for (int a = 0, t = 0; a < m; ++a) if (a != k) ord[t++] = a;
  ord[m - 1] = k;
  int nrot = m - 1 - k;                       /* rotations on rows (q, q+1), q = k..m-2 */
  double* rc = dalloc(nrot > 0 ? nrot : 1);
  double* rs = dalloc(nrot > 0 ? nrot : 1);
  double log_rN = 0.0; int sign_rN = 1;
  double* A = dalloc(qn);
  for (int i = 1; i <= n; ++i) {
    double* Vi = tr->V + chain_ix(S, side, i) * qn;
    if (i == 1) {
      for (int a = 0; a < m; ++a) for (int b = 0; b < m; ++b) A[a * m + b] = Vi[a * m + ord[b]];
    } else {
      memcpy(A, Vi, sizeof(double) * qn);
      for (int t = 0; t < nrot; ++t) {         /* A <- A G_{i-1}^T */
        int q = k + t; double c = rc[t], s = rs[t];
        for (int a = 0; a < m; ++a) {
          double x = A[a * m + q], y = A[a * m + q + 1];
          A[a * m + q] = c * x + s * y;
          A[a * m + q + 1] = -s * x + c * y;
        }
      }
    }
    for (int t = 0; t < nrot; ++t) {           /* G_i: zero the subdiagonal */
      int q = k + t;
      double a = A[q * m + q], b = A[(q + 1) * m + q];
      double r = hypot(a, b), c = 1.0, s = 0.0;
      if (r != 0.0) { c = a / r; s = b / r; }
      rc[t] = c; rs[t] = s;
      for (int col = 0; col < m; ++col) {
        double x = A[q * m + col], y = A[(q + 1) * m + col];
        A[q * m + col] = c * x + s * y;
        A[(q + 1) * m + col] = -s * x + c * y;
      }
      A[q * m + q] = r;
      A[(q + 1) * m + q] = 0.0;
    }
    memcpy(Vi, A, sizeof(double) * qn);
    double* Qi = tr->Q + chain_ix(S, side, i) * pn;  /* Q_i' = Q_i G_i^T */
    for (int row = 0; row < N; ++row)
      for (int t = 0; t < nrot; ++t) {
        int q = k + t; double c = rc[t], s = rs[t];
        double x = Qi[(size_t)row * m + q], y = Qi[(size_t)row * m + q + 1];
        Qi[(size_t)row * m + q] = c * x + s * y;
        Qi[(size_t)row * m + q + 1] = -s * x + c * y;
      }
    double d = A[(m - 1) * m + (m - 1)];
    if (d < 0) sign_rN = -sign_rN;
    log_rN += log(fabs(d));
  }
  /* M^{-1} = G_n T0 U */
  double* Mi = dalloc(qn);
  for (int a = 0; a < m; ++a) for (int b = 0; b < m; ++b) Mi[a * m + b] = T0[a * m + ord[b]];
  for (int t = 0; t < nrot; ++t) {
    int q = k + t; double c = rc[t], s = rs[t];
    for (int col = 0; col < m; ++col) {
      double x = Mi[q * m + col], y = Mi[(q + 1) * m + col];
      Mi[q * m + col] = c * x + s * y;
      Mi[(q + 1) * m + col] = -s * x + c * y;
    }
  }
  double mNN = Mi[(m - 1) * m + (m - 1)];
  tr->log_rem = log(fabs(mNN)) - log_rN;
  tr->sign_rem = ((mNN < 0) ? -1 : 1) * sign_rN;
  if (mNN == 0.0) tr->valid = 0;
  /* downdate (Eq. S12) to the (m-1) x (m-1) inverse of the reduced system */
  int mr = m - 1;
  double* Tp = dalloc((size_t)mr * mr);
  for (int a = 0; a < mr; ++a)
    for (int b = 0; b < mr; ++b)
      Tp[a * (mr ? mr : 1) + b] = Mi[a * m + b] - Mi[a * m + (m - 1)] * Mi[(m - 1) * m + b] / mNN;
  int* occr = (int*)calloc(m, sizeof(int));
  for (int a = 0; a < mr; ++a) occr[a] = S->occ[sigma][ord[a]];
  /* addition of site j to the reduced chain; Q'_i = first mr columns of tr->Q */
  double* q = dalloc(N);
  double* w = dalloc(N);
  double* v = dalloc(m); double* v2 = dalloc(m);
  q[j] = 1.0;
  double log_rho = 0.0;
  for (int i = 1; i <= n && tr->valid; ++i) {
    memcpy(w, q, sizeof(double) * N);
    chain_prop(S, side, sigma, i, w);
    double* Qi = tr->Q + chain_ix(S, side, i) * pn;
    for (int a = 0; a < mr; ++a) { double acc = 0.0; for (int r = 0; r < N; ++r) acc += Qi[(size_t)r * m + a] * w[r]; v[a] = acc; }
    for (int r = 0; r < N; ++r) { double acc = 0.0; for (int a = 0; a < mr; ++a) acc += Qi[(size_t)r * m + a] * v[a]; w[r] -= acc; }
    for (int a = 0; a < mr; ++a) { double acc = 0.0; for (int r = 0; r < N; ++r) acc += Qi[(size_t)r * m + a] * w[r]; v2[a] = acc; }
    for (int r = 0; r < N; ++r) { double acc = 0.0; for (int a = 0; a < mr; ++a) acc += Qi[(size_t)r * m + a] * v2[a]; w[r] -= acc; }
    for (int a = 0; a < mr; ++a) v[a] += v2[a];
    double rho = 0.0;
    for (int r = 0; r < N; ++r) rho += w[r] * w[r];
    rho = sqrt(rho);
    if (rho == 0.0) { tr->valid = 0; break; }
    for (int r = 0; r < N; ++r) q[r] = w[r] / rho;
    for (int r = 0; r < N; ++r) Qi[(size_t)r * m + (m - 1)] = q[r];
    double* Vi = tr->V + chain_ix(S, side, i) * qn;
    for (int a = 0; a < mr; ++a) { Vi[a * m + (m - 1)] = v[a]; Vi[(m - 1) * m + a] = 0.0; }
    Vi[(m - 1) * m + (m - 1)] = rho;
    log_rho += log(rho);
  }
  double s_add = 0.0;
  double* av = dalloc(m); double* bv = dalloc(m);
  if (tr->valid) {
    const double* Qn = tr->Q + chain_ix(S, side, n) * pn;
    for (int a = 0; a < mr; ++a) {
      double acc = 0.0;
      for (int b = 0; b < mr; ++b) acc += Tp[a * mr + b] * q[occr[b]];
      av[a] = acc;
    }
    for (int b = 0; b < mr; ++b) {
      double acc = 0.0;
      for (int a = 0; a < mr; ++a) acc += Qn[(size_t)j * m + a] * Tp[a * mr + b];
      bv[b] = acc;
    }
    s_add = q[j];
    for (int a = 0; a < mr; ++a) s_add -= Qn[(size_t)j * m + a] * av[a];
    if (s_add == 0.0) tr->valid = 0;
  }
  tr->log_add = log(fabs(s_add)) + log_rho;
  tr->sign_add = (s_add < 0) ? -1 : 1;
  tr->logabs = tr->log_rem + tr->log_add;
  tr->sign = tr->sign_rem * tr->sign_add;
  if (!tr->valid) { tr->logabs = -INFINITY; }
  /* bordered inverse (Eq. S8) and the new column order */
  if (tr->valid) {
    for (int a = 0; a < mr; ++a)
      for (int b = 0; b < mr; ++b) tr->Tnew[a * m + b] = Tp[a * mr + b] + av[a] * bv[b] / s_add;
    for (int a = 0; a < mr; ++a) { tr->Tnew[a * m + (m - 1)] = -av[a] / s_add; tr->Tnew[(m - 1) * m + a] = -bv[a] / s_add; }
    tr->Tnew[(m - 1) * m + (m - 1)] = 1.0 / s_add;
    for (int a = 0; a < mr; ++a) tr->occ_new[a] = occr[a];
    tr->occ_new[m - 1] = j;
    double* P = tr->Q + chain_ix(S, side, 0) * pn;
    memset(P, 0, sizeof(double) * pn);
    for (int a = 0; a < m; ++a) P[(size_t)tr->occ_new[a] * m + a] = 1.0;
  }
  free(ord); free(rc); free(rs); free(A); free(Mi); free(Tp); free(occr);
  free(q); free(w); free(v); free(v2); free(av); free(bv);
}

static void free_trial(swap_trial* tr) { free(tr->Q); free(tr->V); free(tr->Tnew); free(tr->occ_new); }

/* T0 = (P^T Q^R_n)^{-1} (side 0) or (P^T Q^L_0)^{-1} (side 1) */
static void pq_inverse(const orc_sim* S, int side, int sigma, double* T0) {
  int m = S->ns[sigma];
  size_t pn = panel(S, sigma);
  double* W = dalloc(sq(S, sigma));
  const double* Qn = side ? S->QL[sigma] : (S->QR[sigma] + S->n * pn);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) W[a * m + b] = Qn[(size_t)S->occ[sigma][a] * m + b];
  double la; int sg;
  inv_lu(W, m, T0, &la, &sg);
  free(W);
}

static int jth_empty(const orc_sim* S, int sigma, int jidx) {
  char* occd = (char*)calloc(S->N, 1);
  for (int a = 0; a < S->ns[sigma]; ++a) occd[S->occ[sigma][a]] = 1;
  int site = -1;
  for (int i = 0, t = 0; i < S->N; ++i)
    if (!occd[i]) { if (t == jidx) { site = i; break; } ++t; }
  free(occd);
  return site;
}

/* N_up then N_dn swap attempts on one chain: side 0 at tau = beta on the
 * right chain after the up pass, side 1 at tau = 0 on the left chain after the
 * down pass (random-number tag 3 and 6). */
static void swap_phase(orc_sim* S, int side) {
  const uint32_t tag = side ? 6u : 3u;
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    if (m == 0 || m == S->N) continue;
    size_t pn = panel(S, sg), qn = sq(S, sg);
    double* T0 = dalloc(qn);
    pq_inverse(S, side, sg, T0);
    for (int att = 0; att < m; ++att) {
      uint32_t ctr[4] = {S->chain, S->sweep, (tag << 24) | ((uint32_t)sg << 16) | (uint32_t)att, 0u}, w[4], w2[4];
      orc_philox(ctr, S->key, w);
      ctr[3] = 1u;
      orc_philox(ctr, S->key, w2);
      int k = (int)(u53(w[0], w[1]) * (double)m);
      double u = u53(w2[0], w2[1]);
      int j;
      double log_hastings = 0.0;
      if (S->swap_mode == 0) {
        int jidx = (int)(u53(w[2], w[3]) * (double)(S->N - m));
        j = jth_empty(S, sg, jidx);
      } else {
        /* target: uniform among the empty neighbours E(i) of i = occ[k]; the
         * reverse move picks i among the empty neighbours E'(j) of j after the
         * move, so the Metropolis-Hastings factor is |E(i)| / |E'(j)| */
        int i = S->occ[sg][k], ne = 0;
        char* occd = (char*)calloc(S->N, 1);
        for (int a = 0; a < m; ++a) occd[S->occ[sg][a]] = 1;
        for (int t = S->nb_off[i]; t < S->nb_off[i + 1]; ++t) ne += !occd[S->nb_site[t]];
        if (ne == 0) {  /* no move: a rejected attempt */
          free(occd);
          S->cnt[2]++;
          continue;
        }
        int jidx = (int)(u53(w[2], w[3]) * (double)ne);
        j = -1;
        for (int t = S->nb_off[i], c = 0; t < S->nb_off[i + 1]; ++t)
          if (!occd[S->nb_site[t]]) { if (c == jidx) { j = S->nb_site[t]; break; } ++c; }
        occd[i] = 0;
        occd[j] = 1;
        int ne2 = 0;
        for (int t = S->nb_off[j]; t < S->nb_off[j + 1]; ++t) ne2 += !occd[S->nb_site[t]];
        free(occd);
        /* mode 2 leaves the factor out on purpose: the tests use it to show
         * that the ED comparison detects a missing Hastings correction */
        log_hastings = (S->swap_mode == 2) ? 0.0 : log((double)ne) - log((double)ne2);
      }
      swap_trial tr;
      swap_core(S, side, sg, k, j, T0, &tr);
      S->cnt[2]++;
      const double lacc = tr.logabs + log_hastings;
      int accept = tr.valid && (lacc >= 0.0 || u < exp(lacc));
      if (accept) {
        S->cnt[3]++;
        memcpy(side ? S->QL[sg] : S->QR[sg], tr.Q, sizeof(double) * (S->n + 1) * pn);
        memcpy(side ? S->VL[sg] : S->VR[sg], tr.V, sizeof(double) * (S->n + 1) * qn);
        memcpy(T0, tr.Tnew, sizeof(double) * qn);
        memcpy(S->occ[sg], tr.occ_new, sizeof(int) * m);
        S->logw += tr.logabs;
        S->sign *= tr.sign;
      }
      free_trial(&tr);
    }
    free(T0);
    /* the next up pass starts the right chain from Q^R_0 = P */
    if (side) fill_P(S, sg, S->QR[sg]);
  }
}

/* ------------------------------------------------------------------------ */
/* Sweeps and hooks                                                          */
/* ------------------------------------------------------------------------ */

void orc_sweep(orc_sim* S, int nsweeps, int measure) {
  for (int t = 0; t < nsweeps; ++t) {
    up_pass(S);
    swap_phase(S, 0);
    down_pass(S, measure);
    if (S->left_swaps) swap_phase(S, 1);
    S->sweep++;
  }
}

/* Ratio of flipping s at (slice l, site i), through the stabilized Green's
 * function at that slice, on freshly built chains. */
double orc_field_ratio(orc_sim* S, int l, int i) {
  orc_build_chains(S);
  int j = 1;
  while (S->bnd[j] <= l) ++j;
  double r = 1.0;
  int8_t s = S->s[(size_t)l * S->N + i];
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    size_t pn = panel(S, sg);
    double* X = dalloc(pn); double* Z = dalloc(pn); double* T = dalloc(sq(S, sg));
    memcpy(X, S->QR[sg] + (j - 1) * pn, sizeof(double) * pn);
    for (int ll = S->bnd[j - 1]; ll <= l; ++ll) { apply_D(S, X, m, ll, sg); if (ll < l) apply_BK(S, X, m); }
    memcpy(Z, S->QL[sg] + j * pn, sizeof(double) * pn);
    for (int ll = S->bnd[j] - 1; ll >= l; --ll) { apply_BKT(S, Z, m); if (ll > l) apply_D(S, Z, m, ll, sg); }
    block_inverse(S, Z, X, m, T);
    double g = g_of(X + (size_t)i * m, T, Z + (size_t)i * m, m);
    r *= 1.0 + delta_of(S, sg, s) * g;
    free(X); free(Z); free(T);
  }
  if (S->charge) r *= (s > 0) ? exp(2.0 * S->lambda) : exp(-2.0 * S->lambda);
  return r;
}

/* Ratio of the swap (remove column k, add site j) for one spin on freshly
 * built chains, walked along the right (side 0) or left (side 1) chain; the
 * removal and addition factors are returned separately. */
double orc_swap_ratio_side(orc_sim* S, int side, int sigma, int k, int j, double* out /* log|r|, sign, log|r_rem|, sign_rem, log|r_add|, sign_add */) {
  orc_build_chains(S);
  double* T0 = dalloc(sq(S, sigma));
  pq_inverse(S, side, sigma, T0);
  swap_trial tr;
  swap_core(S, side, sigma, k, j, T0, &tr);
  out[0] = tr.logabs; out[1] = tr.sign; out[2] = tr.log_rem; out[3] = tr.sign_rem;
  out[4] = tr.log_add; out[5] = tr.sign_add;
  double r = tr.sign * exp(tr.logabs);
  free_trial(&tr); free(T0);
  return r;
}

double orc_swap_ratio(orc_sim* S, int sigma, int k, int j, double* out) {
  return orc_swap_ratio_side(S, 0, sigma, k, j, out);
}

/* Measurement on freshly built chains at block boundary jb (0..n). */
void orc_measure_at(orc_sim* S, int jb, double* obs, double* nn, double* ss) {
  orc_build_chains(S);
  measure_boundary(S, jb, obs, nn, ss);
}

int orc_num_records(const orc_sim* S) { return S->nrec; }
void orc_get_records(const orc_sim* S, double* out) { memcpy(out, S->records, sizeof(double) * (size_t)S->nrec * NOBS); }
void orc_clear_records(orc_sim* S) {
  S->nrec = 0; S->ncorr = 0;
  if (S->corr_nn) { memset(S->corr_nn, 0, sizeof(double) * (size_t)S->N * S->N); memset(S->corr_ss, 0, sizeof(double) * (size_t)S->N * S->N); }
}
long long orc_get_corr(const orc_sim* S, double* nn, double* ss) {
  if (!S->want_corr) return 0;
  memcpy(nn, S->corr_nn, sizeof(double) * (size_t)S->N * S->N);
  memcpy(ss, S->corr_ss, sizeof(double) * (size_t)S->N * S->N);
  return S->ncorr;
}

/* side 0: right chain (j = 0..n, V for j >= 1), side 1: left chain (V for j <= n-1) */
void orc_get_chain(const orc_sim* S, int side, int sigma, int j, double* Q, double* V) {
  size_t pn = panel(S, sigma), qn = sq(S, sigma);
  const double* Qs = side ? S->QL[sigma] : S->QR[sigma];
  const double* Vs = side ? S->VL[sigma] : S->VR[sigma];
  if (Q) memcpy(Q, Qs + j * pn, sizeof(double) * pn);
  if (V) memcpy(V, Vs + j * qn, sizeof(double) * qn);
}

/* Dense B_K (N x N) and the per-slice propagator B_l^sigma = B_K D_l^sigma. */
void orc_get_BK(const orc_sim* S, double* dense) {
  int N = S->N;
  /* columns of B_K = B_K applied to unit vectors; X = I (N x N) as a panel */
  memset(dense, 0, sizeof(double) * (size_t)N * N);
  for (int i = 0; i < N; ++i) dense[(size_t)i * N + i] = 1.0;
  apply_BK(S, dense, N);
}

void orc_stats(const orc_sim* S, long long* out) { for (int k = 0; k < 4; ++k) out[k] = S->cnt[k]; }

/* ints: N, L, tw, n, G, n_up, n_dn, charge, sweep; doubles: lambda */
void orc_info(const orc_sim* S, int* ints, double* dbl) {
  ints[0] = S->N; ints[1] = S->L; ints[2] = S->tw; ints[3] = S->n; ints[4] = S->G;
  ints[5] = S->ns[0]; ints[6] = S->ns[1]; ints[7] = S->charge; ints[8] = (int)S->sweep;
  dbl[0] = S->lambda;
}

void orc_get_families(const orc_sim* S, int* fam) { memcpy(fam, S->fam_of, sizeof(int) * S->nb); }

void orc_set_sweep(orc_sim* S, uint32_t sweep) { S->sweep = sweep; }
void orc_set_swap_mode(orc_sim* S, int mode) { S->swap_mode = mode; }
void orc_set_left_swaps(orc_sim* S, int on) { S->left_swaps = on ? 1 : 0; }

/* ------------------------------------------------------------------------ */
/* Constrained-path inner loop for one Fock state (SM Sec. VI)               */
/* ------------------------------------------------------------------------ */

/* log|det| and sign of the overlap Psi^T Phi of two N x m panels (m = 0: 1). */
static void overlap_det(const double* Psi, const double* Phi, int N, int m, double* la, int* sg) {
  *la = 0.0; *sg = 1;
  if (m == 0) return;
  double* W = dalloc((size_t)m * m); double* Wi = dalloc((size_t)m * m);
  gram(Psi, Phi, N, m, m, W);
  inv_lu(W, m, Wi, la, sg);
  free(W); free(Wi);
}

/* Trial panels Psi_l = (B_K^T)^{L-l} P, l = 0..L-1, per spin (N x m each,
 * columns orthonormalized: a right factor cancels in every ratio). */
static void cp_trials(const orc_sim* S, double* Psi[2]) {
  double* R = dalloc((size_t)S->N * S->N);
  for (int sg = 0; sg < 2; ++sg) {
    int m = S->ns[sg];
    size_t pn = panel(S, sg);
    Psi[sg] = dalloc((size_t)S->L * pn);
    double* X = dalloc(pn);
    fill_P(S, sg, X);
    for (int l = S->L - 1; l >= 0; --l) {
      apply_BKT(S, X, m);
      qr_pos(X, S->N, m, R);
      memcpy(Psi[sg] + (size_t)l * pn, X, sizeof(double) * pn);
    }
    free(X);
  }
  free(R);
}

/* One walker through slice l: at each site i draw s = +-1 with probability
 * proportional to (1/2) max(0, r(s)), r(s) = prod_sigma
 * det(Psi_l^T D_i(s) Phi) / det(Psi_l^T Phi) (times the charge-channel scalar
 * e^{-lambda s} for U < 0), multiply the weight by
 * (1/2) [max(0, r(+1)) + max(0, r(-1))] and apply D_i(s) to row i; then
 * Phi <- B_K Phi and re-orthonormalize (with the trial advanced one slice the
 * kinetic step leaves the overlap unchanged, and a right factor of Phi
 * cancels in every ratio).  Philox counter (c0, c1, tag<<24 | l, i).
 * Returns the slice's weight factor; 0 drops the walker (Phi then unused). */
static double cp_slice(const orc_sim* S, double* const Psi[2], double* Phi[2], double* Tr[2], int l, uint32_t c0,
                       uint32_t c1, uint32_t tag) {
  int N = S->N;
  double factor = 1.0;
  for (int i = 0; i < N; ++i) {
    double a[2];
    for (int t = 0; t < 2; ++t) {
      int8_t s = t ? -1 : 1;
      double r = S->charge ? exp(-S->lambda * s) : 1.0;
      for (int sg = 0; sg < 2; ++sg) {
        int m = S->ns[sg];
        if (m == 0) continue;
        const double* Ps = Psi[sg] + (size_t)l * panel(S, sg);
        double la0, la1; int s0, s1;
        overlap_det(Ps, Phi[sg], N, m, &la0, &s0);
        memcpy(Tr[sg], Phi[sg], sizeof(double) * panel(S, sg));
        for (int c = 0; c < m; ++c) Tr[sg][(size_t)i * m + c] *= dfac(S, sg, s);
        overlap_det(Ps, Tr[sg], N, m, &la1, &s1);
        r *= (double)(s0 * s1) * exp(la1 - la0);
      }
      a[t] = 0.5 * (r > 0.0 ? r : 0.0);
    }
    double tot = a[0] + a[1];
    if (!(tot > 0.0)) return 0.0;
    factor *= tot;
    uint32_t ctr[4] = {c0, c1, (tag << 24) | (uint32_t)l, (uint32_t)i}, w[4];
    orc_philox(ctr, S->key, w);
    int8_t s = (u53(w[0], w[1]) * tot < a[0]) ? 1 : -1;
    for (int sg = 0; sg < 2; ++sg)
      for (int c = 0; c < S->ns[sg]; ++c) Phi[sg][(size_t)i * S->ns[sg] + c] *= dfac(S, sg, s);
  }
  double* R = dalloc((size_t)N * N);
  for (int sg = 0; sg < 2; ++sg) {
    apply_BK(S, Phi[sg], S->ns[sg]);
    qr_pos(Phi[sg], N, S->ns[sg], R);
  }
  free(R);
  return factor;
}

/* n_walkers independent walkers of the inner loop for the current Fock state
 * eta (the columns of P), with the fields sampled afresh.  The trial state
 * at slice l is Psi_l^T = P^T e^{-(beta - tau_l) H_0} = P^T B_K^{L-l}: all
 * that still acts on the walker after the fields of slice l, with the fields
 * off.  A walker starts at Phi = P with weight 1 and goes through the slices
 * (cp_slice); a walker whose factor is 0 has crossed the node of the trial
 * and is dropped (weight 0).  Without such truncation the mean weight is
 * R(eta) = sum_s 2^{-LN} <eta|U(s)|eta> / <eta|e^{-beta H_0}|eta>.  Random
 * numbers: Philox counter (walker, sweep, 7<<24 | slice, site).  Returns the
 * number of dropped walkers; weights go to w_out[n_walkers]. */
int orc_cp_walk(orc_sim* S, int n_walkers, double* w_out) {
  int dropped = 0;
  double* Psi[2]; double* Phi[2]; double* Tr[2];
  cp_trials(S, Psi);
  for (int sg = 0; sg < 2; ++sg) { Phi[sg] = dalloc(panel(S, sg)); Tr[sg] = dalloc(panel(S, sg)); }
  for (int wk = 0; wk < n_walkers; ++wk) {
    double weight = 1.0;
    for (int sg = 0; sg < 2; ++sg) fill_P(S, sg, Phi[sg]);
    for (int l = 0; l < S->L && weight > 0.0; ++l) weight *= cp_slice(S, Psi, Phi, Tr, l, (uint32_t)wk, S->sweep, 7u);
    if (!(weight > 0.0)) { weight = 0.0; dropped++; }
    w_out[wk] = weight;
  }
  for (int sg = 0; sg < 2; ++sg) { free(Psi[sg]); free(Phi[sg]); free(Tr[sg]); }
  return dropped;
}

/* Systematic ("comb") resampling (Kitagawa 1996): n new walkers from n old
 * ones with weights w (total > 0), one uniform u in [0, 1): new walker k
 * copies the first old walker whose cumulative weight exceeds (k + u)/n of
 * the total.  Old walker j is copied floor or ceil of n w_j / sum(w) times,
 * and n w_j / sum(w) times on average over u; weight-0 walkers never. */
void orc_comb(const double* w, int n, double u, int* src_out) {
  double tot = 0.0;
  for (int j = 0; j < n; ++j) tot += w[j];
  double cum = w[0];
  for (int k = 0, src = 0; k < n; ++k) {
    double pos = (k + u) / n * tot;
    while (src < n - 1 && cum <= pos) cum += w[++src];
    src_out[k] = src;
  }
}

/* A branching population of n_walkers for the current Fock state: the
 * walkers go through the slices as in orc_cp_walk; after every comb_every
 * slices (and after the last) the population's mean weight joins the
 * estimate, and n_walkers new walkers are drawn from the old ones with
 * probabilities proportional to their weights (orc_comb).  New walkers carry weight 1; dropped walkers (weight 0) are never drawn.
 * The estimate of R(eta) is the product of the mean weights, an unbiased
 * estimator of the unconstrained R(eta) when nothing is truncated (the
 * normalizing-constant property of sequential Monte Carlo).  run selects
 * the random numbers: Philox counters (slot, run, 8<<24 | slice, site) for
 * the fields and (run, 0xFFFFFFFD, 9<<24 | slice, 0) for the comb.  Returns
 * log of the estimate (-inf when every walker was dropped). */
double orc_cp_population(orc_sim* S, int n_walkers, int comb_every, uint32_t run) {
  double* Psi[2]; double* Phi[2]; double* Nw[2]; double* Tr[2];
  cp_trials(S, Psi);
  for (int sg = 0; sg < 2; ++sg) {
    Phi[sg] = dalloc((size_t)n_walkers * panel(S, sg));
    Nw[sg] = dalloc((size_t)n_walkers * panel(S, sg));
    Tr[sg] = dalloc(panel(S, sg));
    for (int k = 0; k < n_walkers; ++k) fill_P(S, sg, Phi[sg] + (size_t)k * panel(S, sg));
  }
  double* w = dalloc(n_walkers);
  int* src = (int*)calloc(n_walkers, sizeof(int));
  for (int k = 0; k < n_walkers; ++k) w[k] = 1.0;
  double log_est = 0.0;
  for (int l = 0; l < S->L; ++l) {
    for (int k = 0; k < n_walkers; ++k) {
      if (!(w[k] > 0.0)) continue;
      double* Pk[2] = {Phi[0] + (size_t)k * panel(S, 0), Phi[1] + (size_t)k * panel(S, 1)};
      w[k] *= cp_slice(S, Psi, Pk, Tr, l, (uint32_t)k, run, 8u);
    }
    if ((comb_every > 0 && (l + 1) % comb_every == 0) || l == S->L - 1) {
      double tot = 0.0;
      for (int k = 0; k < n_walkers; ++k) tot += w[k];
      if (!(tot > 0.0)) { log_est = -INFINITY; break; }
      log_est += log(tot / n_walkers);
      if (l == S->L - 1) break;
      uint32_t ctr[4] = {run, 0xFFFFFFFDu, (9u << 24) | (uint32_t)l, 0u}, rw[4];
      orc_philox(ctr, S->key, rw);
      orc_comb(w, n_walkers, u53(rw[0], rw[1]), src);
      for (int k = 0; k < n_walkers; ++k)
        for (int sg = 0; sg < 2; ++sg)
          memcpy(Nw[sg] + (size_t)k * panel(S, sg), Phi[sg] + (size_t)src[k] * panel(S, sg),
                 sizeof(double) * panel(S, sg));
      for (int sg = 0; sg < 2; ++sg) { double* t = Phi[sg]; Phi[sg] = Nw[sg]; Nw[sg] = t; }
      for (int k = 0; k < n_walkers; ++k) w[k] = 1.0;
    }
  }
  for (int sg = 0; sg < 2; ++sg) { free(Psi[sg]); free(Phi[sg]); free(Nw[sg]); free(Tr[sg]); }
  free(w); free(src);
  return log_est;
}
