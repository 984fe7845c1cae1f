// Internal view of a host lattice object (family-sorted bond tables built
// when the lattice is created) and the shared error setter.
#pragma once
#include <cmath>
#include <string>

#include "../../include/lecqmc.h"

struct lq_lattice_view {
  int N, nb, G;
  bool has_eps;
  const int* fam_off;      // G + 1 offsets into the sorted bond arrays
  const int* sorted_i;     // bonds sorted by family (stable in build order)
  const int* sorted_j;
  const double* sorted_k;
  const double* eps;       // N onsite terms
  const int* sub;          // N sublattice labels
  const int* nb_off;       // N + 1 offsets into nb_site
  const int* nb_site;      // each site's distinct bond partners, ascending
  // K in compressed rows (bonds summed, onsite term on the diagonal)
  int nnz;
  const int* k_off;
  const int* k_col;
  const double* k_val;
  double k_rownorm;        // max_i sum_j |K_ij|
};

lq_lattice_view lq_lattice_get_view(const lq_lattice* L);
lq_status lq_internal_fail(lq_status s, const std::string& msg);

// Factors of the checkerboard propagator for a Trotter step dtau: the exact
// 2x2 bond exponential e^{-dtau k (|i><j| + |j><i|)} has cosh(dtau k) on the
// diagonal and -sinh(dtau k) off it, and the onsite factor is e^{-dtau eps}.
// Every table is built on the host with these same expressions, so two
// entry points given the same lattice and dtau hold bit-identical tables.
static inline void lq_bond_factors(double dtau, double k, double* c, double* s) {
  *c = std::cosh(dtau * k);
  *s = -std::sinh(dtau * k);
}
static inline double lq_onsite_factor(double dtau, double eps) { return std::exp(-dtau * eps); }

// Checkerboard families in the two-FMA form: bit g is set when every bond of
// family g has the same cosh c_g and the family holds N/2 bonds.  Families
// never repeat a site, so such a family holds every site exactly once and its
// factor is c_g times [[1, t], [t, 1]] blocks with t = -tanh(dtau k_b); the
// scalar c_g commutes with everything and is applied once per slice.
// *cprod is the product of those c_g.  Only the first 32 families qualify.
static inline unsigned lq_uniform_families(const lq_lattice_view& v, double dtau, double* cprod) {
  unsigned mask = 0;
  *cprod = 1.0;
  if (v.N & 1) return 0;
  for (int g = 0; g < v.G && g < 32; ++g) {
    const int b0 = v.fam_off[g], b1 = v.fam_off[g + 1];
    if (2 * (b1 - b0) != v.N) continue;
    double c0, s0, c, s;
    lq_bond_factors(dtau, v.sorted_k[b0], &c0, &s0);
    bool ok = true;
    for (int b = b0; b < b1 && ok; ++b) {
      lq_bond_factors(dtau, v.sorted_k[b], &c, &s);
      ok = c == c0 && v.sorted_i[b] != v.sorted_j[b];
    }
    if (!ok) continue;
    mask |= 1u << g;
    *cprod *= c0;
  }
  return mask;
}
static inline double lq_bond_tanh(double dtau, double k) { return -std::tanh(dtau * k); }

// Degree of the Taylor polynomial that stands for e^{-dtau K} in the exact
// kinetic mode, for theta = dtau max_i sum_j |K_ij| >= ||dtau K||: the
// smallest q whose remainder bound theta^{q+1} / (q+1)! / (1 - theta/(q+2))
// is below 1e-17 e^{-theta}, a lower bound of the smallest singular value of
// e^{-dtau K}, i.e. below 1e-17 relative to every column the propagator
// produces.  Exact chains need theta <= LQ_EXACT_THETA_MAX.
#define LQ_EXACT_THETA_MAX 2.0
static inline int lq_taylor_degree(double theta) {
  double term = theta;  // theta^{q+1} / (q+1)! at q = 0
  for (int q = 1; q <= 64; ++q) {
    term *= theta / (double)(q + 1);
    const double tail = term / (1.0 - theta / (double)(q + 2));
    if (tail <= 1e-17 * std::exp(-theta)) return q;
  }
  return 64;
}
