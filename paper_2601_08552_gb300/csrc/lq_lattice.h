// Internal view of a host lattice object (family-sorted bond tables built
// when the lattice is created) and the shared error setter.
#pragma once
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
};

lq_lattice_view lq_lattice_get_view(const lq_lattice* L);
lq_status lq_internal_fail(lq_status s, const std::string& msg);
