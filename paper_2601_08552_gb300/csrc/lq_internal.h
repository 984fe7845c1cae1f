// Internal hooks of the simulation object used by the serving loop.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/lecqmc.h"
#include "lq_device.h"

struct lq_sim_launch_info {
  LqChainDev* d_chains;  // device descriptors of the simulation's chains
  int n_chains, prec, M, Nmax, buf_bytes;
  size_t arena_bytes;
};
lq_sim_launch_info lq_internal_sim_info(const lq_sim* sim);
// after a foreign launch wrote the descriptors, drop the cached host copy
void lq_internal_sim_invalidate(lq_sim* sim);
// device footprint a one-chain simulation of this lattice and these parameters needs
size_t lq_internal_footprint(const lq_lattice* lat, const lq_params* p);
// sign-weighted means <sign O>/<sign> over per-sweep records and jackknife errors over nbins bins
void lq_internal_obs_stats(const double* rec, int n, int nbins, double* mean, double* err);
