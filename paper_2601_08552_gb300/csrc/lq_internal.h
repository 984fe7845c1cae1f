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
  double cost;           // relative cost of one sweep of chain 0 (L N (m^2 + (3G+1) m) summed over spins)
};
lq_sim_launch_info lq_internal_sim_info(const lq_sim* sim);
// after a foreign launch wrote the descriptors, drop the cached host copy
void lq_internal_sim_invalidate(lq_sim* sim);
// a one-chain simulation whose QR chains are not built yet (the caller runs
// the init and build kernels over a gathered descriptor array)
lq_status lq_internal_sim_create_unbuilt(const lq_lattice* lat, const lq_params* params, uint32_t chain_id,
                                         void* stream, const lq_allocator* alloc, lq_sim** out);
// host copy of the descriptors as uploaded at creation
const LqChainDev* lq_internal_sim_host_desc(const lq_sim* sim);
// device footprint a one-chain simulation of this lattice and these parameters needs
size_t lq_internal_footprint(const lq_lattice* lat, const lq_params* p);
// sign-weighted means <sign O>/<sign> over per-sweep records and jackknife errors over nbins bins
void lq_internal_obs_stats(const double* rec, int n, int nbins, double* mean, double* err);
