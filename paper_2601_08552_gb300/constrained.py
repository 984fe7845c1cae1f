"""Two-stage constrained-path sampling (SM Sec. VI) on the GPU path.

The outer stage samples Fock states eta with the free weight
W_T(eta) = <eta|e^{-beta H_0}|eta>: a U = 0 chain of lq_sim, whose fields are
inert (lambda = 0), so only its particle-hole swaps move and they sample
exactly W_T.  The inner stage estimates, for each sampled eta,
R(eta) = sum_s 2^{-LN} <eta|U(s)|eta> / <eta|e^{-beta H_0}|eta> with a
branching walker population (lq_cp_population).  Averaged over eta ~ W_T,
R estimates Z_U / Z_0 times the Hubbard-Stratonovich constant e^{c L}
(c = dtau U N_e / 2 in the spin channel, dtau |U| (N - N_e) / 2 in the charge
channel): the interacting partition function relative to the free one, the
quantity whose ratio between Fock states the constraint approximates.

Both stages run in the CUDA library; this module only sequences the calls
and averages the estimates.
"""
import numpy as np

from . import lecqmc as lq


def partition_ratio(lattice, params, n_fock, n_walkers=16, comb_every=0, thin=1, burn=5, chain_id=0):
    """Estimate E_{eta ~ W_T}[R(eta)].

    params: the model (U, beta, dtau, n_up, n_dn, n_stab, seed, kinetic).
    n_fock Fock states are taken from the U = 0 chain, thin sweeps apart after
    burn sweeps; each gets a population of n_walkers combed every comb_every
    slices (0: only at the end), with run word k for the k-th state.
    Returns dict(mean, err, r) with r the per-state estimates and err the
    standard error from batch means (eight batches) over the correlated
    outer chain."""
    outer = dict(params, U=0.0, precision=lq.LQ_FP64)
    sim = lq.Sim([lattice], [outer], chain_ids=[chain_id])
    sim.init()
    if burn:
        sim.sweep(burn, measure=False)
    r = np.empty(n_fock)
    for k in range(n_fock):
        sim.sweep(thin, measure=False)
        up, dn = sim.get_fock(0)
        r[k] = np.exp(lq.cp_population(lattice, params, up, dn, n_walkers, comb_every, run=k))
    sim.close()
    nb = 8
    b = r[: (n_fock // nb) * nb].reshape(nb, -1).mean(axis=1)
    return dict(mean=float(r.mean()), err=float(b.std(ddof=1) / np.sqrt(nb)), r=r)
