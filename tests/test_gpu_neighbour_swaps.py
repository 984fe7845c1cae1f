"""Nearest-neighbour Fock-swap proposals (LQ_SWAP_NEIGHBOUR) on the GPU.

The target of a swap is drawn among the empty nearest neighbours of the
removed particle's site, and the Metropolis test carries the
Metropolis-Hastings factor |E(i)| / |E'(j)|.  Trajectories must match the
oracle's (same Philox numbers, same proposals) bit-exactly in the integer
state and within 1e-10 in the records; Monte Carlo averages must match the
exact Trotterized ED on an open chain, where the neighbour counts differ
between the ends and the bulk."""
import numpy as np
import pytest

import exact
from oracle import OBS_NAMES, OracleSim, lattices
from stats import jackknife_ratio
from parity import elem_rel

pytestmark = pytest.mark.gpu

CASES = {
    "open_chain10": dict(lattice=("chain", 10, 1.0, False), U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=4),
    "square4x4_attractive": dict(lattice=("square", 4, 4), U=-4.0, beta=0.8, dtau=0.1, n_up=3, n_dn=3, n_stab=4),
    "flat6": dict(lattice=("flatband", 6), U=2.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5),
    "chain96_m40": dict(lattice=("chain", 96), U=4.0, beta=0.4, dtau=0.1, n_up=40, n_dn=33, n_stab=2),
    "crowded_chain8": dict(lattice=("chain", 8, 1.0, False), U=2.0, beta=0.6, dtau=0.1, n_up=6, n_dn=7, n_stab=3),
}


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_neighbour_swap_trajectory(lq, name, prec):
    spec = CASES[name]
    lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
    o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"], spec["n_stab"], seed=19,
                  chain=6, swap_mode=1)
    L = getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:])
    sim = lq.Sim([L], [dict(spec, precision=prec, seed=19, swap_mode=lq.LQ_SWAP_NEIGHBOUR)], chain_ids=[6])
    sim.init()
    o.sweep(3)
    sim.sweep(3)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    gu, gd = sim.get_fock(0)
    ou, od = o.get_fock()
    assert np.array_equal(gu, ou) and np.array_equal(gd, od)
    assert np.array_equal(sim.stats(0), o.stats())
    tol = 1e-10 if prec == 0 else 1e-5
    rg, ro = sim.records(0), o.records()
    assert elem_rel(rg, ro) < tol


def test_neighbour_swaps_match_trotter_ed(lq):
    """64 chains x 1000 sweeps on an open 6-site chain (U = 4, N_up = 2,
    N_dn = 1) against the exact canonical Trotterized ED."""
    lat_o = lattices.chain(6, 1.0, False)
    U, beta, dtau, nu, nd, tw = 4.0, 1.0, 0.1, 2, 1, 5
    ed = exact.TrotterED(lat_o, U, dtau, round(beta / dtau), nu, nd).observables()
    n = 64
    L = lq.Lattice.chain(6, 1.0, False)
    sim = lq.Sim([L] * n, [dict(U=U, beta=beta, dtau=dtau, n_up=nu, n_dn=nd, n_stab=tw, precision=0, seed=2027,
                                swap_mode=lq.LQ_SWAP_NEIGHBOUR)] * n)
    sim.init()
    sim.sweep(100, measure=False)
    sim.sweep(1000, measure=True)
    sim.sync()
    recs = np.concatenate([sim.records(c) for c in range(n)])
    for name in ("docc", "ekin", "szz_00", "szz_01", "s_par"):
        est, err = jackknife_ratio(recs, OBS_NAMES.index(name), nbins=64)
        assert abs(est - ed[name]) < 4.0 * err + 1e-12, (name, est, err, ed[name])


def test_bad_swap_mode_rejected(lq):
    with pytest.raises(lq.LqError) as e:
        lq.Sim([lq.Lattice.chain(8)], [dict(U=4.0, beta=0.5, dtau=0.1, n_up=2, n_dn=2, n_stab=5, swap_mode=7)])
    assert e.value.status == 1  # LQ_EINVAL
