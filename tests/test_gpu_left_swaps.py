"""Fock swaps at tau = 0 on the left chain (lq_params.left_swaps = 1) on the GPU.

After the down pass a second set of N_up + N_dn swap attempts walks the left
chain from tau = beta down to 0, i.e. the right chain of the transposed
propagator B(beta,0)^T.  Trajectories must match the oracle's (same Philox
numbers, same proposals) bit-exactly in the integer state and within 1e-10
(FP64) or 1e-5 (double-word flips) in the records; the tracked weight must
equal a fresh rebuild; Monte Carlo averages must match the exact
Trotterized ED."""
import numpy as np
import pytest

import exact
from oracle import OBS_NAMES, OracleSim, lattices
from stats import jackknife_ratio
from parity import elem_rel

pytestmark = pytest.mark.gpu

CASES = {
    # tau_w = 3 does not divide L = 10: a short last block on both chains
    "chain8_ragged": dict(lattice=("chain", 8), U=4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=3, n_stab=3),
    "square4x4_attractive": dict(lattice=("square", 4, 4), U=-4.0, beta=0.8, dtau=0.1, n_up=3, n_dn=3, n_stab=4),
    "flat6": dict(lattice=("flatband", 6), U=2.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5),
    "chain9_empty_dn": dict(lattice=("chain", 9), U=4.0, beta=0.5, dtau=0.1, n_up=4, n_dn=0, n_stab=2),
    # above 32 particles per spin: the large-N_sigma kernel instance
    "chain96_m40": dict(lattice=("chain", 96), U=4.0, beta=0.4, dtau=0.1, n_up=40, n_dn=33, n_stab=2),
    "open_chain10_neighbour": dict(lattice=("chain", 10, 1.0, False), U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2,
                                   n_stab=4, swap_mode=1),
}


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def _pair(lq, spec, prec, seed=23, chain=4):
    lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
    o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"], spec["n_stab"], seed=seed,
                  chain=chain, swap_mode=spec.get("swap_mode", 0), left_swaps=True)
    L = getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:])
    p = {k: v for k, v in spec.items() if k != "lattice"}
    sim = lq.Sim([L], [dict(p, precision=prec, seed=seed, left_swaps=1)], chain_ids=[chain])
    sim.init()
    return o, sim


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_left_swap_trajectory(lq, name, prec):
    spec = CASES[name]
    o, sim = _pair(lq, spec, prec)
    o.sweep(3)
    sim.sweep(3)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    gu, gd = sim.get_fock(0)
    ou, od = o.get_fock()
    assert np.array_equal(gu, ou) and np.array_equal(gd, od)
    st = sim.stats(0)
    assert np.array_equal(st, o.stats())
    # two swap phases per sweep: 2 (N_up + N_dn) attempts over sectors that can swap
    assert st[2] == 3 * 2 * sum(m for m in (spec["n_up"], spec["n_dn"]) if 0 < m < o.N)
    tol = 1e-10 if prec == 0 else 1e-5
    rg, ro = sim.records(0), o.records()
    assert elem_rel(rg, ro) < tol
    lt, sg = sim.tracked_weight(0)
    lo, so = o.tracked()
    assert sg == so and abs(lt - lo) < (1e-10 if prec == 0 else 1e-5) * max(1.0, abs(lo))


def test_left_swaps_accept_and_tracked_weight_is_fresh(lq):
    """Accepted left swaps exchange the left chain with the spare right-chain
    buffer; after sweeps the tracked weight equals a rebuild from the fields
    and Fock state, and the chain continues on the oracle's trajectory."""
    o, sim = _pair(lq, CASES["flat6"], 0, seed=31, chain=2)
    o.sweep(4)
    sim.sweep(4)
    sim.sync()
    st = sim.stats(0)
    assert st[3] > 0  # some swaps were accepted
    worst, bad = sim.check_drift(1e-10)
    assert bad == 0 and worst < 1e-10
    o.sweep(2)
    sim.sweep(2)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    assert np.array_equal(sim.stats(0), o.stats())


def test_left_swaps_match_trotter_ed(lq):
    """64 chains x 1000 sweeps on a 6-site ring (U = 4, N_up = 2, N_dn = 1)
    with both swap phases, against the exact canonical Trotterized ED."""
    lat_o = lattices.chain(6)
    U, beta, dtau, nu, nd, tw = 4.0, 1.0, 0.1, 2, 1, 5
    ed = exact.TrotterED(lat_o, U, dtau, round(beta / dtau), nu, nd).observables()
    n = 64
    L = lq.Lattice.chain(6)
    sim = lq.Sim([L] * n, [dict(U=U, beta=beta, dtau=dtau, n_up=nu, n_dn=nd, n_stab=tw, precision=0, seed=2029,
                                left_swaps=1)] * n)
    sim.init()
    sim.sweep(100, measure=False)
    sim.sweep(1000, measure=True)
    sim.sync()
    recs = np.concatenate([sim.records(c) for c in range(n)])
    for name in ("docc", "ekin", "szz_00", "szz_01", "s_par"):
        est, err = jackknife_ratio(recs, OBS_NAMES.index(name), nbins=64)
        assert abs(est - ed[name]) < 4.0 * err + 1e-12, (name, est, err, ed[name])


def test_bad_left_swaps_rejected(lq):
    with pytest.raises(lq.LqError) as e:
        lq.Sim([lq.Lattice.chain(8)], [dict(U=4.0, beta=0.5, dtau=0.1, n_up=2, n_dn=2, n_stab=5, left_swaps=2)])
    assert e.value.status == 1  # LQ_EINVAL
