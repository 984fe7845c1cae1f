"""Reduced-precision paths against the FP64 oracle and the exact Trotterized ED.

LQ_MIXED keeps panels in FP32 (QR, inverses and ratios in FP64); LQ_MIXED_DW
additionally runs the per-site flip algebra in double-word FP32.  Stated
tolerances: ratios and log-weights within 1e-5 relative of the FP64 oracle
on identical configurations; Monte Carlo averages within 4 standard errors
of the exact canonical Trotterized ED.
"""
import numpy as np
import pytest

import exact
from oracle import OBS_NAMES, OracleSim, lattices
from stats import jackknife_ratio
from parity import elem_rel

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


CASES = {
    "square4x4": (("square", 4, 4), dict(U=4.0, beta=2.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5)),
    "chain8_attractive": (("chain", 8), dict(U=-4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=2, n_stab=4)),
    "flat6": (("flatband", 6), dict(U=2.0, beta=2.0, dtau=0.1, n_up=3, n_dn=3, n_stab=8)),
    "square8x8_m16": (("square", 8, 8), dict(U=4.0, beta=1.6, dtau=0.05, n_up=16, n_dn=12, n_stab=8)),
}


def make(lq, name, prec, seed=5, chain=1):
    latspec, spec = CASES[name]
    o = OracleSim(getattr(lattices, latspec[0])(*latspec[1:]), spec["U"], spec["beta"], spec["dtau"], spec["n_up"],
                  spec["n_dn"], spec["n_stab"], seed=seed, chain=chain)
    sim = lq.Sim([getattr(lq.Lattice, latspec[0])(*latspec[1:])], [dict(spec, precision=prec, seed=seed)],
                 chain_ids=[chain])
    sim.init()
    return o, sim


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_precision_ratios_and_weight(lq, name, prec):
    o, sim = make(lq, name, prec)
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < RTOL * max(1.0, abs(lo))
    rng = np.random.default_rng(3)
    for _ in range(5):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
        assert abs(rg - ro) < RTOL * max(1.0, abs(ro))
    occ = o.get_fock()
    for spin in (0, 1):
        empty = [x for x in range(o.N) if x not in set(occ[spin].tolist())]
        for _ in range(3):
            k, j = int(rng.integers(o.ns[spin])), int(empty[rng.integers(len(empty))])
            rg, _ = sim.swap_ratio(0, spin, k, j)
            ro, _ = o.swap_ratio(spin, k, j)
            assert abs(rg - ro) < RTOL * max(1.0, abs(ro))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["square4x4", "flat6", "square8x8_m16"])
def test_reduced_precision_short_trajectory(lq, name, prec):
    """Two sweeps from one seeded state: same accept/reject decisions as the
    FP64 oracle (no ratio lies within the panel error of its uniform here),
    tracked weight and measurements within the stated tolerance."""
    o, sim = make(lq, name, prec, seed=13, chain=4)
    o.sweep(2)
    sim.sweep(2)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    assert np.array_equal(sim.stats(0), o.stats())
    lt, st = sim.tracked_weight(0)
    lo, so = o.tracked()
    assert st == so and abs(lt - lo) < RTOL * max(1.0, abs(lo))
    rg, ro = sim.records(0), o.records()
    assert elem_rel(rg, ro) < RTOL


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_gpu_monte_carlo_matches_trotter_ed(lq, prec):
    """64 chains x 1000 sweeps on the GPU against the exact canonical
    Trotterized ED (repulsive chain, N = 6, N_up = 2, N_dn = 1)."""
    lat_o = lattices.chain(6)
    U, beta, dtau, nu, nd, tw = 4.0, 1.0, 0.1, 2, 1, 5
    ed = exact.TrotterED(lat_o, U, dtau, round(beta / dtau), nu, nd).observables()
    n = 64
    L = lq.Lattice.chain(6)
    sim = lq.Sim([L] * n, [dict(U=U, beta=beta, dtau=dtau, n_up=nu, n_dn=nd, n_stab=tw, precision=prec,
                                seed=2026)] * n)
    sim.init()
    sim.sweep(100, measure=False)
    sim.sweep(1000, measure=True)
    sim.sync()
    recs = np.concatenate([sim.records(c) for c in range(n)])
    for name in ("docc", "ekin", "szz_00", "szz_01", "s_par"):
        est, err = jackknife_ratio(recs, OBS_NAMES.index(name), nbins=64)
        assert abs(est - ed[name]) < 4.0 * err + 1e-12, (name, est, err, ed[name])
