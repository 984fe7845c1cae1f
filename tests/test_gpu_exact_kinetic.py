"""The exact kinetic propagator (lq_params.kinetic = LQ_EXACT) on the GPU.

B_l = e^{-dtau K} e^{-dtau V(s_l)} with e^{-dtau K} itself: the kernels apply
the Taylor polynomial of the sparse -dtau K (Horner's rule, remainder below
1e-17), the oracle the dense matrix exponential.  Same bar as the
checkerboard: FP64 log-weights, ratios and records within 1e-10, integer
state bit-exact over trajectories; FP32 panels within 1e-5.
"""
import numpy as np
import pytest

from oracle import OracleSim, lattices
from parity import elem_rel, norm_rel

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    "chain8_U4_tw3": dict(lattice=("chain", 8), U=4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=3, n_stab=3),
    "square4x4_attractive": dict(lattice=("square", 4, 4), U=-3.0, beta=1.0, dtau=0.1, n_up=3, n_dn=3, n_stab=4),
    # onsite terms on K's diagonal, theta = dtau max_i sum_j |K_ij| = 0.8
    "flat6": dict(lattice=("flatband", 6, 1.0, 1.0, 1.0, 1.0), U=2.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5),
    "square6x6_m20": dict(lattice=("square", 6, 6), U=4.0, beta=0.6, dtau=0.05, n_up=20, n_dn=9, n_stab=4),
    # the large-N_sigma kernel
    "chain96_m40": dict(lattice=("chain", 96), U=4.0, beta=0.3, dtau=0.1, n_up=40, n_dn=33, n_stab=2),
}


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def make(lq, spec, prec=0, seed=7, chain=0):
    lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
    o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"], spec["n_stab"], seed=seed,
                  chain=chain, kinetic="exact")
    L = getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:])
    sim = lq.Sim([L], [dict(spec, precision=prec, seed=seed, kinetic=lq.LQ_EXACT)], chain_ids=[chain])
    return o, sim


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_log_weight_chains_and_ratios(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=5, chain=2)
    sim.init()
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < TOL * max(1.0, abs(lo))
    for side in (0, 1):
        for spin in (0, 1):
            j = 1 if side == 0 else 0
            Qg, Vg = sim.chain_panel(0, side, spin, j)
            Qo, Vo = o.chain_panel(side, spin, j)
            assert norm_rel(Qg, Qo) < TOL and norm_rel(Vg, Vo) < TOL
    rng = np.random.default_rng(3)
    for _ in range(4):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
        assert abs(rg - ro) < TOL * max(1.0, abs(ro))
    occ = o.get_fock()
    for spin in (0, 1):
        if o.ns[spin] in (0, o.N):
            continue
        empty = np.setdiff1d(np.arange(o.N), occ[spin])
        k, j = int(rng.integers(o.ns[spin])), int(empty[rng.integers(len(empty))])
        rg, pg = sim.swap_ratio(0, spin, k, j)
        ro, po = o.swap_ratio(spin, k, j)
        assert abs(rg - ro) < TOL * max(1.0, abs(ro)) and pg[1] == po[1]


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_sweep_trajectory(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=11, chain=3)
    sim.init()
    o.sweep(2)
    sim.sweep(2)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    gu, gd = sim.get_fock(0)
    ou, od = o.get_fock()
    assert np.array_equal(gu, ou) and np.array_equal(gd, od)
    assert np.array_equal(sim.stats(0), o.stats())
    lt, st = sim.tracked_weight(0)
    lo, so = o.tracked()
    assert st == so and abs(lt - lo) < TOL * max(1.0, abs(lo))
    assert elem_rel(sim.records(0), o.records()) < TOL


@pytest.mark.parametrize("prec", [1, 2])
def test_exact_reduced_precision(lq, prec):
    spec = CASES["square4x4_attractive"]
    o, sim = make(lq, spec, prec=prec, seed=13, chain=4)
    sim.init()
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < 1e-5 * max(1.0, abs(lo))
    o.sweep(1)
    sim.sweep(1)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    assert np.array_equal(sim.stats(0), o.stats())
    assert elem_rel(sim.records(0), o.records()) < 1e-5


def test_exact_with_checkerboard_chains_in_one_launch(lq):
    """Chains of both kinetic modes side by side in one simulation."""
    specs = [(CASES["chain8_U4_tw3"], 1), (CASES["flat6"], 0), (CASES["square4x4_attractive"], 1)]
    lats, params, oracles = [], [], []
    for c, (spec, ex) in enumerate(specs):
        lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
        oracles.append(OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"],
                                 spec["n_stab"], seed=21, chain=c, kinetic="exact" if ex else "checkerboard"))
        lats.append(getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:]))
        params.append(dict(spec, precision=0, seed=21, kinetic=ex))
    sim = lq.Sim(lats, params)
    sim.init()
    for o in oracles:
        o.sweep(2)
    sim.sweep(2)
    sim.sync()
    for c, o in enumerate(oracles):
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
        assert elem_rel(sim.records(c), o.records()) < TOL


def test_exact_rejects_large_dtau_norm_and_bad_mode(lq):
    L = lq.Lattice.square(4, 4)
    base = dict(U=4.0, beta=1.2, dtau=0.6, n_up=2, n_dn=2, n_stab=4)  # theta = 0.6 * 4 > 2
    with pytest.raises(lq.LqError) as e:
        lq.Sim([L], [dict(base, kinetic=lq.LQ_EXACT)])
    assert e.value.status == 8
    with pytest.raises(lq.LqError) as e:
        lq.Sim([L], [dict(base, beta=1.2, dtau=0.1, kinetic=7)])
    assert e.value.status == 1
