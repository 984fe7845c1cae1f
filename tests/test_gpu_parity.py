"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 panels: log-weights, ratios, QR chains and observables within 1e-10
relative; integer state (fields, occupations, acceptance counts) bit-exact.
Both sides draw the same Philox4x32-10 numbers, so whole trajectories agree.
"""
import numpy as np
import pytest

from oracle import OracleSim, lattices
from paper_2601_08552_gb300 import inputs
from parity import elem_rel, norm_rel

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p




def make(lq, spec, prec=0, seed=7, chain=0, fields=None, fock=None):
    lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
    o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"], spec["n_stab"], seed=seed,
                  chain=chain, want_corr=False)
    L = getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:])
    p = dict(spec, precision=prec, seed=seed)
    sim = lq.Sim([L], [p], chain_ids=[chain])
    if fields is not None:
        o.set_fields(fields)
        sim.set_fields(0, fields)
    if fock is not None:
        o.set_fock(*fock)
        sim.set_fock(0, *fock)
    return o, sim


CASES = {
    "chain8_U4_tw3": dict(lattice=("chain", 8), U=4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=3, n_stab=3),
    "chain8_Um4": dict(lattice=("chain", 8), U=-4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=2, n_stab=4),
    "square4x4": dict(lattice=("square", 4, 4), U=4.0, beta=2.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5),
    "flat6": dict(lattice=("flatband", 6), U=2.0, beta=2.0, dtau=0.1, n_up=3, n_dn=3, n_stab=8),
    "chain16_cfg": dict(lattice=("chain", 16), U=4.0, beta=4.0, dtau=0.1, n_up=2, n_dn=2, n_stab=10),
    "square6x6_m9": dict(lattice=("square", 6, 6), U=3.0, beta=1.0, dtau=0.1, n_up=9, n_dn=4, n_stab=4),
    "open_chain_one": dict(lattice=("chain", 9, 1.0, False), U=2.0, beta=0.7, dtau=0.1, n_up=1, n_dn=1, n_stab=3),
    "empty_spin": dict(lattice=("chain", 6), U=4.0, beta=0.5, dtau=0.1, n_up=3, n_dn=0, n_stab=2),
    "full_spin": dict(lattice=("chain", 4), U=4.0, beta=0.5, dtau=0.1, n_up=4, n_dn=1, n_stab=2),
    "cross_stitch": dict(lattice=("cross_stitch", 5), U=2.0, beta=1.0, dtau=0.1, n_up=2, n_dn=3, n_stab=5),
    "wide_m32": dict(lattice=("square", 8, 8), U=2.0, beta=0.4, dtau=0.1, n_up=32, n_dn=20, n_stab=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_init_from_seed_matches_oracle(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=123, chain=5)
    sim.init()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    gu, gd = sim.get_fock(0)
    ou, od = o.get_fock()
    assert np.array_equal(gu, ou) and np.array_equal(gd, od)


@pytest.mark.parametrize("name", sorted(CASES))
def test_log_weight_and_chains(lq, name):
    spec = CASES[name]
    rng = np.random.default_rng(sorted(CASES).index(name))
    o, sim = make(lq, spec)
    f = inputs.fields(rng, o.L, o.N)
    fk = (inputs.fock(rng, o.N, spec["n_up"], shuffle=True), inputs.fock(rng, o.N, spec["n_dn"], shuffle=True))
    o.set_fields(f)
    sim.set_fields(0, f)
    o.set_fock(*fk)
    sim.set_fock(0, *fk)
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < TOL * max(1.0, abs(lo))
    for side in (0, 1):
        for spin in (0, 1):
            for j in range(o.n + 1):
                if (side == 0 and j == 0) or (side == 1 and j == o.n):
                    continue
                Qg, Vg = sim.chain_panel(0, side, spin, j)
                Qo, Vo = o.chain_panel(side, spin, j)
                assert norm_rel(Qg, Qo) < TOL and norm_rel(Vg, Vo) < TOL, (side, spin, j)


@pytest.mark.parametrize("name", ["chain8_U4_tw3", "chain8_Um4", "square4x4", "flat6", "square6x6_m9"])
def test_field_ratio(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=3)
    sim.init()
    rng = np.random.default_rng(1)
    for _ in range(6):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
        assert abs(rg - ro) < TOL * max(1.0, abs(ro))


@pytest.mark.parametrize("name", ["chain8_U4_tw3", "chain8_Um4", "square4x4", "flat6", "square6x6_m9",
                                  "open_chain_one", "wide_m32"])
def test_swap_ratio(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=4)
    sim.init()
    rng = np.random.default_rng(2)
    occ = o.get_fock()
    for spin in (0, 1):
        m = o.ns[spin]
        if m == 0 or m == o.N:
            continue
        empty = [x for x in range(o.N) if x not in set(occ[spin].tolist())]
        for _ in range(3):
            k, j = int(rng.integers(m)), int(empty[rng.integers(len(empty))])
            rg, pg = sim.swap_ratio(0, spin, k, j)
            ro, po = o.swap_ratio(spin, k, j)
            assert abs(rg - ro) < TOL * max(1.0, abs(ro))
            assert pg[1] == po[1] and pg[3] == po[3] and pg[5] == po[5]
            assert abs(pg[2] - po[2]) < TOL * max(1, abs(po[2])) and abs(pg[4] - po[4]) < TOL * max(1, abs(po[4]))


@pytest.mark.parametrize("name", sorted(CASES))
def test_sweep_trajectory(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=11, chain=3)
    sim.init()
    ns = 3
    o.sweep(ns)
    sim.sweep(ns)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    gu, gd = sim.get_fock(0)
    ou, od = o.get_fock()
    assert np.array_equal(gu, ou) and np.array_equal(gd, od)
    assert np.array_equal(sim.stats(0), o.stats())
    lt, st = sim.tracked_weight(0)
    lo, so = o.tracked()
    assert st == so and abs(lt - lo) < TOL * max(1.0, abs(lo))
    rg, ro = sim.records(0), o.records()
    assert rg.shape == ro.shape and elem_rel(rg, ro) < TOL


def test_uneven_batch(lq):
    specs = [CASES[k] for k in ("square4x4", "chain8_Um4", "flat6", "chain16_cfg", "cross_stitch", "empty_spin")]
    sims_lat, params, oracles = [], [], []
    for c, spec in enumerate(specs):
        lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
        oracles.append(OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"],
                                 spec["n_stab"], seed=99, chain=c))
        sims_lat.append(getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:]))
        params.append(dict(spec, precision=0, seed=99))
    sim = lq.Sim(sims_lat, params)
    sim.init()
    for c, o in enumerate(oracles):
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        o.sweep(2)
    sim.sweep(2)
    sim.sync()
    for c, o in enumerate(oracles):
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
        assert elem_rel(sim.records(c), o.records()) < TOL


def test_full_size_gas32x32_sampled(lq):
    """The benchmark's workload (256 chains of the 32x32 dilute gas), one sweep
    in the benchmark's launch; chains 0 and 255 re-run by the oracle."""
    w = inputs.WORKLOADS["gas32x32"]
    spec = {k: w[k] for k in ("lattice", "U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
    L = lq.Lattice.square(32, 32)
    n = w["chains"]
    sim = lq.Sim([L] * n, [dict(spec, precision=0, seed=inputs.SEED0)] * n)
    sim.init()
    sim.sweep(1)
    sim.sync()
    lat = lattices.square(32, 32)
    for c in (0, n - 1):
        o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], 8, 8, 8, seed=inputs.SEED0, chain=c)
        o.sweep(1)
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
        assert elem_rel(sim.records(c), o.records()) < TOL
        lt, st = sim.tracked_weight(c)
        lo, so = o.tracked()
        assert st == so and abs(lt - lo) < TOL * abs(lo)


def test_check_drift_resynchronizes(lq):
    """lq_sim_check_drift rebuilds the chains from fields and Fock states:
    after sweeps the drift is at round-off, the tracked weight then equals a
    fresh log|W|, and the rebuilt chains continue on the oracle's trajectory."""
    o, sim = make(lq, CASES["square4x4"], seed=11, chain=3)
    sim.init()
    o.sweep(3)
    sim.sweep(3)
    sim.sync()
    worst, bad = sim.check_drift(1e-10)
    assert bad == 0 and worst < 1e-10
    # the rebuilt (fresh) weight against the oracle's tracked one, which the
    # oracle pins tie to a fresh brute-force weight after sweeps
    lt, st = sim.tracked_weight(0)
    lo, so = o.tracked()
    assert st == so and abs(lt - lo) < TOL * max(1.0, abs(lo))
    o.sweep(2)
    sim.sweep(2)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    assert np.array_equal(sim.stats(0), o.stats())
    with pytest.raises(lq.LqError):
        sim.check_drift(-1.0)


def test_checkpoint_and_resume(lq):
    """Checkpoint = fields, Fock state and sweep counter (the QR chains are
    rebuilt from them).  A chain resumed in a new simulation continues
    exactly as the uninterrupted one: same fields, occupations and accept
    counts, records within 1e-10, tracked weights within 1e-10."""
    spec = CASES["flat6"]
    _, a = make(lq, spec, seed=17, chain=2)
    a.init()
    a.sweep(3)
    a.sync()
    fields = a.get_fields(0)
    up, dn = a.get_fock(0)
    counts3 = a.stats(0).copy()
    _, b = make(lq, spec, seed=17, chain=2)
    b.set_fields(0, fields)
    b.set_fock(0, up, dn)
    b.set_sweep_index(3)
    a.sweep(2)
    b.sweep(2)
    a.sync()
    b.sync()
    assert np.array_equal(a.get_fields(0), b.get_fields(0))
    ua, da = a.get_fock(0)
    ub, db = b.get_fock(0)
    assert np.array_equal(ua, ub) and np.array_equal(da, db)
    assert np.array_equal(a.stats(0) - counts3, b.stats(0))
    assert elem_rel(b.records(0), a.records(0)[3:5]) < TOL
    la, sa = a.tracked_weight(0)
    lb, sb = b.tracked_weight(0)
    assert sa == sb and abs(la - lb) < TOL * max(1.0, abs(la))
