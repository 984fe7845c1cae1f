"""Parity with the CPU oracle for more than 32 particles per spin.

Above 32 particles per spin the kernels keep the m x m matrices in a global
workspace per CTA and flip with a four-warp group per spin (the small path
has one warp per spin and shared-memory matrices).  Same bar as the small
path: FP64 log-weights, ratios and observables within 1e-10 relative,
integer state bit-exact; FP32 panels within 1e-5.
"""
import numpy as np
import pytest

from oracle import OracleSim, lattices
from paper_2601_08552_gb300 import inputs
from parity import elem_rel, norm_rel

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    # both spins above 32
    "chain96_m40_m33": dict(lattice=("chain", 96), U=4.0, beta=0.6, dtau=0.1, n_up=40, n_dn=33, n_stab=3),
    # one spin above 32, one small; attractive (charge channel)
    "square10x10_m48_m7": dict(lattice=("square", 10, 10), U=-3.0, beta=0.4, dtau=0.1, n_up=48, n_dn=7, n_stab=2),
    # an empty spin beside a large one, ragged last block
    "flat40_m60_empty": dict(lattice=("flatband", 40), U=2.0, beta=0.5, dtau=0.1, n_up=60, n_dn=0, n_stab=2),
    # m = 100 and 70 on 144 sites
    "square12x12_m100": dict(lattice=("square", 12, 12), U=4.0, beta=0.2, dtau=0.1, n_up=100, n_dn=70, n_stab=2),
}

# the largest particle numbers, on short imaginary time (the oracle's cost
# grows as L N m^2): the flat-band chain's 3/4 filling at 256 cells (m = 192),
# at 512 cells (m = 384, the largest of the uneven flat-band workload), and the
# library's limit LQ_MAX_PARTICLES = 512.  The scratch matrices, the flip
# window and the vectors of these plans live in the global workspace.
LARGEST = {
    "flat256_m192": dict(lattice=("flatband", 256, 1.0, 1.0, 1.0, 1.0, True), U=2.0, beta=0.2, dtau=0.05,
                         n_up=192, n_dn=192, n_stab=2),
    "flat512_m384": dict(lattice=("flatband", 512, 1.0, 1.0, 1.0, 1.0, False), U=2.0, beta=0.1, dtau=0.05,
                         n_up=384, n_dn=383, n_stab=2),
    "chain1024_m512": dict(lattice=("chain", 1024), U=-2.0, beta=0.1, dtau=0.05, n_up=512, n_dn=500, n_stab=1),
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
                  chain=chain, want_corr=False)
    L = getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:])
    sim = lq.Sim([L], [dict(spec, precision=prec, seed=seed)], chain_ids=[chain])
    return o, sim


@pytest.mark.parametrize("name", sorted(CASES))
def test_log_weight_and_chains_large_m(lq, name):
    spec = CASES[name]
    rng = np.random.default_rng(40 + sorted(CASES).index(name))
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


@pytest.mark.parametrize("name", sorted(CASES))
def test_field_and_swap_ratios_large_m(lq, name):
    spec = CASES[name]
    o, sim = make(lq, spec, seed=3)
    sim.init()
    rng = np.random.default_rng(5)
    for _ in range(4):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
        assert abs(rg - ro) < TOL * max(1.0, abs(ro))
    occ = o.get_fock()
    for spin in (0, 1):
        m = o.ns[spin]
        if m == 0 or m == o.N:
            continue
        empty = [x for x in range(o.N) if x not in set(occ[spin].tolist())]
        for _ in range(2):
            k, j = int(rng.integers(m)), int(empty[rng.integers(len(empty))])
            rg, pg = sim.swap_ratio(0, spin, k, j)
            ro, po = o.swap_ratio(spin, k, j)
            assert abs(rg - ro) < TOL * max(1.0, abs(ro))
            assert pg[1] == po[1] and pg[3] == po[3] and pg[5] == po[5]


@pytest.mark.parametrize("name", sorted(CASES))
def test_sweep_trajectory_large_m(lq, name):
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


def test_mixed_sizes_in_one_launch(lq):
    """Chains of 3 and of 40 particles per spin in one simulation: the launch
    takes the large-m kernel, which must run the small chains too."""
    specs = [dict(lattice=("chain", 12), U=4.0, beta=0.5, dtau=0.1, n_up=3, n_dn=2, n_stab=2),
             CASES["chain96_m40_m33"],
             dict(lattice=("square", 4, 4), U=-2.0, beta=0.4, dtau=0.1, n_up=5, n_dn=5, n_stab=4)]
    lats, params, oracles = [], [], []
    for c, spec in enumerate(specs):
        lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
        oracles.append(OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"],
                                 spec["n_stab"], seed=21, chain=c))
        lats.append(getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:]))
        params.append(dict(spec, precision=0, seed=21))
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


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["chain96_m40_m33", "square10x10_m48_m7"])
def test_reduced_precision_large_m(lq, name, prec):
    spec = CASES[name]
    o, sim = make(lq, spec, prec=prec, seed=13, chain=4)
    sim.init()
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < 1e-5 * max(1.0, abs(lo))
    rng = np.random.default_rng(8)
    for _ in range(3):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
        assert abs(rg - ro) < 1e-5 * max(1.0, abs(ro))
    o.sweep(1)
    sim.sweep(1)
    sim.sync()
    assert np.array_equal(sim.get_fields(0), o.get_fields())
    assert np.array_equal(sim.stats(0), o.stats())
    assert elem_rel(sim.records(0), o.records()) < 1e-5


@pytest.mark.parametrize("name", sorted(LARGEST))
def test_largest_particle_numbers(lq, name):
    """Up to LQ_MAX_PARTICLES per spin: log-weight of freshly built chains,
    a field ratio and a swap ratio through the hooks, then one sweep with its
    trajectory (integer state bit-exact, records and tracked weight within
    1e-10)."""
    spec = LARGEST[name]
    o, sim = make(lq, spec, seed=17, chain=1)
    sim.init()
    lw, sg = sim.log_weight(0)
    lo, so = o.log_weight()
    assert sg == so and abs(lw - lo) < TOL * max(1.0, abs(lo))
    rng = np.random.default_rng(9)
    l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
    rg, ro = sim.field_ratio(0, l, i), o.field_ratio(l, i)
    assert abs(rg - ro) < TOL * max(1.0, abs(ro))
    occ = o.get_fock()
    empty = [x for x in range(o.N) if x not in set(occ[0].tolist())]
    k, j = int(rng.integers(o.ns[0])), int(empty[rng.integers(len(empty))])
    rg, pg = sim.swap_ratio(0, 0, k, j)
    ro, po = o.swap_ratio(0, k, j)
    assert abs(rg - ro) < TOL * max(1.0, abs(ro)) and pg[1] == po[1]
    o.sweep(1)
    sim.sweep(1)
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


def test_beyond_the_particle_limit_is_rejected(lq):
    L = lq.Lattice.chain(1100)
    with pytest.raises(lq.LqError) as e:
        lq.Sim([L], [dict(U=2.0, beta=0.1, dtau=0.05, n_up=lq.LQ_MAX_PARTICLES + 1, n_dn=1, n_stab=1)])
    assert e.value.status == 8
