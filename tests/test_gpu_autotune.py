"""Autotuner of the batched launch (lq_sim_autotune).

The tuner times real sweeps under candidate staging-buffer sizes and keeps
the fastest.  The staging size changes only how work is chunked, so after
tuning every chain still follows the oracle's trajectory: the tuning sweeps
are ordinary sweeps of the chains of each plan class."""
import numpy as np
import pytest

from oracle import OracleSim, lattices
from parity import elem_rel

pytestmark = pytest.mark.gpu

TOL = 1e-10

SPECS = [
    dict(lattice=("square", 4, 4), U=4.0, beta=0.8, dtau=0.1, n_up=3, n_dn=2, n_stab=4),
    dict(lattice=("chain", 96), U=4.0, beta=0.4, dtau=0.1, n_up=40, n_dn=33, n_stab=2),
    dict(lattice=("flatband", 10), U=2.0, beta=0.6, dtau=0.1, n_up=4, n_dn=4, n_stab=3),
]


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def build(lq, seed):
    lats, params, oracles = [], [], []
    for c, spec in enumerate(SPECS):
        lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
        oracles.append(OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"],
                                 spec["n_stab"], seed=seed, chain=c))
        lats.append(getattr(lq.Lattice, spec["lattice"][0])(*spec["lattice"][1:]))
        params.append(dict(spec, precision=0, seed=seed))
    sim = lq.Sim(lats, params)
    sim.init()
    return sim, oracles


def test_autotune_keeps_the_trajectory(lq):
    sim, oracles = build(lq, 31)
    bufs = sim.autotune(1)
    assert bufs[0] > 0 and bufs[1] > 0
    sim.sync()
    for c, o in enumerate(oracles):
        L, N = o.L, o.N
        done = int(sim.stats(c)[0]) // (2 * L * N)  # field attempts -> sweeps the tuner ran
        assert done >= 1
        o.sweep(done)
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
    sim.sweep(2)
    sim.sync()
    for c, o in enumerate(oracles):
        o.sweep(2)
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
        lt, st = sim.tracked_weight(c)
        lo, so = o.tracked()
        assert st == so and abs(lt - lo) < TOL * max(1.0, abs(lo))
        rg = sim.records(c)
        ro = o.records()[-2:]
        assert elem_rel(rg, ro) < TOL


def test_autotune_cache(lq):
    sim, _ = build(lq, 32)
    first = sim.autotune(1)
    sim2, _ = build(lq, 33)
    sim2.sync()
    before = sim2.stats(0).copy()
    again = sim2.autotune(0)  # cached: applies the choice without sweeping
    sim2.sync()
    assert again == first
    assert np.array_equal(sim2.stats(0), before)
    with pytest.raises(lq.LqError):
        sim2.autotune(-1)


@pytest.mark.parametrize("staging,threads", [(24576, 128), (65536, 128), (24576, 256), (204800, 256)])
def test_pinned_launch_configs_keep_the_trajectory(lq, staging, threads):
    """Every launch the autotuner may pick for the small plan class (half-size
    CTAs, four per SM, or full ones; small and large staging buffers) gives
    the oracle's trajectory on the dilute-gas chains."""
    spec = dict(lattice=("square", 16, 16), U=4.0, beta=2.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8)
    n = 64
    lat = lq.Lattice.square(16, 16)
    sim = lq.Sim([lat] * n, [dict(spec, precision=0, seed=5)] * n)
    sim.init()
    for c in (0, 33):
        sim.log_weight(c)
    sim.set_launch_config(0, staging, threads)
    cfg = sim.launch_config()[0]
    assert cfg["threads"] == threads and cfg["staging_bytes"] == staging
    sim.sweep(2)
    sim.sync()
    for c in (0, n - 1):
        o = OracleSim(lattices.square(16, 16), 4.0, 2.0, 0.05, 8, 8, 8, seed=5, chain=c)
        o.sweep(2)
        assert np.array_equal(sim.get_fields(c), o.get_fields())
        assert np.array_equal(sim.stats(c), o.stats())
        assert elem_rel(sim.records(c), o.records()) < TOL
    with pytest.raises(lq.LqError):
        sim.set_launch_config(0, 1024, 256)  # below the plan's minimum
    with pytest.raises(lq.LqError):
        sim.set_launch_config(0, staging, 96)
