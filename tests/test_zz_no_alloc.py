"""The allocation-free single-chain entry point (lq_sweep_noalloc).

Callers that cannot allocate device memory (a plug-in inside a framework
that owns all GPU memory, code that must not call cudaMalloc on its hot path)
pass their own device buffers for fields, occupations and records; all
scratch lives in the library's fixed device array.  Each case runs two calls
in a row through the C ABI and checks them against the regular entry point
(lq_sim_create / lq_sim_sweep) on the same seeded chain: fields and
occupations bit-exact, acceptance counts equal, records within 1e-10 and the
tracked log-weight within 1e-10 (FP64 panels) or 1e-5 (FP32 panels).  Collected
last so that a failure here stops a
-x run only after every other test has run.
"""
import numpy as np
import pytest
from parity import elem_rel, norm_rel

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    "square4x4": (("square", 4, 4), dict(U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=4)),
    "chain8_attractive": (("chain", 8), dict(U=-4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=2, n_stab=3)),
    "flat6_mixed": (("flatband", 6), dict(U=2.0, beta=1.0, dtau=0.1, n_up=3, n_dn=3, n_stab=5, precision=1)),
    "open_chain_neighbour_swaps": (("chain", 10, 1.0, False),
                                   dict(U=4.0, beta=0.8, dtau=0.1, n_up=3, n_dn=2, n_stab=4, swap_mode=1)),
    "square4x4_left_swaps": (("square", 4, 4), dict(U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=4, left_swaps=1)),
    "gas32x32_one_chain": (("square", 32, 32), dict(U=4.0, beta=10.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8)),
    "flat6_exact_kinetic": (("flatband", 6), dict(U=2.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=5, kinetic=1)),
}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as lq

    lq.load()
    return torch, lq




@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_two_calls_match_regular_entry_point(env, name):
    torch = env[0]
    lq = env[1]
    from paper_2601_08552_gb300.lecqmc import sweep_noalloc

    latspec, spec = CASES[name]
    params = dict(spec, seed=77)
    params.setdefault("precision", 0)
    chain = 9
    lat = getattr(lq.Lattice, latspec[0])(*latspec[1:])
    sim = lq.Sim([lat], [params], chain_ids=[chain])
    sim.init()
    f0 = sim.get_fields(0)
    u0, d0 = sim.get_fock(0)
    dev_f = torch.from_numpy(f0.copy()).cuda()
    dev_o = torch.from_numpy(np.concatenate([u0, d0]).astype(np.int32)).cuda()
    nobs = lq.LQ_NOBS
    done = 0
    prev_cnt = np.zeros(4, np.int64)
    for n in (2, 1):
        rec = torch.full((n, nobs), np.nan, dtype=torch.float64, device="cuda")
        lw, sg, cnt = sweep_noalloc(lat, params, chain, done, dev_f, dev_o, n, rec)
        sim.sweep(n)
        sim.sync()
        done += n
        assert np.array_equal(dev_f.cpu().numpy(), sim.get_fields(0))
        u, d = sim.get_fock(0)
        assert np.array_equal(dev_o.cpu().numpy(), np.concatenate([u, d]))
        st = sim.stats(0)
        assert np.array_equal(cnt, st - prev_cnt)
        prev_cnt = st
        assert elem_rel(rec.cpu().numpy(), sim.records(0)[done - n:done]) < TOL
        # each call rebuilds its QR chains, the regular entry point keeps
        # tracking: they agree to the panel precision (FP64 1e-10, FP32 1e-5)
        lt, stg = sim.tracked_weight(0)
        wtol = 1e-10 if params["precision"] == 0 else 1e-5
        assert sg == stg and abs(lw - lt) < wtol * max(1.0, abs(lt))


def test_noalloc_rejects_chains_beyond_its_scratch(env):
    torch = env[0]
    lq = env[1]
    from paper_2601_08552_gb300.lecqmc import LqError, sweep_noalloc

    lat = lq.Lattice.square(64, 64)
    params = dict(U=4.0, beta=16.0, dtau=0.05, n_up=16, n_dn=16, n_stab=8, precision=0, seed=1)
    dev_f = torch.ones((320, 4096), dtype=torch.int8, device="cuda")
    dev_o = torch.arange(32, dtype=torch.int32, device="cuda")
    with pytest.raises(LqError) as e:
        sweep_noalloc(lat, params, 0, 0, dev_f, dev_o, 1, None)
    assert e.value.status == 8 and "LQ_NOALLOC_SCRATCH_BYTES" in str(e.value)
    assert torch.equal(dev_f, torch.ones_like(dev_f))
