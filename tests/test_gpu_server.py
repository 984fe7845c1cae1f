"""Serving loop (lq_server_*): continuous batching of simulation requests.

A request's result must not depend on what else is in the batch: the same
request run alone and in a mix of requests of other sizes gives the same
Monte Carlo result (identical accept counts, observables within 1e-10).
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def wait(srv, ids, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(ids):
        for i in ids:
            if i not in out:
                r = srv.poll(i)
                if r is not None:
                    out[i] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.005)
    return out


def request_mix(lq):
    return [
        (lq.Lattice.square(6, 6), dict(U=4.0, beta=1.0, dtau=0.1, n_up=4, n_dn=3, n_stab=5, seed=9), 6, 3),
        (lq.Lattice.chain(20), dict(U=-3.0, beta=2.0, dtau=0.1, n_up=2, n_dn=2, n_stab=8, seed=4), 9, 11),
        (lq.Lattice.flatband(8), dict(U=2.0, beta=1.5, dtau=0.05, n_up=4, n_dn=4, n_stab=6, seed=5), 4, 2),
        (lq.Lattice.square(10, 10), dict(U=4.0, beta=0.8, dtau=0.1, n_up=12, n_dn=10, n_stab=4, seed=7), 3, 8),
        (lq.Lattice.chain(12), dict(U=2.0, beta=1.0, dtau=0.1, n_up=1, n_dn=3, n_stab=10, seed=2), 12, 5),
    ]


@pytest.mark.parametrize("prec", [0, 2])
def test_result_same_alone_and_in_mix(lq, prec):
    lat = lq.Lattice.square(4, 4)
    params = dict(U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=4, seed=21, precision=prec)
    alone = lq.Server(hbm_budget=1 << 30, precision=prec)
    rid = alone.submit(lat, params, 8, chain_id=77)
    ra = wait(alone, [rid])[rid]
    alone.close()
    mix = lq.Server(hbm_budget=1 << 30, precision=prec)
    ids = []
    for L, p, ns, cid in request_mix(lq):
        ids.append(mix.submit(L, dict(p, precision=prec), ns, chain_id=cid))
    rid2 = mix.submit(lat, params, 8, chain_id=77)
    for L, p, ns, cid in request_mix(lq)[:2]:
        ids.append(mix.submit(L, dict(p, precision=prec, seed=p["seed"] + 100), ns, chain_id=cid + 50))
    res = wait(mix, ids + [rid2])
    rb = res[rid2]
    st = mix.stats()
    mix.close()
    assert ra["status"] == 0 and rb["status"] == 0
    assert ra["n_records"] == rb["n_records"] == 8
    assert np.array_equal(ra["counts"], rb["counts"])
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.max(np.abs(ra["obs_mean"] - rb["obs_mean"])) < tol
    assert ra["sign"] == rb["sign"] and abs(ra["log_weight"] - rb["log_weight"]) < tol * max(1, abs(ra["log_weight"]))
    assert all(r["status"] == 0 for r in res.values())
    assert st["completed"] == st["submitted"] == len(ids) + 1
    assert st["p99_sweep_ms"] >= st["p50_sweep_ms"] > 0 and st["updates_per_s"] > 0


def test_result_matches_regular_entry_point(lq):
    lat = lq.Lattice.chain(10)
    params = dict(U=4.0, beta=1.0, dtau=0.1, n_up=2, n_dn=2, n_stab=5, seed=3, precision=0)
    srv = lq.Server(hbm_budget=1 << 30)
    rid = srv.submit(lat, params, 5, chain_id=4)
    r = wait(srv, [rid])[rid]
    srv.close()
    sim = lq.Sim([lat], [params], chain_ids=[4])
    sim.init()
    sim.sweep(5)
    sim.sync()
    mean, _ = sim.measure(0, n_bins=5)
    assert np.array_equal(r["counts"], sim.stats(0))
    assert np.max(np.abs(r["obs_mean"] - mean)) < 1e-10


def test_queue_full_and_unknown_ids(lq):
    lat = lq.Lattice.square(8, 8)
    params = dict(U=4.0, beta=2.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8, seed=1, precision=0)
    srv = lq.Server(hbm_budget=1 << 30, max_active=1, queue_capacity=2)
    ids = []
    with pytest.raises(lq.LqError) as e:
        for _ in range(50):
            ids.append(srv.submit(lat, params, 50))
    assert e.value.status == 6  # LQ_EBUSY
    with pytest.raises(lq.LqError):
        srv.poll(10 ** 9)
    with pytest.raises(lq.LqError):  # footprint larger than the whole budget
        tiny = lq.Server(hbm_budget=1 << 20)
        tiny.submit(lat, params, 1)
    srv.close()  # finishes the admitted request, drops the queued ones


def test_grouping_of_sweeps_into_launches_does_not_change_results(lq):
    """Tick target 0 (one sweep per launch for a lone request) against 10 s
    (every sweep in one launch): the counter-based random numbers depend on
    (chain, sweep, slice, site) only, so the results agree."""
    lat = lq.Lattice.flatband(10)
    params = dict(U=2.0, beta=1.2, dtau=0.05, n_up=4, n_dn=4, n_stab=8, seed=8, precision=0)
    out = []
    for target in (0.0, 10000.0):
        srv = lq.Server(hbm_budget=1 << 30)
        srv.set_tick_target(target)
        rid = srv.submit(lat, params, 12, chain_id=3)
        out.append((wait(srv, [rid])[rid], srv.stats()))
        srv.close()
    (ra, sa), (rb, sb) = out
    assert sa["ticks"] == 12 and sb["ticks"] == 1
    assert np.array_equal(ra["counts"], rb["counts"])
    assert np.max(np.abs(ra["obs_mean"] - rb["obs_mean"])) < 1e-10
    assert abs(ra["log_weight"] - rb["log_weight"]) < 1e-10 * max(1.0, abs(ra["log_weight"]))
    srv = lq.Server(hbm_budget=1 << 30)
    with pytest.raises(lq.LqError):
        srv.set_tick_target(-1.0)
    srv.close()


def test_large_request_alone_and_in_mix(lq):
    """A request with more than 32 particles per spin runs in its own launch
    of each tick (the large plan) beside small requests: same result alone
    and in the mix."""
    lat = lq.Lattice.chain(96)
    params = dict(U=4.0, beta=0.6, dtau=0.1, n_up=40, n_dn=33, n_stab=3, seed=17, precision=0)
    srv = lq.Server(hbm_budget=1 << 30)
    rid = srv.submit(lat, params, 3, chain_id=5)
    ra = wait(srv, [rid])[rid]
    srv.close()
    srv = lq.Server(hbm_budget=1 << 30)
    ids = [srv.submit(L, dict(p, precision=0), ns, chain_id=cid) for L, p, ns, cid in request_mix(lq)]
    rid2 = srv.submit(lat, params, 3, chain_id=5)
    res = wait(srv, ids + [rid2])
    srv.close()
    rb = res[rid2]
    assert ra["status"] == 0 and rb["status"] == 0 and all(r["status"] == 0 for r in res.values())
    assert np.array_equal(ra["counts"], rb["counts"])
    assert np.max(np.abs(ra["obs_mean"] - rb["obs_mean"])) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_request_admitted_mid_run_after_memory_frees(lq, prec):
    """Continuous batching: a long request A and a medium one B are on the
    device when the tested request C arrives.  The budget holds A with either
    B or C but not all three, so C waits at the head of the queue until B
    retires, then runs beside A.  C's result equals the same request run
    alone (FP64 1e-10, LQ_MIXED 1e-5; the kernels draw counter-based random
    numbers, so identical in practice)."""
    la, lb, lc = lq.Lattice.square(8, 8), lq.Lattice.square(6, 6), lq.Lattice.square(4, 4)
    pa = dict(U=4.0, beta=2.0, dtau=0.1, n_up=4, n_dn=4, n_stab=5, seed=31, precision=prec)
    pb = dict(U=-2.0, beta=2.0, dtau=0.1, n_up=6, n_dn=6, n_stab=5, seed=32, precision=prec)
    pc = dict(U=4.0, beta=1.0, dtau=0.1, n_up=3, n_dn=2, n_stab=4, seed=21, precision=prec)
    fa, fb, fc = (lq.Server.footprint(l, p) for l, p in ((la, pa), (lb, pb), (lc, pc)))
    budget = fa + max(fb, fc)
    assert fa + fb + fc > budget
    alone = lq.Server(hbm_budget=1 << 30, precision=prec)
    rid = alone.submit(lc, pc, 8, chain_id=77)
    ref = wait(alone, [rid])[rid]
    alone.close()

    srv = lq.Server(hbm_budget=budget, precision=prec)
    ida = srv.submit(la, pa, 600, chain_id=1)
    idb = srv.submit(lb, pb, 150, chain_id=2)
    t0 = time.time()
    while srv.stats()["active"] < 2:
        assert time.time() - t0 < 60, "A and B were not both admitted"
        time.sleep(0.001)
    assert srv.poll(idb) is None  # B still runs when C arrives
    idc = srv.submit(lc, pc, 8, chain_id=77)
    rc = wait(srv, [idc], timeout=300)[idc]
    a_running = srv.poll(ida) is None  # A outlives C
    rest = wait(srv, [ida, idb], timeout=300)
    st = srv.stats()
    srv.close()
    assert rc["status"] == 0 and all(r["status"] == 0 for r in rest.values())
    assert rc["waited_for_memory"] == 1 and rc["active_at_admit"] >= 1 and a_running
    assert rc["queue_ms"] > 0 and rc["wall_ms_per_sweep"] > 0
    assert np.array_equal(ref["counts"], rc["counts"]) and ref["n_records"] == rc["n_records"] == 8
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.max(np.abs(ref["obs_mean"] - rc["obs_mean"])) < tol
    assert ref["sign"] == rc["sign"] and abs(ref["log_weight"] - rc["log_weight"]) < tol * max(1, abs(ref["log_weight"]))
    assert st["sweeps"] == 600 + 150 + 8 and st["p99_wall_sweep_ms"] >= st["p50_wall_sweep_ms"] > 0
