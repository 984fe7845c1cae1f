#!/usr/bin/env python
"""Benchmark of the LEC-QMC sweep on GB300: Hubbard-Stratonovich field
updates per second and sweeps per second, FP64 panels (the headline) and the
mixed FP32-panel path on the same workload, with per-sweep latency.

A step is one sweep of every chain of the workload (one persistent launch).
Workload (synthetic, the dilute 2D Hubbard gas): 32x32 periodic square
lattice, t = 1, U = +4, beta = 10, dtau = 0.05 (L = 200 slices), N_up = N_dn
= 8, QR every 8 slices, 256 independent seeded chains.  Its device state
(about 3 GB) is far larger than the 129 MB L2, so no flush is needed between
steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs its own 256 chains (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HS field updates/sec & sweeps/sec vs plain FP64 same GPU; p50/p99 sweep latency"
UNIT = "field-updates/s"
# The FP64 roof is measured in the run (lq_device_fp64_rate: independent FMA chains on every SM, CUDA
# events).  Only if that probe fails does the line fall back to the unit-count figure: 0.5 FP64 FMA per
# cycle per sub-partition x 4 x 152 SMs x 2.07 GHz x 2 flops = 1.26 TFLOP/s.
FP64_FALLBACK_TFLOPS = 1.26
WORKLOAD = "gas32x32"


def workload_desc(w, n_chains):
    return ("dilute 2D Hubbard gas: %dx%d periodic square, t=1, U=%+.0f, beta=%g, dtau=%g (L=%d), N_up=N_dn=%d, "
            "QR every %d slices, %d chains" % (w["lattice"][1], w["lattice"][2], w["U"], w["beta"], w["dtau"],
                                               round(w["beta"] / w["dtau"]), w["n_up"], w["n_stab"], n_chains))


# ---------------------------------------------------------------------------
# CPU oracle legs (spawned worker processes, one chain each)
# ---------------------------------------------------------------------------
def _oracle_worker(conn, spec, seed, chain):
    sys.path.insert(0, ROOT)
    from oracle import OracleSim, lattices

    lat = getattr(lattices, spec["lattice"][0])(*spec["lattice"][1:])
    o = OracleSim(lat, spec["U"], spec["beta"], spec["dtau"], spec["n_up"], spec["n_dn"], spec["n_stab"], seed=seed,
                  chain=chain, max_records=1024)
    conn.send("ready")
    while True:
        cmd = conn.recv()
        if cmd is None:
            break
        t0 = time.perf_counter()
        o.sweep(int(cmd))
        conn.send((int(o.stats()[0]), time.perf_counter() - t0))
    conn.close()


class OraclePool:
    def __init__(self, spec, seed, n):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for c in range(n):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, spec, seed, c), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for a in self.conns:
            assert a.recv() == "ready"

    def step(self, nsweeps=1):
        t0 = time.perf_counter()
        for a in self.conns:
            a.send(nsweeps)
        res = [a.recv() for a in self.conns]
        return time.perf_counter() - t0, res

    def close(self):
        for a in self.conns:
            a.send(None)
        for p in self.procs:
            p.join(timeout=10)


def host_cores():
    """Cores this process may run on (nproc)."""
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


ORACLE_CAP = 16


def oracle_cores():
    """Oracle processes: one per host core, at most ORACLE_CAP."""
    return max(1, min(ORACLE_CAP, host_cores()))


def run_reference(args, spec, n_chains):
    """--impl reference: the oracle as it stands, on the host cores."""
    from paper_2601_08552_gb300 import inputs

    P = oracle_cores()
    pool = OraclePool(spec, inputs.SEED0, P)
    upd = 2 * round(spec["beta"] / spec["dtau"]) * spec["lattice"][1] * spec["lattice"][2]
    for _ in range(args.warmup):
        pool.step(1)
    times = []
    for _ in range(args.steps):
        dt, _ = pool.step(1)
        times.append(dt)
    pool.close()
    tot = sum(times)
    value = P * upd * args.steps / tot
    sample = "%d of the %d chains (one per host core), 1 sweep per chain per step" % (P, n_chains)
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * tot / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=workload_desc(spec, n_chains), sample=sample),
                sweeps_per_s=P * args.steps / tot,
                cpu_baseline=dict(value=value, unit=UNIT, cores=P, nproc=host_cores(), core_cap=ORACLE_CAP,
                                  kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def cpu_baseline(spec, n_chains, target_s=12.0):
    """The oracle as it stands on the host cores: one single-threaded process
    per core (P = nproc, at most ORACLE_CAP), each sweeping its own chain of
    the workload; one untimed sweep, then as many timed sweeps as fill about
    target_s of wall time."""
    from paper_2601_08552_gb300 import inputs

    P = oracle_cores()
    pool = OraclePool(spec, inputs.SEED0, P)
    upd = 2 * round(spec["beta"] / spec["dtau"]) * spec["lattice"][1] * spec["lattice"][2]
    dt1, _ = pool.step(1)
    k = max(2, min(200, int(target_s / max(dt1, 1e-3))))
    dt, _ = pool.step(k)
    pool.close()
    sample = ("%d chains of the %d-chain workload (one process per host core), %d timed sweeps each after one "
              "untimed, %.1f s wall" % (P, n_chains, k, dt))
    return dict(value=P * upd * k / dt, unit=UNIT, cores=P, nproc=host_cores(), core_cap=ORACLE_CAP, kind="oracle",
                sample=sample, sweeps_per_s=P * k / dt)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", bus_id], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


# ---------------------------------------------------------------------------
# the GPU leg
# ---------------------------------------------------------------------------
def algorithmic_fp64_flops(spec, n_chains, accepts, attempts, G_bonds, prec):
    """FP64 flops of one sweep of all chains: field-flip algebra (Sherman-
    Morrison ratio and rank-1 update), and for FP64 panels the slice
    propagation, the block Gram matrices and CholeskyQR2.  The square
    lattice's checkerboard families share one cosh each and hold every site
    once, so a bond costs two FMAs per column (x_i + t x_j, x_j + t x_i) and
    the cosh product and the field factor one multiply per element."""
    N = spec["lattice"][1] * spec["lattice"][2]
    L = round(spec["beta"] / spec["dtau"])
    n = -(-L // spec["n_stab"])
    ms = (spec["n_up"], spec["n_dn"])
    a = accepts / max(attempts, 1)
    per_attempt = sum(2 * m * m + 2 * m for m in ms) + a * sum(4 * m * m + m for m in ms)
    flips = 2 * L * N * per_attempt
    if prec == 0:
        prop = sum(4 * L * (4 * G_bonds * m + 2 * N * m) for m in ms)
        qr = sum(2 * n * 6 * N * m * m for m in ms)
        gram = sum(2 * n * 2 * N * m * m for m in ms)
    else:
        prop = gram = 0
        qr = sum(2 * n * 6 * N * m * m for m in ms)
    return n_chains * (flips + prop + qr + gram)


def kernel_source_hash():
    """Hash of the device code (the kernels and the structs they read), with
    comments and whitespace removed: the committed DRAM traffic is used only
    while the code it was measured on is unchanged."""
    import re

    h = hashlib.sha256()
    for f in ("lq_device.h", "lq_sweep.cuh", "lq_kernels.cu", "lq_kernels.h"):
        with open(os.path.join(ROOT, "paper_2601_08552_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_fp64_peak(lq):
    """The FP64 roof measured in this run by lq_device_fp64_rate (independent
    FMA chains on every SM, grown to about 300 ms, CUDA events), else the
    unit-count figure."""
    try:
        t, cyc = lq.device_fp64_rate(300.0)
        return t, ("measured in this run: lq_device_fp64_rate, FP64 FMA chains on every SM, CUDA events "
                   "(%.3f TFLOP/s)" % t), cyc
    except Exception as e:  # the probe failed: say so and use the unit-count figure
        return FP64_FALLBACK_TFLOPS, "fallback (probe failed: %s): 0.5 FMA/cycle/sub-partition x 4 x 152 x " \
                                     "2.07 GHz x 2" % e, None


def measured_hbm_gbs():
    """The pod's measured copy bandwidth (MEASURED_PEAKS.json beside this
    file), else the earlier GB300 measurement of 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def profiled_traffic(kind):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
    p = os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get(kind)


def serving_leg(lq, inputs, prec, rate=200.0, window_s=5.0, n_sweeps=10, seed=None):
    """Continuous batching through lq_server_*: a seeded Poisson stream of
    Hubbard runs of differing size, admitted by device footprint while
    earlier requests run.  The request mix is the serving workload's shape
    scaled down so that the leg takes seconds: N in [64, 1024], N_up = N_dn
    in [2, 16], beta in [1, 4], n_sweeps sweeps per request."""
    rng = np.random.default_rng(inputs.SEED0 + 5 if seed is None else seed)
    reqs = inputs.serving_mix(rng, rate, window_s, n_range=(64, 1024), ns_range=(2, 16), beta_range=(1.0, 4.0),
                              n_sweeps=n_sweeps)
    lats = {}
    srv = lq.Server(hbm_budget=64 << 30, precision=prec, max_active=304, queue_capacity=len(reqs) + 16)
    pending, results, i = {}, [], 0
    t0 = time.perf_counter()
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i]["t"] <= now:
            r = reqs[i]
            if r["lattice"] not in lats:
                lats[r["lattice"]] = getattr(lq.Lattice, r["lattice"][0])(*r["lattice"][1:])
            params = {k: r[k] for k in ("U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
            params.update(precision=prec, seed=inputs.SEED0)
            pending[srv.submit(lats[r["lattice"]], params, r["n_sweeps"], chain_id=i)] = i
            i += 1
        for rid in list(pending):
            res = srv.poll(rid)
            if res is not None:
                results.append(res)
                del pending[rid]
        if now > 600:
            raise RuntimeError("serving leg did not drain")
        time.sleep(0.005)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    tot = [r["total_ms"] for r in results]
    que = [r["queue_ms"] for r in results]
    return dict(requests=len(reqs), offered_rate_per_s=len(reqs) / window_s, completed=len(results),
                failed=sum(1 for r in results if r["status"] != 0), wall_s=wall,
                p50_sweep_ms=st["p50_sweep_ms"], p99_sweep_ms=st["p99_sweep_ms"], updates_per_s=st["updates_per_s"],
                unit=UNIT, request_p50_ms=float(np.percentile(tot, 50)), request_p99_ms=float(np.percentile(tot, 99)),
                queue_p50_ms=float(np.percentile(que, 50)), queue_p99_ms=float(np.percentile(que, 99)),
                device_busy_s=st["busy_s"], host_admit_s=st["admit_s"], host_retire_s=st["retire_s"],
                p50_tick_ms=st["p50_tick_ms"], p99_tick_ms=st["p99_tick_ms"], launches=st["ticks"],
                mix="Poisson %.0f/s for %.0f s; square (Lx, Ly even) or flat-band chain 50/50, N in [64, 1024], "
                    "N_up=N_dn in [2, 16], U in [-6, 6], beta in [1, 4], dtau 0.05, QR every 8, %d sweeps each"
                    % (rate, window_s, n_sweeps),
                precision=prec)


# ---------------------------------------------------------------------------
# multi-rank helpers (one process per GPU; chains are independent, so ranks
# share nothing but the timing reduction)
# ---------------------------------------------------------------------------
def rank_chain_ids(rank, n_chains):
    """Philox chain words of this rank's chains: disjoint across ranks."""
    return [rank * n_chains + c for c in range(n_chains)]


def max_over_ranks(torch, dist, x, device):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units_per_rank_step, steps, max_ms):
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    return world * units_per_rank_step * steps / (max_ms * 1e-3)


def uneven_leg(lq, inputs, torch, stream, prec=0, n_chains=608, steps=2, warmup=1, autotune=True):
    """Hundreds of flat-band chains of uneven N, N_sigma and beta advancing in
    one persistent launch per plan class.  The paper-shaped batch (cells
    U[64, 512], beta U[4, 40]) costs minutes per sweep, so the leg draws
    cells U[16, 128] and beta U[1, 4] with the same filling law (N_sigma
    from 2 to 48, both plan classes present)."""
    rng = np.random.default_rng(inputs.SEED0 + 4)
    specs = inputs.flatband_batch(rng, n_chains, cells=(16, 128), beta_range=(1.0, 4.0))
    lats = [lq.Lattice.flatband(*sp["lattice"][1:]) for sp in specs]
    params = [dict({k: sp[k] for k in ("U", "beta", "dtau", "n_up", "n_dn", "n_stab")}, precision=prec,
                   seed=inputs.SEED0) for sp in specs]
    sim = lq.Sim(lats, params, stream=stream.cuda_stream)
    sim.init()
    bufs = sim.autotune(1 if autotune else 0)
    for _ in range(warmup):
        sim.sweep(1, measure=True)
    per = time_steps(torch, sim, steps, stream)
    upd = sum(2 * round(p["beta"] / p["dtau"]) * L.N for p, L in zip(params, lats))
    ns = np.array([p["n_up"] for p in params])
    Ns = np.array([L.N for L in lats])
    sim.close()
    return dict(chains=n_chains, value=upd * steps / (sum(per) * 1e-3), unit=UNIT,
                sweeps_per_s=n_chains * steps / (sum(per) * 1e-3), ms_per_sweep=float(np.mean(per)),
                n_sigma_range=[int(ns.min()), int(ns.max())], chains_above_32=int((ns > 32).sum()),
                N_range=[int(Ns.min()), int(Ns.max())], precision="FP64", staging_bytes_per_class=list(bufs),
                mix="BCL flat-band chains, cells U[16, 128], filling U[1/4, 3/4] of the flat band split by spin, "
                    "beta U[1, 4], dtau 0.05, U=2, half periodic")


def gas64_leg(lq, inputs, torch, stream, fp64_peak, warmup=1, steps=2, n_chains=None):
    """The mixed-precision configuration at full size: 64x64 periodic square
    (N = 4096), N_up = N_dn = 16, U = +4, beta = 16 (L = 320), QR every 8
    slices, 512 chains in one launch.  FP64, LQ_MIXED (FP32 panels, FP64
    algebra and ratios) and LQ_MIXED_DW run from identical seeded states (same
    seeds, so the same initial fields and Fock states); each reports its rate,
    its ratio to FP64, the log-weight error of its freshly built chains
    against FP64's on those states, and its chain-mean observables against
    FP64's in standard errors."""
    w = inputs.WORKLOADS["gas64x64"]
    spec = {k: w[k] for k in ("lattice", "U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
    n = n_chains or w["chains"]
    lat = lq.Lattice.square(64, 64)
    N, L = lat.N, round(spec["beta"] / spec["dtau"])
    upd = n * 2 * L * N
    out, lw0, obs = {}, {}, {}
    for prec, key in ((0, "fp64"), (1, "mixed"), (2, "mixed_dw")):
        sim = lq.Sim([lat] * n, [dict(spec, precision=prec, seed=inputs.SEED0)] * n, stream=stream.cuda_stream)
        sim.init()
        lw0[prec] = np.array([sim.log_weight(c)[0] for c in range(4)])
        for _ in range(warmup):
            sim.sweep(1, measure=True)
        sim.sync()
        st0 = sum(sim.stats(c) for c in range(n))
        pr0 = sum(sim.profile(c) for c in range(n))
        per = time_steps(torch, sim, steps, stream)
        sim.sync()
        d = sum(sim.stats(c) for c in range(n)) - st0
        pr = sum(sim.profile(c) for c in range(n)) - pr0
        tot = max(float(pr[:6].sum()), 1.0)
        shares = {k: round(float(pr[i]) / tot, 4) for i, k in
                  enumerate(["flips", "propagation", "qr", "block_inverse", "swaps", "measure"])}
        obs[prec] = np.stack([sim.records(c).mean(axis=0) for c in range(n)])
        ms = float(np.mean(per))
        r = dict(value=upd / (ms * 1e-3), unit=UNIT, sweeps_per_s=n / (ms * 1e-3), ms_per_sweep=ms,
                 field_accept=float(d[1] / max(d[0], 1)), swap_accept=float(d[3] / max(d[2], 1)),
                 phase_cycle_share=shares)
        if prec < 2:  # LQ_MIXED_DW runs the flip algebra in double-word FP32, not on the FP64 pipe
            flops = algorithmic_fp64_flops(spec, n, d[1], d[0], lat.n_bonds, prec)
            r["fp64_alu"] = dict(achieved=flops / (ms * 1e-3) / 1e12, peak=fp64_peak, unit="TFLOP/s",
                                 frac=flops / (ms * 1e-3) / 1e12 / fp64_peak)
        # propagation streams every N x N_sigma panel through the SM once per slice and
        # panel (read and write): its bytes over the wall time the phase takes
        b = 4 if prec else 8
        prop_bytes = n * sum(4 * L * 2 * N * m * b for m in (spec["n_up"], spec["n_dn"]))
        prop_s = ms * 1e-3 * shares["propagation"]
        hbm_peak, _ = measured_hbm_gbs()
        r["propagation_effective_gbs"] = dict(achieved=prop_bytes / max(prop_s, 1e-12) / 1e9, peak=hbm_peak,
                                              frac=prop_bytes / max(prop_s, 1e-12) / 1e9 / hbm_peak,
                                              note="panel bytes (read + write per slice) over the sweep time "
                                                   "times the propagation share of the cycles")
        if prec:
            r["speedup_vs_fp64"] = r["value"] / out["fp64"]["value"]
            r["logw_max_rel_err_vs_fp64"] = float(np.max(np.abs(lw0[prec] - lw0[0]) /
                                                         np.maximum(1.0, np.abs(lw0[0]))))
            r["observables_vs_fp64"] = observable_deviation(obs[prec], obs[0])
        out[key] = r
        sim.close()
        del sim
    out["workload"] = ("64x64 periodic square, t=1, U=+4, beta=16, dtau=0.05 (L=320), N_up=N_dn=16, QR every 8, "
                       "%d chains in one launch; %d warm-up and %d timed sweeps per precision, identical seeded "
                       "initial states" % (n, warmup, steps))
    return out


def cp_leg(lq, inputs, torch, n_walkers=304, comb_every=8):
    """The constrained-path inner loop on the headline lattice: for a seeded
    Fock state of the 32x32 gas (N_up = N_dn = 8, U = +4, beta = 10, dtau =
    0.05, L = 200), n_walkers independent walkers (lq_cp_walk) and a
    branching population of the same size combed every comb_every slices
    (lq_cp_population).  A walker samples one field per site and slice, so the
    rate is field samples per second (walkers x L x N over the call's wall
    time, set-up included)."""
    from paper_2601_08552_gb300.lecqmc import cp_population, cp_walk

    rng = np.random.default_rng(inputs.SEED0 + 7)
    lat = lq.Lattice.square(32, 32)
    up, dn = inputs.fock(rng, 1024, 8), inputs.fock(rng, 1024, 8)
    p = dict(U=4.0, beta=10.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8, seed=inputs.SEED0)
    samples = n_walkers * 200 * 1024
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lw, dropped = cp_walk(lat, p, up, dn, n_walkers)
    t_walk = time.perf_counter() - t0
    t0 = time.perf_counter()
    est = cp_population(lat, p, up, dn, n_walkers, comb_every, run=1)
    t_pop = time.perf_counter() - t0
    alive = np.isfinite(lw)
    return dict(walkers=n_walkers, field_samples_per_s=samples / t_walk, walk_s=t_walk, dropped=int(dropped),
                log_mean_weight=float(np.log(np.mean(np.exp(lw[alive] - lw[alive].max()))) + lw[alive].max())
                if alive.any() else None,
                population_field_samples_per_s=samples / t_pop, population_s=t_pop, comb_every=comb_every,
                population_log_estimate=est, precision="FP64",
                workload="32x32 periodic square, U=+4, beta=10, dtau=0.05 (L=200), N_up=N_dn=8, one seeded Fock "
                         "state; one CTA per walker")


def uneven_full_leg(lq, inputs, torch, stream, beta_scale=0.1, n_chains=1024, check_chains=2):
    """The paper-shaped uneven batch in one lq_sim_sweep call: 1024 BCL
    flat-band chains, cells U[64, 512] (N = 128 to 1024), filling U[1/4, 3/4]
    of the flat band split by spin (N_sigma = f N_cells, up to 384), U = 2,
    half periodic, with beta drawn from U[4, 40] and then scaled by beta_scale
    (rounded to whole slices): the work of a chain grows linearly with its
    slices, so the full-beta sweep time is the measured one over beta_scale.
    One autotuned sweep is timed; the check_chains cheapest chains are re-run
    by the oracle from the same seeds (fields, occupations and counts
    bit-exact)."""
    from oracle import OracleSim, lattices

    rng = np.random.default_rng(inputs.SEED0 + 4)
    specs = inputs.flatband_batch(rng, n_chains, cells=(64, 512), beta_range=(4.0, 40.0))
    for sp in specs:
        sp["beta"] = max(0.05, round(sp["beta"] * beta_scale / 0.05) * 0.05)
    lats = [lq.Lattice.flatband(*sp["lattice"][1:]) for sp in specs]
    params = [dict({k: sp[k] for k in ("U", "beta", "dtau", "n_up", "n_dn", "n_stab")}, precision=0,
                   seed=inputs.SEED0) for sp in specs]
    sim = lq.Sim(lats, params, stream=stream.cuda_stream)
    sim.init()
    cfg0 = sim.launch_config()
    per = time_steps(torch, sim, 1, stream)
    sim.sync()
    ns = np.array([p["n_up"] for p in params])
    Ns = np.array([L.N for L in lats])
    Ls = np.array([round(p["beta"] / p["dtau"]) for p in params])
    upd = int(np.sum(2 * Ls * Ns))
    cost = Ls * Ns * ns.astype(float) ** 2
    parity = []
    for c in np.argsort(cost)[:check_chains]:
        sp = specs[c]
        lat = lattices.flatband(*sp["lattice"][1:])
        o = OracleSim(lat, sp["U"], sp["beta"], sp["dtau"], sp["n_up"], sp["n_dn"], sp["n_stab"], seed=inputs.SEED0,
                      chain=int(c))
        o.sweep(1)
        gu, gd = sim.get_fock(int(c))
        ou, od = o.get_fock()
        parity.append(dict(chain=int(c), N=int(Ns[c]), n_sigma=int(ns[c]), L=int(Ls[c]),
                           fields=bool(np.array_equal(sim.get_fields(int(c)), o.get_fields())),
                           fock=bool(np.array_equal(gu, ou) and np.array_equal(gd, od)),
                           counts=bool(np.array_equal(sim.stats(int(c)), o.stats()))))
    sim.close()
    return dict(chains=n_chains, ms_per_sweep=per[0], beta_scale=beta_scale,
                full_beta_ms_per_sweep_estimate=per[0] / beta_scale, value=upd / (per[0] * 1e-3), unit=UNIT,
                n_sigma_range=[int(ns.min()), int(ns.max())], chains_above_32=int((ns > 32).sum()),
                N_range=[int(Ns.min()), int(Ns.max())], L_range=[int(Ls.min()), int(Ls.max())],
                launch=cfg0, oracle_parity=parity, precision="FP64",
                mix="BCL flat-band chains, cells U[64, 512], filling U[1/4, 3/4] of the flat band split by spin "
                    "(N_sigma = f N_cells), beta U[4, 40] x %g, dtau 0.05, U=2, half periodic" % beta_scale)


def chain16_leg(lq, inputs, torch, stream, warm=200, sweeps=1000):
    """The single-chain FP64 run on the 16-site Hubbard chain (N_up = N_dn = 2,
    U = 4, beta = 4, dtau = 0.1, QR every 10): `warm` unmeasured sweeps, then
    `sweeps` measured sweeps in one launch timed by CUDA events; beside it the
    oracle on one host core (a spawned process) on the same chain for about
    5 s of sweeps.  One chain occupies one CTA, so this is the latency of a
    sweep, not a throughput figure."""
    w = inputs.WORKLOADS["chain16"]
    spec = {k: w[k] for k in ("lattice", "U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
    N = spec["lattice"][1]
    L = round(spec["beta"] / spec["dtau"])
    lat = lq.Lattice.chain(N)
    sim = lq.Sim([lat], [dict(spec, precision=0, seed=inputs.SEED0)], stream=stream.cuda_stream)
    sim.init()
    sim.sweep(warm, measure=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.sweep(sweeps, measure=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = sim.stats(0)
    sim.close()
    upd = 2 * L * N
    out = dict(value=upd * sweeps / (ms * 1e-3), unit=UNIT, sweeps_per_s=sweeps / (ms * 1e-3), ms_per_sweep=ms / sweeps,
               field_accept=float(st[1] / max(st[0], 1)), swap_accept=float(st[3] / max(st[2], 1)),
               sweeps=sweeps, warm=warm, precision="FP64",
               workload="1D periodic Hubbard chain N=16, t=1, N_up=N_dn=2, U=4, beta=4, dtau=0.1 (L=40), QR every 10, "
                        "1 chain, %d + %d sweeps" % (warm, sweeps))
    pool = OraclePool(spec, inputs.SEED0, 1)
    dt1, _ = pool.step(1)
    k = max(2, min(5000, int(5.0 / max(dt1, 1e-4))))
    dt, _ = pool.step(k)
    pool.close()
    out["oracle_1core"] = dict(value=upd * k / dt, unit=UNIT, sweeps_per_s=k / dt, cores=1, kind="oracle",
                               sample="the same chain, %d timed sweeps after one untimed, %.1f s wall" % (k, dt))
    return out


def observable_deviation(a, b):
    """Chain-mean observables of two runs from the same seeded states: the
    largest |difference| over the measured observables in units of the
    combined standard error across chains (the FP64 run as reference)."""
    from paper_2601_08552_gb300 import OBS_NAMES

    ma, mb = a.mean(axis=0), b.mean(axis=0)
    se = np.sqrt(a.var(axis=0, ddof=1) / len(a) + b.var(axis=0, ddof=1) / len(b))
    dev = {}
    for k, name in enumerate(OBS_NAMES):
        if se[k] > 0:
            dev[name] = float(abs(ma[k] - mb[k]) / se[k])
    return dict(max_sigma=max(dev.values()) if dev else 0.0, sigma=dev,
                max_rel=float(np.max(np.abs(ma - mb) / np.maximum(np.abs(mb), 1e-300))))


def time_steps(torch, sim, steps, stream):
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        sim.sweep(1, measure=True)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return per


def nsigma_scan(lq, torch, stream, sizes=(16, 32, 33, 48, 64, 96, 128, 192, 256, 384), cells=256, L_slices=40):
    """Cost of a sweep against N_sigma: 152 flat-band chains (one per SM) of
    `cells` cells (N = 2 cells, BCL t1 = t2 = t3 = t4 = 1, periodic), U = 2,
    dtau = 0.05, L = L_slices, QR every 8, FP64; one untimed and one timed
    sweep per N_sigma.  Reports microseconds per site and chain (the sweep
    time over 2 L N sites) and the phase shares, with the swap removal and
    addition sub-phases."""
    out = []
    for ns in sizes:
        if ns > cells:
            continue
        lat = lq.Lattice.flatband(cells, 1.0, 1.0, 1.0, 1.0, True)
        p = dict(U=2.0, beta=L_slices * 0.05, dtau=0.05, n_up=ns, n_dn=ns, n_stab=8, precision=0, seed=1)
        n = 152
        sim = lq.Sim([lat] * n, [p] * n, stream=stream.cuda_stream)
        sim.init()
        sim.sweep(1, measure=False)
        sim.sync()
        pr0 = sum(sim.profile(c) for c in range(n))
        per = time_steps(torch, sim, 1, stream)
        pr = sum(sim.profile(c) for c in range(n)) - pr0
        tot = max(float(pr[:6].sum()), 1.0)
        out.append(dict(n_sigma=ns, us_per_site=1e3 * per[0] / (2 * L_slices * lat.N),
                        flips=round(float(pr[0]) / tot, 3), propagation=round(float(pr[1]) / tot, 3),
                        qr=round(float(pr[2] + pr[3]) / tot, 3), swaps=round(float(pr[4]) / tot, 3),
                        swap_removal=round(float(pr[6]) / tot, 3), swap_addition=round(float(pr[7]) / tot, 3)))
        sim.close()
    return dict(workload="152 BCL flat-band chains of %d cells (N = %d), U = 2, dtau = 0.05, L = %d, QR every 8, "
                         "FP64, one sweep" % (cells, 2 * cells, L_slices), rows=out)


def gram_scan(lq, sizes=((1024, 16), (1024, 64), (4096, 16), (4096, 64), (4096, 128), (16384, 64)), n_panels=304):
    """The sweep's Gram contraction W = A^T B of two N x m panels, one per CTA
    (304 CTAs: two per SM, as the sweep runs), on the FP64 CUDA cores, the
    FP64 tensor cores (DMMA), FP32 panels with FP64 CUDA-core accumulation,
    and FP32 panels on the TF32 tensor cores with the three-product split."""
    from paper_2601_08552_gb300.lecqmc import GRAM_VARIANTS, probe_gram

    rows = []
    for N, m in sizes:
        r = dict(N=N, m=m)
        for v, name in enumerate(GRAM_VARIANTS):
            us, err = probe_gram(N, m, v, n_panels)
            r[name] = dict(us=us, gflops=2.0 * N * m * m * n_panels / (us * 1e-6) / 1e9, max_rel_err=err)
        rows.append(r)
    return dict(panels_per_launch=n_panels, rows=rows)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--chains", type=int, default=0, help="override the chain count (small profiling cases)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-gas64", action="store_true", help="skip the 64x64 mixed-precision leg (512 chains)")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline FP64 leg and its e2e (small profiling cases)")
    ap.add_argument("--gram-scan", action="store_true",
                    help="only the Gram study: CUDA cores against tensor cores (DMMA, 3xTF32)")
    ap.add_argument("--uneven-full", action="store_true",
                    help="only the paper-shaped uneven flat-band batch (1024 chains, N_sigma up to 384), beta scaled")
    ap.add_argument("--nsigma-scan", action="store_true",
                    help="only the cost-against-N_sigma study (flat-band chains, one sweep per N_sigma)")
    ap.add_argument("--nsigma-sizes", default="",
                    help="comma-separated N_sigma values for --nsigma-scan (default: 16 to 384)")
    ap.add_argument("--serving-window", type=float, default=10.0)
    ap.add_argument("--workload", default=WORKLOAD, choices=["gas32x32", "gas64x64"],
                    help="gas64x64: the 64x64 mixed-precision comparison (512 chains, ~10 s per sweep)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.headline_only:
        args.no_mixed = args.no_serving = args.no_uneven = args.no_gas64 = True

    from paper_2601_08552_gb300 import inputs

    w = inputs.WORKLOADS[args.workload]
    spec = {k: w[k] for k in ("lattice", "U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
    n_chains = args.chains or w["chains"]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, spec, n_chains)
        return

    # the CPU baseline runs first, in spawned processes, before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not (args.nsigma_scan or args.gram_scan or
                                                                      args.uneven_full):
        cpu = cpu_baseline(spec, n_chains)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2601_08552_gb300 as lq

    stream = torch.cuda.current_stream()
    if args.nsigma_scan:
        kw = dict(sizes=tuple(int(x) for x in args.nsigma_sizes.split(","))) if args.nsigma_sizes else {}
        print(json.dumps(dict(study="cost against N_sigma", **nsigma_scan(lq, torch, stream, **kw))), flush=True)
        return
    if args.uneven_full:
        print(json.dumps(dict(study="paper-shaped uneven batch", **uneven_full_leg(lq, inputs, torch, stream))),
              flush=True)
        return
    if args.gram_scan:
        print(json.dumps(dict(study="Gram contractions: CUDA cores and tensor cores", **gram_scan(lq))), flush=True)
        return
    lat = lq.Lattice.square(spec["lattice"][1], spec["lattice"][2])
    N = lat.N
    L = round(spec["beta"] / spec["dtau"])
    upd_per_step = n_chains * 2 * L * N

    def make(prec, sp=spec):
        ids = rank_chain_ids(rank, n_chains)
        s = lq.Sim([lat] * n_chains, [dict(sp, precision=prec, seed=inputs.SEED0)] * n_chains, chain_ids=ids,
                   stream=stream.cuda_stream)
        s.init()
        return s

    def run(prec, sp=spec):
        sim = make(prec, sp)
        # log-weights of the first chains on their seeded initial fields (identical across precisions)
        lw0 = np.array([sim.log_weight(c)[0] for c in range(min(8, n_chains))])
        run.lw0[prec] = lw0
        # the autotuner's timed candidates are ordinary (unmeasured) sweeps: part of the warm-up
        run.tuned[prec] = sim.autotune(0 if args.no_autotune else 1)
        for _ in range(args.warmup):
            sim.sweep(1, measure=True)
        sim.sync()
        st0 = sum(sim.stats(c) for c in range(n_chains))
        pr0 = sum(sim.profile(c) for c in range(n_chains))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        props = torch.cuda.get_device_properties(local)
        bus = "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
        clk = ClockSampler(bus) if (prec == 0 and sp is spec) else None
        per = time_steps(torch, sim, args.steps, stream)
        clocks = clk.stop() if clk else None
        total_ms = max_over_ranks(torch, dist, sum(per), "cuda")
        sim.sync()
        st1 = sum(sim.stats(c) for c in range(n_chains))
        d = st1 - st0
        pr = sum(sim.profile(c) for c in range(n_chains)) - pr0
        tot = max(float(pr[:6].sum()), 1.0)
        phases = {k: round(float(pr[i]) / tot, 4) for i, k in
                  enumerate(["flips", "propagation", "qr", "block_inverse", "swaps", "measure"])}
        if pr[8:12].sum() > 0:  # parts of the flips (chains of up to 32 particles per spin)
            phases.update({k: round(float(pr[8 + i]) / tot, 4) for i, k in
                           enumerate(["flip_staging", "flip_first_window", "flip_serial_chain", "flip_loop_rest"])})
        # per-chain means of the measured observables (warm-up and timed sweeps)
        if sp is spec:
            run.obs[prec] = np.stack([sim.records(c).mean(axis=0) for c in range(n_chains)])
        return sim, per, total_ms, clocks, d, phases

    run.lw0 = {}
    run.tuned = {}
    run.obs = {}
    sim, per, total_ms, clocks, dstat, phases = run(0)
    value = aggregate_rate(world, upd_per_step, args.steps, total_ms)
    sweeps = world * n_chains * args.steps / (total_ms * 1e-3)
    flops = algorithmic_fp64_flops(spec, n_chains, dstat[1], dstat[0], lat.n_bonds, 0)
    kern_ms = total_ms / args.steps
    achieved = flops / (kern_ms * 1e-3) / 1e12
    fp64_peak, peak_src, issue = measured_fp64_peak(lq)
    roofline = dict(bound="alu", achieved=achieved, peak=fp64_peak, unit="TFLOP/s",
                    frac=achieved / fp64_peak, traffic=profiled_traffic("fp64_bytes_per_launch"),
                    kernel="lq::sweep_kernel<double, false>", flops_per_launch=flops, peak_source=peak_src,
                    fp64_issue_cycles=issue)
    if roofline["traffic"]:
        # the same kernel against DRAM: profiled bytes per launch over the launch time
        hbm_peak, hbm_src = measured_hbm_gbs()
        hbm_ach = roofline["traffic"] / (kern_ms * 1e-3) / 1e9
        roofline["hbm"] = dict(achieved=hbm_ach, peak=hbm_peak, unit="GB/s", frac=hbm_ach / hbm_peak, source=hbm_src)

    # end to end through the C ABI on pinned host buffers
    n_occ = spec["n_up"] + spec["n_dn"]
    hf = torch.empty(n_chains * L * N, dtype=torch.int8, pin_memory=True)
    ho = torch.empty(n_chains * n_occ, dtype=torch.int32, pin_memory=True)
    for c in range(n_chains):
        hf[c * L * N:(c + 1) * L * N] = torch.from_numpy(sim.get_fields(c).ravel())
        u, dn = sim.get_fock(c)
        ho[c * n_occ:(c + 1) * n_occ] = torch.from_numpy(np.concatenate([u, dn]).astype(np.int32))
    hf_out = torch.empty_like(hf).pin_memory()
    ho_out = torch.empty_like(ho).pin_memory()
    rec = torch.empty(n_chains * lq.LQ_NOBS, dtype=torch.float64, pin_memory=True)
    e2e_times = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        sim.run_host(hf, ho, 1, True, hf_out, ho_out, rec)
        dt = time.perf_counter() - t0
        hf, hf_out = hf_out, hf
        ho, ho_out = ho_out, ho
        if k > 0:
            e2e_times.append(dt)
    e2e_s = max_over_ranks(torch, dist, max(sum(e2e_times), 1e-12), "cuda")
    e2e = dict(value=world * upd_per_step * len(e2e_times) / e2e_s, unit=UNIT,
               h2d_bytes_per_step=int(hf.numel() + 4 * ho.numel()),
               d2h_bytes_per_step=int(hf.numel() + 4 * ho.numel() + 8 * rec.numel()),
               call="lq_sim_run_host (upload, QR-chain rebuild, 1 sweep, download)")
    bytes_dev = sim.device_bytes()
    sim.close()
    del sim

    mixed = None
    if not args.no_mixed:
        mixed = {}
        for prec, key, desc in ((1, "mixed", "FP32 panels; FP64 QR, inverses, flip algebra, ratios"),
                                (2, "mixed_dw", "FP32 panels; double-word FP32 flip algebra; FP64 QR, inverses, "
                                                "log-weights")):
            msim, mper, mtotal, _, mstat, mphases = run(prec)
            d = dict(value=world * upd_per_step * args.steps / (mtotal * 1e-3), unit=UNIT,
                     sweeps_per_s=world * n_chains * args.steps / (mtotal * 1e-3),
                     p50_ms=float(np.percentile(mper, 50)), p99_ms=float(np.percentile(mper, 99)),
                     field_accept=float(mstat[1] / max(mstat[0], 1)), phase_cycle_share=mphases, precision=desc)
            d["speedup_vs_fp64"] = d["value"] / value
            d["logw_max_rel_err_vs_fp64"] = float(np.max(np.abs(run.lw0[prec] - run.lw0[0]) /
                                                         np.maximum(1.0, np.abs(run.lw0[0]))))
            d["observables_vs_fp64"] = observable_deviation(run.obs[prec], run.obs[0])
            mixed[key] = d
            msim.close()

    # the second run of the 32x32 gas: attractive U = -4 (charge-channel fields)
    attractive = None
    if not args.headline_only and args.workload + "_attractive" in inputs.WORKLOADS:
        wa = inputs.WORKLOADS[args.workload + "_attractive"]
        spa = {k: wa[k] for k in ("lattice", "U", "beta", "dtau", "n_up", "n_dn", "n_stab")}
        asim, aper, atotal, _, astat, aphases = run(0, spa)
        attractive = dict(value=world * upd_per_step * args.steps / (atotal * 1e-3), unit=UNIT, U=spa["U"],
                          sweeps_per_s=world * n_chains * args.steps / (atotal * 1e-3),
                          p50_ms=float(np.percentile(aper, 50)), p99_ms=float(np.percentile(aper, 99)),
                          field_accept=float(astat[1] / max(astat[0], 1)),
                          swap_accept=float(astat[3] / max(astat[2], 1)), phase_cycle_share=aphases, precision="FP64")
        asim.close()

    uneven = None
    if not args.no_uneven and args.workload == WORKLOAD:
        uneven = uneven_leg(lq, inputs, torch, stream, autotune=not args.no_autotune)

    # nearest-neighbour Fock-swap proposals on the same workload (FP64)
    neighbour = None
    if not args.headline_only and args.workload == WORKLOAD:
        spn = dict(spec, swap_mode=1)
        nsim, nper, ntotal, _, nstat, nphases = run(0, spn)
        neighbour = dict(value=world * upd_per_step * args.steps / (ntotal * 1e-3), unit=UNIT,
                         swap_accept=float(nstat[3] / max(nstat[2], 1)),
                         swap_accept_uniform=float(dstat[3] / max(dstat[2], 1)),
                         field_accept=float(nstat[1] / max(nstat[0], 1)), phase_cycle_share=nphases,
                         proposal="target uniform among the empty nearest neighbours, Metropolis-Hastings factor",
                         precision="FP64")
        nsim.close()

    # a second swap phase per sweep at tau = 0 on the left chain (FP64): twice
    # the Fock-swap attempts, at the cost of one more swap phase
    left = None
    if not args.headline_only and args.workload == WORKLOAD:
        spl = dict(spec, left_swaps=1)
        lsim, lper, ltotal, _, lstat, lphases = run(0, spl)
        left = dict(value=world * upd_per_step * args.steps / (ltotal * 1e-3), unit=UNIT,
                    swap_accept=float(lstat[3] / max(lstat[2], 1)),
                    swap_attempts_vs_one_phase=float(lstat[2]) / max(float(dstat[2]), 1.0),
                    rate_vs_one_phase=(world * upd_per_step * args.steps / (ltotal * 1e-3)) / value,
                    field_accept=float(lstat[1] / max(lstat[0], 1)), phase_cycle_share=lphases,
                    swaps="N_up + N_dn attempts after the up pass (tau = beta, right chain) and again after the "
                          "down pass (tau = 0, left chain)", precision="FP64")
        lsim.close()

    cp = None
    if not args.headline_only and args.workload == WORKLOAD:
        cp = cp_leg(lq, inputs, torch)

    chain16 = None
    if not args.headline_only and args.workload == WORKLOAD:
        chain16 = chain16_leg(lq, inputs, torch, stream)

    gas64 = None
    if not args.no_gas64 and args.workload == WORKLOAD:
        gas64 = gas64_leg(lq, inputs, torch, stream, roofline["peak"])

    serving = None
    if not args.no_serving and world == 1 and args.workload == WORKLOAD:
        # the same request stream served in LQ_MIXED and in plain FP64
        serving = serving_leg(lq, inputs, 1, window_s=args.serving_window)
        serving_fp64 = serving_leg(lq, inputs, 0, window_s=args.serving_window)
        serving["fp64"] = {k: serving_fp64[k] for k in ("updates_per_s", "p50_sweep_ms", "p99_sweep_ms",
                                                        "request_p50_ms", "request_p99_ms", "completed", "wall_s",
                                                        "device_busy_s")}
        serving["mixed_vs_fp64_updates"] = serving["updates_per_s"] / max(serving_fp64["updates_per_s"], 1e-9)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f64", data="synthetic",
                    config=dict(workload=workload_desc(spec, n_chains), chains_per_gpu=n_chains, N=N, L=L,
                                n_up=spec["n_up"], n_dn=spec["n_dn"], n_stab=spec["n_stab"], U=spec["U"],
                                l2="device state %.1f GB per GPU >> 129 MB L2; no flush" % (bytes_dev / 1e9),
                                staging_bytes=run.tuned.get(0, (0, 0))[0],
                                autotune="staging buffer picked by lq_sim_autotune (1 sweep per candidate, warm-up)"
                                if not args.no_autotune else "off",
                                parallelism="independent chains, %d per GPU" % n_chains),
                    sweeps_per_s=sweeps, p50_ms=float(np.percentile(per, 50)), p99_ms=float(np.percentile(per, 99)),
                    field_accept=float(dstat[1] / max(dstat[0], 1)),
                    swap_accept=float(dstat[3] / max(dstat[2], 1)), phase_cycle_share=phases,
                    roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=args.steps, clocks=clocks,
                    reduced_precision=mixed, attractive=attractive, neighbour_swaps=neighbour, left_swaps=left,
                    uneven_flatband=uneven, gas64x64=gas64, constrained_path=cp, chain16=chain16,
                    serving=serving)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
