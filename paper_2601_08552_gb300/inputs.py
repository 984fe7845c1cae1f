"""Seeded synthetic inputs shared by the tests and the benchmark.

Pure data generation (numpy Generator draws): field configurations, Fock
states, and the workload shapes of the benchmark configurations.  Nothing
here computes any part of the method.
"""
import numpy as np

SEED0 = 20260108


def fields(rng, L, N):
    """Uniform +-1 Hubbard-Stratonovich fields, L x N int8."""
    return np.where(rng.random((L, N)) < 0.5, 1, -1).astype(np.int8)


def fock(rng, N, n, shuffle=False):
    """n distinct occupied sites out of N (ascending unless shuffled)."""
    occ = rng.choice(N, size=n, replace=False)
    if not shuffle:
        occ = np.sort(occ)
    return occ.astype(np.int32)


# Workload shapes (synthetic, shaped like the paper's dilute Hubbard gas and
# flat-band chain).  "lattice" is (builder name, args...).
WORKLOADS = {
    "chain16": dict(lattice=("chain", 16), U=4.0, beta=4.0, dtau=0.1, n_up=2, n_dn=2, n_stab=10, chains=1),
    "gas32x32": dict(lattice=("square", 32, 32), U=4.0, beta=10.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8, chains=256),
    "gas32x32_attractive": dict(lattice=("square", 32, 32), U=-4.0, beta=10.0, dtau=0.05, n_up=8, n_dn=8, n_stab=8,
                                chains=256),
    "gas64x64": dict(lattice=("square", 64, 64), U=4.0, beta=16.0, dtau=0.05, n_up=16, n_dn=16, n_stab=8, chains=512),
}


def flatband_batch(rng, n_chains, periodic_frac=0.5, cells=(64, 512), beta_range=(4.0, 40.0)):
    """Uneven flat-band chains: cells uniform in `cells` (U[64, 512] in the
    paper-shaped workload), filling f uniform in [1/4, 3/4] of the flat band
    split evenly by spin, beta uniform in beta_range (U[4, 40]), dtau 0.05,
    U = 2; half of the chains periodic.  The flat band has one state per cell
    and spin, and half filling is N_e = N_up + N_dn = N_cells (the paper's
    half-filling condition), so N_up = N_dn = f * N_cells."""
    out = []
    for _ in range(n_chains):
        nc = int(rng.integers(cells[0], cells[1] + 1))
        f = rng.uniform(0.25, 0.75)
        ns = max(1, int(round(f * nc)))
        beta = float(np.round(rng.uniform(*beta_range) / 0.05) * 0.05)
        out.append(dict(lattice=("flatband", nc, 1.0, 1.0, 1.0, 1.0, bool(rng.random() < periodic_frac)), U=2.0,
                        beta=beta, dtau=0.05, n_up=ns, n_dn=ns, n_stab=8))
    return out


def serving_mix(rng, rate_per_s, window_s, n_range=(256, 16384), ns_range=(4, 64), beta_range=(2.0, 20.0),
                n_sweeps=100, dtau=0.05, n_stab=8):
    """Poisson request stream of Hubbard runs: arrival times (s) with mean rate
    rate_per_s over window_s, each a square lattice (Lx, Ly even, N = Lx*Ly in
    n_range) or a flat-band chain (2 sites per cell) with equal probability,
    N_up = N_dn uniform in ns_range (at most N/4), U uniform in [-6, 6], beta
    uniform in beta_range rounded to a whole number of QR blocks."""
    out, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= window_s:
            return out
        n_target = int(rng.integers(n_range[0], n_range[1] + 1))
        if rng.random() < 0.5:
            lx = max(2, 2 * int(round(np.sqrt(n_target) / 2)))
            ly = max(2, 2 * int(round(n_target / lx / 2)))
            lattice, N = ("square", lx, ly), lx * ly
        else:
            nc = max(2, n_target // 2)
            lattice, N = ("flatband", nc, 1.0, 1.0, 1.0, 1.0, True), 2 * nc
        ns = int(rng.integers(ns_range[0], ns_range[1] + 1))
        ns = max(1, min(ns, N // 4))
        blocks = max(1, int(round(rng.uniform(*beta_range) / (dtau * n_stab))))
        out.append(dict(t=t, lattice=lattice, U=float(rng.uniform(-6.0, 6.0)), beta=blocks * n_stab * dtau,
                        dtau=dtau, n_up=ns, n_dn=ns, n_stab=n_stab, n_sweeps=n_sweeps))
