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


def flatband_batch(rng, n_chains, periodic_frac=0.5):
    """Uneven flat-band chains: cells U[64, 512], filling U[1/4, 3/4] of the flat
    band split evenly by spin, beta U[4, 40], dtau 0.05, U = 2."""
    out = []
    for _ in range(n_chains):
        nc = int(rng.integers(64, 513))
        f = rng.uniform(0.25, 0.75)
        ns = max(1, int(round(f * nc / 2)))
        beta = float(np.round(rng.uniform(4.0, 40.0) / 0.05) * 0.05)
        out.append(dict(lattice=("flatband", nc, 1.0, 1.0, 1.0, 1.0, bool(rng.random() < periodic_frac)), U=2.0,
                        beta=beta, dtau=0.05, n_up=ns, n_dn=ns, n_stab=8))
    return out
