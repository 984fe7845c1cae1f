"""Validation runs of the paper's two applications on the GPU path.

* Sign in the dilute limit (main text, Fig. 2): <sign> of the 2D repulsive
  Hubbard gas at fixed particle number and temperature as the linear size L
  grows (density N_e / L^2 falls).
* Flat-band ferromagnetism (main text, Fig. 4; SM Secs. IV-V): the BCL chain
  at half filling of its flat lowest band (N_e = number of cells,
  N_up = N_dn), where the in-plane S^par(q=0) grows as T -> 0 and the
  A1-sublattice S^zz(q=0) tends to 1/16 (SM Eq. S33).  With S^z_tot = 0 in
  this sector, S^zz_11 + S^zz_22 + 2 S^zz_12 = 0 holds per measurement.

  python -m paper_2601_08552_gb300.physics [--chains C --sweeps S]

prints one JSON line per point.  Estimates are sign-weighted means with
errors from the spread of the per-chain means.
"""
import argparse
import json

import numpy as np

from . import OBS_NAMES
from . import lecqmc as lq


def _estimate(recs_by_chain, name):
    """Sign-weighted mean <sign O>/<sign> over chains, error from the spread
    of the chains' ratios (chains are independent Markov chains)."""
    k, s = OBS_NAMES.index(name), OBS_NAMES.index("sign")
    num = np.array([r[:, k].mean() for r in recs_by_chain])
    den = np.array([r[:, s].mean() for r in recs_by_chain])
    est = num.mean() / den.mean()
    # delete-one jackknife over chains
    n = len(num)
    jk = np.array([(num.sum() - num[c]) / (den.sum() - den[c]) for c in range(n)])
    err = np.sqrt((n - 1) / n * np.sum((jk - jk.mean()) ** 2))
    return float(est), float(err)


def _run(lat, params, chains, warm, sweeps):
    sim = lq.Sim([lat] * chains, [params] * chains)
    sim.init()
    sim.sweep(warm, measure=False)
    sim.sweep(sweeps, measure=True)
    sim.sync()
    recs = [sim.records(c) for c in range(chains)]
    sim.close()
    return recs


def sign_vs_size(sizes=(4, 6, 8, 12, 16, 24, 32), n_sigma=8, U=4.0, beta=10.0, dtau=0.05, chains=128, warm=50,
                 sweeps=200, seed=20260108):
    out = []
    for Ls in sizes:
        lat = lq.Lattice.square(Ls, Ls)
        p = dict(U=U, beta=beta, dtau=dtau, n_up=n_sigma, n_dn=n_sigma, n_stab=8, precision=lq.LQ_FP64, seed=seed)
        recs = _run(lat, p, chains, warm, sweeps)
        sgn = np.array([r[:, 0].mean() for r in recs])
        out.append(dict(study="sign_vs_size", L=Ls, N=Ls * Ls, n_up=n_sigma, n_dn=n_sigma, U=U, beta=beta,
                        sign=float(sgn.mean()), sign_err=float(sgn.std(ddof=1) / np.sqrt(len(sgn))),
                        chains=chains, sweeps=sweeps))
    return out


def flatband_ferro(cells=16, betas=(1.0, 2.0, 4.0, 8.0, 16.0, 32.0), U=2.0, dtau=0.05, chains=128, warm=50,
                   sweeps=200, seed=20260108):
    out = []
    lat = lq.Lattice.flatband(cells)  # t1 = t4 = -0.2, t2 = t3 = 1
    ns = cells // 2                   # half filling of the flat band: N_e = cells
    for beta in betas:
        p = dict(U=U, beta=beta, dtau=dtau, n_up=ns, n_dn=ns, n_stab=8, precision=lq.LQ_FP64, seed=seed)
        recs = _run(lat, p, chains, warm, sweeps)
        row = dict(study="flatband_ferro", cells=cells, N=2 * cells, n_up=ns, n_dn=ns, U=U, beta=beta, chains=chains,
                   sweeps=sweeps)
        for name in ("sign", "szz_00", "szz_11", "szz_01", "s_par", "docc"):
            if name == "sign":
                sgn = np.array([r[:, 0].mean() for r in recs])
                row["sign"], row["sign_err"] = float(sgn.mean()), float(sgn.std(ddof=1) / np.sqrt(len(sgn)))
            else:
                row[name], row[name + "_err"] = _estimate(recs, name)
        allr = np.concatenate(recs)
        k0, k1, k2 = (OBS_NAMES.index(x) for x in ("szz_00", "szz_11", "szz_01"))
        row["sum_rule_max_abs"] = float(np.max(np.abs(allr[:, k0] + allr[:, k1] + 2 * allr[:, k2])))
        out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=128)
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--warm", type=int, default=50)
    ap.add_argument("--study", choices=["sign", "flatband", "both"], default="both")
    a = ap.parse_args()
    lq.load()
    rows = []
    if a.study in ("flatband", "both"):
        rows += flatband_ferro(chains=a.chains, sweeps=a.sweeps, warm=a.warm)
    if a.study in ("sign", "both"):
        rows += sign_vs_size(chains=a.chains, sweeps=a.sweeps, warm=a.warm)
    for r in rows:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
