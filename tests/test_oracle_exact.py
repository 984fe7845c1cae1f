"""Pins of the oracle's exact kinetic mode (CPU only).

In this mode B_l = e^{-dtau K} e^{-dtau V(s_l)} (Eq. 1) with e^{-dtau K}
itself instead of the checkerboard product.  The oracle applies the dense
matrix exponential of K (scipy's expm); every reference here builds
e^{-dtau K} from the eigendecomposition of K instead, so a mistake in the
oracle's use of the exponential (a transposed operand, a missing onsite
term, dtau instead of -dtau) fails them:

* U = 0: the weight of a Fock state is det[P^T e^{-beta K} P] in closed form;
* fixed fields: log|W| against the brute-force determinant of the dense
  product of the slices, and the field and swap ratios against brute-force
  determinant ratios;
* the tracked weight after sweeps against a fresh brute-force weight;
* Monte Carlo against the Trotterized canonical ED with T_K built from the
  same exact exponential;
* the checkerboard's splitting error against the exact mode shrinks with
  dtau at fixed beta (the mode switch changes the propagator, by the
  amount a Trotter splitting should).
"""
import numpy as np
import pytest

import exact
from oracle import OBS_NAMES, OracleSim, lattices
from stats import jackknife_ratio

CASES = [
    (lattices.chain(8), 4.0, 1.0, 0.1, 2, 3, 3),
    (lattices.square(3, 4), -3.0, 0.8, 0.1, 3, 3, 4),
    (lattices.flatband(4), 2.0, 1.0, 0.1, 2, 2, 5),  # onsite terms on the diagonal of K
    (lattices.chain(7, 1.0, False), 0.0, 1.5, 0.1, 2, 1, 5),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_exact_log_weight_matches_brute_force(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=5 + case, kinetic="exact")
    s = o.get_fields()
    up, dn = o.get_fock()
    ref, sg = exact.log_weight(lat, U, dtau, s, up, dn, BK=exact.exact_BK_eigh(lat, dtau))
    lw, so = o.log_weight()
    assert so == sg and abs(lw - ref) < 1e-10 * max(1.0, abs(ref))
    # the checkerboard weight of the same configuration is a different number
    lc, _ = exact.log_weight(lat, U, dtau, s, up, dn)
    if lat["N"] > 2 and U != 0.0:
        assert abs(lc - ref) > 1e-6


def test_exact_free_weight_closed_form():
    """At U = 0 all slices multiply to e^{-beta K}: the weight of eta is
    det[P^T e^{-beta K} P], e^{-beta K} from the spectrum of K."""
    lat = lattices.square(3, 3)
    beta, dtau = 1.2, 0.1
    o = OracleSim(lat, 0.0, beta, dtau, 3, 2, 4, seed=2, kinetic="exact")
    up, dn = o.get_fock()
    E = exact.exact_BK_eigh(lat, beta)
    ref = sum(np.linalg.slogdet(E[np.ix_(occ, occ)])[1] for occ in (up, dn))
    lw, sg = o.log_weight()
    assert sg == 1 and abs(lw - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_exact_ratios_match_brute_force(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=41 + case, kinetic="exact")
    BK = exact.exact_BK_eigh(lat, dtau)
    s = o.get_fields()
    occ = o.get_fock()
    lw0, sg0 = exact.log_weight(lat, U, dtau, s, occ[0], occ[1], BK=BK)
    rng = np.random.default_rng(case)
    for _ in range(4):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        s2 = s.copy()
        s2[l, i] = -s2[l, i]
        lw1, sg1 = exact.log_weight(lat, U, dtau, s2, occ[0], occ[1], BK=BK)
        ref = sg0 * sg1 * np.exp(lw1 - lw0)
        assert abs(o.field_ratio(l, i) - ref) < 1e-10 * max(1.0, abs(ref))
    for spin in (0, 1):
        B = exact.dense_B(lat, U, dtau, s, spin, BK)
        cur = list(occ[spin])
        if not cur or len(cur) == o.N:
            continue
        empty = [x for x in range(o.N) if x not in cur]
        for _ in range(3):
            k = int(rng.integers(len(cur)))
            j = int(empty[rng.integers(len(empty))])
            new = cur[:k] + cur[k + 1:] + [j]
            ref = np.linalg.det(B[np.ix_(new, new)]) / np.linalg.det(B[np.ix_(cur, cur)])
            for side in ("right", "left"):
                r, _ = o.swap_ratio(spin, k, j, side=side)
                assert abs(r - ref) < 1e-10 * max(1.0, abs(ref)), side


@pytest.mark.parametrize("case", range(len(CASES)))
def test_exact_tracked_weight_equals_fresh_after_sweeps(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=61 + case, kinetic="exact", left_swaps=(case % 2 == 1))
    o.sweep(3)
    lt, st = o.tracked()
    up, dn = o.get_fock()
    ref, sg = exact.log_weight(lat, U, dtau, o.get_fields(), up, dn, BK=exact.exact_BK_eigh(lat, dtau))
    assert st == sg and abs(lt - ref) < 1e-10 * max(1.0, abs(ref))


@pytest.mark.parametrize("U,lat,nu,nd", [(4.0, lattices.chain(6), 2, 1), (-4.0, lattices.square(3, 2), 1, 2)])
def test_exact_mc_matches_trotter_ed(U, lat, nu, nd):
    beta, dtau, tw, nsweep = 1.0, 0.1, 5, 20000
    L = int(round(beta / dtau))
    ed = exact.TrotterED(lat, U, dtau, L, nu, nd, BK=exact.exact_BK_eigh(lat, dtau)).observables()
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=7, max_records=nsweep, kinetic="exact")
    o.sweep(nsweep // 10, measure=False)
    o.sweep(nsweep)
    recs = o.records()
    for name in ("docc", "ekin", "szz_00", "s_par"):
        est, err = jackknife_ratio(recs, OBS_NAMES.index(name))
        assert abs(est - ed[name]) < 5 * err + 1e-12, (name, est, err, ed[name])


def test_checkerboard_error_shrinks_with_dtau():
    lat = lattices.square(3, 4)
    beta = 1.0
    rng = np.random.default_rng(3)
    up, dn = np.sort(rng.choice(12, 3, replace=False)), np.sort(rng.choice(12, 2, replace=False))
    diffs = []
    for dtau in (0.1, 0.05, 0.025):
        L = int(round(beta / dtau))
        s = np.ones((L, 12), np.int8)
        w_ex, _ = exact.log_weight(lat, 0.0, dtau, s, up, dn, BK=exact.exact_BK_eigh(lat, dtau))
        o = OracleSim(lat, 0.0, beta, dtau, 3, 2, 5, kinetic="exact")
        o.set_fields(s)
        o.set_fock(up, dn)
        lw, _ = o.log_weight()
        assert abs(lw - w_ex) < 1e-10 * max(1.0, abs(w_ex))
        w_cb, _ = exact.log_weight(lat, 0.0, dtau, s, up, dn)
        diffs.append(abs(w_cb - w_ex))
    assert diffs[0] > 1.5 * diffs[1] > 2.25 * diffs[2] > 0
