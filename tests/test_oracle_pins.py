"""Pins of the CPU oracle against things other than itself (CPU only).

Each check compares the oracle's stabilized-QR algorithm with an independent
reference: published Philox test vectors, closed-form lattice spectra,
scipy's matrix exponential, brute-force determinants (numpy, mpmath),
exhaustive enumeration of Eq. (1), the Trotterized canonical ED and the
canonical free-fermion trace.
"""
import os

import numpy as np
import pytest

import exact
from oracle import OBS_NAMES, OracleSim, lattices, philox4x32_10
from stats import jackknife_ratio

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------- lattices

def test_chain_and_square_spectra():
    for N in (8, 10):
        ev = np.sort(np.linalg.eigvalsh(lattices.dense_K(lattices.chain(N, t=1.3))))
        ref = np.sort(-2 * 1.3 * np.cos(2 * np.pi * np.arange(N) / N))
        assert np.allclose(ev, ref, atol=1e-12)
    Lx, Ly = 4, 6
    ev = np.sort(np.linalg.eigvalsh(lattices.dense_K(lattices.square(Lx, Ly))))
    kx, ky = np.meshgrid(2 * np.pi * np.arange(Lx) / Lx, 2 * np.pi * np.arange(Ly) / Ly)
    assert np.allclose(ev, np.sort((-2 * (np.cos(kx) + np.cos(ky))).ravel()), atol=1e-12)


@pytest.mark.parametrize("t", [(-0.2, 1.0, 1.0, -0.2), (1.0, 1.0, 1.0, 1.0), (0.3, -0.7, 1.1, 0.4)])
def test_flatband_exactly_flat_lowest_band(t):
    n = 12
    ev = np.sort(np.linalg.eigvalsh(lattices.dense_K(lattices.flatband(n, *t))))
    assert np.allclose(ev[:n], 0.0, atol=1e-12)          # H_eff = S S^dag has a zero mode per k
    ks = 2 * np.pi * np.arange(n) / n
    upper = np.sort(np.abs(t[0] + t[1] * np.exp(-1j * ks)) ** 2 + np.abs(t[2] + t[3] * np.exp(-1j * ks)) ** 2)
    assert np.allclose(ev[n:], upper, atol=1e-12)        # |S1|^2 + |S2|^2


def test_cross_stitch_flat_band_inside():
    ev = np.linalg.eigvalsh(lattices.dense_K(lattices.cross_stitch(16)))
    assert np.sum(np.abs(ev - 1.0) < 1e-12) == 16        # flat band at +t_intra
    assert ev.min() < -4.9 and ev.max() > 2.9


@pytest.mark.parametrize("lat", [lattices.square(4, 4), lattices.flatband(5), lattices.chain(9, periodic=False),
                                 lattices.chain(7), lattices.cross_stitch(4)])
def test_checkerboard_BK_matches_expm(lat):
    o = OracleSim(lat, 4.0, 1.0, 0.1, 1, 1, 5)
    assert np.abs(o.BK() - exact.dense_BK(lat, 0.1)).max() < 1e-14
    fam = o.families()
    for g in range(o.G):
        sites = np.concatenate([lat["bi"][fam == g], lat["bj"][fam == g]])
        assert len(sites) == len(set(sites.tolist()))
    # first-order check against the exact exponential of K
    import scipy.linalg as sla
    d = 1e-3
    o2 = OracleSim(lat, 0.0, d, d, 1, 1, 1)
    K = lattices.dense_K(lat)
    assert np.abs(o2.BK() - sla.expm(-d * K)).max() < 10 * d * d * np.abs(K).max() ** 2 * o.G


# ---------------------------------------------------------------- weights

CASES = [
    (lattices.chain(8), 4.0, 1.0, 0.1, 2, 3, 3),
    (lattices.chain(8), -4.0, 1.0, 0.1, 2, 3, 4),
    (lattices.square(3, 4), 2.0, 0.8, 0.1, 3, 2, 8),
    (lattices.flatband(4), 2.0, 1.0, 0.05, 2, 2, 6),
    (lattices.chain(6, periodic=False), 3.0, 0.7, 0.1, 1, 1, 3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_log_weight_matches_brute_force(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=11 + case, chain=case)
    s = o.get_fields()
    up, dn = o.get_fock()
    ref = exact.log_weight(lat, U, dtau, s, up, dn)
    for side in ("right", "left"):
        lw, sg = o.log_weight(side)
        assert sg == ref[1]
        assert abs(lw - ref[0]) < 1e-10 * max(1.0, abs(ref[0]))


def test_log_weight_low_temperature_mpmath():
    lat = lattices.chain(8)
    o = OracleSim(lat, 4.0, 6.0, 0.1, 2, 2, 10, seed=5)
    s = o.get_fields()
    up, dn = o.get_fock()
    ref = exact.log_weight_mp(lat, 4.0, 0.1, s, up, dn)
    lw, sg = o.log_weight()
    assert sg == ref[1] and abs(lw - ref[0]) < 1e-9 * abs(ref[0])


@pytest.mark.parametrize("case", range(len(CASES)))
def test_field_ratio_matches_brute_force(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=21 + case)
    s = o.get_fields()
    up, dn = o.get_fock()
    lw0, sg0 = exact.log_weight(lat, U, dtau, s, up, dn)
    rng = np.random.default_rng(case)
    for _ in range(6):
        l, i = int(rng.integers(o.L)), int(rng.integers(o.N))
        s2 = s.copy()
        s2[l, i] = -s2[l, i]
        lw1, sg1 = exact.log_weight(lat, U, dtau, s2, up, dn)
        ref = sg0 * sg1 * np.exp(lw1 - lw0)
        assert abs(o.field_ratio(l, i) - ref) < 1e-10 * max(1.0, abs(ref))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_swap_ratio_matches_brute_force(case):
    lat, U, beta, dtau, nu, nd, tw = CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=31 + case)
    s = o.get_fields()
    occ = o.get_fock()
    rng = np.random.default_rng(100 + case)
    for spin in (0, 1):
        B = exact.dense_B(lat, U, dtau, s, spin)
        cur = list(occ[spin])
        A = B[np.ix_(cur, cur)]
        empty = [x for x in range(o.N) if x not in cur]
        for _ in range(4):
            k = int(rng.integers(len(cur)))
            j = int(empty[rng.integers(len(empty))])
            new = cur[:k] + cur[k + 1:] + [j]
            ref = np.linalg.det(B[np.ix_(new, new)]) / np.linalg.det(A)
            # the same ratio walked along the right chain (tau = beta) and along
            # the left chain (tau = 0, the transposed propagator)
            for side in ("right", "left"):
                r, parts = o.swap_ratio(spin, k, j, side=side)
                assert abs(r - ref) < 1e-10 * max(1.0, abs(ref)), side
                # removal factor = [(P^T B P)^{-1}]_kk (cofactor identity)
                rem = parts[3] * np.exp(parts[2])
                assert abs(rem - np.linalg.inv(A)[k, k]) < 1e-10 * max(1.0, abs(rem)), side


def test_chain_invariants():
    lat, U, beta, dtau = lattices.square(4, 4), 4.0, 2.0, 0.1
    o = OracleSim(lat, U, beta, dtau, 3, 2, 4, seed=9)
    o.sweep(2)
    o.build_chains()
    s = o.get_fields()
    BK = exact.dense_BK(lat, dtau)
    lam = exact.hs_lambda(U, dtau)
    bnd = [min(j * o.tw, o.L) for j in range(o.n + 1)]
    for spin in (0, 1):
        sp = 1.0 if spin == 0 else -1.0
        for j in range(1, o.n + 1):
            Qp, _ = o.chain_panel(0, spin, j - 1)
            Q, V = o.chain_panel(0, spin, j)
            assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-13
            assert np.allclose(np.tril(V, -1), 0) and np.all(np.diag(V) >= 0)
            Bi = np.eye(o.N)
            for l in range(bnd[j - 1], bnd[j]):
                Bi = BK @ (np.exp(sp * lam * s[l])[:, None] * Bi)
            assert np.abs(Bi @ Qp - Q @ V).max() < 1e-12 * np.abs(V).max()


# ---------------------------------------------------------------- sweeps

SWEEP_CASES = [
    (lattices.chain(8), 4.0, 1.0, 0.1, 2, 3, 3),       # tau_w does not divide L
    (lattices.chain(8), -4.0, 1.0, 0.1, 2, 2, 5),      # charge channel
    (lattices.chain(6), 0.0, 1.0, 0.1, 2, 1, 5),       # U = 0
    (lattices.square(3, 3), 3.0, 1.0, 0.1, 1, 1, 5),   # one particle per spin
    (lattices.chain(5), 4.0, 0.5, 0.1, 2, 0, 2),       # empty spin sector
    (lattices.chain(4), 4.0, 0.5, 0.1, 4, 1, 2),       # full spin sector (no swaps)
    (lattices.flatband(4), 2.0, 2.0, 0.1, 2, 2, 8),
]


@pytest.mark.parametrize("case", range(len(SWEEP_CASES)))
def test_tracked_weight_equals_fresh_after_sweeps(case):
    lat, U, beta, dtau, nu, nd, tw = SWEEP_CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=41 + case)
    o.sweep(4)
    lt, st = o.tracked()
    s = o.get_fields()
    up, dn = o.get_fock()
    ref = exact.log_weight(lat, U, dtau, s, up, dn)
    assert st == ref[1]
    assert abs(lt - ref[0]) < 1e-9 * max(1.0, abs(ref[0]))
    st_ = o.stats()
    assert st_[0] == 4 * 2 * o.L * o.N
    assert st_[2] == 4 * sum(m for m in (nu, nd) if 0 < m < o.N)


@pytest.mark.parametrize("case", range(len(SWEEP_CASES)))
def test_tracked_weight_equals_fresh_with_left_swaps(case):
    """A second swap phase at tau = 0 on the left chain after the down pass:
    the tracked weight still equals the dense determinant, both chains agree,
    and each sweep makes twice the swap attempts."""
    lat, U, beta, dtau, nu, nd, tw = SWEEP_CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=41 + case, left_swaps=True)
    o.sweep(4)
    lt, st = o.tracked()
    s = o.get_fields()
    up, dn = o.get_fock()
    ref = exact.log_weight(lat, U, dtau, s, up, dn)
    assert st == ref[1]
    assert abs(lt - ref[0]) < 1e-9 * max(1.0, abs(ref[0]))
    # the left chain the left swaps edited in place, against the dense weight
    lw, sg = o.log_weight("left")
    assert sg == ref[1] and abs(lw - ref[0]) < 1e-9 * max(1.0, abs(ref[0]))
    st_ = o.stats()
    assert st_[2] == 8 * sum(m for m in (nu, nd) if 0 < m < o.N)


WICK_CASES = [
    (lattices.chain(6), 4.0, 1.0, 0.1, 2, 1, 3),
    (lattices.square(3, 2), -4.0, 0.8, 0.1, 2, 2, 3),     # charge channel
    (lattices.flatband(3), 2.0, 1.0, 0.1, 2, 2, 4),       # two sublattices
]


@pytest.mark.parametrize("case", range(len(WICK_CASES)))
def test_measure_matches_dense_wick(case):
    lat, U, beta, dtau, nu, nd, tw = WICK_CASES[case]
    o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=3 + case)
    s = o.get_fields()
    up, dn = o.get_fock()
    for jb in range(o.n + 1):
        obs, nn, ss = o.measure_at(jb, corr=True)
        w = exact.wick_observables(lat, U, dtau, s, list(up), list(dn), boundary_slice=min(jb * o.tw, o.L))
        assert obs[0] == w["sign"]
        for k, name in enumerate(OBS_NAMES[1:], start=1):
            assert abs(obs[k] / obs[0] - w[name]) < 1e-12
        assert np.abs(nn / obs[0] - w["nn"]).max() < 1e-12
        assert np.abs(ss / obs[0] - w["ss"]).max() < 1e-12


def test_enumeration_equals_trotter_ed():
    lat, U, dtau, L = lattices.chain(4), 4.0, 0.25, 2
    names = OBS_NAMES[1:]
    ex = exact.enumerate_exact(lat, U, dtau, L, 1, 1, names)
    ed = exact.TrotterED(lat, U, dtau, L, 1, 1).observables()
    for k in names:
        assert abs(ex[k] - ed[k]) < 1e-12


def test_enumeration_equals_trotter_ed_attractive():
    lat, U, dtau, L = lattices.chain(4, periodic=False), -3.0, 0.25, 2
    names = ["docc", "ekin", "szz_00", "s_par"]
    ex = exact.enumerate_exact(lat, U, dtau, L, 1, 1, names)
    ed = exact.TrotterED(lat, U, dtau, L, 1, 1).observables()
    for k in names:
        assert abs(ex[k] - ed[k]) < 1e-12


def test_ed_canonical_free_trace():
    lat, dtau, L = lattices.chain(7), 0.1, 12
    ed = exact.TrotterED(lat, 0.0, dtau, L, 3, 2)
    A = np.linalg.matrix_power(exact.dense_BK(lat, dtau), L)
    Z = exact.canonical_free_Z(A, 3) * exact.canonical_free_Z(A, 2)
    assert abs(ed.Z - Z) < 1e-10 * abs(Z)


def _mc_records(lat, U, beta, dtau, nu, nd, tw, nsweep, seed, chains=1, swap_mode=0, left_swaps=False):
    recs = []
    for c in range(chains):
        o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=seed, chain=c, max_records=nsweep, swap_mode=swap_mode,
                      left_swaps=left_swaps)
        o.sweep(nsweep // 10, measure=False)
        o.sweep(nsweep)
        recs.append(o.records())
    return np.concatenate(recs)


def _mc_vs_ed(lat, U, beta, dtau, nu, nd, tw, nsweep, names, seed, nsig=5.0, chains=1, swap_mode=0,
              left_swaps=False):
    L = int(round(beta / dtau))
    ed = exact.TrotterED(lat, U, dtau, L, nu, nd).observables()
    recs = []
    for c in range(chains):
        o = OracleSim(lat, U, beta, dtau, nu, nd, tw, seed=seed, chain=c, max_records=nsweep, swap_mode=swap_mode,
                      left_swaps=left_swaps)
        o.sweep(nsweep // 10, measure=False)
        o.sweep(nsweep)
        recs.append(o.records())
    recs = np.concatenate(recs)
    for name in names:
        col = OBS_NAMES.index(name)
        est, err = jackknife_ratio(recs, col)
        assert abs(est - ed[name]) < nsig * err + 1e-12, (name, est, err, ed[name])


def test_mc_matches_trotter_ed_repulsive():
    _mc_vs_ed(lattices.chain(6), 4.0, 1.0, 0.1, 2, 1, 5, 20000, ["docc", "ekin", "szz_00", "szz_01", "s_par"], seed=1)


def test_mc_matches_trotter_ed_attractive():
    _mc_vs_ed(lattices.square(3, 2), -4.0, 1.0, 0.1, 1, 2, 5, 20000, ["docc", "ekin", "szz_00", "s_par"], seed=2)


def test_mc_matches_trotter_ed_free_fermions():
    # at U = 0 the fields are inert and only the Fock-state swaps sample
    _mc_vs_ed(lattices.chain(7), 0.0, 2.0, 0.1, 2, 2, 5, 20000, ["ekin", "szz_00", "s_par"], seed=3)


def test_mc_matches_trotter_ed_flatband():
    _mc_vs_ed(lattices.flatband(3), 2.0, 2.0, 0.1, 2, 1, 5, 10000, ["docc", "ekin", "szz_00", "szz_11"], seed=4)


# Nearest-neighbour Fock-swap proposals (target uniform among the empty
# neighbours of the removed particle's site, Metropolis-Hastings factor
# |E(i)| / |E'(j)|).  Open chains make the neighbour counts uneven (the end
# sites have one neighbour), so a wrong factor biases the density profile and
# with it the kinetic energy.
def test_mc_matches_trotter_ed_nearest_neighbour_swaps_free():
    _mc_vs_ed(lattices.chain(7, 1.0, False), 0.0, 2.0, 0.1, 2, 2, 5, 20000, ["ekin", "szz_00", "s_par"], seed=3,
              swap_mode=1)


def test_mc_matches_trotter_ed_nearest_neighbour_swaps_repulsive():
    _mc_vs_ed(lattices.chain(6, 1.0, False), 4.0, 1.0, 0.1, 2, 1, 5, 20000, ["docc", "ekin", "szz_00", "s_par"],
              seed=1, swap_mode=1)


# Left-chain swaps at tau = 0 (a second set of attempts per sweep): the chain
# samples the same weight, so the same exact values hold.
def test_mc_matches_trotter_ed_left_swaps_free():
    _mc_vs_ed(lattices.chain(7), 0.0, 2.0, 0.1, 2, 2, 5, 20000, ["ekin", "szz_00", "s_par"], seed=3, left_swaps=True)


def test_mc_matches_trotter_ed_left_swaps_repulsive():
    _mc_vs_ed(lattices.chain(6), 4.0, 1.0, 0.1, 2, 1, 5, 20000, ["docc", "ekin", "szz_00", "szz_01", "s_par"], seed=1,
              left_swaps=True)


def test_mc_matches_trotter_ed_left_swaps_nearest_neighbour():
    _mc_vs_ed(lattices.chain(6, 1.0, False), 4.0, 1.0, 0.1, 2, 1, 5, 20000, ["docc", "ekin", "szz_00", "s_par"],
              seed=1, swap_mode=1, left_swaps=True)


def test_missing_hastings_factor_is_detected():
    """Planted mistake: the same proposal without the Hastings factor (oracle
    mode 2) must miss the exact kinetic energy by many standard errors."""
    lat = lattices.chain(7, 1.0, False)
    ed = exact.TrotterED(lat, 0.0, 0.1, 20, 2, 2).observables()
    recs = _mc_records(lat, 0.0, 2.0, 0.1, 2, 2, 5, 20000, seed=3, swap_mode=2)
    est, err = jackknife_ratio(recs, OBS_NAMES.index("ekin"))
    assert abs(est - ed["ekin"]) > 10.0 * err
