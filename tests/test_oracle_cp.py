"""Pins of the oracle's constrained-path inner loop (SM Sec. VI), CPU only.

For a fixed Fock state eta the walk estimates
R(eta) = sum_s 2^{-LN} <eta|U(s)|eta> / <eta|e^{-beta H_0}|eta>, truncating
walkers whose overlap with the trial would change sign.  Where no walker can
be truncated the estimate is unbiased, and R(eta) is known exactly from the
Trotterized ED:
  * U < 0 with the same Fock state for both spins: both spins see the same
    charge-channel fields, so each site ratio is a square times e^{-lambda s};
  * one particle per spin with hoppings of one sign: B_K and the field
    factors are entrywise positive, so every overlap is positive;
  * U = 0: every ratio is exactly 1.
The ED value is itself pinned to the plain sum over all HS fields.
"""
import itertools

import numpy as np
import pytest

import exact
from oracle import OracleSim, lattices


def exact_ratio(lat, U, dtau, L, up, dn):
    """R(eta) from the Trotterized ED.  The HS sum of one site's factors is
    e^{-dtau U n_up n_dn} times e^{dtau U (n_up + n_dn)/2} (U > 0, spin
    channel) or e^{-dtau |U| (n_up + n_dn - 1)/2} (U < 0, charge channel),
    so the field average of U(s) is the ED transfer matrix times a constant
    fixed by N_e and N."""
    N = lat["N"]
    ne = len(up) + len(dn)
    ed = exact.TrotterED(lat, U, dtau, L, len(up), len(dn))
    idx = ed.bu.index(tuple(up)) * len(ed.bd) + ed.bd.index(tuple(dn))
    c = dtau * U * ne / 2.0 if U >= 0 else -dtau * abs(U) * (ne - N) / 2.0
    lw0, s0 = exact.log_weight(lat, 0.0, dtau, np.ones((L, N), np.int8), list(up), list(dn))
    return float(ed.T[idx, idx] * np.exp(c * L - lw0) * s0)


def enumerated_ratio(lat, U, dtau, L, up, dn):
    """The same ratio as the plain average over all 2^{LN} field configurations."""
    N = lat["N"]
    lw0, s0 = exact.log_weight(lat, 0.0, dtau, np.ones((L, N), np.int8), list(up), list(dn))
    acc = 0.0
    for bits in itertools.product((1, -1), repeat=L * N):
        s = np.array(bits, dtype=np.int8).reshape(L, N)
        lw, sg = exact.log_weight(lat, U, dtau, s, list(up), list(dn))
        acc += sg * np.exp(lw - lw0)
    return s0 * acc / 2.0 ** (L * N)


@pytest.mark.parametrize("U", [2.0, -2.0])
def test_exact_ratio_equals_field_enumeration(U):
    lat = lattices.chain(4)
    for up, dn in (((0,), (2,)), ((0, 1), (1, 3))):
        ref = enumerated_ratio(lat, U, 0.1, 3, up, dn)
        assert abs(exact_ratio(lat, U, 0.1, 3, up, dn) - ref) < 1e-11 * max(1.0, abs(ref))


def _walk(lat, U, beta, dtau, up, dn, n_walkers, seed=5):
    o = OracleSim(lat, U, beta, dtau, len(up), len(dn), 4, seed=seed)
    o.set_fock(np.array(up), np.array(dn))
    return o.cp_walk(n_walkers)


def _assert_unbiased(w, ref, nsig=5.0):
    err = w.std(ddof=1) / np.sqrt(len(w))
    assert abs(w.mean() - ref) < nsig * err, (w.mean(), err, ref)


def test_cp_walk_attractive_same_fock_state_is_exact():
    lat, U, beta, dtau = lattices.chain(6), -3.0, 0.6, 0.1
    up = dn = (0, 3)
    w, dropped = _walk(lat, U, beta, dtau, up, dn, 20000)
    assert dropped == 0 and np.all(w > 0)
    _assert_unbiased(w, exact_ratio(lat, U, dtau, 6, up, dn))


def test_cp_walk_one_particle_per_spin_is_exact():
    lat, U, beta, dtau = lattices.chain(6), 4.0, 0.8, 0.1
    up, dn = (1,), (4,)
    w, dropped = _walk(lat, U, beta, dtau, up, dn, 20000)
    assert dropped == 0 and np.all(w > 0)
    _assert_unbiased(w, exact_ratio(lat, U, dtau, 8, up, dn))


def test_cp_walk_flatband_attractive_is_exact():
    lat, U, beta, dtau = lattices.flatband(3), -2.0, 0.5, 0.1
    up = dn = (0, 5)
    w, dropped = _walk(lat, U, beta, dtau, up, dn, 20000)
    assert dropped == 0
    _assert_unbiased(w, exact_ratio(lat, U, dtau, 5, up, dn))


def test_cp_walk_free_fermions_weight_one():
    w, dropped = _walk(lattices.square(3, 2), 0.0, 0.5, 0.1, (0, 4), (1,), 50)
    assert dropped == 0 and np.max(np.abs(w - 1.0)) < 1e-12


def test_cp_walk_weights_nonnegative_with_constraint():
    """Repulsive, two particles per spin in different states: the constraint
    may act (no exact value then); weights stay finite and non-negative."""
    w, dropped = _walk(lattices.chain(6), 4.0, 1.0, 0.1, (0, 1), (2, 4), 2000)
    assert np.all(np.isfinite(w)) and np.all(w >= 0.0)
    assert dropped == int(np.sum(w == 0.0))


def _population(lat, U, beta, dtau, up, dn, n_walkers, comb_every, runs, seed=5):
    o = OracleSim(lat, U, beta, dtau, len(up), len(dn), 4, seed=seed)
    o.set_fock(np.array(up), np.array(dn))
    return np.exp([o.cp_population(n_walkers, comb_every, run=r) for r in runs])


@pytest.mark.parametrize("comb_every", [1, 3])
def test_cp_population_with_comb_is_unbiased(comb_every):
    """Branching populations (systematic resampling every comb_every slices):
    the product of the population's mean weights averages to the exact R(eta)
    where nothing is truncated."""
    lat, U, beta, dtau = lattices.chain(6), -3.0, 0.6, 0.1
    up = dn = (0, 3)
    est = _population(lat, U, beta, dtau, up, dn, 8, comb_every, range(3000))
    assert np.all(est > 0)
    _assert_unbiased(est, exact_ratio(lat, U, dtau, 6, up, dn))


def test_cp_population_one_particle_per_spin():
    lat, U, beta, dtau = lattices.chain(6), 4.0, 0.8, 0.1
    up, dn = (1,), (4,)
    est = _population(lat, U, beta, dtau, up, dn, 8, 2, range(2000))
    _assert_unbiased(est, exact_ratio(lat, U, dtau, 8, up, dn))


def test_comb_resampling_law():
    """Systematic resampling: n new walkers, old walker j copied floor or ceil
    of n w_j / W times (never when w_j = 0), and n w_j / W times on average
    over the uniform (checked exactly on a fine grid of u)."""
    from oracle import comb

    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 16):
        w = rng.exponential(size=n)
        if n > 2:
            w[[1, n - 1]] = 0.0
        expect = n * w / w.sum()
        grid = (np.arange(4096) + 0.5) / 4096
        mean = np.zeros(n)
        for u in grid:
            src = comb(w, u)
            assert len(src) == n and np.all(np.diff(src) >= 0)
            cnt = np.bincount(src, minlength=n)
            assert np.all((cnt == np.floor(expect)) | (cnt == np.ceil(expect)))
            assert np.all(cnt[w == 0] == 0)
            mean += cnt / len(grid)
        assert np.max(np.abs(mean - expect)) < 2.0 / 4096
