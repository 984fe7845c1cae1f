"""The constrained-path inner loop (SM Sec. VI) on the GPU: lq_cp_walk and
lq_cp_population against the oracle's orc_cp_walk and orc_cp_population on
the same seeds and Fock states.

Both draw the same Philox numbers, so each walker takes the same field values
at every site: the dropped walkers must be the same, each surviving walker's
log-weight within 1e-10, and a population's log-estimate within 1e-10
(FP64).  The GPU's overlap ratios come from the matrix-determinant lemma with
a Sherman-Morrison inverse, the oracle's from full determinants, so the
comparison also checks that algebra.  Cases: no truncation possible (the
attractive model with the same Fock state for both spins, one particle per
spin), free fermions (every weight 1), a repulsive case with two particles
per spin in different states, the flat band, the exact kinetic propagator,
and more than 32 particles per spin.  A Monte Carlo check ties the GPU population to the
exact R(eta) of the Trotterized ED where nothing is truncated.
"""
import numpy as np
import pytest

from oracle import OracleSim, lattices

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    "attractive_same_fock": (("chain", 6), -3.0, 0.6, 0.1, (0, 3), (0, 3), "checkerboard"),
    "one_particle_per_spin": (("chain", 6), 4.0, 0.8, 0.1, (1,), (4,), "checkerboard"),
    "free_fermions": (("square", 3, 2), 0.0, 0.5, 0.1, (0, 4), (1,), "checkerboard"),
    "repulsive_two_per_spin": (("chain", 6), 4.0, 1.0, 0.1, (0, 1), (2, 4), "checkerboard"),
    "flatband_attractive": (("flatband", 3), -2.0, 0.5, 0.1, (0, 5), (0, 5), "checkerboard"),
    "square4x4_exact_kinetic": (("square", 4, 4), 3.0, 0.6, 0.1, (0, 5, 10), (3, 6), "exact"),
    "chain80_m36": (("chain", 80), 2.0, 0.2, 0.1, tuple(range(0, 72, 2)), tuple(range(1, 70, 2)), "checkerboard"),
}


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def setup(lq, name, seed=5):
    spec, U, beta, dtau, up, dn, kin = CASES[name]
    lat = getattr(lattices, spec[0])(*spec[1:])
    o = OracleSim(lat, U, beta, dtau, len(up), len(dn), 4, seed=seed, kinetic=kin)
    o.set_fock(np.array(up), np.array(dn))
    L = getattr(lq.Lattice, spec[0])(*spec[1:])
    params = dict(U=U, beta=beta, dtau=dtau, n_up=len(up), n_dn=len(dn), n_stab=4, seed=seed,
                  kinetic=lq.LQ_EXACT if kin == "exact" else lq.LQ_CHECKERBOARD)
    return o, L, params, up, dn


@pytest.mark.parametrize("name", sorted(CASES))
def test_cp_walk_matches_oracle(lq, name):
    from paper_2601_08552_gb300.lecqmc import cp_walk

    o, L, params, up, dn = setup(lq, name)
    n = 64 if not name.startswith("chain80") else 8
    wo, do = o.cp_walk(n)
    lg, dg = cp_walk(L, params, up, dn, n)
    assert dg == do
    alive = wo > 0
    assert np.array_equal(np.isfinite(lg), alive)
    lo = np.log(wo[alive])
    assert np.max(np.abs(lg[alive] - lo) / np.maximum(1.0, np.abs(lo)), initial=0.0) < TOL
    if name == "free_fermions":
        assert np.max(np.abs(lg)) < 1e-12


@pytest.mark.parametrize("comb_every", [0, 1, 3])
@pytest.mark.parametrize("name", ["attractive_same_fock", "repulsive_two_per_spin", "square4x4_exact_kinetic"])
def test_cp_population_matches_oracle(lq, name, comb_every):
    from paper_2601_08552_gb300.lecqmc import cp_population

    o, L, params, up, dn = setup(lq, name)
    for run in range(3):
        eo = o.cp_population(16, comb_every, run=run)
        eg = cp_population(L, params, up, dn, 16, comb_every, run=run)
        if np.isfinite(eo):
            assert abs(eg - eo) < TOL * max(1.0, abs(eo)), (run, eg, eo)
        else:
            assert not np.isfinite(eg)


def test_cp_population_mean_is_exact_ratio(lq):
    """Where nothing is truncated the population's estimate averages to the
    exact R(eta) of the Trotterized ED (an independent pin of the GPU path)."""
    import exact
    from paper_2601_08552_gb300.lecqmc import cp_population

    spec, U, beta, dtau, up, dn, _ = CASES["attractive_same_fock"]
    lat = lattices.chain(6)
    Lq = lq.Lattice.chain(6)
    Lsl = int(round(beta / dtau))
    N, ne = lat["N"], len(up) + len(dn)
    ed = exact.TrotterED(lat, U, dtau, Lsl, len(up), len(dn))
    idx = ed.bu.index(tuple(up)) * len(ed.bd) + ed.bd.index(tuple(dn))
    c = -dtau * abs(U) * (ne - N) / 2.0
    lw0, s0 = exact.log_weight(lat, 0.0, dtau, np.ones((Lsl, N), np.int8), list(up), list(dn))
    ref = float(ed.T[idx, idx] * np.exp(c * Lsl - lw0) * s0)
    params = dict(U=U, beta=beta, dtau=dtau, n_up=2, n_dn=2, n_stab=4, seed=9)
    est = np.exp([cp_population(Lq, params, up, dn, 8, 2, run=r) for r in range(400)])
    err = est.std(ddof=1) / np.sqrt(len(est))
    assert abs(est.mean() - ref) < 5 * err, (est.mean(), err, ref)


def test_cp_rejects_reduced_precision_and_bad_occupations(lq):
    from paper_2601_08552_gb300.lecqmc import LqError

    L = lq.Lattice.chain(6)
    p = dict(U=2.0, beta=0.5, dtau=0.1, n_up=2, n_dn=1, n_stab=4, seed=1)
    lib = lq.load()
    import ctypes as C

    from paper_2601_08552_gb300.lecqmc import _params_struct

    ps = _params_struct(dict(p, precision=1))
    u = (C.c_int32 * 2)(0, 1)
    d = (C.c_int32 * 1)(2)
    out = (C.c_double * 4)()
    assert lib.lq_cp_walk(L.h, C.byref(ps), u, d, 4, 0, out, None) == 8
    from paper_2601_08552_gb300.lecqmc import cp_walk

    with pytest.raises(LqError):
        cp_walk(L, p, [0, 0], [2], 4)


@pytest.mark.parametrize("U,up_dn", [(4.0, (1, 1)), (-3.0, (1, 1))])
def test_two_stage_partition_ratio_is_exact(lq, U, up_dn):
    """The outer stage (Fock states from the U = 0 chain, which samples the
    free weight W_T) and the inner populations together estimate
    e^{cL} Z_U / Z_0 of the Trotterized ED."""
    import exact
    from paper_2601_08552_gb300.constrained import partition_ratio

    lat = lattices.chain(6)
    beta, dtau = 0.8, 0.1
    Lsl = int(round(beta / dtau))
    nu, nd = up_dn
    ne, N = nu + nd, lat["N"]
    c = dtau * U * ne / 2.0 if U >= 0 else dtau * abs(U) * (N - ne) / 2.0
    ref = np.exp(c * Lsl) * exact.TrotterED(lat, U, dtau, Lsl, nu, nd).Z / exact.TrotterED(lat, 0.0, dtau, Lsl, nu,
                                                                                         nd).Z
    params = dict(U=U, beta=beta, dtau=dtau, n_up=nu, n_dn=nd, n_stab=4, seed=17)
    est = partition_ratio(lq.Lattice.chain(6), params, 400, n_walkers=8, comb_every=2, thin=2)
    print(est["mean"], est["err"], ref)
    assert abs(est["mean"] - ref) < 5 * est["err"] + 1e-12
