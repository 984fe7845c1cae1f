"""Independent exact references used to pin the oracle (no oracle code here).

* ``dense_B``: B_sigma(beta,0) = prod_l B_K D_l as dense matrices, with B_K
  built from scipy's expm of each checkerboard family (Eq. 1).
* ``TrotterED``: the canonical-ensemble Trotterized transfer matrix on the
  fixed (N_up, N_dn) sector.  One slice is T_K T_U with T_K the
  N_sigma-th compound matrices of B_K (the many-body action of a one-body
  propagator on Slater determinants) and T_U = exp(-dtau U sum n_up n_dn).
  Summing the discrete HS fields of each slice reproduces T_U up to
  constants in the canonical ensemble, so Monte Carlo averages of the
  Trotterized weight equal Tr[O T^L] / Tr[T^L] exactly.
* ``enumerate_exact``: brute-force sum over all (eta, s) of
  det[P^T B P] * O(eta, s) on tiny systems (Eq. 1), with the Wick estimators
  evaluated from dense Green's functions.
"""
import itertools

import numpy as np
import scipy.linalg as sla


def families(lat):
    """Greedy checkerboard families in bond order (lowest family with both sites free)."""
    used = []
    fam = []
    for i, j in zip(lat["bi"], lat["bj"]):
        g = 0
        while True:
            if g == len(used):
                used.append(set())
            if i not in used[g] and j not in used[g]:
                break
            g += 1
        used[g].update((int(i), int(j)))
        fam.append(g)
    return np.array(fam, dtype=np.int32), len(used)


def dense_BK(lat, dtau):
    """B_K = E_{G-1} ... E_0 C_eps with E_g = expm(-dtau K_g), computed with scipy."""
    N = lat["N"]
    fam, G = families(lat)
    B = np.diag(np.exp(-dtau * np.asarray(lat["eps"], dtype=float)))
    for g in range(G):
        Kg = np.zeros((N, N))
        for b in np.where(fam == g)[0]:
            i, j, k = lat["bi"][b], lat["bj"][b], lat["kb"][b]
            Kg[i, j] += k
            Kg[j, i] += k
        B = sla.expm(-dtau * Kg) @ B
    return B


def exact_BK_eigh(lat, dtau):
    """e^{-dtau K} from the eigendecomposition of the dense K (V diag(e^{-dtau
    k}) V^T): independent of the Pade approximant behind scipy's expm."""
    from oracle.lattices import dense_K

    k, V = np.linalg.eigh(dense_K(lat))
    return (V * np.exp(-dtau * k)) @ V.T


def hs_lambda(U, dtau):
    return float(np.arccosh(np.exp(dtau * abs(U) / 2.0)))


def dense_B(lat, U, dtau, s, spin, BK=None):
    """B_sigma(beta, 0) = B_{L-1} ... B_0 with B_l = B_K diag(e^{sigma' lambda s_l})."""
    if BK is None:
        BK = dense_BK(lat, dtau)
    lam = hs_lambda(U, dtau)
    sp = 1.0 if (U < 0 or spin == 0) else -1.0
    B = np.eye(lat["N"])
    for l in range(s.shape[0]):
        B = BK @ (np.exp(sp * lam * s[l])[:, None] * B)
    return B


def log_weight(lat, U, dtau, s, occ_up, occ_dn, BK=None):
    """log|W| and sign of W = prod_sigma det[P^T B_sigma P] (times e^{-lambda sum s} for U < 0);
    BK: the kinetic propagator (default: the checkerboard product)."""
    if BK is None:
        BK = dense_BK(lat, dtau)
    lw, sg = 0.0, 1.0
    for spin, occ in ((0, occ_up), (1, occ_dn)):
        B = dense_B(lat, U, dtau, s, spin, BK)
        if len(occ):
            sgn, la = np.linalg.slogdet(B[np.ix_(occ, occ)])
            lw += la
            sg *= sgn
    if U < 0:
        lw += -hs_lambda(U, dtau) * float(np.sum(s))
    return lw, int(sg)


def log_weight_mp(lat, U, dtau, s, occ_up, occ_dn, dps=60):
    """The same weight in mpmath arithmetic (for low temperatures)."""
    import mpmath as mp

    mp.mp.dps = dps
    N = lat["N"]
    fam, G = families(lat)
    lam = mp.acosh(mp.e ** (mp.mpf(dtau) * abs(U) / 2))
    Es = []
    for g in range(G):
        E = mp.eye(N)
        for b in np.where(fam == g)[0]:
            i, j, k = int(lat["bi"][b]), int(lat["bj"][b]), mp.mpf(float(lat["kb"][b]))
            c, sh = mp.cosh(mp.mpf(dtau) * k), -mp.sinh(mp.mpf(dtau) * k)
            E[i, i] = c
            E[j, j] = c
            E[i, j] = sh
            E[j, i] = sh
        Es.append(E)
    Ceps = mp.diag([mp.e ** (-mp.mpf(dtau) * mp.mpf(float(e))) for e in lat["eps"]])
    BK = Ceps
    for E in Es:
        BK = E * BK
    lw = mp.mpf(0)
    sg = 1
    for spin, occ in ((0, occ_up), (1, occ_dn)):
        sp = 1 if (U < 0 or spin == 0) else -1
        B = mp.eye(N)
        for l in range(s.shape[0]):
            D = mp.diag([mp.e ** (sp * lam * int(x)) for x in s[l]])
            B = BK * (D * B)
        if len(occ):
            M = mp.matrix([[B[int(a), int(b)] for b in occ] for a in occ])
            d = mp.det(M)
            lw += mp.log(abs(d))
            sg *= 1 if d > 0 else -1
    if U < 0:
        lw += -lam * int(np.sum(s))
    return float(lw), sg


# --------------------------------------------------------------------------
# canonical many-body basis and operators
# --------------------------------------------------------------------------

def basis(N, k):
    return [tuple(c) for c in itertools.combinations(range(N), k)]


def compound(B, states):
    """k-th compound matrix of B on the given k-subsets: det B[S, S']."""
    n = len(states)
    C = np.empty((n, n))
    if n and len(states[0]) == 0:
        return np.ones((1, 1))
    for a, Sa in enumerate(states):
        rows = B[list(Sa), :]
        for b, Sb in enumerate(states):
            C[a, b] = np.linalg.det(rows[:, list(Sb)])
    return C


def hop(states, N, i, j):
    """Matrix of c_i^dag c_j on ascending-ordered k-particle states."""
    idx = {S: a for a, S in enumerate(states)}
    n = len(states)
    M = np.zeros((n, n))
    for b, S in enumerate(states):
        if j not in S:
            continue
        sign = (-1) ** S.index(j)
        rest = [x for x in S if x != j]
        if i in rest:
            continue
        new = sorted(rest + [i])
        sign *= (-1) ** new.index(i)
        M[idx[tuple(new)], b] += sign
    return M


class TrotterED:
    """Trotterized canonical ensemble on the (N_up, N_dn) sector."""

    def __init__(self, lat, U, dtau, L, n_up, n_dn, BK=None):
        self.lat = lat
        N = lat["N"]
        self.N = N
        self.bu = basis(N, n_up)
        self.bd = basis(N, n_dn)
        if BK is None:
            BK = dense_BK(lat, dtau)
        Cu = compound(BK, self.bu)
        Cd = compound(BK, self.bd)
        self.nu = np.array([[1.0 if i in S else 0.0 for i in range(N)] for S in self.bu]).reshape(len(self.bu), N)
        self.nd = np.array([[1.0 if i in S else 0.0 for i in range(N)] for S in self.bd]).reshape(len(self.bd), N)
        # product basis index = a * len(bd) + b
        nup = np.repeat(self.nu, len(self.bd), axis=0)
        ndn = np.tile(self.nd, (len(self.bu), 1))
        self.nup, self.ndn = nup, ndn
        docc = (nup * ndn).sum(axis=1)
        TK = np.kron(Cu, Cd)
        TU = np.exp(-dtau * U * docc)
        T1 = TK * TU[None, :]
        self.T = np.linalg.matrix_power(T1, L)
        self.Z = np.trace(self.T)

    def expect(self, O):
        return float(np.trace(O @ self.T) / self.Z)

    def expect_diag(self, d):
        return float(np.dot(d, np.diag(self.T)) / self.Z)

    def _op_up(self, i, j):
        return np.kron(hop(self.bu, self.N, i, j), np.eye(len(self.bd)))

    def _op_dn(self, i, j):
        return np.kron(np.eye(len(self.bu)), hop(self.bd, self.N, i, j))

    def observables(self, corr=False):
        lat, N = self.lat, self.N
        nup, ndn = self.nup, self.ndn
        out = {}
        out["n_up"] = self.expect_diag(nup.sum(1))
        out["n_dn"] = self.expect_diag(ndn.sum(1))
        out["docc"] = self.expect_diag((nup * ndn).sum(1)) / N
        ek = 0.0
        for i, j, k in zip(lat["bi"], lat["bj"], lat["kb"]):
            for op in (self._op_up, self._op_dn):
                ek += k * (self.expect(op(i, j)) + self.expect(op(j, i)))
        ek += self.expect_diag(((nup + ndn) * np.asarray(lat["eps"])[None, :]).sum(1))
        out["ekin"] = ek / N
        sub = np.asarray(lat["sub"])
        sz = 0.5 * (nup - ndn)
        ncell = N / 2.0
        for a, b, name in ((0, 0, "szz_00"), (1, 1, "szz_11"), (0, 1, "szz_01")):
            out[name] = self.expect_diag(sz[:, sub == a].sum(1) * sz[:, sub == b].sum(1)) / ncell
        # S+_i S-_j = (c^dag_iu c_ju)(c_id c^dag_jd) and its spin mirror
        tot = 0.0
        for i in range(N):
            for j in range(N):
                cdc_dn = (np.eye(len(self.bd)) if i == j else 0.0) - hop(self.bd, N, j, i)
                Opm = np.kron(hop(self.bu, N, i, j), cdc_dn)
                cdc_up = (np.eye(len(self.bu)) if i == j else 0.0) - hop(self.bu, N, j, i)
                Omp = np.kron(cdc_up, hop(self.bd, N, i, j))
                tot += self.expect(Opm) + self.expect(Omp)
        out["s_par"] = 0.5 * tot / ncell
        if corr:
            nn = np.zeros((N, N))
            ss = np.zeros((N, N))
            ntot = nup + ndn
            for i in range(N):
                for j in range(N):
                    nn[i, j] = self.expect_diag(ntot[:, i] * ntot[:, j])
                    zz = self.expect_diag(sz[:, i] * sz[:, j])
                    cdc_dn = (np.eye(len(self.bd)) if i == j else 0.0) - hop(self.bd, N, j, i)
                    cdc_up = (np.eye(len(self.bu)) if i == j else 0.0) - hop(self.bu, N, j, i)
                    pm = self.expect(np.kron(hop(self.bu, N, i, j), cdc_dn))
                    mp_ = self.expect(np.kron(cdc_up, hop(self.bd, N, i, j)))
                    ss[i, j] = zz + 0.5 * (pm + mp_)
            out["nn"] = nn
            out["ss"] = ss
        return out


# --------------------------------------------------------------------------
# per-configuration Wick estimators from dense matrices
# --------------------------------------------------------------------------

def wick_observables(lat, U, dtau, s, occ_up, occ_dn, boundary_slice=0):
    """Observables of one configuration at the slice boundary ``boundary_slice``
    (O inserted between B_{b-1} and B_b), from dense propagators.

    rho_ij = <c_i^dag c_j> = [R (L R)^{-1} L]_{ji} with R = B(b,0) P and
    L = P^T B(beta, b)."""
    N = lat["N"]
    BK = dense_BK(lat, dtau)
    lam = hs_lambda(U, dtau)
    rho = []
    sgn = 1.0
    for spin, occ in ((0, occ_up), (1, occ_dn)):
        sp = 1.0 if (U < 0 or spin == 0) else -1.0
        Bs = [BK @ np.diag(np.exp(sp * lam * s[l])) for l in range(s.shape[0])]
        P = np.zeros((N, len(occ)))
        for a, i in enumerate(occ):
            P[i, a] = 1.0
        R = P.copy()
        for l in range(boundary_slice):
            R = Bs[l] @ R
        Lm = P.T.copy()
        for l in range(s.shape[0] - 1, boundary_slice - 1, -1):
            Lm = Lm @ Bs[l]
        W = Lm @ R
        if len(occ):
            sgn *= np.sign(np.linalg.det(W))
            rho.append((R @ np.linalg.inv(W) @ Lm).T)
        else:
            rho.append(np.zeros((N, N)))
    ru, rd = rho
    nu, nd = np.diag(ru), np.diag(rd)
    out = {"sign": sgn, "n_up": nu.sum(), "n_dn": nd.sum(), "docc": (nu * nd).sum() / N}
    K = np.diag(np.asarray(lat["eps"], dtype=float))
    for i, j, k in zip(lat["bi"], lat["bj"], lat["kb"]):
        K[i, j] += k
        K[j, i] += k
    out["ekin"] = (np.sum(K * ru) + np.sum(K * rd)) / N
    I = np.eye(N)
    # <n^s_i n^s_j> = n_i n_j + rho_ij (delta_ij - rho_ji)
    same = [np.outer(np.diag(r), np.diag(r)) + r * (I - r.T) for r in (ru, rd)]
    cross = np.outer(nu, nd) + np.outer(nd, nu)
    zz = 0.25 * (same[0] + same[1] - cross)
    pm = ru * (I - rd.T)
    mp_ = rd * (I - ru.T)
    sub = np.asarray(lat["sub"])
    ncell = N / 2.0
    for a, b, name in ((0, 0, "szz_00"), (1, 1, "szz_11"), (0, 1, "szz_01")):
        out[name] = zz[np.ix_(sub == a, sub == b)].sum() / ncell
    out["s_par"] = 0.5 * (pm.sum() + mp_.sum()) / ncell
    out["nn"] = same[0] + same[1] + cross
    out["ss"] = zz + 0.5 * (pm + mp_)
    return out


def enumerate_exact(lat, U, dtau, L, n_up, n_dn, names):
    """Sum over all Fock states and all HS fields of W * O / sum W."""
    N = lat["N"]
    BK = dense_BK(lat, dtau)
    lam = hs_lambda(U, dtau)
    num = {k: 0.0 for k in names}
    den = 0.0
    for bits in range(2 ** (N * L)):
        s = np.array([1 if (bits >> k) & 1 else -1 for k in range(N * L)], dtype=np.int8).reshape(L, N)
        Bsp = []
        for spin in (0, 1):
            sp = 1.0 if (U < 0 or spin == 0) else -1.0
            B = np.eye(N)
            for l in range(L):
                B = BK @ (np.exp(sp * lam * s[l])[:, None] * B)
            Bsp.append(B)
        cfac = np.exp(-lam * s.sum()) if U < 0 else 1.0
        for ou in itertools.combinations(range(N), n_up):
            wu = np.linalg.det(Bsp[0][np.ix_(ou, ou)]) if n_up else 1.0
            for od in itertools.combinations(range(N), n_dn):
                wd = np.linalg.det(Bsp[1][np.ix_(od, od)]) if n_dn else 1.0
                w = wu * wd * cfac
                if w == 0.0:
                    continue
                obs = wick_observables(lat, U, dtau, s, list(ou), list(od))
                den += w
                for k in names:
                    num[k] += w * obs[k]
    return {k: num[k] / den for k in names}


def canonical_free_Z(A, k):
    """Canonical trace of a one-body operator with matrix A on k fermions:
    the elementary symmetric polynomial e_k of the eigenvalues of A."""
    ev = np.linalg.eigvals(A)
    coeffs = np.poly(ev)  # prod (x - ev) = sum (-1)^m e_m x^{n-m}
    return float(np.real(((-1) ** k) * coeffs[k]))
