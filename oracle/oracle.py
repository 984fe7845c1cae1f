"""ctypes binding of the C oracle (test infrastructure only).

``build_oracle()`` compiles ``lq_oracle.c`` with gcc into ``oracle/_build``;
``OracleSim`` wraps one Markov chain of the canonical-ensemble DQMC with the
stabilized QR update.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblq_oracle.so")
_lib = None

NOBS = 9
OBS_NAMES = ["sign", "n_up", "n_dn", "docc", "ekin", "szz_00", "szz_11", "szz_01", "s_par"]


def build_oracle(force=False):
    """Compile the oracle shared library (plain C, -O2, no machine-specific flags)."""
    src = os.path.join(_HERE, "lq_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build_oracle())
    P = C.c_void_p
    ip = C.POINTER(C.c_int)
    dp = C.POINTER(C.c_double)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.c_int, C.c_int, ip, ip, dp, dp, ip, C.c_double, C.c_double, C.c_double,
                               C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_int]
    lib.orc_destroy.argtypes = [P]
    lib.orc_philox.argtypes = [C.POINTER(C.c_uint32)] * 3
    for name in ("orc_init_from_seed", "orc_build_chains"):
        getattr(lib, name).argtypes = [P]
        getattr(lib, name).restype = C.c_int
    lib.orc_set_fields.argtypes = [P, C.POINTER(C.c_int8)]
    lib.orc_set_fields.restype = C.c_int
    lib.orc_get_fields.argtypes = [P, C.POINTER(C.c_int8)]
    lib.orc_set_fock.argtypes = [P, ip, ip]
    lib.orc_set_fock.restype = C.c_int
    lib.orc_get_fock.argtypes = [P, ip, ip]
    lib.orc_log_weight.argtypes = [P, dp, ip]
    lib.orc_log_weight_left.argtypes = [P, dp, ip]
    lib.orc_tracked.argtypes = [P, dp, ip]
    lib.orc_sweep.argtypes = [P, C.c_int, C.c_int]
    lib.orc_field_ratio.argtypes = [P, C.c_int, C.c_int]
    lib.orc_field_ratio.restype = C.c_double
    lib.orc_swap_ratio.argtypes = [P, C.c_int, C.c_int, C.c_int, dp]
    lib.orc_swap_ratio.restype = C.c_double
    lib.orc_swap_ratio_side.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, dp]
    lib.orc_swap_ratio_side.restype = C.c_double
    lib.orc_measure_at.argtypes = [P, C.c_int, dp, dp, dp]
    lib.orc_num_records.argtypes = [P]
    lib.orc_num_records.restype = C.c_int
    lib.orc_get_records.argtypes = [P, dp]
    lib.orc_clear_records.argtypes = [P]
    lib.orc_get_corr.argtypes = [P, dp, dp]
    lib.orc_get_corr.restype = C.c_longlong
    lib.orc_get_chain.argtypes = [P, C.c_int, C.c_int, C.c_int, dp, dp]
    lib.orc_get_BK.argtypes = [P, dp]
    lib.orc_set_dense_BK.argtypes = [P, dp]
    lib.orc_stats.argtypes = [P, C.POINTER(C.c_longlong)]
    lib.orc_info.argtypes = [P, ip, dp]
    lib.orc_get_families.argtypes = [P, ip]
    lib.orc_set_swap_mode.argtypes = [P, C.c_int]
    lib.orc_set_left_swaps.argtypes = [P, C.c_int]
    lib.orc_cp_walk.argtypes = [P, C.c_int, dp]
    lib.orc_cp_walk.restype = C.c_int
    lib.orc_cp_population.argtypes = [P, C.c_int, C.c_int, C.c_uint32]
    lib.orc_cp_population.restype = C.c_double
    lib.orc_comb.argtypes = [dp, C.c_int, C.c_double, ip]
    lib.orc_set_sweep.argtypes = [P, C.c_uint32]
    _lib = lib
    return lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def comb(w, u):
    """Systematic resampling of the oracle: indices of the old walkers that
    the len(w) new walkers copy, for one uniform u in [0, 1)."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(len(w), dtype=np.int32)
    lib.orc_comb(_ptr(w, C.c_double), len(w), float(u), _ptr(out, C.c_int))
    return out


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


class OracleSim:
    """One chain of the oracle.  ``lat`` is a dict from ``oracle.lattices``."""

    def __init__(self, lat, U, beta, dtau, n_up, n_dn, n_stab, seed=0, chain=0,
                 max_records=100000, want_corr=False, init="seed", swap_mode=0, left_swaps=False,
                 kinetic="checkerboard"):
        lib = _load()
        self.lib = lib
        self.lat = lat
        self._bi = np.ascontiguousarray(lat["bi"], dtype=np.int32)
        self._bj = np.ascontiguousarray(lat["bj"], dtype=np.int32)
        self._kb = np.ascontiguousarray(lat["kb"], dtype=np.float64)
        self._eps = np.ascontiguousarray(lat["eps"], dtype=np.float64)
        self._sub = np.ascontiguousarray(lat["sub"], dtype=np.int32)
        h = lib.orc_create(int(lat["N"]), len(self._bi), _ptr(self._bi, C.c_int), _ptr(self._bj, C.c_int),
                           _ptr(self._kb, C.c_double), _ptr(self._eps, C.c_double), _ptr(self._sub, C.c_int),
                           float(U), float(beta), float(dtau), int(n_up), int(n_dn), int(n_stab),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, int(chain), int(max_records), int(bool(want_corr)))
        if not h:
            raise ValueError("invalid oracle parameters")
        self.h = C.c_void_p(h)
        ints = np.zeros(9, dtype=np.int32)
        dbl = np.zeros(1)
        lib.orc_info(self.h, _ptr(ints, C.c_int), _ptr(dbl, C.c_double))
        self.N, self.L, self.tw, self.n, self.G, self.n_up, self.n_dn, self.charge = [int(x) for x in ints[:8]]
        self.lam = float(dbl[0])
        self.ns = (self.n_up, self.n_dn)
        if kinetic == "exact":
            # Eq. 1 with e^{-dtau K} itself: the dense matrix exponential of the hopping matrix
            from scipy.linalg import expm

            from .lattices import dense_K

            self._BK = np.ascontiguousarray(expm(-float(dtau) * dense_K(lat)))
            lib.orc_set_dense_BK(self.h, _ptr(self._BK, C.c_double))
        elif kinetic != "checkerboard":
            raise ValueError("kinetic must be 'checkerboard' or 'exact'")
        lib.orc_set_swap_mode(self.h, int(swap_mode))  # 0 uniform target, 1 empty nearest neighbour
        lib.orc_set_left_swaps(self.h, int(bool(left_swaps)))  # second swap phase at tau = 0
        if init == "seed":
            lib.orc_init_from_seed(self.h)
        else:
            lib.orc_build_chains(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and self.lib is not None:
            self.lib.orc_destroy(h)
            self.h = None

    # configuration ---------------------------------------------------------
    def set_fields(self, s):
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(self.L, self.N)
        if self.lib.orc_set_fields(self.h, _ptr(s, C.c_int8)) != 0:
            raise ValueError("fields must be +-1")

    def get_fields(self):
        s = np.zeros((self.L, self.N), dtype=np.int8)
        self.lib.orc_get_fields(self.h, _ptr(s, C.c_int8))
        return s

    def set_fock(self, occ_up, occ_dn):
        u = np.ascontiguousarray(occ_up, dtype=np.int32)
        d = np.ascontiguousarray(occ_dn, dtype=np.int32)
        if len(u) != self.n_up or len(d) != self.n_dn or self.lib.orc_set_fock(self.h, _ptr(u, C.c_int), _ptr(d, C.c_int)) != 0:
            raise ValueError("bad occupation lists")

    def get_fock(self):
        u = np.zeros(max(self.n_up, 1), dtype=np.int32)
        d = np.zeros(max(self.n_dn, 1), dtype=np.int32)
        self.lib.orc_get_fock(self.h, _ptr(u, C.c_int), _ptr(d, C.c_int))
        return u[: self.n_up].copy(), d[: self.n_dn].copy()

    def set_sweep(self, k):
        self.lib.orc_set_sweep(self.h, int(k))

    # weights and hooks -----------------------------------------------------
    def log_weight(self, side="right"):
        la = C.c_double()
        sg = C.c_int()
        fn = self.lib.orc_log_weight if side == "right" else self.lib.orc_log_weight_left
        fn(self.h, C.byref(la), C.byref(sg))
        return la.value, sg.value

    def tracked(self):
        la = C.c_double()
        sg = C.c_int()
        self.lib.orc_tracked(self.h, C.byref(la), C.byref(sg))
        return la.value, sg.value

    def build_chains(self):
        self.lib.orc_build_chains(self.h)

    def field_ratio(self, l, i):
        return self.lib.orc_field_ratio(self.h, int(l), int(i))

    def swap_ratio(self, spin, k, j, side="right"):
        """Swap ratio on freshly built chains, walked along the right chain
        (tau = beta end) or the left chain (tau = 0 end)."""
        out = np.zeros(6)
        r = self.lib.orc_swap_ratio_side(self.h, 0 if side == "right" else 1, int(spin), int(k), int(j),
                                         _ptr(out, C.c_double))
        return r, out

    def cp_walk(self, n_walkers):
        """Constrained-path inner loop for the current Fock state: the final
        weights of n_walkers independent walkers and how many were dropped."""
        w = np.zeros(max(int(n_walkers), 1))
        dropped = self.lib.orc_cp_walk(self.h, int(n_walkers), _ptr(w, C.c_double))
        return w[: int(n_walkers)].copy(), int(dropped)

    def cp_population(self, n_walkers, comb_every, run=0):
        """Branching population with comb resampling every comb_every slices:
        log of its estimate of R(eta) (-inf if every walker was dropped)."""
        return float(self.lib.orc_cp_population(self.h, int(n_walkers), int(comb_every), int(run)))

    def measure_at(self, jb, corr=False):
        obs = np.zeros(NOBS)
        if corr:
            nn = np.zeros((self.N, self.N))
            ss = np.zeros((self.N, self.N))
            self.lib.orc_measure_at(self.h, int(jb), _ptr(obs, C.c_double), _ptr(nn, C.c_double), _ptr(ss, C.c_double))
            return obs, nn, ss
        self.lib.orc_measure_at(self.h, int(jb), _ptr(obs, C.c_double), None, None)
        return obs

    # sweeps ----------------------------------------------------------------
    def sweep(self, n=1, measure=True):
        self.lib.orc_sweep(self.h, int(n), int(bool(measure)))

    def records(self):
        k = self.lib.orc_num_records(self.h)
        out = np.zeros((k, NOBS))
        if k:
            self.lib.orc_get_records(self.h, _ptr(out, C.c_double))
        return out

    def clear_records(self):
        self.lib.orc_clear_records(self.h)

    def corr(self):
        nn = np.zeros((self.N, self.N))
        ss = np.zeros((self.N, self.N))
        cnt = self.lib.orc_get_corr(self.h, _ptr(nn, C.c_double), _ptr(ss, C.c_double))
        return nn, ss, int(cnt)

    def stats(self):
        out = np.zeros(4, dtype=np.int64)
        self.lib.orc_stats(self.h, out.ctypes.data_as(C.POINTER(C.c_longlong)))
        return out

    def chain_panel(self, side, spin, j):
        m = self.ns[spin]
        Q = np.zeros((self.N, m))
        V = np.zeros((m, m))
        self.lib.orc_get_chain(self.h, int(side), int(spin), int(j), _ptr(Q, C.c_double), _ptr(V, C.c_double))
        return Q, V

    def BK(self):
        out = np.zeros((self.N, self.N))
        self.lib.orc_get_BK(self.h, _ptr(out, C.c_double))
        return out

    def families(self):
        fam = np.zeros(max(len(self._bi), 1), dtype=np.int32)
        self.lib.orc_get_families(self.h, _ptr(fam, C.c_int))
        return fam[: len(self._bi)]
