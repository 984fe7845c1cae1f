"""Thin ctypes binding of the C ABI in include/lecqmc.h.

Argument marshalling only: every step of the sweep runs in the sm_103a
kernels of liblecqmc.so.  PyTorch supplies the CUDA stream and, through its
caching allocator, the device memory.  There is no CPU fallback: without the
built library (or without a GPU) the calls raise.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

LQ_FP64 = 0
LQ_MIXED = 1
LQ_MIXED_DW = 2
LQ_SWAP_UNIFORM = 0
LQ_SWAP_NEIGHBOUR = 1
LQ_CHECKERBOARD = 0
LQ_EXACT = 1
LQ_NOBS = 9
OBS_NAMES = ["sign", "n_up", "n_dn", "docc", "ekin", "szz_00", "szz_11", "szz_01", "s_par"]
LQ_MAX_PARTICLES = 512

_STATUS = {0: "LQ_OK", 1: "LQ_EINVAL", 2: "LQ_ENOMEM", 3: "LQ_ECUDA", 4: "LQ_ENUMERIC", 5: "LQ_ETIMEOUT",
           6: "LQ_EBUSY", 7: "LQ_ENOTFOUND", 8: "LQ_EUNSUPPORTED"}

EXPORTS = [
    "lq_lattice_from_bonds", "lq_lattice_chain", "lq_lattice_square", "lq_lattice_flatband",
    "lq_lattice_cross_stitch", "lq_lattice_info", "lq_lattice_bonds", "lq_lattice_destroy",
    "lq_sim_create", "lq_sim_init", "lq_sim_set_fields", "lq_sim_get_fields", "lq_sim_set_fock",
    "lq_sim_get_fock", "lq_sim_set_sweep_index", "lq_sim_sweep", "lq_sim_autotune", "lq_sim_launch_config",
    "lq_sim_set_launch_config",
    "lq_sim_run_host", "lq_sim_sync",
    "lq_sim_log_weight",
    "lq_sim_tracked_weight", "lq_sim_field_ratio", "lq_sim_swap_ratio", "lq_sim_records",
    "lq_sim_clear_records", "lq_sim_stats", "lq_sim_profile", "lq_sim_chain_panel", "lq_sim_chain_info",
    "lq_sim_device_bytes", "lq_sim_destroy", "lq_sim_measure", "lq_sim_check_drift", "lq_server_create",
    "lq_server_submit",
    "lq_server_poll", "lq_server_stats", "lq_server_set_tick_target", "lq_server_destroy", "lq_sweep_noalloc",
    "lq_device_fp64_rate", "lq_test_quotient", "lq_request_footprint", "lq_cp_walk", "lq_cp_population",
    "lq_probe_gram",
    "lq_last_error", "lq_version",
]


class LqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [("U", C.c_double), ("beta", C.c_double), ("dtau", C.c_double), ("n_up", C.c_int32),
                ("n_dn", C.c_int32), ("n_stab", C.c_int32), ("precision", C.c_int32), ("seed", C.c_uint64),
                ("swap_mode", C.c_int32), ("left_swaps", C.c_int32), ("kinetic", C.c_int32)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class Request(C.Structure):
    _fields_ = [("lattice", C.c_void_p), ("params", Params), ("n_sweeps", C.c_int32), ("chain_id", C.c_uint32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_records", C.c_int32), ("obs_mean", C.c_double * 9),
                ("obs_err", C.c_double * 9), ("log_weight", C.c_double), ("sign", C.c_int32),
                ("counts", C.c_int64 * 4), ("queue_ms", C.c_double), ("total_ms", C.c_double),
                ("sweep_ms_mean", C.c_double), ("wall_ms_per_sweep", C.c_double), ("active_at_admit", C.c_int32),
                ("waited_for_memory", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("p50_sweep_ms", C.c_double), ("p99_sweep_ms", C.c_double), ("p50_tick_ms", C.c_double),
                ("p99_tick_ms", C.c_double), ("updates_per_s", C.c_double), ("busy_s", C.c_double),
                ("wall_s", C.c_double), ("admit_s", C.c_double), ("retire_s", C.c_double), ("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("active", C.c_int64), ("queued", C.c_int64), ("ticks", C.c_int64),
                ("hbm_in_use", C.c_size_t), ("p50_wall_sweep_ms", C.c_double), ("p99_wall_sweep_ms", C.c_double),
                ("sweeps", C.c_int64)]


class Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


_lib = None


def load(build_if_missing=True):
    """Load liblecqmc.so (building it with nvcc if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise ImportError("liblecqmc.so is not built (run paper_2601_08552_gb300/build.py)")
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, dbl, u32 = C.c_int32, C.c_double, C.c_uint32
    pi32, pdbl = C.POINTER(C.c_int32), C.POINTER(C.c_double)
    lib.lq_last_error.restype = C.c_char_p
    lib.lq_version.restype = C.c_char_p
    sig = {
        "lq_lattice_from_bonds": [i32, i32, pi32, pi32, pdbl, pdbl, pi32, C.POINTER(P)],
        "lq_lattice_chain": [i32, dbl, i32, C.POINTER(P)],
        "lq_lattice_square": [i32, i32, dbl, i32, C.POINTER(P)],
        "lq_lattice_flatband": [i32, dbl, dbl, dbl, dbl, i32, C.POINTER(P)],
        "lq_lattice_cross_stitch": [i32, dbl, dbl, dbl, i32, C.POINTER(P)],
        "lq_lattice_info": [P, pi32, pi32, pi32],
        "lq_lattice_bonds": [P, pi32, pi32, pdbl, pi32],
        "lq_lattice_destroy": [P],
        "lq_sim_create": [C.POINTER(P), C.POINTER(Params), i32, C.POINTER(u32), P, C.POINTER(Allocator),
                          C.POINTER(P)],
        "lq_sim_init": [P],
        "lq_sim_set_fields": [P, i32, C.POINTER(C.c_int8)],
        "lq_sim_get_fields": [P, i32, C.POINTER(C.c_int8)],
        "lq_sim_set_fock": [P, i32, pi32, pi32],
        "lq_sim_get_fock": [P, i32, pi32, pi32],
        "lq_sim_set_sweep_index": [P, u32],
        "lq_sim_sweep": [P, i32, i32],
        "lq_sim_autotune": [P, i32, pi32],
        "lq_sim_launch_config": [P, pi32],
        "lq_sim_set_launch_config": [P, i32, i32, i32],
        "lq_sim_run_host": [P, C.POINTER(C.c_int8), pi32, i32, i32, C.POINTER(C.c_int8), pi32, pdbl],
        "lq_sim_sync": [P],
        "lq_sim_log_weight": [P, i32, pdbl, pi32],
        "lq_sim_tracked_weight": [P, i32, pdbl, pi32],
        "lq_sim_field_ratio": [P, i32, i32, i32, pdbl],
        "lq_sim_swap_ratio": [P, i32, i32, i32, i32, pdbl, pdbl],
        "lq_sim_records": [P, i32, i32, pi32, pdbl],
        "lq_sim_clear_records": [P],
        "lq_sim_stats": [P, i32, C.POINTER(C.c_int64)],
        "lq_sim_profile": [P, i32, C.POINTER(C.c_int64)],
        "lq_sim_chain_panel": [P, i32, i32, i32, i32, pdbl, pdbl],
        "lq_sim_chain_info": [P, i32, pi32],
        "lq_sim_device_bytes": [P, C.POINTER(C.c_size_t)],
        "lq_sim_destroy": [P],
        "lq_sweep_noalloc": [P, C.POINTER(Params), u32, u32, P, P, i32, P, P, pdbl, pi32, C.POINTER(C.c_int64)],
        "lq_sim_measure": [P, i32, i32, pdbl, pdbl],
        "lq_sim_check_drift": [P, dbl, pdbl, pi32],
        "lq_server_create": [i32, C.c_size_t, i32, i32, i32, C.POINTER(P)],
        "lq_server_submit": [P, C.POINTER(Request), C.POINTER(C.c_uint64)],
        "lq_server_poll": [P, C.c_uint64, C.POINTER(Result)],
        "lq_server_stats": [P, C.POINTER(ServerStats)],
        "lq_server_set_tick_target": [P, dbl],
        "lq_server_destroy": [P],
        "lq_device_fp64_rate": [dbl, pdbl, pdbl],
        "lq_test_quotient": [i32, pdbl, pdbl, pdbl, pdbl],
        "lq_request_footprint": [P, C.POINTER(Params), C.POINTER(C.c_size_t)],
        "lq_cp_walk": [P, C.POINTER(Params), pi32, pi32, i32, u32, pdbl, pi32],
        "lq_cp_population": [P, C.POINTER(Params), pi32, pi32, i32, i32, u32, pdbl],
        "lq_probe_gram": [i32, i32, i32, i32, pdbl, pdbl],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise LqError(status, _lib.lq_last_error().decode())


def _addr(a):
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Lattice:
    """A hopping matrix in checkerboard form (see include/lecqmc.h)."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)
        n, nb, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib.lq_lattice_info(self.h, C.byref(n), C.byref(nb), C.byref(g)))
        self.N, self.n_bonds, self.n_families = n.value, nb.value, g.value

    @classmethod
    def _make(cls, fn, *args):
        load()
        out = C.c_void_p()
        _check(fn(*args, C.byref(out)))
        return cls(out.value)

    @classmethod
    def from_bonds(cls, n_sites, bi, bj, kij, onsite=None, sublattice=None):
        load()
        bi = np.ascontiguousarray(bi, dtype=np.int32)
        bj = np.ascontiguousarray(bj, dtype=np.int32)
        kij = np.ascontiguousarray(kij, dtype=np.float64)
        on = None if onsite is None else np.ascontiguousarray(onsite, dtype=np.float64)
        sb = None if sublattice is None else np.ascontiguousarray(sublattice, dtype=np.int32)
        return cls._make(_lib.lq_lattice_from_bonds, int(n_sites), len(bi), _p(bi, C.c_int32), _p(bj, C.c_int32),
                         _p(kij, C.c_double), None if on is None else _p(on, C.c_double),
                         None if sb is None else _p(sb, C.c_int32))

    @classmethod
    def chain(cls, n, t=1.0, periodic=True):
        return cls._make(load().lq_lattice_chain, int(n), float(t), int(bool(periodic)))

    @classmethod
    def square(cls, lx, ly, t=1.0, periodic=True):
        return cls._make(load().lq_lattice_square, int(lx), int(ly), float(t), int(bool(periodic)))

    @classmethod
    def flatband(cls, n_cells, t1=-0.2, t2=1.0, t3=1.0, t4=-0.2, periodic=True):
        return cls._make(load().lq_lattice_flatband, int(n_cells), float(t1), float(t2), float(t3), float(t4),
                         int(bool(periodic)))

    @classmethod
    def cross_stitch(cls, n_cells, t_intra=1.0, t_leg=1.0, t_cross=1.0, periodic=True):
        return cls._make(load().lq_lattice_cross_stitch, int(n_cells), float(t_intra), float(t_leg),
                         float(t_cross), int(bool(periodic)))

    def bonds(self):
        bi = np.zeros(max(self.n_bonds, 1), np.int32)
        bj = np.zeros_like(bi)
        k = np.zeros(max(self.n_bonds, 1))
        f = np.zeros_like(bi)
        _check(_lib.lq_lattice_bonds(self.h, _p(bi, C.c_int32), _p(bj, C.c_int32), _p(k, C.c_double),
                                     _p(f, C.c_int32)))
        nb = self.n_bonds
        return bi[:nb], bj[:nb], k[:nb], f[:nb]

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.lq_lattice_destroy(self.h)
            self.h = None


def sweep_noalloc(lattice, params, chain_id, sweep_index, dev_fields, dev_occ, n_sweeps, dev_records=None,
                  stream=None, want_state=True):
    """Allocation-free single-chain sweep (lq_sweep_noalloc): dev_fields (int8
    L x N), dev_occ (int32 n_up + n_dn) and dev_records (float64 n_sweeps x
    LQ_NOBS, optional) are caller-owned CUDA tensors, updated in place.
    Returns (log|W|, sign, counts4) when want_state."""
    load()
    import torch

    p = _params_struct(params)
    _check_noalloc_buffers(torch, lattice, params, dev_fields, dev_occ, n_sweeps, dev_records)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    lw, sg = C.c_double(), C.c_int32()
    cnt = np.zeros(4, np.int64)
    _check(_lib.lq_sweep_noalloc(lattice.h, C.byref(p), int(chain_id), int(sweep_index),
                                 C.c_void_p(dev_fields.data_ptr()), C.c_void_p(dev_occ.data_ptr()), int(n_sweeps),
                                 C.c_void_p(dev_records.data_ptr()) if dev_records is not None else None,
                                 C.c_void_p(stream),
                                 C.byref(lw) if want_state else None, C.byref(sg) if want_state else None,
                                 cnt.ctypes.data_as(C.POINTER(C.c_int64)) if want_state else None))
    return (lw.value, sg.value, cnt) if want_state else None


def _check_noalloc_buffers(torch, lattice, params, dev_fields, dev_occ, n_sweeps, dev_records):
    """The C entry point receives raw device pointers and cannot check them:
    every buffer must be a contiguous CUDA tensor of the right dtype and
    element count on the current device, or the kernels would write out of
    bounds.  Raises ValueError on any mismatch."""
    L = int(round(float(params["beta"]) / float(params["dtau"])))
    want = [("dev_fields", dev_fields, torch.int8, L * lattice.N),
            ("dev_occ", dev_occ, torch.int32, int(params["n_up"]) + int(params["n_dn"]))]
    if dev_records is not None:
        want.append(("dev_records", dev_records, torch.float64, int(n_sweeps) * LQ_NOBS))
    for name, t, dtype, numel in want:
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != dtype:
            raise ValueError("%s must have dtype %s, not %s" % (name, dtype, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() != numel:
            raise ValueError("%s must hold %d elements, not %d" % (name, numel, t.numel()))
    for name, t, _, _ in want:
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        dev = torch.cuda.current_device()
        if t.device.index != dev:
            raise ValueError("%s must be on the current device (cuda:%d), not %s" % (name, dev, t.device))


def device_fp64_rate(ms=200.0):
    """Measured FP64 FMA throughput of the current device (lq_device_fp64_rate):
    (TFLOP/s, {issue cycles of FP64 and FP32 FMA warp instructions, latencies
    of dependent FP64 FMA, multiply, reciprocal seed, conversion pair, 64-bit
    shuffle and shared-memory load})."""
    load()
    t = C.c_double()
    cyc = np.zeros(9)
    _check(_lib.lq_device_fp64_rate(float(ms), C.byref(t), _p(cyc, C.c_double)))
    names = ["dfma_1lane", "dfma_32lanes", "ffma_32lanes", "latency_dfma", "latency_dmul", "latency_rcp64",
             "latency_cvt_f32_f64_f32", "latency_shfl64", "latency_lds"]
    return t.value, {k: float(v) for k, v in zip(names, cyc)}


def flip_quotient(d, r):
    """The flip loop's FP64 quotient d/r and the IEEE quotient, evaluated on
    the device (lq_test_quotient)."""
    load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    q = np.zeros_like(d)
    qi = np.zeros_like(d)
    _check(_lib.lq_test_quotient(len(d), _p(d, C.c_double), _p(r, C.c_double), _p(q, C.c_double),
                                 _p(qi, C.c_double)))
    return q, qi


def cp_walk(lattice, params, occ_up, occ_dn, n_walkers, sweep_word=0):
    """Constrained-path inner loop (lq_cp_walk): log of each walker's final
    weight (-inf when dropped) and the number dropped."""
    load()
    p = _params_struct(dict(params, precision=LQ_FP64))
    u = np.ascontiguousarray(occ_up, dtype=np.int32)
    d = np.ascontiguousarray(occ_dn, dtype=np.int32)
    lw = np.zeros(max(int(n_walkers), 1))
    dropped = C.c_int32()
    _check(_lib.lq_cp_walk(lattice.h, C.byref(p), _p(u, C.c_int32) if len(u) else None,
                           _p(d, C.c_int32) if len(d) else None, int(n_walkers), int(sweep_word),
                           _p(lw, C.c_double), C.byref(dropped)))
    return lw[: int(n_walkers)].copy(), dropped.value


def cp_population(lattice, params, occ_up, occ_dn, n_walkers, comb_every, run=0):
    """Branching constrained-path population (lq_cp_population): log of its
    estimate of R(eta)."""
    load()
    p = _params_struct(dict(params, precision=LQ_FP64))
    u = np.ascontiguousarray(occ_up, dtype=np.int32)
    d = np.ascontiguousarray(occ_dn, dtype=np.int32)
    est = C.c_double()
    _check(_lib.lq_cp_population(lattice.h, C.byref(p), _p(u, C.c_int32) if len(u) else None,
                                 _p(d, C.c_int32) if len(d) else None, int(n_walkers), int(comb_every), int(run),
                                 C.byref(est)))
    return est.value


GRAM_VARIANTS = ["fp64_cuda_core", "fp64_dmma", "fp32_panels_cuda_core", "fp32_panels_3xtf32"]


def probe_gram(N, m, variant, n_panels=304):
    """Time one N x m Gram per CTA in one of GRAM_VARIANTS (lq_probe_gram):
    (microseconds per launch, largest error relative to the Gram's scale)."""
    load()
    us, err = C.c_double(), C.c_double()
    _check(_lib.lq_probe_gram(int(N), int(m), int(variant), int(n_panels), C.byref(us), C.byref(err)))
    return us.value, err.value


def _torch_allocator():
    """lq_allocator backed by PyTorch's CUDA caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(ctx, nbytes, stream):
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream))

    def _free(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = Allocator()
    a.ctx = None
    a.alloc = _ALLOC_FN(_alloc)
    a.free = _FREE_FN(_free)
    return a


class Sim:
    """A batch of independent Markov chains on one GPU."""

    def __init__(self, lattices, params, chain_ids=None, stream=None, use_torch_allocator=True):
        load()
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("lecqmc needs a CUDA GPU; there is no CPU fallback")
        n = len(lattices)
        if len(params) != n:
            raise ValueError("one params entry per lattice")
        self._lattices = list(lattices)
        lh = (C.c_void_p * n)(*[l.h.value for l in lattices])
        pp = (Params * n)()
        for c, p in enumerate(params):
            pp[c] = _params_struct(p)
        ids = None
        if chain_ids is not None:
            ids = (C.c_uint32 * n)(*[int(x) for x in chain_ids])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._alloc = _torch_allocator() if use_torch_allocator else None
        out = C.c_void_p()
        _check(_lib.lq_sim_create(C.cast(lh, C.POINTER(C.c_void_p)), pp, n, ids, C.c_void_p(stream),
                                  C.byref(self._alloc) if self._alloc is not None else None, C.byref(out)))
        self.h = out
        self.n_chains = n
        self.info = []
        for c in range(n):
            a = np.zeros(6, np.int32)
            _check(_lib.lq_sim_chain_info(self.h, c, _p(a, C.c_int32)))
            self.info.append(dict(N=int(a[0]), L=int(a[1]), tw=int(a[2]), n=int(a[3]), n_up=int(a[4]),
                                  n_dn=int(a[5])))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.lq_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self):
        _check(_lib.lq_sim_init(self.h))

    def set_fields(self, c, s):
        i = self.info[c]
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(i["L"], i["N"])
        _check(_lib.lq_sim_set_fields(self.h, c, _p(s, C.c_int8)))

    def get_fields(self, c):
        i = self.info[c]
        s = np.zeros((i["L"], i["N"]), np.int8)
        _check(_lib.lq_sim_get_fields(self.h, c, _p(s, C.c_int8)))
        return s

    def set_fock(self, c, occ_up, occ_dn):
        u = np.ascontiguousarray(occ_up, dtype=np.int32)
        d = np.ascontiguousarray(occ_dn, dtype=np.int32)
        i = self.info[c]
        if len(u) != i["n_up"] or len(d) != i["n_dn"]:
            raise ValueError("occupation lists must have n_up / n_dn entries")
        _check(_lib.lq_sim_set_fock(self.h, c, _p(u, C.c_int32) if len(u) else None,
                                    _p(d, C.c_int32) if len(d) else None))

    def get_fock(self, c):
        i = self.info[c]
        u = np.zeros(max(i["n_up"], 1), np.int32)
        d = np.zeros(max(i["n_dn"], 1), np.int32)
        _check(_lib.lq_sim_get_fock(self.h, c, _p(u, C.c_int32), _p(d, C.c_int32)))
        return u[: i["n_up"]].copy(), d[: i["n_dn"]].copy()

    def set_sweep_index(self, k):
        _check(_lib.lq_sim_set_sweep_index(self.h, int(k)))

    def sweep(self, n=1, measure=True):
        _check(_lib.lq_sim_sweep(self.h, int(n), int(bool(measure))))

    def check_drift(self, tol=1e-8):
        """Rebuild every chain from its fields and Fock state and compare the
        fresh log|W| with the tracked one; returns (largest relative drift,
        number of drifted chains) or raises LqError (LQ_ENUMERIC) on drift."""
        worst, bad = C.c_double(), C.c_int32()
        _check(_lib.lq_sim_check_drift(self.h, float(tol), C.byref(worst), C.byref(bad)))
        return worst.value, bad.value

    def autotune(self, sweeps_per_candidate=1):
        """Time each plan class's candidate staging buffers on real (unmeasured)
        sweeps and keep the fastest; returns the chosen bytes per class."""
        out = (C.c_int32 * 2)()
        _check(_lib.lq_sim_autotune(self.h, int(sweeps_per_candidate), out))
        return int(out[0]), int(out[1])

    def launch_config(self):
        """Per plan class (small, large): chains, staging bytes, threads per
        CTA and grid of its sweep launch."""
        out = np.zeros(8, np.int32)
        _check(_lib.lq_sim_launch_config(self.h, _p(out, C.c_int32)))
        keys = ("chains", "staging_bytes", "threads", "grid")
        return [dict(zip(keys, (int(x) for x in out[4 * k:4 * k + 4]))) for k in range(2)]

    def set_launch_config(self, plan_class, staging_bytes, threads=256):
        """Pin a plan class's launch (staging bytes, threads per CTA)."""
        _check(_lib.lq_sim_set_launch_config(self.h, int(plan_class), int(staging_bytes), int(threads)))

    def run_host(self, fields, occ, n_sweeps, measure=True, fields_out=None, occ_out=None, records_out=None):
        """Batch call on host arrays (ideally pinned): fields int8 (all chains
        concatenated), occ int32 (n_up then n_dn per chain)."""
        f = fields
        o = occ
        _check(_lib.lq_sim_run_host(
            self.h, C.cast(f.data_ptr() if hasattr(f, "data_ptr") else f.ctypes.data, C.POINTER(C.c_int8)),
            C.cast(o.data_ptr() if hasattr(o, "data_ptr") else o.ctypes.data, C.POINTER(C.c_int32)), int(n_sweeps),
            int(bool(measure)),
            None if fields_out is None else C.cast(_addr(fields_out), C.POINTER(C.c_int8)),
            None if occ_out is None else C.cast(_addr(occ_out), C.POINTER(C.c_int32)),
            None if records_out is None else C.cast(_addr(records_out), C.POINTER(C.c_double))))

    def sync(self):
        _check(_lib.lq_sim_sync(self.h))

    def log_weight(self, c):
        la, sg = C.c_double(), C.c_int32()
        _check(_lib.lq_sim_log_weight(self.h, c, C.byref(la), C.byref(sg)))
        return la.value, sg.value

    def tracked_weight(self, c):
        la, sg = C.c_double(), C.c_int32()
        _check(_lib.lq_sim_tracked_weight(self.h, c, C.byref(la), C.byref(sg)))
        return la.value, sg.value

    def field_ratio(self, c, l, i):
        r = C.c_double()
        _check(_lib.lq_sim_field_ratio(self.h, c, int(l), int(i), C.byref(r)))
        return r.value

    def swap_ratio(self, c, spin, k, j):
        r = C.c_double()
        parts = np.zeros(6)
        _check(_lib.lq_sim_swap_ratio(self.h, c, int(spin), int(k), int(j), C.byref(r), _p(parts, C.c_double)))
        return r.value, parts

    def records(self, c, max_rows=1 << 16):
        n = C.c_int32()
        out = np.zeros((max_rows, LQ_NOBS))
        _check(_lib.lq_sim_records(self.h, c, max_rows, C.byref(n), _p(out, C.c_double)))
        return out[: min(n.value, max_rows)].copy()

    def clear_records(self):
        _check(_lib.lq_sim_clear_records(self.h))

    def stats(self, c):
        out = np.zeros(4, np.int64)
        _check(_lib.lq_sim_stats(self.h, c, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def profile(self, c):
        """SM cycles per phase: flips, propagation, QR, block inverse, swaps,
        measurement; swap removal and addition; flip staging, window
        products, serial chain, recurrences and T update."""
        out = np.zeros(12, np.int64)
        _check(_lib.lq_sim_profile(self.h, c, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def measure(self, c, n_bins=16):
        """Sign-weighted means and jackknife errors over chain c's records."""
        mean = np.zeros(LQ_NOBS)
        err = np.zeros(LQ_NOBS)
        _check(_lib.lq_sim_measure(self.h, c, int(n_bins), _p(mean, C.c_double), _p(err, C.c_double)))
        return mean, err

    def chain_panel(self, c, side, spin, j):
        i = self.info[c]
        m = i["n_up"] if spin == 0 else i["n_dn"]
        Q = np.zeros((i["N"], max(m, 1)))
        V = np.zeros((max(m, 1), max(m, 1)))
        _check(_lib.lq_sim_chain_panel(self.h, c, side, spin, j, _p(Q, C.c_double), _p(V, C.c_double)))
        return Q[:, :m].copy(), V[:m, :m].copy()

    def device_bytes(self):
        b = C.c_size_t()
        _check(_lib.lq_sim_device_bytes(self.h, C.byref(b)))
        return b.value


def _params_struct(p):
    return Params(float(p["U"]), float(p["beta"]), float(p["dtau"]), int(p["n_up"]), int(p["n_dn"]),
                  int(p["n_stab"]), int(p.get("precision", LQ_FP64)), int(p.get("seed", 0)) & (2**64 - 1),
                  int(p.get("swap_mode", LQ_SWAP_UNIFORM)), int(p.get("left_swaps", 0)),
                  int(p.get("kinetic", LQ_CHECKERBOARD)))


class Server:
    """Continuous-batching serving loop (lq_server_*)."""

    def __init__(self, hbm_budget, precision=LQ_FP64, max_active=256, queue_capacity=4096, device=0):
        load()
        out = C.c_void_p()
        _check(_lib.lq_server_create(int(device), int(hbm_budget), int(precision), int(max_active),
                                     int(queue_capacity), C.byref(out)))
        self.h = out
        self._keep = {}

    def submit(self, lattice, params, n_sweeps, chain_id=0):
        req = Request(lattice.h.value, _params_struct(params), int(n_sweeps), int(chain_id))
        rid = C.c_uint64()
        _check(_lib.lq_server_submit(self.h, C.byref(req), C.byref(rid)))
        return rid.value

    def poll(self, rid):
        """The request's result dict, or None while it runs."""
        r = Result()
        st = _lib.lq_server_poll(self.h, C.c_uint64(rid), C.byref(r))
        if st == 7:
            return None
        _check(st)
        return dict(status=r.status, n_records=r.n_records, obs_mean=np.array(r.obs_mean[:]),
                    obs_err=np.array(r.obs_err[:]), log_weight=r.log_weight, sign=r.sign,
                    counts=np.array(r.counts[:]), queue_ms=r.queue_ms, total_ms=r.total_ms,
                    sweep_ms_mean=r.sweep_ms_mean, wall_ms_per_sweep=r.wall_ms_per_sweep,
                    active_at_admit=r.active_at_admit, waited_for_memory=r.waited_for_memory)

    @staticmethod
    def footprint(lattice, params):
        """Device bytes a request holds while admitted (lq_request_footprint)."""
        load()
        b = C.c_size_t()
        p = _params_struct(params)
        _check(_lib.lq_request_footprint(lattice.h, C.byref(p), C.byref(b)))
        return b.value

    def set_tick_target(self, ms):
        _check(_lib.lq_server_set_tick_target(self.h, float(ms)))

    def stats(self):
        s = ServerStats()
        _check(_lib.lq_server_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.lq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
