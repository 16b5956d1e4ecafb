"""Python binding of the gbfmm CUDA library (argument marshalling only).

The force solve of Mukherjee et al. (2021), Section 2, runs entirely in the
library's kernels; this module passes device pointers of torch tensors (or
host numpy buffers) through the C ABI declared in ``include/gbfmm.h``.
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbfmm.so")
_lock = threading.Lock()
_lib = None

FMM_PRECISION_FP64 = 0
FMM_PRECISION_MIXED = 1
FMM_FLAG_FP64_LOCALS = 1
FMM_FLAG_P2P_LOADS = 2

STATUS = {0: "FMM_OK", -1: "FMM_ERR_ARG", -2: "FMM_ERR_CUDA", -3: "FMM_ERR_OOM", -4: "FMM_ERR_NONFINITE",
          -5: "FMM_ERR_COINCIDENT", -6: "FMM_ERR_CAPACITY", -7: "FMM_ERR_TIMEOUT"}


class FmmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("eps", ctypes.c_double), ("leaf_size", ctypes.c_int),
                ("precision", ctypes.c_int), ("G", ctypes.c_double), ("flags", ctypes.c_uint),
                ("fault_inject", ctypes.c_uint), ("soft", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnodes", ctypes.c_int32), ("nleaves", ctypes.c_int32),
                ("nlevels", ctypes.c_int32), ("n_far", ctypes.c_int64), ("n_near", ctypes.c_int64),
                ("n_m2l", ctypes.c_int64), ("n_p2p", ctypes.c_int64), ("p2p_interactions", ctypes.c_int64),
                ("ms_tree", ctypes.c_double), ("ms_upward", ctypes.c_double), ("ms_estimate", ctypes.c_double),
                ("ms_walk", ctypes.c_double), ("ms_m2l", ctypes.c_double), ("ms_downward", ctypes.c_double),
                ("ms_leaf", ctypes.c_double), ("ms_total", ctypes.c_double), ("walk_iters", ctypes.c_int32),
                ("regrows", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("graph_replays", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ms_jerk", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    from . import build_lib as _b  # noqa: PLC0415
    return _b.build(force=force)


def lib():
    """The loaded CUDA library; builds it from source if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                build()
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
            L.fmm_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Config)]
            L.fmm_destroy.argtypes = [vp]
            L.fmm_destroy.restype = None
            L.fmm_solve.argtypes = [vp, i64] + [dp] * 8 + [vp]
            L.fmm_solve_host.argtypes = [vp, i64] + [dp] * 8 + [vp]
            L.fmm_solve_batch.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)] + [dp] * 8 + [vp]
            L.fmm_solve_graph.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), i64] + [dp] * 8 + [vp]
            L.fmm_solve_jerk.argtypes = [vp, i64] + [dp] * 14 + [vp]
            L.fmm_direct.argtypes = [vp, i64, dp, dp, dp, dp, i64, dp, dp, dp, dp, dp, vp]
            L.fmm_timesteps.argtypes = [vp, i64] + [dp] * 7 + [ctypes.c_double, ctypes.c_int32, dp, vp]
            L.fmm_hold.argtypes = [vp, i64] + [dp] * 7 + [ctypes.c_double, i64, ctypes.c_double, ctypes.c_int32,
                                                          ctypes.c_double, i64, i64, ctypes.POINTER(ctypes.c_int64),
                                                          vp]
            L.fmm_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
            L.fmm_export_tree.argtypes = [vp] + [dp] * 8
            L.fmm_export_geometry.argtypes = [vp] + [dp] * 6
            L.fmm_export_pairs.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp]
            L.fmm_export_swap.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), dp, dp]
            L.fmm_morton_sort_noalloc.argtypes = [i64, dp, dp, dp, dp, dp, dp, vp]
            L.fmm_fma_peak.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp]
            L.fmm_last_error.argtypes = [vp]
            L.fmm_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch  # noqa: PLC0415
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


@dataclass
class Config:
    p: int = 8
    eps: float = 1e-7
    leaf_size: int = 64
    precision: int = FMM_PRECISION_MIXED
    G: float = 1.0
    fault_inject: int = 0
    soft: float = 0.0
    flags: int = 0


class FMM:
    """One solver context (fmm_create/fmm_destroy) on the current CUDA device."""

    def __init__(self, p=8, eps=1e-7, leaf_size=64, precision="mixed", G=1.0, fault_inject=0, soft=0.0,
                 fp64_locals=False, p2p_bulk=True):
        """fp64_locals: in mixed precision, run M2L, L2L and L2P in FP64 on FP64
        coefficients (FMM_FLAG_FP64_LOCALS); P2P stays FP32. p2p_bulk: stage the
        FP32 P2P sources by bulk copies (the default; False sets
        FMM_FLAG_P2P_LOADS, per-lane loads)."""
        if isinstance(precision, str):
            precision = {"fp64": FMM_PRECISION_FP64, "mixed": FMM_PRECISION_MIXED}[precision]
        flags = (FMM_FLAG_FP64_LOCALS if fp64_locals else 0) | (0 if p2p_bulk else FMM_FLAG_P2P_LOADS)
        self.config = Config(p, eps, leaf_size, precision, G, fault_inject, soft, flags)
        cfg = _Config(p, eps, leaf_size, precision, G, flags, fault_inject, soft)
        h = ctypes.c_void_p()
        rc = lib().fmm_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != 0:
            raise FmmError(rc, lib().fmm_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _check(self, rc):
        if rc != 0:
            raise FmmError(rc, lib().fmm_last_error(self._h).decode())

    # -- solves -----------------------------------------------------------
    def solve(self, x, y, z, m, out=None, stream=None):
        """Accelerations and potentials of n bodies; device FP64 tensors in,
        (ax, ay, az, pot) device FP64 tensors out, in the same order."""
        import torch  # noqa: PLC0415
        n = x.numel()
        for t in (x, y, z, m):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("x, y, z, m must be contiguous CUDA float64 tensors of equal length")
        if out is None:
            out = tuple(torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(4))
        ax, ay, az, pot = out
        self._check(lib().fmm_solve(self._h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(ax), _ptr(ay),
                                    _ptr(az), _ptr(pot), _stream_handle(stream)))
        return ax, ay, az, pot

    def solve_host(self, pos: np.ndarray, mass: np.ndarray, stream=0):
        """Same solve from host arrays: pos (n,3) and mass (n,); returns
        (acc (n,3), pot (n,)) numpy arrays. Copies happen inside the call."""
        pos = np.asarray(pos, dtype=np.float64)
        cols = [np.ascontiguousarray(pos[:, d]) for d in range(3)]
        m = np.ascontiguousarray(mass, dtype=np.float64)
        n = len(m)
        outs = [np.empty(n) for _ in range(4)]
        self._check(lib().fmm_solve_host(self._h, n, *[c.ctypes.data for c in cols], m.ctypes.data,
                                         *[o.ctypes.data for o in outs], stream))
        return np.stack(outs[:3], axis=1), outs[3]

    def solve_batch(self, offsets, x, y, z, m, out=None, stream=None):
        """Independent clusters in one pass: cluster c is bodies offsets[c] ..
        offsets[c+1]-1 of the device FP64 tensors x, y, z, m; no force acts
        between clusters. Returns (ax, ay, az, pot) like solve()."""
        import torch  # noqa: PLC0415
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        n = x.numel()
        for t in (x, y, z, m):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("x, y, z, m must be contiguous CUDA float64 tensors of equal length")
        if len(offs) < 1 or offs[-1] != n:
            raise ValueError("offsets must have nclusters + 1 entries ending at len(x)")
        if out is None:
            out = tuple(torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(4))
        ax, ay, az, pot = out
        self._check(lib().fmm_solve_batch(self._h, len(offs) - 1, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(ax), _ptr(ay), _ptr(az),
                                          _ptr(pot), _stream_handle(stream)))
        return ax, ay, az, pot

    def solve_graph(self, x, y, z, m, out=None, offsets=None, stream=None):
        """solve() (or solve_batch() with offsets) replayed from a captured CUDA
        graph: the first call with given tensors solves, plans and captures;
        later calls with the same tensors replay the graph (see fmm_solve_graph).
        The output tensors must be passed in (out) to be reused between calls."""
        import torch  # noqa: PLC0415
        n = x.numel()
        for t in (x, y, z, m):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("x, y, z, m must be contiguous CUDA float64 tensors of equal length")
        if out is None:
            out = tuple(torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(4))
        ax, ay, az, pot = out
        if offsets is None:
            optr, ncl = None, 1
        else:
            offs = np.ascontiguousarray(offsets, dtype=np.int64)
            optr, ncl = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(offs) - 1
        self._check(lib().fmm_solve_graph(self._h, ncl, optr, n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(ax),
                                          _ptr(ay), _ptr(az), _ptr(pot), _stream_handle(stream)))
        return ax, ay, az, pot

    def solve_jerk(self, x, y, z, vx, vy, vz, m, out=None, stream=None):
        """Accelerations, potentials and jerks (the time derivative of the
        acceleration) of bodies moving with velocities (vx, vy, vz): device FP64
        tensors in, (ax, ay, az, pot, jx, jy, jz) out (see fmm_solve_jerk)."""
        import torch  # noqa: PLC0415
        n = x.numel()
        for t in (x, y, z, vx, vy, vz, m):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("positions, velocities and masses must be contiguous CUDA float64 tensors "
                                 "of equal length")
        if out is None:
            out = tuple(torch.empty(n, dtype=torch.float64, device=x.device) for _ in range(7))
        self._check(lib().fmm_solve_jerk(self._h, n, *(_ptr(t) for t in (x, y, z, vx, vy, vz, m)),
                                         *(_ptr(o) for o in out), _stream_handle(stream)))
        return out

    def hold(self, x, y, z, vx, vy, vz, m, dt, nsteps, eta=0.025, symmetrize=True, dt_min=1e-9,
             direct_below=4096, device_below=1024, stream=None):
        """nsteps HOLD steps (fmm_hold) on device FP64 tensors, positions and
        velocities updated in place; returns the run's counters. Sets of at
        most device_below bodies evolve inside one GPU block (0: none)."""
        import torch  # noqa: PLC0415
        n = x.numel()
        for t in (x, y, z, vx, vy, vz, m):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("positions, velocities and masses must be contiguous CUDA float64 tensors "
                                 "of equal length")
        st = (ctypes.c_int64 * 5)()
        self._check(lib().fmm_hold(self._h, n, *(_ptr(t) for t in (x, y, z, vx, vy, vz, m)), float(dt), int(nsteps),
                                   float(eta), int(bool(symmetrize)), float(dt_min), int(direct_below),
                                   int(device_below), st,
                                   _stream_handle(stream)))
        return dict(zip(("kicks", "fmm_solves", "direct_solves", "max_depth", "splits"), list(st)))

    def timesteps(self, x, y, z, vx, vy, vz, m, eta, symmetrize=True, stream=None):
        """Per-body HOLD step sizes (see fmm_timesteps) of device FP64 tensors."""
        import torch  # noqa: PLC0415
        tau = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
        self._check(lib().fmm_timesteps(self._h, x.numel(), *(_ptr(t) for t in (x, y, z, vx, vy, vz, m)),
                                        float(eta), int(bool(symmetrize)), _ptr(tau), _stream_handle(stream)))
        return tau

    def direct(self, x, y, z, m, targets=None, stream=None):
        """FP64 direct sum at device int64 target indices (all bodies if None)."""
        import torch  # noqa: PLC0415
        n = x.numel()
        nt = n if targets is None else targets.numel()
        out = tuple(torch.empty(nt, dtype=torch.float64, device=x.device) for _ in range(4))
        self._check(lib().fmm_direct(self._h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), nt, _ptr(targets),
                                     *[_ptr(o) for o in out], _stream_handle(stream)))
        return out

    # -- inspection -------------------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        self._check(lib().fmm_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def export_tree(self):
        s = self.stats()
        n, nn = s["n"], s["nnodes"]
        keys = np.zeros(n, np.uint64)
        perm = np.zeros(n, np.int64)
        arrs = {k: np.zeros(nn, np.int32) for k in ("level", "begin", "end", "parent", "first_child", "nchild")}
        self._check(lib().fmm_export_tree(self._h, keys.ctypes.data, perm.ctypes.data,
                                          *[arrs[k].ctypes.data for k in ("level", "begin", "end", "parent",
                                                                          "first_child", "nchild")]))
        arrs["keys"], arrs["perm"] = keys, perm
        return arrs

    def export_geometry(self):
        s = self.stats()
        n, nn, p = s["n"], s["nnodes"], self.config.p
        out = {"M": np.zeros(nn), "z": np.zeros((nn, 3)), "r": np.zeros(nn), "P": np.zeros((nn, p + 1)),
               "fmin": np.zeros(nn, np.float32), "f": np.zeros(n, np.float32)}
        self._check(lib().fmm_export_geometry(self._h, *[out[k].ctypes.data for k in ("M", "z", "r", "P", "fmin", "f")]))
        return out

    def export_pairs(self, which: str):
        code = {"far": 0, "near": 1, "m2l": 2, "p2p": 3}[which]
        cnt = ctypes.c_int64()
        self._check(lib().fmm_export_pairs(self._h, code, ctypes.byref(cnt), None))
        out = np.zeros((cnt.value, 2), np.int32)
        self._check(lib().fmm_export_pairs(self._h, code, ctypes.byref(cnt), out.ctypes.data))
        return out


def export_swap():
    """The swap-matrix table compiled into the library: (cos blocks, sin blocks)."""
    nc, ns = ctypes.c_int64(), ctypes.c_int64()
    lib().fmm_export_swap(ctypes.byref(nc), ctypes.byref(ns), None, None)
    c, s = np.zeros(nc.value), np.zeros(ns.value)
    lib().fmm_export_swap(ctypes.byref(nc), ctypes.byref(ns), c.ctypes.data, s.ctypes.data)
    return c, s


NOALLOC_MAX_N = 262144


def morton_sort_noalloc(x, y, z, stream=None):
    """Bounding cube, Morton keys and sort of up to 262144 bodies without any
    device allocation inside the library (fmm_morton_sort_noalloc): returns
    device tensors (keys as int64 holding the unsigned keys, perm int64, box
    float64[4] = cube centre and half-size)."""
    import torch  # noqa: PLC0415
    n = x.numel()
    for t in (x, y, z):
        if (t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n
                or t.device != x.device):
            raise ValueError("x, y, z must be contiguous CUDA float64 tensors of equal length on one device")
    with torch.cuda.device(x.device):  # the library uses the current device's scratch and launches there
        keys = torch.empty(n, dtype=torch.int64, device=x.device)
        perm = torch.empty(n, dtype=torch.int64, device=x.device)
        box = torch.empty(4, dtype=torch.float64, device=x.device)
        rc = lib().fmm_morton_sort_noalloc(n, _ptr(x), _ptr(y), _ptr(z), _ptr(keys), _ptr(perm), _ptr(box),
                                           _stream_handle(stream))
    if rc != 0:
        raise FmmError(rc, lib().fmm_last_error(None).decode())
    return keys, perm, box
