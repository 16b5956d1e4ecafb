"""ctypes shim over the C oracle (``fmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module to check the GPU library. The
GPU library never imports it.

The oracle is a plain CPU implementation of the FMM force solve of
Mukherjee et al. (2021), Section 2, in FP64 (the scalar-force estimate f of
Sec. 2.3 in FP32 with a fixed order), plus an O(N^2) FP64 direct sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

NCOEF = lambda p: (p + 1) * (p + 2) // 2  # noqa: E731  complex coefficients, m >= 0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no fused multiply-add)."""
    src = os.path.join(_HERE, "fmm_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_run.restype = ctypes.c_void_p
            L.orc_run.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.orc_free.argtypes = [ctypes.c_void_p]
            L.orc_status.argtypes = [ctypes.c_void_p]
            L.orc_nnodes.argtypes = [ctypes.c_void_p]
            L.orc_nlevels.argtypes = [ctypes.c_void_p]
            L.orc_mac_tests.argtypes = [ctypes.c_void_p]
            L.orc_mac_tests.restype = ctypes.c_double
            L.orc_npairs.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_npairs.restype = ctypes.c_int64
            L.orc_copy.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            L.orc_regular.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_void_p]
            L.orc_irregular.argtypes = L.orc_regular.argtypes
            L.orc_p2m.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            for f in (L.orc_m2m, L.orc_m2l, L.orc_l2l):
                f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, ctypes.c_void_p]
            L.orc_l2p.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp, dp, dp, dp]
            L.orc_eval_multipole.argtypes = [ctypes.c_int, ctypes.c_void_p] + [ctypes.c_double] * 6
            L.orc_eval_multipole.restype = ctypes.c_double
            L.orc_direct.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp, dp, dp, dp]
            L.orc_direct_jerk.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                          dp, dp, dp]
            L.orc_regular_grad.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_p2m_dipole.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            L.orc_l2p_hessian.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, dp]
            L.orc_jerk.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, dp]
            L.orc_tau_pair.argtypes = [ctypes.c_double] * 9 + [ctypes.c_int]
            L.orc_tau_pair.restype = ctypes.c_double
            L.orc_hold.argtypes = [ctypes.c_int64] + [dp] * 7 + [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.c_double,
                                                                                     ctypes.c_int64, ctypes.c_double,
                                                                                     ctypes.POINTER(ctypes.c_int64)]
            L.orc_taus.argtypes = [ctypes.c_int64] + [dp] * 7 + [ctypes.c_double] * 2 + [ctypes.c_int, dp]
            L.orc_energy.argtypes = [ctypes.c_int64] + [dp] * 7 + [ctypes.c_double] * 2
            L.orc_energy.restype = ctypes.c_double
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_mac_values.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_num_threads(int(k))


# --------------------------------------------------------------- harmonics

def regular(p: int, x: float, y: float, z: float) -> np.ndarray:
    """Upsilon_n^m(x,y,z) for 0 <= m <= n <= p, complex, index n(n+1)/2 + m."""
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    lib().orc_regular(p, x, y, z, out.ctypes.data)
    return out


def irregular(p: int, x: float, y: float, z: float) -> np.ndarray:
    """Theta_n^m(x,y,z) for 0 <= m <= n <= p, complex, index n(n+1)/2 + m."""
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    lib().orc_irregular(p, x, y, z, out.ctypes.data)
    return out


def p2m(p, pos, mass, center):
    pos = _c(pos)
    x, y, z = (np.ascontiguousarray(pos[:, d]) for d in range(3))
    m = _c(mass)
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    lib().orc_p2m(p, len(m), _dp(x), _dp(y), _dp(z), _dp(m), *map(float, center), out.ctypes.data)
    return out


def m2m(p, M, shift):
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    lib().orc_m2m(p, M.ctypes.data, *map(float, shift), out.ctypes.data)
    return out


def m2l(p, M, r):
    """Local coefficients about z_B of a multipole about z_A, r = z_A - z_B."""
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    lib().orc_m2l(p, M.ctypes.data, *map(float, r), out.ctypes.data)
    return out


def l2l(p, F, shift):
    out = np.zeros(NCOEF(p), dtype=np.complex128)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    lib().orc_l2l(p, F.ctypes.data, *map(float, shift), out.ctypes.data)
    return out


def l2p(p, F, d):
    """(phi, ax, ay, az) of a local expansion at offset d, without G."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    vals = [ctypes.c_double() for _ in range(4)]
    lib().orc_l2p(p, F.ctypes.data, *map(float, d), *[ctypes.byref(v) for v in vals])
    return tuple(v.value for v in vals)


def eval_multipole(p, M, center, x):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    return lib().orc_eval_multipole(p, M.ctypes.data, *map(float, center), *map(float, x))


# -------------------------------------------------------------- direct sum

def direct(pos, mass, G=1.0, targets=None, soft=0.0):
    """FP64 O(N^2) accelerations (N,3) and potentials (N,) at the targets
    (Plummer-softened with length soft > 0, Appendix B)."""
    pos = _c(pos)
    x, y, z = (np.ascontiguousarray(pos[:, d]) for d in range(3))
    m = _c(mass)
    n = len(m)
    if targets is None:
        nt, tp = n, None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = len(tg), tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    ax, ay, az, pot = (np.zeros(nt) for _ in range(4))
    lib().orc_direct(n, _dp(x), _dp(y), _dp(z), _dp(m), G, float(soft), nt, tp, _dp(ax), _dp(ay), _dp(az),
                     _dp(pot))
    return np.stack([ax, ay, az], axis=1), pot


def direct_jerk(pos, vel, mass, G=1.0, targets=None, soft=0.0):
    """FP64 O(N^2) jerks (N,3), the time derivative of the direct-sum accelerations."""
    pos, vel = _c(pos), _c(vel)
    x, y, z = (np.ascontiguousarray(pos[:, d]) for d in range(3))
    vx, vy, vz = (np.ascontiguousarray(vel[:, d]) for d in range(3))
    m = _c(mass)
    n = len(m)
    if targets is None:
        nt, tp = n, None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = len(tg), tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    jx, jy, jz = (np.zeros(nt) for _ in range(3))
    lib().orc_direct_jerk(n, _dp(x), _dp(y), _dp(z), _dp(vx), _dp(vy), _dp(vz), _dp(m), G, float(soft), nt, tp,
                          _dp(jx), _dp(jy), _dp(jz))
    return np.stack([jx, jy, jz], axis=1)


def regular_grad(p, x, y, z):
    """d/dx, d/dy, d/dz of Upsilon_n^m at (x, y, z), each packed like regular()."""
    g = [np.zeros(NCOEF(p), dtype=np.complex128) for _ in range(3)]
    lib().orc_regular_grad(p, x, y, z, *(a.ctypes.data for a in g))
    return g


def p2m_dipole(p, pos, dip, center):
    """Multipoles -sum_j D_j . grad Upsilon_n^m(x_j - c) of point dipoles D_j at x_j."""
    pos, dip = _c(pos), _c(dip)
    cols = [np.ascontiguousarray(pos[:, d]) for d in range(3)] + [np.ascontiguousarray(dip[:, d]) for d in range(3)]
    M = np.zeros(NCOEF(p), dtype=np.complex128)
    lib().orc_p2m_dipole(p, len(pos), *(_dp(a) for a in cols), *map(float, center), M.ctypes.data)
    return M


def l2p_hessian(p, F, d):
    """(xx, yy, zz, xy, xz, yz) second derivatives of sum conj(Upsilon(d)) F at d."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    h = np.zeros(6)
    lib().orc_l2p_hessian(p, F.ctypes.data, *map(float, d), _dp(h))
    return h


# ------------------------------------------------------------- integrator

def tau_pair(r, v, mij, G=1.0, eta=0.03, sym=False):
    """Step size of a pair (Appendix A): separation r, relative velocity v."""
    return lib().orc_tau_pair(*map(float, r), *map(float, v), float(mij), float(G), float(eta), int(bool(sym)))


def taus(pos, vel, mass, eta=0.03, sym=False, G=1.0):
    """Per-body step size: min over the other bodies of tau_pair."""
    pos, vel = _c(pos), _c(vel)
    cols = [np.ascontiguousarray(pos[:, d]) for d in range(3)] + [np.ascontiguousarray(vel[:, d]) for d in range(3)]
    out = np.zeros(len(mass))
    lib().orc_taus(len(mass), *(_dp(a) for a in cols), _dp(_c(mass)), float(G), float(eta), int(bool(sym)), _dp(out))
    return out


def hold(pos, vel, mass, dt, nsteps, eta=0.03, sym=True, G=1.0, soft=0.0, dt_min=0.0):
    """nsteps HOLD steps (Appendix A) with direct FP64 forces. Returns the new
    positions and velocities and {kicks, pair force evaluations, deepest level}."""
    pos, vel = _c(pos).copy(), _c(vel).copy()
    cols = [np.ascontiguousarray(pos[:, d]) for d in range(3)] + [np.ascontiguousarray(vel[:, d]) for d in range(3)]
    m = _c(mass)
    st = np.zeros(3, dtype=np.int64)
    lib().orc_hold(len(m), *(_dp(a) for a in cols), _dp(m), float(G), float(soft), float(eta), int(bool(sym)),
                   float(dt), int(nsteps), float(dt_min), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return (np.stack(cols[:3], 1), np.stack(cols[3:], 1),
            {"kicks": int(st[0]), "pair_forces": int(st[1]), "max_depth": int(st[2])})


def energy(pos, vel, mass, G=1.0, soft=0.0):
    """Kinetic plus potential energy, direct FP64."""
    pos, vel = _c(pos), _c(vel)
    cols = [np.ascontiguousarray(pos[:, d]) for d in range(3)] + [np.ascontiguousarray(vel[:, d]) for d in range(3)]
    return lib().orc_energy(len(mass), *(_dp(a) for a in cols), _dp(_c(mass)), float(G), float(soft))


# ------------------------------------------------------------------- solve

STAGE_TREE, STAGE_F, STAGE_LISTS, STAGE_FULL = 1, 2, 3, 4


class OracleRun:
    """Result of one oracle solve; every intermediate is kept."""

    def __init__(self, pos, mass, p=8, eps=1e-7, leaf_size=64, G=1.0, stage=STAGE_FULL, soft=0.0):
        pos = _c(pos)
        self._x, self._y, self._z = (np.ascontiguousarray(pos[:, d]) for d in range(3))
        self._m = _c(mass)
        self.n = len(self._m)
        self.p, self.eps, self.leaf_size, self.G, self.stage = p, eps, leaf_size, G, stage
        self.soft = float(soft)
        L = lib()
        self._h = L.orc_run(self.n, _dp(self._x), _dp(self._y), _dp(self._z), _dp(self._m),
                            p, eps, leaf_size, G, self.soft, stage)
        self.status = L.orc_status(self._h)
        self.nnodes = L.orc_nnodes(self._h)
        self.nlevels = L.orc_nlevels(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    def _get(self, which, dtype, shape):
        out = np.zeros(shape, dtype=dtype)
        lib().orc_copy(self._h, which, out.ctypes.data)
        return out

    @property
    def mac_tests(self):
        return lib().orc_mac_tests(self._h)

    def npairs(self, which):
        return lib().orc_npairs(self._h, {"far": 0, "near": 1, "m2l": 2, "p2p": 3}[which])

    def tree(self):
        nn = self.nnodes
        return {
            "keys": self._get(0, np.uint64, self.n),
            "perm": self._get(1, np.int64, self.n),
            "level": self._get(2, np.int32, nn),
            "begin": self._get(3, np.int32, nn),
            "end": self._get(4, np.int32, nn),
            "parent": self._get(5, np.int32, nn),
            "first_child": self._get(6, np.int32, nn),
            "nchild": self._get(7, np.int32, nn),
            "level_start": self._get(25, np.int32, self.nlevels + 1),
            "box": self._get(24, np.float64, 4),
        }

    def geometry(self):
        nn = self.nnodes
        return {
            "M": self._get(8, np.float64, nn),
            "S": self._get(26, np.float64, (nn, 3)),
            "z": self._get(9, np.float64, (nn, 3)),
            "r": self._get(10, np.float64, nn),
            "P": self._get(11, np.float64, (nn, self.p + 1)),
            "f": self._get(12, np.float32, self.n),
            "fmin": self._get(13, np.float32, nn),
        }

    def multipoles(self):
        return self._get(18, np.complex128, (self.nnodes, NCOEF(self.p)))

    def locals(self):
        return self._get(19, np.complex128, (self.nnodes, NCOEF(self.p)))

    def pairs(self, which):
        code = {"far": 14, "near": 15, "m2l": 16, "p2p": 17}[which]
        return self._get(code, np.int32, (self.npairs(which), 2))

    def mac_values(self, a, b):
        """(E_AB M_A/r^2, E_BA M_B/r^2, eps f_B, eps f_A, theta test) of Sec. 2.3, then the
        softening bounds A->B and B->A (0 without softening)."""
        out = np.zeros(7)
        lib().orc_mac_values(self._h, int(a), int(b), _dp(out))
        return out

    def forces(self):
        acc = np.stack([self._get(20 + d, np.float64, self.n) for d in range(3)], axis=1)
        return acc, self._get(23, np.float64, self.n)

    def jerk(self, vel):
        """Jerks (N,3) of the bodies moving with velocities vel (N,3), on this
        solve's tree and lists (needs a full solve)."""
        vel = _c(vel)
        v = [np.ascontiguousarray(vel[:, d]) for d in range(3)]
        j = [np.zeros(self.n) for _ in range(3)]
        rc = lib().orc_jerk(self._h, *(_dp(a) for a in v), *(_dp(a) for a in j))
        if rc != 0:
            raise RuntimeError("the jerk needs a full solve")
        return np.stack(j, axis=1)


def fmm(pos, mass, p=8, eps=1e-7, leaf_size=64, G=1.0, soft=0.0):
    """Accelerations (N,3) and potentials (N,) from the oracle FMM."""
    run = OracleRun(pos, mass, p=p, eps=eps, leaf_size=leaf_size, G=G, stage=STAGE_FULL, soft=soft)
    if run.status != 0:
        raise RuntimeError(f"oracle status {run.status}")
    return run.forces()


def rel_errors(acc, acc_ref):
    """Per-particle relative acceleration error |a - a_ref| / |a_ref| (Sec. 3.1.1)."""
    return np.linalg.norm(acc - acc_ref, axis=1) / np.linalg.norm(acc_ref, axis=1)


def error_stats(acc, acc_ref):
    d = rel_errors(acc, acc_ref)
    return {
        "median": float(np.median(d)),
        "p99": float(np.percentile(d, 99)),
        "p9999": float(np.percentile(d, 99.99)),
        "rms": float(np.sqrt(np.mean(d * d))),
        "max": float(d.max()),
    }
