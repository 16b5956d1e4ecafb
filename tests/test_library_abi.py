"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every function declared in include/gbfmm.h, and carries a correct swap table
(Sec. 2.4). No GPU compute is called here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest
from scipy.special import lpmv

import paper_2012_02207_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "gbfmm.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(fmm_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_function():
    path = gb.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name


def test_create_rejects_bad_config_without_a_gpu():
    """Argument checks run before any device call."""
    L = gb.lib()
    h = ctypes.c_void_p()
    for bad in (dict(p=0), dict(p=31), dict(eps=-1.0), dict(leaf_size=0), dict(precision=7),
                dict(p=20, precision=1), dict(soft=-1e-3), dict(soft=float("inf")), dict(soft=float("nan")),
                dict(flags=4), dict(flags=1, precision=0)):
        cfg = dict(p=8, eps=1e-7, leaf_size=64, precision=1, G=1.0, flags=0, fault_inject=0, soft=0.0)
        cfg.update(bad)
        c = gb._Config(**cfg)
        assert L.fmm_create(ctypes.byref(h), ctypes.byref(c)) == -1, bad
        assert L.fmm_last_error(None)


def _shat(n, m, x, y, z):
    """Schmidt semi-normalised r^n P_n^m e^{im phi} from scipy (independent of
    the generator): sqrt((n-m)!/(n+m)!) r^n Pbar_n^m(cos t) e^{i m phi}."""
    r = math.sqrt(x * x + y * y + z * z)
    ct, ph = z / r, math.atan2(y, x)
    pbar = (-1) ** m * lpmv(m, n, ct)
    return math.sqrt(math.factorial(n - m) / math.factorial(n + m)) * r ** n * pbar * np.exp(1j * m * ph)


def _blocks(n):
    cos_t, sin_t = gb.export_swap()
    co = n * (n + 1) * (2 * n + 1) // 6
    so = (n - 1) * n * (2 * n - 1) // 6 if n > 0 else 0
    A = cos_t[co:co + (n + 1) ** 2].reshape(n + 1, n + 1)
    B = sin_t[so:so + n * n].reshape(n, n)
    return A, B


def test_swap_table_size_covers_p30():
    cos_t, sin_t = gb.export_swap()
    assert len(cos_t) == sum((n + 1) ** 2 for n in range(31))
    assert len(sin_t) == sum(n * n for n in range(31))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 17, 24, 30])
def test_swap_matrices_reproduce_swapped_harmonics(n):
    """c_n^m(z,y,x) = sum A[m][m'] c_n^{m'}(x,y,z), s likewise with B."""
    A, B = _blocks(n)
    rng = np.random.default_rng(n)
    for _ in range(4):
        x, y, z = rng.normal(size=3)
        orig = np.array([_shat(n, m, x, y, z) for m in range(n + 1)])
        swp = np.array([_shat(n, m, z, y, x) for m in range(n + 1)])
        tol = 1e-10 * max(1.0, np.abs(orig).max())
        assert np.allclose(A @ orig.real, swp.real, atol=tol)
        if n:
            assert np.allclose(B @ orig.imag[1:], swp.imag[1:], atol=tol)


@pytest.mark.parametrize("n", [1, 4, 9, 16, 30])
def test_swap_is_an_involution_with_parity_zeros(n):
    A, B = _blocks(n)
    assert np.allclose(A @ A, np.eye(n + 1), atol=1e-12)
    assert np.allclose(B @ B, np.eye(n), atol=1e-12)
    for m in range(n + 1):
        for j in range(n + 1):
            if (j + m + n) % 2:
                assert A[m, j] == 0.0
    for m in range(1, n + 1):
        for j in range(1, n + 1):
            if (j + m + n) % 2 == 0:
                assert B[m - 1, j - 1] == 0.0


def test_every_context_call_rejects_a_null_context_without_a_gpu():
    """FMM_ERR_ARG (-1), before any device call, for a NULL context."""
    L = gb.lib()
    calls = {
        "fmm_solve": (None, 10) + (None,) * 8 + (None,),
        "fmm_solve_host": (None, 10) + (None,) * 8 + (None,),
        "fmm_solve_batch": (None, 1, None) + (None,) * 8 + (None,),
        "fmm_solve_graph": (None, 1, None, 10) + (None,) * 8 + (None,),
        "fmm_solve_jerk": (None, 10) + (None,) * 14 + (None,),
        "fmm_direct": (None, 10, None, None, None, None, 10, None, None, None, None, None, None),
        "fmm_timesteps": (None, 10) + (None,) * 7 + (0.03, 1, None, None),
        "fmm_hold": (None, 10) + (None,) * 7 + (0.01, 1, 0.03, 1, 1e-9, 4096, 1024, None, None),
        "fmm_get_stats": (None, None),
        "fmm_export_tree": (None,) + (None,) * 8,
        "fmm_export_geometry": (None,) + (None,) * 6,
        "fmm_export_pairs": (None, 0, None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == -1, name
    L.fmm_destroy(None)  # allowed, does nothing
    assert isinstance(L.fmm_last_error(None), bytes)


def test_noalloc_wrapper_rejects_host_tensors_before_calling_the_library():
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        gb.morton_sort_noalloc(x, x, x)
