"""Jerks through the FMM: the CUDA path against the CPU oracle.

The GPU and the oracle compute j_i = G [-grad chi + H v_i + near_i] on the
same tree and lists. chi is the potential of the point dipoles m_j v_j, H
the Hessian of the local expansion, near_i the direct jerk over the P2P
pairs. FP64 mode is compared with the oracle's FMM jerk per body, against
the scale J_i = sum_j m_j |v_ij| / r_ij^3 (the jerk's analogue of the
scalar force f_i; bodies near the centre have |j| far below the sum of their
terms). Mixed precision is compared with the oracle's direct jerk.
"""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_02207_gb300 as gb  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def solve_jerk(pos, vel, m, **kw):
    f = gb.FMM(**kw)
    out = f.solve_jerk(*(dev(pos[:, d]) for d in range(3)), *(dev(vel[:, d]) for d in range(3)), dev(m))
    torch.cuda.synchronize()
    o = [t.cpu().numpy() for t in out]
    return f, np.stack(o[:3], 1), o[3], np.stack(o[4:], 1)


def jerk_scale(pos, vel, m, soft=0.0):
    n = len(m)
    J = np.zeros(n)
    for i in range(0, n, 256):
        d = pos[None, :, :] - pos[i:i + 256, None, :]
        u = vel[None, :, :] - vel[i:i + 256, None, :]
        r2 = (d * d).sum(-1) + soft * soft
        r2[r2 == soft * soft] = np.inf  # the body itself
        J[i:i + 256] = (m[None, :] * np.linalg.norm(u, axis=-1) / r2 ** 1.5).sum(1)
    return J


@pytest.mark.parametrize("n,p,eps", [(4096, 8, 1e-7), (20000, 10, 1e-8), (3000, 16, 1e-9), (2000, 3, 1e-6)])
def test_fp64_jerk_matches_oracle_fmm(n, p, eps):
    pos, vel, m = ics.plummer(n, 300 + n + p)
    m = ics.kroupa_masses(n, 400 + n)
    f, acc, pot, jerk = solve_jerk(pos, vel, m, p=p, eps=eps, precision="fp64", G=1.3)
    run = oracle.OracleRun(pos, m, p=p, eps=eps, G=1.3)
    ojerk = run.jerk(vel)
    oacc, _ = run.forces()
    J = 1.3 * jerk_scale(pos, vel, m)
    d = np.linalg.norm(jerk - ojerk, axis=1)
    assert np.max(d / J) <= 1e-12, np.max(d / J)
    assert np.median(d / np.linalg.norm(ojerk, axis=1)) <= 1e-13
    # the accelerations are those of the ordinary solve
    ref = gb.FMM(p=p, eps=eps, precision="fp64", G=1.3).solve(*(dev(pos[:, d]) for d in range(3)), dev(m))
    assert np.array_equal(acc, np.stack([t.cpu().numpy() for t in ref[:3]], 1))
    assert f.stats()["ms_jerk"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("soft", [0.0, 0.01])
def test_all_direct_jerk_equals_the_direct_jerk(precision, soft):
    n = 3000
    pos, vel, m = ics.plummer(n, 45)
    _, _, _, jerk = solve_jerk(pos, vel, m, p=4, eps=0.0, leaf_size=16, precision=precision, soft=soft)
    jd = oracle.direct_jerk(pos, vel, m, soft=soft)
    J = jerk_scale(pos, vel, m, soft)
    rel = np.linalg.norm(jerk - jd, axis=1) / J
    assert np.max(rel) <= (1e-13 if precision == "fp64" else 1e-5), np.max(rel)


@pytest.mark.parametrize("p,eps", [(8, 1e-7), (10, 1e-8), (12, 1e-8)])
def test_mixed_jerk_error_vs_direct(p, eps):
    n = 30000
    pos, vel, _ = ics.plummer(n, 46)
    m = ics.kroupa_masses(n, 47)
    _, _, _, jm = solve_jerk(pos, vel, m, p=p, eps=eps, precision="mixed")
    _, _, _, j64 = solve_jerk(pos, vel, m, p=p, eps=eps, precision="fp64")
    jd = oracle.direct_jerk(pos, vel, m)
    s_mixed = oracle.error_stats(jm, jd)
    s_fp64 = oracle.error_stats(j64, jd)
    # the far field of the jerk is second derivatives; FP32 adds ~1e-6 to the
    # FP64 truncation error (p >= 12: the FP32 M2L's wider rounding)
    assert s_fp64["median"] < 20 * eps, s_fp64
    assert s_mixed["median"] <= s_fp64["median"] + (3e-7 if p <= 10 else 1e-6), (s_mixed, s_fp64)
    assert s_mixed["rms"] <= s_fp64["rms"] + (3e-6 if p <= 10 else 1e-5), (s_mixed, s_fp64)
