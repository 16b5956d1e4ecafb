"""The leapfrog driver around the force solve (energy bookkeeping of Sec. 4.2)
against the same integrator run on the CPU with the oracle's FP64 direct
forces."""
import numpy as np
import pytest

import ics
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_02207_gb300 as gb  # noqa: E402
from paper_2012_02207_gb300 import leapfrog  # noqa: E402

DEV = torch.device("cuda:0")


def cpu_leapfrog(pos, vel, m, dt, steps, soft=0.0):
    pos, vel = pos.copy(), vel.copy()
    acc, pot = oracle.direct(pos, m, soft=soft)
    es = [0.5 * (m * (vel * vel).sum(1)).sum() + 0.5 * (m * pot).sum()]
    for _ in range(steps):
        vel += 0.5 * dt * acc
        pos += dt * vel
        acc, pot = oracle.direct(pos, m, soft=soft)
        vel += 0.5 * dt * acc
        es.append(0.5 * (m * (vel * vel).sum(1)).sum() + 0.5 * (m * pot).sum())
    return pos, vel, np.array(es)


@pytest.mark.parametrize("soft", [0.0, 1.0 / 4097])
def test_leapfrog_tracks_direct_integration_and_conserves_energy(soft):
    """soft = 1/N is Appendix B's softening length."""
    n, dt, steps = 4096, 1.0 / 1024, 12
    pos, vel, m = ics.nucleus(n, 5)
    P, V, M = (torch.tensor(a, device=DEV) for a in (pos, vel, m))
    fmm = gb.FMM(p=10, eps=1e-8, precision="mixed", soft=soft)
    es = np.array(leapfrog.integrate(fmm, P, V, M, dt, steps))
    ref_pos, ref_vel, ref_es = cpu_leapfrog(pos, vel, m, dt, steps, soft=soft)
    # Henon-unit Plummer plus a point mass: E0 is close to -1/4 (more bound by the point mass)
    assert -0.4 < es[0] < -0.2
    assert np.allclose(es, ref_es, rtol=1e-6, atol=0)
    assert np.abs(P.cpu().numpy() - ref_pos).max() < 1e-9
    assert np.abs(V.cpu().numpy() - ref_vel).max() < 1e-7
    assert np.abs(es / es[0] - 1).max() < 1e-5
