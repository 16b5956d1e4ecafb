"""The HOLD integrator of Appendix A on the GPU (fmm_hold, fmm_timesteps)
against the oracle's HOLD with direct FP64 forces.

The step sizes are bit-exact (FP64, the same operations, no contraction), so
both sides split every set the same way. The direct-force run then follows
the oracle's trajectory to round-off; the FMM-force run to the FMM's
accuracy.
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


def cols(a):
    return [torch.tensor(np.ascontiguousarray(a[:, d]), dtype=torch.float64, device=DEV) for d in range(3)]


def run_gpu(pos, vel, m, dt, nsteps, **kw):
    f = gb.FMM(p=kw.pop("p", 10), eps=kw.pop("eps", 1e-8), precision=kw.pop("precision", "fp64"),
               G=kw.pop("G", 1.0), soft=kw.pop("soft", 0.0))
    X, V = cols(pos), cols(vel)
    M = torch.tensor(m, dtype=torch.float64, device=DEV)
    st = f.hold(*X, *V, M, dt, nsteps, **kw)
    return (np.stack([t.cpu().numpy() for t in X], 1), np.stack([t.cpu().numpy() for t in V], 1), st)


@pytest.mark.parametrize("sym", [False, True])
def test_step_sizes_are_bit_exact(sym):
    pos, vel, _ = ics.plummer(1000, 61)
    m = ics.kroupa_masses(1000, 62)
    f = gb.FMM(p=4, G=1.3)
    tau = f.timesteps(*cols(pos), *cols(vel), torch.tensor(m, device=DEV), eta=0.03, symmetrize=sym).cpu().numpy()
    assert np.array_equal(tau, oracle.taus(pos, vel, m, eta=0.03, sym=sym, G=1.3))


@pytest.mark.parametrize("sym", [False, True])
def test_hold_with_direct_forces_follows_the_oracle(sym):
    """The host-driven recursion (no set evolves inside one block)."""
    pos, vel, m = ics.plummer(100, 63)
    p, v, st = run_gpu(pos, vel, m, 1 / 64, 16, eta=0.03, symmetrize=sym, dt_min=1e-9, direct_below=1 << 30,
                       device_below=0)
    op, ov, ost = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=16, eta=0.03, sym=sym, dt_min=1e-9)
    assert st["kicks"] == ost["kicks"] and st["max_depth"] == ost["max_depth"] and st["fmm_solves"] == 0
    assert st["max_depth"] >= 3
    assert np.abs(p - op).max() < 1e-11 and np.abs(v - ov).max() < 1e-9
    P0, P1 = (m[:, None] * vel).sum(0), (m[:, None] * v).sum(0)
    assert np.abs(P1 - P0).max() < 1e-13 * (m[:, None] * np.abs(v)).sum()


@pytest.mark.parametrize("sym,soft,G", [(False, 0.0, 1.0), (True, 0.0, 1.0), (True, 2e-3, 1.3)])
def test_device_resident_hold_reproduces_the_oracle_bit_for_bit(sym, soft, G):
    """The whole recursion inside one block: the same splits (bit-exact step
    sizes), and forces with the oracle's operations in the oracle's order, so
    positions and velocities equal the oracle's bit for bit after 16 steps
    of several levels each."""
    pos, vel, m = ics.plummer(100, 63)
    p, v, st = run_gpu(pos, vel, m, 1 / 64, 16, eta=0.03, symmetrize=sym, dt_min=1e-9, direct_below=1 << 30,
                       device_below=1024, G=G, soft=soft)
    op, ov, ost = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=16, eta=0.03, sym=sym, G=G, soft=soft, dt_min=1e-9)
    assert st["kicks"] == ost["kicks"] and st["max_depth"] == ost["max_depth"] >= 3
    assert st["fmm_solves"] == 0 and st["splits"] > 16
    assert np.array_equal(p, op) and np.array_equal(v, ov)


def test_device_resident_sets_below_the_host_recursion():
    """Sets above 64 bodies split on the host, smaller ones evolve inside one
    block: the same kicks and depth as the oracle, and its trajectory to
    round-off."""
    pos, vel, m = ics.plummer(600, 65)
    p, v, st = run_gpu(pos, vel, m, 1 / 64, 8, eta=0.03, symmetrize=True, dt_min=1e-9, direct_below=1 << 30,
                       device_below=64)
    op, ov, ost = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=8, eta=0.03, sym=True, dt_min=1e-9)
    assert st["kicks"] == ost["kicks"] and st["max_depth"] == ost["max_depth"]
    assert np.abs(p - op).max() < 1e-10 and np.abs(v - ov).max() < 1e-8


def test_hold_with_fmm_forces_tracks_the_oracle():
    """Sets of 256 or more bodies use the FMM (fast from slow as the
    difference of two solves); the run stays within the FMM's accuracy of the
    direct-force oracle and conserves energy as well."""
    pos, vel, m = ics.plummer(2000, 64)
    E0 = oracle.energy(pos, vel, m)
    p, v, st = run_gpu(pos, vel, m, 1 / 64, 8, eta=0.05, symmetrize=True, dt_min=1e-9, direct_below=256,
                       p=12, eps=1e-10)
    op, ov, ost = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=8, eta=0.05, sym=True, dt_min=1e-9)
    assert st["fmm_solves"] > 0 and st["direct_solves"] > 0
    assert np.abs(p - op).max() < 1e-6 and np.abs(v - ov).max() < 1e-4
    dE_gpu = abs(oracle.energy(p, v, m) / E0 - 1)
    dE_orc = abs(oracle.energy(op, ov, m) / E0 - 1)
    assert dE_gpu < 2 * dE_orc + 1e-9, (dE_gpu, dE_orc)
