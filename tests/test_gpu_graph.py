"""fmm_solve_graph: the solve replayed from a captured CUDA graph.

A replay must give exactly the result of an ordinary solve of the same
bodies: when they are the bodies it was captured with, when they moved a
little (sizes within the planned capacities), and, through the fallback,
when they moved so much that the plan no longer fits.
"""
import numpy as np
import pytest

import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_02207_gb300 as gb  # noqa: E402

DEV = torch.device("cuda:0")


def to_dev(pos, m):
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), dtype=torch.float64, device=DEV) for d in range(3)]
    return cols + [torch.tensor(np.ascontiguousarray(m), dtype=torch.float64, device=DEV)]


def host(out):
    return torch.stack(out[:3], 1).cpu().numpy(), out[3].cpu().numpy()


def reference(cols, mt, offsets=None, **kw):
    f = gb.FMM(**kw)
    if offsets is None:
        return host(f.solve(*cols, mt))
    return host(f.solve_batch(offsets, *cols, mt))


@pytest.mark.parametrize("precision,p,eps", [("mixed", 10, 2e-8), ("fp64", 8, 1e-7)])
def test_replay_equals_solve_and_follows_moving_bodies(precision, p, eps):
    pos, vel, m = ics.plummer(20000, 31)
    x, y, z, mt = to_dev(pos, m)
    kw = dict(p=p, eps=eps, precision=precision)
    f = gb.FMM(**kw)
    out = tuple(torch.empty_like(x) for _ in range(4))
    a0, p0 = host(f.solve_graph(x, y, z, mt, out=out))  # ordinary solve, plan, capture
    assert f.stats()["graph_replays"] == 0
    ra, rp = reference([x, y, z], mt, **kw)
    assert np.array_equal(a0, ra) and np.array_equal(p0, rp)
    for _ in range(2):
        a1, p1 = host(f.solve_graph(x, y, z, mt, out=out))
        assert f.stats()["graph_replays"] == 1
        assert np.array_equal(a1, ra) and np.array_equal(p1, rp)
    # a small step of the bodies: the same graph, the new result
    v = [torch.tensor(vel[:, d], device=DEV) for d in range(3)]
    for step in range(3):
        for c, vc in zip((x, y, z), v):
            c.add_(1e-3 * vc)
        a2, p2 = host(f.solve_graph(x, y, z, mt, out=out))
        assert f.stats()["graph_replays"] == 1, step
        ra2, rp2 = reference([x, y, z], mt, **kw)
        assert np.array_equal(a2, ra2) and np.array_equal(p2, rp2)
        st = f.stats()
        assert st["p2p_interactions"] > 0 and st["n_m2l"] > 0 and st["nnodes"] > 0


def test_fallback_and_new_capture_when_the_tree_changes():
    pos, _, m = ics.plummer(20000, 32)
    x, y, z, mt = to_dev(pos, m)
    kw = dict(p=8, eps=1e-7, precision="mixed")
    f = gb.FMM(**kw)
    out = tuple(torch.empty_like(x) for _ in range(4))
    f.solve_graph(x, y, z, mt, out=out)
    f.solve_graph(x, y, z, mt, out=out)
    assert f.stats()["graph_replays"] == 1
    # squeeze the inner half of the cluster into a tiny core: many more nodes and levels
    r = torch.sqrt(x * x + y * y + z * z)
    inner = r < r.median()
    for c in (x, y, z):
        c[inner] *= 1e-3
    a, p = host(f.solve_graph(x, y, z, mt, out=out))
    assert f.stats()["graph_replays"] == 0  # the plan did not fit: ordinary solve
    ra, rp = reference([x, y, z], mt, **kw)
    assert np.array_equal(a, ra) and np.array_equal(p, rp)
    a, p = host(f.solve_graph(x, y, z, mt, out=out))  # captured again for the new sizes
    assert f.stats()["graph_replays"] == 1
    assert np.array_equal(a, ra) and np.array_equal(p, rp)


def test_replayed_forest_equals_batch():
    offsets, pos, m, sizes, _ = ics.ensemble(12, 33, log2n_lo=8, log2n_hi=12)
    x, y, z, mt = to_dev(pos, m)
    kw = dict(p=10, eps=2e-8, precision="mixed")
    f = gb.FMM(**kw)
    out = tuple(torch.empty_like(x) for _ in range(4))
    f.solve_graph(x, y, z, mt, out=out, offsets=offsets)
    a, p = host(f.solve_graph(x, y, z, mt, out=out, offsets=offsets))
    assert f.stats()["graph_replays"] == 1
    ra, rp = reference([x, y, z], mt, offsets=offsets, **kw)
    assert np.array_equal(a, ra) and np.array_equal(p, rp)


def test_new_pointers_mean_a_new_capture():
    pos, _, m = ics.plummer(5000, 34)
    x, y, z, mt = to_dev(pos, m)
    f = gb.FMM(p=8, eps=1e-7)
    keep = [f.solve_graph(x, y, z, mt)]  # new output tensors, the old ones kept alive: new addresses
    keep.append(f.solve_graph(x, y, z, mt))
    assert f.stats()["graph_replays"] == 0
    out = tuple(torch.empty_like(x) for _ in range(4))
    f.solve_graph(x, y, z, mt, out=out)
    a, p = host(f.solve_graph(x, y, z, mt, out=out))
    assert f.stats()["graph_replays"] == 1
    ra, rp = reference([x, y, z], mt, p=8, eps=1e-7)
    assert np.array_equal(a, ra) and np.array_equal(p, rp)
