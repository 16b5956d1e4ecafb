"""Ensemble solves: many independent clusters in one pipeline pass (a forest).

Every cluster of a batch must come out exactly as if it had been solved on
its own: the forest's nodes of cluster c, taken in order, are the oracle's
octree of that cluster, and the forces equal those of a separate solve bit
for bit (every kernel works per node, in the same order inside a cluster).
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


def to_dev(pos, m):
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), dtype=torch.float64, device=DEV) for d in range(3)]
    return cols + [torch.tensor(np.ascontiguousarray(m), dtype=torch.float64, device=DEV)]


def host(out):
    ax, ay, az, pot = out
    return torch.stack([ax, ay, az], 1).cpu().numpy(), pot.cpu().numpy()


def separate(pos, m, offsets, **kw):
    acc = np.zeros_like(pos)
    pot = np.zeros(len(m))
    for c in range(len(offsets) - 1):
        sl = slice(int(offsets[c]), int(offsets[c + 1]))
        if sl.stop == sl.start:
            continue
        f = gb.FMM(**kw)
        acc[sl], pot[sl] = host(f.solve(*to_dev(pos[sl], m[sl])))
    return acc, pot


def odd_ensemble():
    """Clusters of uneven size, including an empty one, single bodies, a
    cluster below the leaf size and two clusters with identical positions."""
    parts = []
    for n, seed, rv in ((3000, 21, 1.0), (0, 0, 1.0), (1, 22, 1.0), (40, 23, 0.5), (5000, 24, 2.0),
                        (5000, 24, 2.0), (2, 25, 1.0), (12000, 26, 0.7)):
        if n == 0:
            parts.append((np.zeros((0, 3)), np.zeros(0)))
            continue
        p, _, m = ics.plummer(n, seed, virial_radius=rv)
        parts.append((p, m))
    sizes = np.array([len(m) for _, m in parts], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = np.concatenate([p for p, _ in parts])
    mass = np.concatenate([m for _, m in parts])
    return offsets, pos, mass


@pytest.mark.parametrize("precision,p,eps", [("fp64", 8, 1e-7), ("mixed", 10, 1e-8), ("mixed", 6, 1e-7)])
def test_batch_equals_separate_solves(precision, p, eps):
    offsets, pos, m = odd_ensemble()
    f = gb.FMM(p=p, eps=eps, precision=precision)
    acc, pot = host(f.solve_batch(offsets, *to_dev(pos, m)))
    sacc, spot = separate(pos, m, offsets, p=p, eps=eps, precision=precision)
    assert np.array_equal(acc, sacc)
    assert np.array_equal(pot, spot)


def test_batch_forest_is_the_oracle_octree_of_every_cluster():
    offsets, pos, m = odd_ensemble()
    leaf = 32
    f = gb.FMM(p=6, eps=1e-6, leaf_size=leaf)
    f.solve_batch(offsets, *to_dev(pos, m))
    gt = f.export_tree()
    nonempty = [c for c in range(len(offsets) - 1) if offsets[c + 1] > offsets[c]]
    # the roots come first, one per non-empty cluster, in cluster order
    roots = np.flatnonzero(gt["level"] == 0)
    assert np.array_equal(roots, np.arange(len(nonempty)))
    assert np.array_equal(gt["begin"][roots], offsets[nonempty])
    for c in nonempty:
        b, e = int(offsets[c]), int(offsets[c + 1])
        ot = oracle.OracleRun(pos[b:e], m[b:e], p=6, eps=1e-6, leaf_size=leaf, stage=oracle.STAGE_TREE).tree()
        assert np.array_equal(gt["keys"][b:e], ot["keys"])
        assert np.array_equal(gt["perm"][b:e] - b, ot["perm"])
        nodes = np.flatnonzero((gt["begin"] >= b) & (gt["begin"] < e))
        assert len(nodes) == len(ot["level"])
        pos_of = {int(k): i for i, k in enumerate(nodes)}  # forest index -> oracle index
        assert np.array_equal(gt["level"][nodes], ot["level"])
        assert np.array_equal(gt["begin"][nodes] - b, ot["begin"])
        assert np.array_equal(gt["end"][nodes] - b, ot["end"])
        assert np.array_equal(gt["nchild"][nodes], ot["nchild"])
        par = np.array([pos_of[int(q)] if q >= 0 else -1 for q in gt["parent"][nodes]])
        assert np.array_equal(par, ot["parent"])
        fc = np.array([pos_of[int(q)] if q >= 0 else -1 for q in gt["first_child"][nodes]])
        assert np.array_equal(fc, ot["first_child"])


def test_batch_is_one_pass_and_meets_the_error_target():
    offsets, pos, m, sizes, _ = ics.ensemble(24, 4, log2n_lo=10, log2n_hi=14)
    f = gb.FMM(p=10, eps=1e-8, precision="mixed")
    cols = to_dev(pos, m)
    acc, _ = host(f.solve_batch(offsets, *cols))
    launches_batch = f.stats()["kernel_launches"]
    g = gb.FMM(p=10, eps=1e-8, precision="mixed")
    sl = slice(int(offsets[0]), int(offsets[1]))
    g.solve(*to_dev(pos[sl], m[sl]))
    # one pass over the forest: about the launches of one solve, not one per cluster
    assert launches_batch < 2 * g.stats()["kernel_launches"] + 16
    for c in range(len(sizes)):
        b, e = int(offsets[c]), int(offsets[c + 1])
        dacc, _ = oracle.direct(pos[b:e], m[b:e])
        d = np.linalg.norm(acc[b:e] - dacc, axis=1) / np.linalg.norm(dacc, axis=1)
        assert np.sqrt((d * d).mean()) <= 1e-6


def test_batch_rejects_bad_offsets():
    offsets, pos, m = odd_ensemble()
    f = gb.FMM()
    cols = to_dev(pos, m)
    bad = offsets.copy()
    bad[3], bad[4] = bad[4], bad[3]
    with pytest.raises(gb.FmmError):
        f.solve_batch(bad, *cols)
    # the context stays usable
    acc, _ = host(f.solve_batch(offsets, *cols))
    assert np.isfinite(acc).all()
