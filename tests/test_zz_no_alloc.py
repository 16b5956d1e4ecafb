"""The no-allocation Morton sort (fmm_morton_sort_noalloc).

Some callers cannot call cudaMalloc while they use the library (a device
budget owned by another allocator, a loop that must not allocate), so the
library offers the first stage of the tree build, the bounding cube and the
sorted Morton keys, with all of its scratch in a static device array. This
checks it, through the C ABI, against the keys and permutation that the
regular solve builds its octree from, on two calls in a row of different
sizes (the static scratch keeps the previous call's contents).
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


def _cols(pos):
    return [torch.tensor(np.ascontiguousarray(pos[:, d]), dtype=torch.float64, device=DEV) for d in range(3)]


def _solver_tree(pos):
    f = gb.FMM(p=4, eps=1e-6, precision="mixed")
    m = torch.full((len(pos),), 1.0 / len(pos), dtype=torch.float64, device=DEV)
    f.solve(*_cols(pos), m)
    t = f.export_tree()
    return t["keys"], t["perm"]


def test_noalloc_morton_sort_matches_the_solver_twice_in_a_row():
    inputs = [ics.plummer(5000, 71)[0], ics.plummer(gb.NOALLOC_MAX_N, 72)[0]]
    outs = []
    for pos in inputs:  # two calls in a row before any check
        keys, perm, box = gb.morton_sort_noalloc(*_cols(pos))
        torch.cuda.synchronize()
        outs.append((keys.cpu().numpy().view(np.uint64), perm.cpu().numpy(), box.cpu().numpy()))
    for pos, (keys, perm, box) in zip(inputs, outs):
        ref_keys, ref_perm = _solver_tree(pos)
        assert np.array_equal(keys, ref_keys)
        assert np.array_equal(perm, ref_perm)
        mn, mx = pos.min(0), pos.max(0)
        assert np.array_equal(box[:3], 0.5 * (mn + mx))
        assert box[3] == (0.5 * (mx - mn)).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(gb.NOALLOC_MAX_N + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(gb.FmmError) as e:
        gb.morton_sort_noalloc(x, x, x)
    assert e.value.status == -1
    assert "262144" in str(e.value)
