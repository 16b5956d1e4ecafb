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


def test_noalloc_wrapper_rejects_wrong_tensors():
    x = torch.zeros(10, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        gb.morton_sort_noalloc(x.float(), x, x)
    with pytest.raises(ValueError):
        gb.morton_sort_noalloc(x, x[:9], x)
    with pytest.raises(ValueError):
        gb.morton_sort_noalloc(x, torch.zeros(20, dtype=torch.float64, device=DEV)[::2], x)


def _raw_call(x, y, z, keys, perm, box):
    """fmm_morton_sort_noalloc straight through the C ABI, outputs preallocated."""
    n = x.numel()
    return gb.lib().fmm_morton_sort_noalloc(n, x.data_ptr(), y.data_ptr(), z.data_ptr(), keys.data_ptr(),
                                            perm.data_ptr(), box.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)


def test_noalloc_single_body_nan_then_valid_and_no_device_allocation():
    """One body: h = 0 becomes 1 (the cube of side 2 centred on it), so each
    axis quantises to 2^20 and the key is the digit 7 at level 1. A NaN
    position reports FMM_ERR_NONFINITE; the next valid call succeeds, so the
    error word left in the shared scratch was cleared. Repeated calls leave
    the device's free memory unchanged: nothing is allocated."""
    one = [torch.tensor([v], dtype=torch.float64, device=DEV) for v in (0.25, -1.5, 3.0)]
    keys = torch.empty(4096, dtype=torch.int64, device=DEV)
    perm = torch.empty(4096, dtype=torch.int64, device=DEV)
    box = torch.empty(4, dtype=torch.float64, device=DEV)
    assert _raw_call(*one, keys, perm, box) == 0
    torch.cuda.synchronize()
    assert int(keys[0].item()) == 7 << 60 and int(perm[0].item()) == 0
    assert box.cpu().tolist() == [0.25, -1.5, 3.0, 1.0]
    pos = ics.plummer(4096, 73)[0]
    cols = _cols(pos)
    bad = cols[0].clone()
    bad[100] = float("nan")
    assert _raw_call(bad, cols[1], cols[2], keys, perm, box) == -4
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(DEV)[0]
    for _ in range(3):
        assert _raw_call(*cols, keys, perm, box) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(DEV)[0] == free0
    ref_keys, ref_perm = _solver_tree(pos)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref_keys)
    assert np.array_equal(perm.cpu().numpy(), ref_perm)
