"""The eps x p accuracy grid (Sec. 3.1.1; results Sec. 4.1) on the GPU solver.

On the paper's workload (a Plummer sphere of 1e5 bodies), in FP64 mode and
on a subset of the grid, the solver must show what the paper reports. At
orders p >= 8 the median relative force error is below the tolerance. Along a row of fixed eps the error falls as p grows.
In the lower-left corner (eps <= 1e-13, low p) the MAC opens the tree down
to direct summation, which is more accurate than the high orders. The
reference is the FP64 direct sum, which the parity tests pin to the oracle.
"""
import pytest

import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_02207_gb300 import accuracy_grid  # noqa: E402


def test_grid_reproduces_the_papers_trends():
    n = 100000
    pos, _, m = ics.plummer(n, 6)
    orders, eps_list = [4, 8, 16], [1e-13, 1e-10, 1e-7, 1e-4]
    recs = accuracy_grid.run_grid(pos, m, orders, eps_list, precision="fp64", repeats=1)
    cell = {(r["p"], r["eps"]): r for r in recs}
    for p in (8, 16):
        for eps in eps_list:
            assert cell[(p, eps)]["median"] < eps, (p, eps, cell[(p, eps)]["median"])
    for eps in (1e-7, 1e-4):
        med = [cell[(p, eps)]["median"] for p in orders]
        assert med[0] > med[1] > med[2], (eps, med)
    # the lower-left corner: p = 4 at eps = 1e-13 is all direct summation
    corner = cell[(4, 1e-13)]
    assert corner["n_m2l"] == 0 or corner["p2p_interactions"] > 0.9 * n * (n - 1)
    assert corner["median"] < cell[(16, 1e-13)]["median"]
    # the tail: the 99.99th percentile lies well above the median
    for r in recs:
        assert r["p9999"] >= r["median"] and r["max"] >= r["p9999"]
    # the table helper lays out one row per eps and one column per p
    t = accuracy_grid.table(recs, "median")
    assert t.count("\n") == len(eps_list) + 1
