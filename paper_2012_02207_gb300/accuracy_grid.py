"""Force-error and timing grid over the MAC tolerance eps and the order p.

The paper's accuracy study (Sec. 3.1.1, results in Sec. 4.1, timing heat
maps in Sec. 4.4) solves one Plummer sphere of 1e5 bodies for every (eps, p)
of a grid. For each solve it reports the distribution of the relative force
error |a_direct - a_fmm| / |a_direct|: median, 99th and 99.99th percentiles,
RMS and maximum. It also reports the time of the force solve (the "Poisson
step").

This module runs that grid with the GPU solver. The reference forces are the
FP64 direct sum over all bodies (fmm_direct). Times are CUDA-event times of
one complete solve, tree build included, the minimum over a few repeats.
Besides the error statistics, each cell records the list sizes and the P2P
interaction count. These show where a small eps opens the tree down to
direct summation.

    python -m paper_2012_02207_gb300.accuracy_grid --precision fp64 --out grid.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

EPS_DECADES = [10.0 ** -k for k in range(13, 2, -1)]  # 1e-13 .. 1e-3
ORDERS = [4, 6, 8, 10, 12, 14, 16, 18, 20]


def error_stats(acc, ref):
    """Median, 99th and 99.99th percentiles, RMS and max of |a - a_ref| / |a_ref|."""
    import torch  # noqa: PLC0415
    d = torch.linalg.norm(acc - ref, dim=1) / torch.linalg.norm(ref, dim=1)
    q = torch.quantile(d.double().cpu(), torch.tensor([0.5, 0.99, 0.9999], dtype=torch.float64)).tolist()
    return {"median": q[0], "p99": q[1], "p9999": q[2], "rms": float(torch.sqrt((d * d).mean())),
            "max": float(d.max())}


def run_grid(pos, mass, orders, eps_list, precision="fp64", leaf_size=64, repeats=3, log=None):
    """Solve once per (p, eps); return a list of per-cell records."""
    import torch  # noqa: PLC0415

    from . import FMM  # noqa: PLC0415

    dev = torch.device("cuda:0")
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), device=dev) for d in range(3)]
    mt = torch.tensor(np.ascontiguousarray(mass), device=dev)
    dax, day, daz, _ = FMM(p=4).direct(*cols, mt)
    ref = torch.stack([dax, day, daz], 1)
    out = []
    for p in orders:
        for eps in eps_list:
            f = FMM(p=p, eps=eps, leaf_size=leaf_size, precision=precision)
            res = f.solve(*cols, mt)
            ts = []
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                res = f.solve(*cols, mt)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            st = f.stats()
            rec = {"p": p, "eps": eps, "precision": precision, "ms": min(ts),
                   "n_m2l": st["n_m2l"], "n_p2p": st["n_p2p"], "p2p_interactions": st["p2p_interactions"],
                   "nnodes": st["nnodes"]}
            rec.update(error_stats(torch.stack(res[:3], 1), ref))
            out.append(rec)
            if log:
                log(f"p={p:2d} eps={eps:.0e} median={rec['median']:.2e} p99={rec['p99']:.2e} "
                    f"p99.99={rec['p9999']:.2e} rms={rec['rms']:.2e} max={rec['max']:.2e} ms={rec['ms']:.2f} "
                    f"p2p/N^2={rec['p2p_interactions'] / float(len(mass)) ** 2:.3f}")
    return out


def table(records, key, fmt="{:.1e}"):
    """Markdown heat-map table of one statistic: rows eps, columns p."""
    orders = sorted({r["p"] for r in records})
    eps_list = sorted({r["eps"] for r in records})
    cell = {(r["p"], r["eps"]): r[key] for r in records}
    lines = ["| eps \\ p | " + " | ".join(str(p) for p in orders) + " |",
             "|---" * (len(orders) + 1) + "|"]
    for e in eps_list:
        vals = [fmt.format(cell[(p, e)]) if (p, e) in cell else "" for p in orders]
        lines.append(f"| {e:.0e} | " + " | ".join(vals) + " |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--seed", type=int, default=6)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--orders", type=int, nargs="*", default=None)
    ap.add_argument("--eps", type=float, nargs="*", default=None)
    ap.add_argument("--leaf-size", type=int, default=64)
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import ics  # noqa: PLC0415

    pos, _, mass = ics.plummer(a.n, a.seed)
    orders = a.orders or [p for p in ORDERS if a.precision == "fp64" or p <= 16]
    eps_list = a.eps or EPS_DECADES
    recs = run_grid(pos, mass, orders, eps_list, a.precision, a.leaf_size, a.repeats,
                    log=lambda s: print(s, flush=True))
    for key, title in [("median", "median"), ("p9999", "99.99th percentile"), ("ms", "solve time, ms")]:
        print(f"\n{title} ({a.precision}, N = {a.n})\n")
        print(table(recs, key, "{:.2f}" if key == "ms" else "{:.1e}"))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump({"n": a.n, "seed": a.seed, "leaf_size": a.leaf_size, "records": recs}, fh, indent=1)
    bad = [r for r in recs if not all(math.isfinite(r[k]) for k in ("median", "rms", "max"))]
    return 1 if bad else 0


if __name__ == "__main__":
    raise SystemExit(main())
