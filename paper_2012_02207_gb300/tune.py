"""Choose the MAC tolerance eps for a target RMS force error.

For each expansion order p this scans eps (half-decades by default, or the
values given with --eps) from large to small and keeps the largest eps whose RMS relative acceleration error
|a_fmm - a_direct| / |a_direct| (Sec. 3.1.1) over a fixed sample of bodies is
at most the target. The reference is the FP64 direct sum (fmm_direct) at the
sampled bodies. The RMS is dominated by a few large-error bodies, so the
sample should be large (the default is 131072 bodies).

    python -m paper_2012_02207_gb300.tune --out tuned_eps.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

EPS_GRID = [1e-5, 3e-6, 1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9]


def _errors(acc, ref):
    import torch  # noqa: PLC0415
    d = torch.linalg.norm(acc - ref, dim=1) / torch.linalg.norm(ref, dim=1)
    return float(torch.sqrt((d * d).mean())), float(d.median()), float(d.max())


def tune(pos, mass, orders, target=1e-6, precision="mixed", sample=131072, seed=0, leaf_size=64, steps=3,
         grid=EPS_GRID):
    """Return {p: {"eps", "rms", "median", "max", "ms"}} for each order."""
    import torch  # noqa: PLC0415

    from . import FMM  # noqa: PLC0415

    dev = torch.device("cuda:0")
    n = len(mass)
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), device=dev) for d in range(3)]
    mt = torch.tensor(np.ascontiguousarray(mass), device=dev)
    idx = torch.tensor(np.sort(np.random.default_rng(seed).choice(n, min(sample, n), replace=False)), device=dev)
    ref = FMM(p=4)
    dax, day, daz, _ = ref.direct(*cols, mt, targets=idx)
    dref = torch.stack([dax, day, daz], 1)
    out = {}
    for p in orders:
        best = None
        for eps in sorted(grid, reverse=True):
            f = FMM(p=p, eps=eps, leaf_size=leaf_size, precision=precision)
            res = f.solve(*cols, mt)
            ts = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                res = f.solve(*cols, mt)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            rms, med, mx = _errors(torch.stack(res[:3], 1)[idx], dref)
            rec = {"eps": eps, "rms": rms, "median": med, "max": mx, "ms": min(ts)}
            print(f"p={p} eps={eps:.3g} {precision} rms={rms:.3e} median={med:.3e} max={mx:.3e} ms={min(ts):.2f}",
                  flush=True)
            if rms <= target:
                best = rec
                break
        out[p] = best
    return out


def full_rms(pos, mass, p, eps, precision="mixed", leaf_size=64, chunk=1 << 17):
    """RMS relative acceleration error over ALL bodies against the FP64
    direct sum (O(N^2): about a minute at N = 2^20 on one GPU)."""
    import torch  # noqa: PLC0415

    from . import FMM  # noqa: PLC0415
    dev = torch.device("cuda:0")
    n = len(mass)
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), device=dev) for d in range(3)]
    mt = torch.tensor(np.ascontiguousarray(mass), device=dev)
    acc = torch.stack(FMM(p=p, eps=eps, leaf_size=leaf_size, precision=precision).solve(*cols, mt)[:3], 1)
    ref = FMM(p=4)
    s2 = 0.0
    for s in range(0, n, chunk):
        idx = torch.arange(s, min(n, s + chunk), device=dev, dtype=torch.int64)
        ax, ay, az, _ = ref.direct(*cols, mt, targets=idx)
        d = torch.stack([ax, ay, az], 1)
        e = torch.linalg.norm(acc[s:s + chunk] - d, dim=1) / torch.linalg.norm(d, dim=1)
        s2 += float((e * e).sum())
    return (s2 / n) ** 0.5


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import ics  # noqa: PLC0415

    ap = argparse.ArgumentParser()
    ap.add_argument("--orders", default="6,8,10,12,14")
    ap.add_argument("--target", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--sample", type=int, default=131072)
    ap.add_argument("--eps", default=None, help="comma-separated eps values to scan (default: half-decades)")
    ap.add_argument("--verify-full", action="store_true",
                    help="also measure the chosen configurations' RMS over all bodies")
    ap.add_argument("--leaf", default="64", help="comma-separated leaf sizes to scan")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    grid = [float(x) for x in args.eps.split(",")] if args.eps else EPS_GRID
    pos, m = ics.config_inputs("kroupa1m")
    by_leaf = {}
    for leaf in [int(x) for x in args.leaf.split(",")]:
        print(f"leaf size {leaf}", flush=True)
        res = tune(pos, m, [int(x) for x in args.orders.split(",")], args.target, args.precision, args.sample,
                   leaf_size=leaf, grid=grid)
        if args.verify_full:
            for p_, rec in res.items():
                if rec:
                    rec["rms_all_bodies"] = full_rms(pos, m, p_, rec["eps"], args.precision, leaf_size=leaf)
                    print(f"p={p_} leaf={leaf} eps={rec['eps']:.3g} rms over all bodies "
                          f"{rec['rms_all_bodies']:.3e}", flush=True)
        by_leaf[leaf] = res
    # the fastest (leaf, p) whose sample RMS met the target
    ok = [(rec["ms"], leaf, p_) for leaf, res in by_leaf.items() for p_, rec in res.items() if rec]
    fastest = min(ok) if ok else None
    doc = {"workload": "plummer_kroupa_n1048576 (positions seed 2, Kroupa masses seed 3)",
           "target_rms": args.target, "precision": args.precision, "sample": args.sample,
           "reference": "FP64 direct sum at the sampled bodies"}
    if len(by_leaf) == 1:
        doc["leaf_size"] = next(iter(by_leaf))
        doc["orders"] = {str(k): v for k, v in next(iter(by_leaf.values())).items()}
    else:
        doc["by_leaf"] = {str(lf): {str(k): v for k, v in res.items()} for lf, res in by_leaf.items()}
    if fastest:
        doc["fastest"] = {"leaf_size": fastest[1], "p": fastest[2], "ms": fastest[0]}
    text = json.dumps(doc, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")


if __name__ == "__main__":
    main()
