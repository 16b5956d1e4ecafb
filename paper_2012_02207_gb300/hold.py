"""Energy test of the HOLD integrator (Appendix A) on the GPU.

Appendix A of the paper integrates ten N = 100 Plummer models for 50 N-body
time units and finds that the time-symmetrized step size conserves energy
better than the plain one. This driver repeats that test with `fmm_hold`:
per realization and step-size rule, it reports the relative energy error
|E(t) - E0| / |E0| once per time unit, its maximum and its final value, and
the wall time. Forces come from the FP64 direct sum below --direct-below
bodies per set and from the FMM above (the latter for large N).

    python -m paper_2012_02207_gb300.hold                                      # 3 models, 10 units
    python -m paper_2012_02207_gb300.hold --realizations 10 --t-end 50         # the paper's setting

At N = 100 the GPU run is bound by launch and round-trip latency (about 2 s
per time unit and model), so the paper's full setting takes about half an
hour.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def energy(fmm, X, V, M, direct=True):
    """Kinetic plus potential energy (the potential from the direct sum or the
    FMM solve, each body's pair terms counted once)."""
    pot = fmm.direct(*X, M)[3] if direct else fmm.solve(*X, M)[3]
    ek = 0.5 * (M * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2])).sum()
    return float(ek + 0.5 * (M * pot).sum())


def run(pos, vel, mass, t_end, dt, eta, sym, soft, direct_below, p, eps, device_below=1024):
    import torch  # noqa: PLC0415

    from . import FMM  # noqa: PLC0415
    dev = torch.device("cuda:0")
    X = [torch.tensor(pos[:, d].copy(), dtype=torch.float64, device=dev) for d in range(3)]
    V = [torch.tensor(vel[:, d].copy(), dtype=torch.float64, device=dev) for d in range(3)]
    M = torch.tensor(mass, dtype=torch.float64, device=dev)
    f = FMM(p=p, eps=eps, precision="fp64", soft=soft)
    direct = len(mass) <= 65536
    E0 = energy(f, X, V, M, direct)
    steps_per_unit = int(round(1.0 / dt))
    errs, totals = [], {}
    t0 = time.perf_counter()
    for _ in range(int(round(t_end))):
        st = f.hold(*X, *V, M, dt, steps_per_unit, eta=eta, symmetrize=sym, dt_min=1e-9, direct_below=direct_below,
                    device_below=device_below)
        for k, v in st.items():
            totals[k] = max(totals.get(k, 0), v) if k == "max_depth" else totals.get(k, 0) + v
        E = energy(f, X, V, M, direct)
        errs.append(abs(E / E0 - 1.0))
    torch.cuda.synchronize()
    return {"E0": E0, "rel_energy_error_per_unit": errs, "max_rel_energy_error": max(errs),
            "final_rel_energy_error": errs[-1], "wall_s": time.perf_counter() - t0, "counters": totals}


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np  # noqa: PLC0415

    import ics  # noqa: PLC0415

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100)
    ap.add_argument("--realizations", type=int, default=3)
    ap.add_argument("--seed", type=int, default=100, help="realization r uses seed + r")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--dt", type=float, default=1.0 / 16, help="top-level step")
    ap.add_argument("--eta", type=float, default=0.025, help="step-size accuracy (Table 1: 0.025)")
    ap.add_argument("--soft", type=float, default=0.0)
    ap.add_argument("--direct-below", type=int, default=4096)
    ap.add_argument("--device-below", type=int, default=1024,
                    help="sets of at most this many bodies evolve inside one GPU block (0: none)")
    ap.add_argument("--p", type=int, default=12)
    ap.add_argument("--eps", type=float, default=1e-10)
    ap.add_argument("--sym", default="both", choices=["both", "on", "off"])
    args = ap.parse_args()
    rules = {"both": [False, True], "on": [True], "off": [False]}[args.sym]
    out = {"n": args.n, "t_end": args.t_end, "dt": args.dt, "eta": args.eta, "soft": args.soft, "runs": {}}
    for sym in rules:
        key = "symmetrized" if sym else "plain"
        runs = []
        for r in range(args.realizations):
            pos, vel, m = ics.plummer(args.n, args.seed + r)
            res = run(pos, vel, m, args.t_end, args.dt, args.eta, sym, args.soft, args.direct_below, args.p,
                      args.eps, args.device_below)
            runs.append(res)
            print(json.dumps({"rule": key, "realization": r, "max": res["max_rel_energy_error"],
                              "final": res["final_rel_energy_error"], "wall_s": res["wall_s"],
                              "counters": res["counters"]}), file=sys.stderr, flush=True)
        out["runs"][key] = {"median_max_rel_energy_error": float(np.median([r["max_rel_energy_error"] for r in runs])),
                            "median_final_rel_energy_error": float(np.median([r["final_rel_energy_error"] for r in runs])),
                            "wall_s": sum(r["wall_s"] for r in runs), "realizations": runs}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
