"""Global-step kick-drift-kick leapfrog around the force solve.

This is a measurement driver, not the paper's integrator (the paper uses a
HOLD hierarchical individual-time-step scheme, Appendix A). It steps a
cluster with a fixed time step, calls one FMM force solve per step, and
reports the relative energy error |E(t) - E0| / |E0| with
E = sum_i m_i v_i^2 / 2 + sum_i m_i phi_i / 2 (the energy bookkeeping of
Sec. 4.2).

    python -m paper_2012_02207_gb300.leapfrog --n 8388608 --steps 100 --dt 0.0009765625
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def energy(v, m, pot):
    """Kinetic plus potential energy (pot = phi_i without the 1/2)."""
    import torch  # noqa: PLC0415
    return float((0.5 * m * (v * v).sum(1)).sum() + 0.5 * (m * pot).sum())


def integrate(fmm, pos, vel, mass, dt, steps, callback=None, direct=False):
    """KDK leapfrog in place on device tensors pos (n,3), vel (n,3), mass (n,).
    direct=True takes the forces from the FP64 direct sum instead of the FMM.

    Returns the list of energies at steps 0..steps."""
    import torch  # noqa: PLC0415

    def forces(cols):
        return fmm.direct(*cols, mass) if direct else fmm.solve(*cols, mass)
    cols = [pos[:, d].contiguous() for d in range(3)]
    ax, ay, az, pot = forces(cols)
    acc = torch.stack([ax, ay, az], 1)
    energies = [energy(vel, mass, pot)]
    for s in range(steps):
        vel += 0.5 * dt * acc
        pos += dt * vel
        cols = [pos[:, d].contiguous() for d in range(3)]
        ax, ay, az, pot = forces(cols)
        acc = torch.stack([ax, ay, az], 1)
        vel += 0.5 * dt * acc
        energies.append(energy(vel, mass, pot))
        if callback:
            callback(s + 1, energies[-1])
    return energies


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np  # noqa: PLC0415
    import torch  # noqa: PLC0415

    import ics  # noqa: PLC0415

    from . import FMM  # noqa: PLC0415

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8388608)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--dt", type=float, default=1.0 / 1024)
    ap.add_argument("--p", type=int, default=12)
    ap.add_argument("--eps", type=float, default=2e-8, help="MAC tolerance (the tuned value for p = 12 at N = 2^20)")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--bh-mass", type=float, default=0.01, help="central point mass (0: a plain Plummer sphere)")
    ap.add_argument("--forces", default="fmm", choices=["fmm", "direct"],
                    help="force solve: the mixed-precision FMM, or the FP64 direct sum (O(N^2), a reference)")
    ap.add_argument("--soft", type=float, default=0.0,
                    help="Plummer softening length (Appendix B uses 1/N); 0: Newtonian")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    if args.bh_mass > 0:
        pos, vel, m = ics.nucleus(args.n, args.seed, bh_mass=args.bh_mass)
    else:
        pos, vel, m = ics.plummer(args.n, args.seed)
    dev = torch.device("cuda:0")
    P = torch.tensor(pos, device=dev)
    V = torch.tensor(vel, device=dev)
    M = torch.tensor(m, device=dev)
    fmm = FMM(p=args.p, eps=args.eps, precision=args.precision, soft=args.soft)
    t0 = time.perf_counter()
    es = integrate(fmm, P, V, M, args.dt, args.steps, direct=args.forces == "direct")
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    drift = [abs(e - es[0]) / abs(es[0]) for e in es]
    name = f"nucleus_plummer_n{args.n}_plus_point_mass_{args.bh_mass:g}" if args.bh_mass > 0 else f"plummer_n{args.n}"
    print(json.dumps({"workload": name, "n_bodies": len(m), "forces": args.forces, "p": args.p,
                      "eps": args.eps, "soft": args.soft, "precision": args.precision, "dt": args.dt,
                      "steps": args.steps, "E0": es[0], "E_final": es[-1],
                      "max_rel_energy_error": max(drift), "final_rel_energy_error": drift[-1],
                      "wall_s": wall, "solves_per_s": (args.steps + 1) / wall}))


if __name__ == "__main__":
    main()
