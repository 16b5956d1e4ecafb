"""Benchmark: particles/s of one FMM force solve at N = 2^20.

Workload (Mukherjee et al. 2021 method; synthetic inputs standing in for the
paper's MCLUSTER Plummer models): Plummer sphere, N = 1,048,576, Henon units,
seed 2, Kroupa IMF masses (seed 3) renormalised to M = 1; mixed precision,
expansion order p and MAC tolerance eps chosen so that the RMS relative
acceleration error against the FP64 direct sum is <= 1e-6; leaf size 64. The
same solve in FP64 mode runs beside it for the mixed-vs-FP64 comparison.

One step = one complete force solve (tree build included) on inputs already
resident in HBM. The inputs (32 MB) fit in L2, so L2 is flushed before every
timed solve by writing a 512 MB buffer; the flush is outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbfmm|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_BODIES = 1 << 20
# fastest tuned configurations (paper_2012_02207_gb300/tuned_eps.json): per precision, the order and
# the largest eps whose RMS over all 2^20 bodies is <= 9e-7 (mixed: 8.3e-7, FP64: 7.5e-7)
P_DEFAULT = 10
EPS_DEFAULT = 2.8e-8
P_FP64 = 12
EPS_FP64 = 4e-8
LEAF = 64
SAMPLE_N = 1 << 16          # bounded CPU sample for the oracle timings
METRIC = "particles/s per FMM force solve at N=1e6: mixed vs FP64 at RMS err<=1e-6"
# config 3's orders, each at its tuned eps (paper_2012_02207_gb300/tuned_eps.json, mixed precision)
CONFIG3_ORDERS = (6, 10, 14)
# config 4 (the ensemble of 256 clusters): the autotuner's pick over all clusters
ENSEMBLE_PICK = {"leaf": 128, "p": 12, "eps": 3e-8}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def tuned_eps(p, precision="mixed"):
    with open(os.path.join(ROOT, "paper_2012_02207_gb300", "tuned_eps.json")) as fh:
        return json.load(fh)[precision][str(p)]["eps"]


def measured_fma_peaks(gb, local):
    """FP32 and FP64 FMA throughput of this GPU (fmm_fma_peak: independent FMA
    chains on every lane, about 200 ms per launch), with the SM clock sampled
    while they run."""
    import ctypes  # noqa: PLC0415

    import torch  # noqa: PLC0415
    L = gb.lib()
    out = {}
    with ClockSampler(local) as clk:
        for name, prec in (("fp32", gb.FMM_PRECISION_MIXED), ("fp64", gb.FMM_PRECISION_FP64)):
            v = ctypes.c_double()
            rc = L.fmm_fma_peak(prec, 200.0, ctypes.byref(v), torch.cuda.current_stream().cuda_stream)
            if rc != 0:
                raise gb.FmmError(rc, L.fmm_last_error(None).decode())
            out[name] = v.value
    out["clocks"] = clk.summary()
    return out


def m2l_flops(p):
    """Algorithmic flops of one directed rotation-accelerated M2L at order p,
    counting a linear combination of t non-zero terms as t multiplies and
    t - 1 adds: four z-rotations (the powers of e^{i angle} and a complex
    product on every m >= 1 coefficient), four swaps (the cosine and sine
    blocks' non-zero entries by parity; the swap right after the
    z-translation only over its non-zero inputs, F'_n^m with m <= p - n), the
    z-translation (the powers of u and v, u^k times each input, one
    combination per output and its scale) and the accumulation of the
    (p+1)^2 result."""
    def lin(t):
        return 2 * t - 1 if t > 0 else 0

    rot = sum(6 + 6 * (p - m + 1) for m in range(1, p + 1))

    def swap(after_z):
        f = 0
        for n in range(1, p + 1):
            jmax = min(n, p - n) if after_z else n
            f += sum(lin(sum(1 for j in range(jmax + 1) if (j + m + n) % 2 == 0)) for m in range(n + 1))
            f += sum(lin(sum(1 for j in range(1, jmax + 1) if (j + m + n) % 2 == 1)) for m in range(1, n + 1))
        return f
    trans = 2 * p
    for m in range(p + 1):
        parts = 2 if m else 1
        trans += parts * (p - m + 1)
        for n in range(m, p + 1):
            t = max(0, p - n - m + 1)
            trans += parts * (lin(t) + (1 if t else 0))
    return 4 * rot + 3 * swap(False) + swap(True) + trans + (p + 1) ** 2


P2P_FLOPS = 20  # per directed body-body interaction (the usual gravity-kernel count)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(name):
    """DRAM bytes per launch of a kernel from an ncu capture summarised in
    profiles/traffic.json, or None when the kernel's sources have changed
    since the capture (their hash no longer matches) or there is none."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(name)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for rel in rec["files"]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest() == rec["sources_sha256"] else None


def workload():
    import ics
    pos, m = ics.config_inputs("kroupa1m")
    return pos, m


def cpu_sample(p, eps):
    """The oracle FMM on a bounded sample of the same workload."""
    import ics
    import oracle
    pos, _, _ = ics.plummer(SAMPLE_N, 2)
    m = ics.kroupa_masses(SAMPLE_N, 3)
    t0 = time.perf_counter()
    oracle.fmm(pos, m, p=p, eps=eps, leaf_size=LEAF)
    dt = time.perf_counter() - t0
    return SAMPLE_N / dt, dt, oracle.num_threads()


def replica_throughput(ms_local, n, world, dist=None, device=None):
    """Whole-job throughput of N independent replicas (one per rank): every
    rank solved n bodies; the job takes as long as the slowest rank.
    Returns (particles/s over all ranks, the max ms over ranks)."""
    ms = ms_local
    if dist is not None:
        import torch  # noqa: PLC0415
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return n * world / (ms * 1e-3), ms


def arm_config(p, eps, world):
    """The GPU arm's workload: the 2^20-body Plummer/Kroupa solve."""
    return {"workload": "plummer_kroupa_n1048576_mixed", "n": 1 << 20, "p": p, "eps": eps, "leaf_size": LEAF,
            "precision": "mixed", "l2": "flushed (512 MB write) before each step", "parallelism": f"replicas{world}"}


def reference_config(p, eps, world):
    """The reference arm's workload as it runs: the oracle (about 23 s per
    2^20-body solve on 16 cores) times a 65536-body Plummer/Kroupa sphere drawn
    like the GPU arm's, so that --steps K --warmup W ends within minutes."""
    return {"workload": f"plummer_kroupa_n{SAMPLE_N}_oracle_sample", "n": SAMPLE_N, "p": p, "eps": eps,
            "leaf_size": LEAF, "precision": "fp64", "sample_of": "plummer_kroupa_n1048576_mixed",
            "parallelism": f"replicas{world}"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, eps = args.p, args.eps
    for _ in range(args.warmup):
        cpu_sample(p, eps)
    vals, times = [], []
    cores = 1
    for _ in range(args.steps):
        v, dt, cores = cpu_sample(p, eps)
        vals.append(v)
        times.append(dt)
    value = SAMPLE_N * len(times) / sum(times)
    # the same solve once on a single core, beside the all-core figure
    import oracle  # noqa: PLC0415
    oracle.set_num_threads(1)
    v1, dt1, _ = cpu_sample(p, eps)
    oracle.set_num_threads(cores)
    sample = (f"oracle FMM (FP64, OpenMP) per step on a Plummer sphere of N={SAMPLE_N} drawn like the workload "
              f"(positions seed 2, Kroupa masses seed 3), p={p}, eps={eps}")
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": reference_config(p, eps, world),
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "value_1_core": v1, "ms_1_core": 1e3 * dt1},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_table():
    """Oracle timings on this host at configs 1-3 (all cores, and one core for
    configs 1 and 3), plus the FP64 direct sum's rate at N = 2^20 from 2048
    sampled targets (N^2 pair interactions would take about an hour)."""
    import platform  # noqa: PLC0415

    import ics  # noqa: PLC0415
    import oracle  # noqa: PLC0415
    cores = oracle.num_threads()
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines() if ln.startswith("Model name")), "")
    except OSError:
        pass
    rows = []

    def time_fmm(name, pos, m, p, eps, threads):
        oracle.set_num_threads(threads)
        t0 = time.perf_counter()
        oracle.fmm(pos, m, p=p, eps=eps, leaf_size=LEAF)
        dt = time.perf_counter() - t0
        rows.append({"row": name, "n": len(m), "p": p, "eps": eps, "threads": threads, "s": dt,
                     "particles_per_s": len(m) / dt})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)

    pos1, m1 = ics.config_inputs("plummer4k")
    time_fmm("config1 oracle FMM", pos1, m1, 8, 1e-7, cores)
    time_fmm("config1 oracle FMM", pos1, m1, 8, 1e-7, 1)
    pos2, m2 = ics.config_inputs("plummer1m")
    time_fmm("config2 oracle FMM (equal masses)", pos2, m2, P_FP64, EPS_FP64, cores)
    pos3, m3 = ics.config_inputs("kroupa1m")
    time_fmm("config3 oracle FMM (Kroupa masses)", pos3, m3, P_DEFAULT, EPS_DEFAULT, cores)
    time_fmm("config3 oracle FMM (Kroupa masses)", pos3, m3, P_DEFAULT, EPS_DEFAULT, 1)
    oracle.set_num_threads(cores)
    tg = np.sort(np.random.default_rng(0).choice(len(m3), 2048, replace=False))
    t0 = time.perf_counter()
    oracle.direct(pos3, m3, targets=tg)
    dt = time.perf_counter() - t0
    pairs_per_s = len(tg) * (len(m3) - 1) / dt
    rows.append({"row": "FP64 direct sum, N = 2^20", "threads": cores, "sampled_targets": len(tg), "s": dt,
                 "pair_interactions_per_s": pairs_per_s,
                 "full_solve_s_extrapolated": len(m3) * (len(m3) - 1) / pairs_per_s})
    print(json.dumps({"cpu_model": model, "machine": platform.machine(), "cores": cores, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbfmm", choices=["gbfmm", "reference"])
    ap.add_argument("--p", type=int, default=P_DEFAULT)
    ap.add_argument("--eps", type=float, default=EPS_DEFAULT)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--p64", type=int, default=P_FP64)
    ap.add_argument("--eps64", type=float, default=EPS_FP64)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the config-3 orders, the ensemble and the FMA peaks (profiling runs)")
    ap.add_argument("--err-sample", type=int, default=0,
                    help="bodies in the force-error check (0: all bodies)")
    ap.add_argument("--p2p-loads", action="store_true",
                    help="stage the P2P sources by per-lane loads (FMM_FLAG_P2P_LOADS) instead of bulk copies")
    ap.add_argument("--cpu-table", action="store_true",
                    help="only time the oracle at configs 1-3 on this host and print one JSON line")
    args = ap.parse_args()
    if args.cpu_table:
        cpu_table()
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import paper_2012_02207_gb300 as gb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = dist_mod

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    pos, m = workload()
    n = len(m)
    cols = [torch.tensor(np.ascontiguousarray(pos[:, d]), device=dev) for d in range(3)]
    mt = torch.tensor(m, device=dev)
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed_solves(solver, steps, warmup):
        for _ in range(warmup):
            solver.solve(*cols, mt, out=outs)
        barrier()
        times, stats = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(*cols, mt, out=outs)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(solver.stats())
        barrier()
        return times, stats

    mixed = gb.FMM(p=args.p, eps=args.eps, leaf_size=LEAF, precision="mixed", p2p_bulk=not args.p2p_loads)
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        times, stats = timed_solves(mixed, args.steps, args.warmup)
        wall = time.perf_counter() - wall0
    clocks = clk.summary()
    value, ms = replica_throughput(sum(times) / len(times), n, world, dist, dev)

    # accuracy of this exact run over ALL bodies against the FP64 direct sum on
    # the GPU (O(N^2), about half a minute at N = 2^20; untimed). The RMS is
    # dominated by a few outliers, so a sample of bodies can miss or catch them.
    if args.err_sample > 0:
        rng = np.random.default_rng(0)
        sample = torch.tensor(np.sort(rng.choice(n, min(args.err_sample, n), replace=False)), device=dev)
    else:
        sample = torch.arange(n, device=dev)
    dref = torch.empty(len(sample), 3, dtype=torch.float64, device=dev)
    for c0 in range(0, len(sample), 1 << 17):
        sl = slice(c0, min(len(sample), c0 + (1 << 17)))
        dax, day, daz, _ = mixed.direct(*cols, mt, targets=sample[sl])
        dref[sl] = torch.stack([dax, day, daz], 1)

    def err_stats(ax, ay, az):
        a = torch.stack([ax, ay, az], 1)[sample]
        d = torch.linalg.norm(a - dref, dim=1) / torch.linalg.norm(dref, dim=1)
        q = torch.quantile(d.float(), torch.tensor([0.99, 0.9999], device=dev)).tolist() if len(d) <= 1 << 24 else [None, None]
        return {"rms": float(torch.sqrt((d * d).mean()).item()), "median": float(d.median().item()),
                "p99": q[0], "p9999": q[1], "max": float(d.max().item())}

    mixed.solve(*cols, mt, out=outs)
    e_mixed = err_stats(*outs[:3])

    # FP64 mode on the same inputs (slow; a few steps)
    fp64 = gb.FMM(p=args.p64, eps=args.eps64, leaf_size=LEAF, precision="fp64")
    t64, s64 = timed_solves(fp64, args.fp64_steps, 1)
    ms64 = sum(t64) / len(t64)
    e64 = err_stats(*outs[:3])
    value64 = n / (ms64 * 1e-3)

    # end to end through the host entry point (pinned host buffers)
    hin = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(4)]
    for h, c in zip(hin, cols + [mt]):
        h.copy_(c.cpu())
    hout = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(4)]
    L = gb.lib()
    e2e_times = []
    for i in range(args.warmup + max(3, args.steps // 2)):
        barrier()
        t0 = time.perf_counter()
        rc = L.fmm_solve_host(mixed._h, n, *[h.data_ptr() for h in hin], *[o.data_ptr() for o in hout],
                              stream.cuda_stream)
        t1 = time.perf_counter()
        if rc != 0:
            raise gb.FmmError(rc, L.fmm_last_error(mixed._h).decode())
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_value = n * world / (sum(e2e_times) / len(e2e_times))

    extras = {}
    if not args.no_extras:
        # config 3 at its three orders, each at its tuned eps: time and error over all bodies
        c3 = {}
        for p3 in CONFIG3_ORDERS:
            eps3 = tuned_eps(p3)
            f3 = gb.FMM(p=p3, eps=eps3, leaf_size=LEAF, precision="mixed")
            t3, s3 = timed_solves(f3, 3, 1)
            c3[str(p3)] = {"eps": eps3, "ms_per_solve": statistics.median(t3),
                           "particles_per_s": n / (statistics.median(t3) * 1e-3), **err_stats(*outs[:3])}
            del f3
        extras["config3_orders"] = c3
        # config 3 as written: FP64 coefficients (M2L, L2L, L2P in FP64) with the FP32 P2P, same p and eps
        f64l = gb.FMM(p=args.p, eps=args.eps, leaf_size=LEAF, precision="mixed", fp64_locals=True)
        tl, sl = timed_solves(f64l, 2, 1)
        extras["config3_fp64_locals"] = {
            "p": args.p, "eps": args.eps, "ms_per_solve": statistics.median(tl),
            "particles_per_s": n / (statistics.median(tl) * 1e-3), **err_stats(*outs[:3]),
            "phases_ms": {k: sl[-1][k] for k in ("ms_m2l", "ms_downward", "ms_leaf", "ms_total")}}
        del f64l
        # config 4: the 256-cluster ensemble as one forest at the autotuner's pick
        from paper_2012_02207_gb300.ensemble import Ensemble, pick_staging  # noqa: PLC0415
        import ics  # noqa: PLC0415
        offsets, epos, emass, _, _ = ics.ensemble(256, 4)
        ens = Ensemble(offsets, epos, emass, sample=512)
        pick, staging_ms = pick_staging(ens, ENSEMBLE_PICK, log=lambda s: None)
        bulk = pick["p2p_staging"] == "bulk"
        fe = gb.FMM(p=pick["p"], eps=pick["eps"], leaf_size=pick["leaf"], precision="mixed", p2p_bulk=bulk)
        eout, ems = ens.time_batch(fe, steps=5)
        erms = ens.errors(eout)
        ge = gb.FMM(p=pick["p"], eps=pick["eps"], leaf_size=pick["leaf"], precision="mixed", p2p_bulk=bulk)
        _, ems_graph, replayed = ens.time_graph(ge)
        extras["config4_ensemble"] = {
            "clusters": 256, "n_bodies": ens.n, **ENSEMBLE_PICK, "p2p_staging": pick["p2p_staging"],
            "staging_ms": staging_ms, "forest_ms": ems,
            "forest_particles_per_s": ens.n / (ems * 1e-3), "graph_replay_ms_host": ems_graph,
            "graph_replayed": replayed, "kernel_launches": fe.stats()["kernel_launches"],
            "worst_cluster_rms": float(erms.max()), "median_cluster_rms": float(np.median(erms)),
            "error_sample": "512 bodies per cluster (all bodies of smaller clusters) against the FP64 direct sum"}
        del ens, fe, ge, eout
        torch.cuda.empty_cache()

    # roofline of the dominant phase: the FP32 pipe in mixed precision, against
    # the FP32 FMA throughput measured on this GPU in this run
    st = stats[-1]
    p = args.p
    phase_ms = {"m2l": statistics.median(s["ms_m2l"] for s in stats),
                "leaf_p2p_l2p": statistics.median(s["ms_leaf"] for s in stats)}
    flops = {"m2l": 2 * st["n_m2l"] * m2l_flops(p), "leaf_p2p_l2p": P2P_FLOPS * st["p2p_interactions"]}
    dom = max(phase_ms, key=phase_ms.get)
    peaks = measured_fma_peaks(gb, local)
    peak = peaks["fp32"]
    achieved = flops[dom] / (phase_ms[dom] * 1e-3) / 1e12
    # P2P by the method's count: mutual pair interactions (Newton's third law, Sec. 2.3)
    p2p_mutual = P2P_FLOPS * st["p2p_interactions"] / 2 / (phase_ms["leaf_p2p_l2p"] * 1e-3) / 1e12

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, cores = cpu_sample(p, args.eps)
        cpu = {"value": v, "unit": "particles/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle FMM (FP64, OpenMP) on one Plummer/Kroupa solve of N={SAMPLE_N} drawn like the "
                         f"workload (positions seed 2, masses seed 3), p={p}, eps={args.eps}: {dt:.2f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": arm_config(p, args.eps, world),
            "fp64": {"value": value64, "ms_per_step": ms64, "steps": args.fp64_steps, "rms_err": e64["rms"],
                     "median_err": e64["median"], "p": args.p64, "eps": args.eps64,
                     "phases_ms": {k: s64[-1][k] for k in ("ms_tree", "ms_upward", "ms_estimate", "ms_walk",
                                                          "ms_m2l", "ms_downward", "ms_leaf", "ms_total")}},
            "speedup_vs_fp64": value / value64,
            "rms_err": e_mixed["rms"], "median_err": e_mixed["median"], "err_stats": e_mixed,
            "err_bodies": int(len(sample)),
            "phases_ms": {k: statistics.median(s[k] for s in stats) for k in
                          ("ms_tree", "ms_upward", "ms_estimate", "ms_walk", "ms_m2l", "ms_downward", "ms_leaf",
                           "ms_total")},
            "counts": {k: st[k] for k in ("nnodes", "nlevels", "n_far", "n_near", "n_m2l", "n_p2p",
                                          "p2p_interactions", "walk_iters")},
            "roofline": {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": kernel_traffic(dom),
                         "peak_note": "FP32 FMA throughput measured in this run (fmm_fma_peak) at SM clock "
                                      f"{peaks['clocks'].get('sm_mhz')} MHz"},
            "roofline_p2p_mutual": {"achieved": p2p_mutual, "peak": peak, "unit": "TFLOP/s",
                                    "frac": p2p_mutual / peak,
                                    "note": "leaf phase (P2P + L2P) by the method's count: 20 flops per mutual pair"},
            "measured_peaks": {"fp32_tflops": peaks["fp32"], "fp64_tflops": peaks["fp64"],
                               "clocks": peaks["clocks"]},
            "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": 32 * n,
                    "d2h_bytes_per_step": 32 * n},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clocks, "wall_s_timed": wall,
            "cpu_baseline": cpu, **extras,
        }), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
