"""Benchmark: RLT2 dual-ascent iterations/s and size-(n-2) LAPs/s at n = 20.

Workload: single QAP, n = 20, F and D symmetric with zero diagonal and uniform
integers 0..99 (seed 2), B = 0; every iteration solves 144,400 Z-LAPs of size
18, 400 Y-LAPs of size 19 and one X-LAP of size 20 and moves reduced costs over
the 46.8 M-entry z array (374 MB FP64, larger than L2, so no L2 flush is
needed between steps).  A step is one full dual-ascent iteration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the CPU oracle (the plain FP64
C implementation the tests check the GPU against) on the host cores.
Multi-GPU runs are independent replicas (one QAP per rank, no collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1710_03732_gb300 import instances as I  # noqa: E402

METRIC = "RLT2 dual-ascent iters/s and size-(n-2) LAPs/s at n=20, plain vs warm-started"
WORKLOAD = "QAP n=20, F,D symmetric dense uniform 0..99 (seed 2), B=0; S1 dual ascent, canonical duals"
CFG = 3
KERNELS = ["move_y", "move_z", "lap_z", "lap_y", "lap_x", "finalize"]
# FP64 ALU peak: 1.25 TFLOP/s nominal GB300 FP64 = 2 flop per FMA -> 0.625e12
# FP64 instructions (lane-ops) per second over 152 SMs at 2.07 GHz, i.e. about
# 2 FP64 lane-ops per clock per SM; every DADD/DSUB/DMUL/DFMA counts as one op.
FP64_PEAK_GOPS = 625.0
FP64_UNIT = "G FP64 ops/s (one DADD/DSUB/DMUL/DFMA lane = 1 op)"
# 64-bit integer add peak: GB300 retires 128 32-bit integer add lanes per clock
# per SM (measured 127.2 with add.s32) and a 64-bit add is two of them (low
# word, then high word with carry; measured 63.8 add.s64 lanes per clock per
# SM), so 64 lane-ops x 152 SMs x 2.07 GHz.
INT64_PEAK_GOPS = 64 * 152 * 2.07
INT64_UNIT = "G int64 ops/s (one 64-bit add/sub lane = 1 op)"


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# source files that define each profiled kernel (its traffic figure stays valid
# until one of them changes)
KERNEL_SOURCES = {
    "lap_z": ["lap.cu", "rlt2_lap.cuh", "rlt2_internal.h"],
    "move_z": ["rlt2_ascent.cuh", "rlt2_internal.h"],
}


def _code_only(text: str) -> str:
    """The source without comments, trailing blanks and empty lines."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def source_digest(kernel: str) -> str:
    """Digest of the code (comments excluded) of the files that define a kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1710_03732_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_digest(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[3] == want:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to $RLT2_CLOCKS_DIR (kept) or a temporary folder
        import tempfile
        folder = os.environ.get("RLT2_CLOCKS_DIR") or tempfile.mkdtemp(prefix="rlt2_clocks_")
        self.path = os.path.join(folder, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], p[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_step(O, st, prm, out, warm: bool, threads: int):
    """One oracle iteration; with warm, every LAP starts from the previous
    iteration's row duals (Z, Y and X), the start the GPU's `value` uses."""
    w = warm and out is not None
    return O.iterate(st, prm, 1, threads=threads, u0z=out.xi.copy() if w else None,
                     u0y=out.gamma.copy() if w else None, u0x=out.alpha.copy() if w else None)


def cpu_oracle_baseline(inst, iters: int, budget_s: float, warm: bool = True):
    """The CPU oracle as it stands, all host cores (OpenMP over LAPs and z
    classes), warm (previous duals, like `value`) or cold (like `plain_cold`)."""
    import oracle as O
    threads = max(1, O.max_threads() or 1)
    st = O.setup(inst.F, inst.D, inst.B)
    prm = O.params_array()
    t0 = time.perf_counter()
    done = 0
    lbs = []
    out = None
    while done < iters:
        out = oracle_step(O, st, prm, out, warm, threads)
        lbs.append(st.const + out.lb)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done, dt, threads, lbs


def cpu_oracle_detail():
    """The oracle on one core at n = 20 (first 2 iterations) and on all cores at
    n = 30 (first iteration, setup excluded): CPU timings of the method itself,
    bounded to about 20 s."""
    import oracle as O
    threads = max(1, O.max_threads() or 1)
    prm = O.params_array()
    inst20 = I.config(CFG)
    st = O.setup(inst20.F, inst20.D, inst20.B)
    out = oracle_step(O, st, prm, None, True, threads)  # the first (cold) solve, untimed
    t0 = time.perf_counter()
    for _ in range(2):
        out = oracle_step(O, st, prm, out, True, 1)
    one = 2 / (time.perf_counter() - t0)
    del st
    inst30 = I.config(5)
    st = O.setup(inst30.F, inst30.D, inst30.B)
    t0 = time.perf_counter()
    O.iterate(st, prm, 1, threads=threads)
    s30 = time.perf_counter() - t0
    del st
    return {"n20_one_core_iters_per_s": one, "n30_all_cores_s_per_iter": s30, "cores": threads,
            "cpu": cpu_model(),
            "note": "CPU oracle, setup excluded: n = 20 iterations 2-3 warm-started from the previous duals "
                    "on one core; n = 30 the first (cold) iteration on all cores"}


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    inst = I.config(CFG)
    # warm-up iterations are part of the same trajectory; each timed step is one
    # full oracle iteration (144,400 Z-LAPs + 400 Y-LAPs + X-LAP + the moves)
    budget = float(os.environ.get("RLT2_REF_BUDGET_S", "150"))
    import oracle as O
    threads = max(1, O.max_threads() or 1)
    st = O.setup(inst.F, inst.D, inst.B)
    prm = O.params_array()
    out = None  # warm starts from the previous iteration's duals, as the GPU arm's `value`
    for _ in range(args.warmup):
        out = oracle_step(O, st, prm, out, True, threads)
    t0 = time.perf_counter()
    steps = 0
    while steps < args.steps:
        out = oracle_step(O, st, prm, out, True, threads)
        steps += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    value = steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": 20, "iterations": steps, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": threads, "kind": "oracle",
                         "sample": f"{steps} consecutive oracle iterations after {args.warmup} warm-up, every "
                                   f"LAP warm-started from the previous iteration's duals as in the GPU arm's "
                                   f"value (capped at {budget:.0f} s); CPU: {cpu_model()}"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_device_run(R, torch, inst, warm: int, steps: int, warmup: int, barrier, mode: int = 1, pipeline: int = 0,
                     timing: bool = True):
    """`steps` iterations after `warmup`, timed with CUDA events on the context's
    stream every 50 iterations.  timing: also CUDA events around every kernel
    launch (the per-kernel times; iterations are then launched kernel by kernel
    instead of replayed as a graph, so the run itself is a little slower)."""
    prm = R.params(dual_mode=mode, warm=warm, feas_tol=0.0, pipeline=pipeline)
    ctx = R.Context(inst.F, inst.D, inst.B, prm=prm)
    ctx.iterate(warmup)
    s0 = ctx.stats()
    ctx.set_timing(timing)
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # events every 50 iterations: the first and last windows show how the
    # iteration time grows as the costs spread (the paper's observation, Section 5)
    chunk = 50
    marks = [torch.cuda.Event(enable_timing=True)]
    marks[0].record(stream)
    left = steps
    while left > 0:
        k = min(chunk, left)
        ctx.iterate_async(k)
        marks.append(torch.cuda.Event(enable_timing=True))
        marks[-1].record(stream)
        left -= k
    torch.cuda.synchronize()
    barrier()
    ms = marks[0].elapsed_time(marks[-1])
    windows = [(min(chunk, steps - chunk * w), marks[w].elapsed_time(marks[w + 1])) for w in range(len(marks) - 1)]
    s1 = ctx.stats()
    kt = ctx.kernel_times()
    lb, best, ub, _, _, its = ctx.bound()
    ctx.close()
    d = s1 - s0
    return dict(ms=ms, stats=d, kt=kt, lb=lb, best=best, ub=ub, iters=its, T=ctx.T, n=ctx.n, windows=windows,
                warm=warm, mode=mode)


def run_profile_case(args):
    """Minimal commands for ncu captures."""
    import torch
    from paper_1710_03732_gb300 import rlt2 as R
    R.lib()
    if args.profile == "nodes":
        inst = I.config(4)
        lb, _, its, st = R.rlt2_bound_nodes(inst.F, inst.D, inst.partials[:16], args.warmup + args.steps,
                                            prm=R.params(feas_tol=0.0, warm=1))
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "16 nodes of config 4", "iterations": int(its.sum()), "stats": st}))
        return 0
    if args.profile == "train":
        mlp, rows = training_samples(R, torch)
        hist = mlp.fit(args.warmup + args.steps, batch_rows=16384)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "training steps of the H = 256 network, 16,384 rows each",
                          "samples": rows, "steps": args.warmup + args.steps, "loss_last": float(hist[-1])}))
        mlp.close()
        return 0
    if args.profile == "gemm":
        # the training GEMMs at the largest batch one call takes (2^18 rows):
        # forward, loss and backward per call, no update
        mlp, rows = training_samples(R, torch)
        big = 1 << 18
        for _ in range(args.warmup):
            mlp.grad(big)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            mlp.grad(big)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "gradients of the H = 256 network on 262,144 rows per call",
                          "samples": rows, "calls": args.warmup + args.steps,
                          "ms_per_call": e0.elapsed_time(e1) / max(1, args.steps)}))
        mlp.close()
        return 0
    if args.profile in ("n22", "n30"):
        # the root problem of the n=22 grid (config 4's QAP) or the n=30 grid, warm
        # starts, launched kernel by kernel with CUDA events around every launch
        inst = I.config(4 if args.profile == "n22" else 5)
        with R.Context(inst.F, inst.D, inst.B, prm=R.params(dual_mode=1, warm=1, feas_tol=0.0)) as ctx:
            ctx.iterate(args.warmup)
            ctx.set_timing(True)
            hist, got = ctx.iterate(args.steps)
            kt = ctx.kernel_times()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": inst.name, "warm": 1, "iterations": args.warmup + got,
                          "ms_per_iteration": {k: v[0] / max(1, v[1]) for k, v in kt.items() if v[1] > 0}}))
        return 0
    inst = I.config(CFG)
    mlp = None
    warm = 0 if args.profile == "cold" else 1
    if args.profile == "learned":
        mlp = R.Mlp(256)
        mlp.load(os.path.join(ROOT, "paper_1710_03732_gb300", "weights", "warmstart_h256.npz"))
        warm = 2
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(dual_mode=1, warm=warm, feas_tol=0.0)) as ctx:
        if mlp is not None:
            ctx.set_mlp(mlp)
        hist, got = ctx.iterate(args.warmup + args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": WORKLOAD, "warm": warm, "iterations": got, "lb_last": float(hist[got - 1])}))
    return 0


def training_samples(R, torch, ntiles: int = 24000):
    """An H = 256 network with (tile, canonical dual) samples of the n = 20
    workload: 24,000 tiles of iteration 3 with the duals of iteration 2 as the
    previous ones (432,000 rows)."""
    inst = I.config(CFG)
    mlp = R.Mlp(256, seed=5)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0)) as ctx:
        T, m = ctx.T, ctx.n - 2
        ctx.iterate(2)
        prev = torch.empty(T * m, dtype=torch.float64, device="cuda")
        R.rlt2_duals(ctx.ctx, xi=prev, on_device=1)
        ctx.iterate(1)
        D = torch.empty(ctx.E, dtype=torch.float64, device="cuda")
        xi = torch.empty(T * m, dtype=torch.float64, device="cuda")
        R.rlt2_export_state(ctx.ctx, Dhat=D, on_device=1)
        R.rlt2_duals(ctx.ctx, xi=xi, on_device=1)
        mlp.add_samples(D.view(T, m, m)[:ntiles].contiguous(), xi.view(T, m)[:ntiles].contiguous(),
                        prev.view(T, m)[:ntiles].contiguous())
        del D, xi, prev
    return mlp, ntiles * 18


def training_rate(R, torch):
    """AdamW training steps of the H = 256 network (16,384 rows each; forward,
    backward and update, the GEMMs on tcgen05), timed with CUDA events."""
    mlp, rows = training_samples(R, torch)
    H, B = 256, 16384
    mlp.fit(5, batch_rows=B)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 100
    e0.record()
    hist = mlp.fit(steps, batch_rows=B)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    gemm_flop = 2.0 * B * (64 * H + H * H) + 2.0 * B * (H * H + H * H + 64 * H)
    mlp.close()
    return {"workload": "AdamW steps of the 34-256-256-1 network, 16,384 rows each, samples from the n=20 workload",
            "samples": rows, "ms_per_step": ms, "rows_per_s": B / (ms * 1e-3),
            "gemm_tflops_whole_step": gemm_flop / (ms * 1e-3) / 1e12, "loss_last": float(hist[-1]),
            "note": "the whole step (features gather, five GEMMs, loss, column sums, AdamW) timed; the "
                    "per-GEMM rates are in the launch-list profile"}


def variant_runs(R, torch, iters: int = 300):
    """S1 / F1 / S2 / F2, each with and without the Type 4 rule (annealing at
    4 % of the best upper bound the S1 run found, cooled by 0.99 every 100
    iterations, draws from instances.sa_draws seed 5): iterations per second over
    the whole run from the first solve, best and last bound, Z augmenting
    searches per iteration (canonical duals, previous-iteration warm starts; the
    time includes the one-time CUDA-graph capture)."""
    inst = I.config(CFG)
    res = {"workload": WORKLOAD, "iterations": iters}
    kf, kl, ng = I.sa_draws(inst.n, iters, 5)
    ub = None
    for name, variant, two_phase, sa in [("S1", 0, 0, False), ("F1", 1, 0, False), ("S2", 0, 1, False),
                                         ("F2", 1, 1, False), ("S1+SA", 0, 0, True), ("F1+SA", 1, 0, True),
                                         ("S2+SA", 0, 1, True), ("F2+SA", 1, 1, True)]:
        prm = R.params(feas_tol=0.0, warm=1, variant=variant, two_phase=two_phase, ub=ub if sa else 0.0)
        with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
            if sa:
                ctx.set_sa(kf, kl, ng)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbs, done = ctx.iterate(iters)
            dt = time.perf_counter() - t0
            _, best, ubf, _, _, _ = ctx.bound()
            st = ctx.stats()
        if name == "S1":
            ub = float(ubf)
            res["ub_for_annealing"] = ub
        res[name] = {"iters_per_s": done / dt, "best_lb": float(best), "lb_last": float(lbs[done - 1]),
                     "z_aug_per_iter": float(st[1]) / done, "drops": int(np.sum(np.diff(lbs[:done]) < 0))}
    # half-Z-LAP scheme (Section 5): 72,200 of the 144,400 Z-LAPs per iteration
    with R.Context(inst.F, inst.D, inst.B, prm=R.half_z_params(feas_tol=0.0, warm=1)) as ctx:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbs, done = ctx.iterate(iters)
        dt = time.perf_counter() - t0
        _, best, _, _, _, _ = ctx.bound()
        st = ctx.stats()
        ctx.set_timing(True)
        ctx.iterate(20)
        kt = ctx.kernel_times()
    res["S1 half-Z"] = {"iters_per_s": done / dt, "best_lb": float(best), "lb_last": float(lbs[done - 1]),
                        "z_aug_per_iter": float(st[1]) / done, "drops": int(np.sum(np.diff(lbs[:done]) < 0)),
                        "z_laps_per_iter": ctx.T // 2,
                        "lap_z_ms": kt["lap_z"][0] / max(1, kt["lap_z"][1]),
                        "move_z_ms": kt["move_z"][0] / max(1, kt["move_z"][1])}
    return res


def run_bnb_hard():
    """Branch and bound to proven optimality on a Nugent-like n = 20 instance."""
    import torch
    from paper_1710_03732_gb300 import rlt2 as R
    R.lib()
    inst = I.grid_instance("n20_grid4x5", 4, 5, 9, 0.5, 12, 1)
    res = {"workload": "QAP n=20, D = Manhattan 4x5 grid, F symmetric 0..9 at density 0.5 (seed 12), B = 0"}
    runs = ((64, 1, "warm"), (64, 0, "warm_one_at_a_time"), (-1, 1, "cold"))
    if os.environ.get("RLT2_BNB_RUNS"):
        runs = tuple(r for r in runs if r[2] in os.environ["RLT2_BNB_RUNS"].split(","))
    for wd, batch, tag in runs:
        # batch: the children of a branched node bounded together (rlt2_iterate_many)
        opts = R.bnb_options(iters_root=300, iters_node=60, warm_depth=wd, time_limit_s=600.0, batch_children=batch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, perm, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(warm=1, stall_window=25),
                                               opts=opts)
        dt = time.perf_counter() - t0
        res[tag] = dict(best=best, perm=[int(x) for x in perm], root_lb=rlb, seconds=dt,
                        nodes_per_s=st["bounded"] / dt, **{k: int(v) for k, v in st.items()})
    print(json.dumps(res), flush=True)
    return 0


def bnb_runs(R, torch):
    """rlt2_bnb_solve on the n = 12 grid workload and on n = 12 and n = 14
    random instances (F 0..9 at density 0.7, asymmetric, with B; seeds 70, 71):
    seconds, nodes, ascent iterations, proven optimality; warm (parent
    multipliers) against cold children; each capped at 60 s."""
    res = {}
    cases = [("n12_grid3x4", I.config(2)),
             ("n12_random_seed70", I.random_instance(12, 70, with_b=True, asymmetric=True)),
             ("n14_random_seed71", I.random_instance(14, 71, with_b=True, asymmetric=True))]
    for name, inst in cases:
        for wd, tag in ((64, "warm"), (-1, "cold")):
            opts = R.bnb_options(iters_root=300, iters_node=100, warm_depth=wd, time_limit_s=60.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            best, _, rlb, st = R.rlt2_bnb_solve(inst.F, inst.D, inst.B, prm=R.params(warm=1, stall_window=25),
                                                opts=opts)
            dt = time.perf_counter() - t0
            res[f"{name}_{tag}"] = dict(best=best, root_lb=rlb, seconds=dt, **{k: int(v) for k, v in st.items()})
    return res


def extra_workloads(R, torch):
    """The other configurations, measured after the headline timed region:
    config 4 (64 branch-and-bound nodes of a 2x11-grid QAP with n = 22, depths
    4..8, bounded in one batched launch sequence), config 5 (n = 30, 5x6 grid)
    and the learned warm start's augmenting searches on the n = 20 workload."""
    out = {}
    wpath = os.path.join(ROOT, "paper_1710_03732_gb300", "weights", "warmstart_h256.npz")
    mlp = None
    if os.path.exists(wpath):
        mlp = R.Mlp(256)
        mlp.load(wpath)
    # config 4: batched node bounding, cold / previous duals / learned
    inst = I.config(4)
    iters = 30
    c4 = {"workload": "n=22 2x11 grid, F 0..9 @0.6 (seed 3), 64 nodes at depths 4..8 (residual 14..18)",
          "iterations_per_node": iters}
    for warm in (0, 1, 2):
        if warm == 2 and mlp is None:
            continue
        prm = R.params(feas_tol=0.0, warm=warm)
        # warm-up that also tunes the Z-stage shape of every size present (the table is kept)
        R.rlt2_bound_nodes(inst.F, inst.D, inst.partials, 6, prm=prm, mlp=mlp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lb, _, its, st = R.rlt2_bound_nodes(inst.F, inst.D, inst.partials, iters, prm=prm, mlp=mlp)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c4[["cold", "warm", "learned"][warm]] = {"node_iters_per_s": float(its.sum() / dt), "seconds": dt,
                                                 "z_aug": int(st["z_aug"]), "lb_sum": float(lb.sum()),
                                                 "z_lanes_per_lap": int(st["group"]), "z_warps_per_block": int(st["wpb"])}
    c4["z_shape_per_size"] = R.rlt2_node_tuning()
    out["config4_nodes"] = c4
    # config 5: n = 30
    inst = I.config(5)
    c5 = {"workload": "n=30 5x6 grid, F 0..9 @0.5 (seed 4); 756,900 Z-LAPs of size 28, 4.75 GB z array"}
    for warm in (0, 1, 2):
        if warm == 2 and mlp is None:
            continue
        with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=warm)) as ctx:
            if warm == 2:
                ctx.set_mlp(mlp)
            ctx.iterate(3)
            s0 = ctx.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbs, _ = ctx.iterate(10)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            s1 = ctx.stats()
            c5[["cold", "warm", "learned"][warm]] = {"iters_per_s": 10 / dt, "lb_after_13": float(lbs[-1]),
                                                     "z_aug_per_lap": float((s1[1] - s0[1]) / (10 * ctx.T))}
    out["config5_n30"] = c5
    # Section 3.4 variants on the headline workload: speed and bound reached
    out["variants_n20"] = variant_runs(R, torch)
    # branch and bound to optimality (Section 4)
    out["branch_and_bound"] = bnb_runs(R, torch)
    out["mlp_training"] = training_rate(R, torch)
    # learned start on the headline workload: augmenting searches, identical bounds
    if mlp is not None:
        inst = I.config(CFG)
        lw = {"iterations": 20}
        for warm in (0, 1, 2):
            with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=warm)) as ctx:
                if warm == 2:
                    ctx.set_mlp(mlp)
                ctx.iterate(4)
                s0 = ctx.stats()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lbs, _ = ctx.iterate(16)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                lw[["cold", "warm", "learned"][warm]] = {"z_aug": int(ctx.stats()[1] - s0[1]), "lb_last": float(lbs[-1]),
                                                         "ms_per_iteration": 1e3 * dt / 16}
                if warm == 2:
                    # inference alone on this state's tiles (CUDA events): the network's cost per iteration
                    T, m = ctx.T, ctx.n - 2
                    D = torch.empty(ctx.E, dtype=torch.float64, device="cuda")
                    xi = torch.empty(T * m, dtype=torch.float64, device="cuda")
                    R.rlt2_export_state(ctx.ctx, Dhat=D, on_device=1)
                    R.rlt2_duals(ctx.ctx, xi=xi, on_device=1)
                    u0 = torch.empty(T, m, dtype=torch.float64, device="cuda")
                    mlp.predict(D.view(T, m, m), u0, xi.view(T, m))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(5):
                        mlp.predict(D.view(T, m, m), u0, xi.view(T, m))
                    e1.record()
                    torch.cuda.synchronize()
                    lw["learned"]["inference_ms_per_iteration"] = e0.elapsed_time(e1) / 5
                    del D, xi, u0
        lw["learned_saves_vs_cold"] = 1.0 - lw["learned"]["z_aug"] / lw["cold"]["z_aug"]
        lw["warm_saves_vs_cold"] = 1.0 - lw["warm"]["z_aug"] / lw["cold"]["z_aug"]
        # break-even: the inference time per iteration below which the learned
        # start would match the other start's iteration time (negative: it loses
        # even with free inference)
        solve = lw["learned"]["ms_per_iteration"] - lw["learned"]["inference_ms_per_iteration"]
        lw["break_even_inference_ms"] = {"vs_cold": lw["cold"]["ms_per_iteration"] - solve,
                                         "vs_previous_duals": lw["warm"]["ms_per_iteration"] - solve}
        out["learned_warm_start_n20"] = lw
        mlp.close()
    return out


def rank_max(x: float, dist, device: str) -> float:
    """Max of x over all ranks (x itself on one process): the timed region of a
    replicated run ends when the slowest rank ends."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, slowest_ms: float) -> float:
    """Replicas: every rank processes the same units; the whole job processed
    world * units in the slowest rank's time."""
    return world * units_per_rank / (slowest_ms / 1000.0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the config 4 / config 5 / learned measurements")
    ap.add_argument("--bnb-hard", action="store_true",
                    help="only solve a Nugent-like n=20 QAP (4x5 grid, F 0..9 at density 0.5, seed 12) to proven "
                         "optimality with rlt2_bnb_solve and print its statistics (about two minutes)")
    ap.add_argument("--profile", nargs="?", const="n20",
                    choices=["n20", "cold", "n22", "n30", "nodes", "learned", "train", "gemm"],
                    help="only run a small case for ncu captures: n20 = warmup+steps iterations of the n=20 "
                         "workload (graph replay, warm start); cold = the same with cold LAPs; "
                         "n22 / n30 = warmup+steps iterations of the n=22 "
                         "grid QAP's root or the n=30 grid QAP, warm, with per-kernel times; "
                         "nodes = 16 nodes of the n=22 grid QAP; "
                         "learned = n=20 with the learned warm start; train = AdamW steps of the H=256 "
                         "network (16,384 rows); gemm = its gradients on 262,144 rows per call")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile_case(args)
    if args.bnb_hard:
        return run_bnb_hard()

    rank, world, local = env_rank()
    inst = I.config(CFG)
    cpu = None
    cpu_cold = None
    cpu_detail = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it, dt, threads, _ = cpu_oracle_baseline(inst, 40, 15.0, warm=True)
        cpu = {"value": it / dt, "unit": "iters/s", "cores": threads, "kind": "oracle",
               "sample": f"first {it} iterations of the same n=20 workload, every LAP warm-started from the "
                         f"previous iteration's duals (the start of `value`), all host cores ({cpu_model()})"}
        itc, dtc, _, _ = cpu_oracle_baseline(inst, 20, 8.0, warm=False)
        cpu_cold = {"value": itc / dtc, "unit": "iters/s", "cores": threads, "kind": "oracle",
                    "sample": f"first {itc} iterations, cold LAPs (the start of `plain_cold`), all host cores"}
        cpu_detail = cpu_oracle_detail()

    import torch
    from paper_1710_03732_gb300 import build as B
    from paper_1710_03732_gb300 import rlt2 as R
    if not os.path.exists(R.LIB_PATH):
        B.build()
    R.lib()
    torch.cuda.set_device(local)
    # roofline denominators measured on this device in this run (instruction
    # throughputs of the pipes the two hot kernels are bound by)
    rates = R.rlt2_probe_rates()
    int64_peak = rates["iadd64"]
    # the z move's FP64 mix per entry: 2 + 5/6 add/sub, 2 fused multiply-adds
    fp64_move_peak = (4 + 5.0 / 6.0) / ((2 + 5.0 / 6.0) / rates["dadd"] + 2.0 / rates["dfma"])
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    with ClockSampler(local) as clocks:
        # the headline runs: graph replay, no per-kernel events
        cold = timed_device_run(R, torch, inst, 0, args.steps, args.warmup, barrier, timing=False)
        warm = timed_device_run(R, torch, inst, 1, args.steps, args.warmup, barrier, timing=False)
        # the same warm run again with CUDA events around every launch: the per-kernel
        # times of the rooflines and the kernel breakdown
        warm_k = timed_device_run(R, torch, inst, 1, args.steps, args.warmup, barrier)
        warm["kt"] = warm_k["kt"]
        # the same ascent with the canonical duals computed in FP64 (dual_mode 2)
        f64 = timed_device_run(R, torch, inst, 1, args.steps, args.warmup, barrier, mode=2)
        # the z move and the next Z-LAPs as one launch (rlt2_params.pipeline)
        pcold = timed_device_run(R, torch, inst, 0, args.steps, args.warmup, barrier, pipeline=1)
        pwarm = timed_device_run(R, torch, inst, 1, args.steps, args.warmup, barrier, pipeline=1)
    clk = clocks.summary()

    # end to end through the C ABI with host buffers: create (H2D of F, D, B and
    # the setup kernels), K iterations with the bound of every iteration read back
    # to host memory, destroy
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    prm = R.params(dual_mode=1, warm=1, feas_tol=0.0)
    with R.Context(inst.F, inst.D, inst.B, prm=prm) as ctx:
        hist, got = ctx.iterate(args.steps)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()

    def per_rank_max(x):
        return rank_max(x, dist, "cuda")

    warm_ms = per_rank_max(warm["ms"])
    warm_k_ms = per_rank_max(warm_k["ms"])
    cold_ms = per_rank_max(cold["ms"])
    f64_ms = per_rank_max(f64["ms"])
    pcold_ms = per_rank_max(pcold["ms"])
    pwarm_ms = per_rank_max(pwarm["ms"])
    e2e_s = per_rank_max(e2e_s)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    n, T = warm["n"], warm["T"]
    m = n - 2
    steps = args.steps

    def lap_z_roofline(r):
        ms_lz, cnt = r["kt"]["lap_z"]
        cnt = max(cnt, 1)
        avg_ms = ms_lz / cnt
        aug, relax = int(r["stats"][1]), int(r["stats"][2])  # totals over the timed launches
        # Additions the method needs in one Z-stage launch (64-bit integer ones
        # in the fixed-point form, FP64 ones in dual_mode 2): 3 per label
        # relaxation (only unscanned columns count; the m start labels of a
        # search, which the counter includes, take 2), 3 per column per search
        # for the dual update and row duals; per LAP, m^2 for the warm start's column
        # reduction (c - u_r), m - 1 for the optimum, and for the canonical duals
        # 2 m^2 for the reduced tile, (m-1)(m-2)/2 Dijkstra relaxations and 3 m
        # for the final row and column duals
        per_lap = (m * m if r["warm"] else 0) + (m - 1) + 2 * m * m + (m - 1) * (m - 2) // 2 + 3 * m
        per_launch = (3 * relax + 2 * m * aug) / cnt + T * per_lap
        achieved = per_launch / (avg_ms * 1e-3) / 1e9
        return avg_ms, per_launch, achieved

    avg_lz, fl_lz, ach_lz = lap_z_roofline(warm)
    avg_lz64, fl_lz64, ach_lz64 = lap_z_roofline(f64)
    mz_ms = warm["kt"]["move_z"][0] / max(warm["kt"]["move_z"][1], 1)
    E = T * m * m
    # folded uniform z move (kz = 1, equal phi): per entry 2 for s = (D - xi) - psi',
    # 5/6 for the class sum S, 2 fused multiply-adds for D' = fma(-(1+phi), s, fma(phi, S, D))
    mz_ops = E * (4 + 5.0 / 6.0)
    mz_bytes = E * 16 + 2 * T * m * 8  # D^ read + write, xi and psi' read once
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    traffic = profiled_traffic("lap_z", "n20")
    traffic_mz = profiled_traffic("move_z", "n20")
    total_kernel_ms = sum(v[0] for v in warm["kt"].values())
    launches = sum(v[1] for v in warm["kt"].values())
    line = {
        "metric": METRIC,
        "value": whole_job_rate(world, steps, warm_ms),
        "unit": "iters/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": warm_ms / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+i64",
        "dtype_note": "FP64 state and multiplier moves (bit-exact with the oracle's operation order); "
                      "LAPs in exact 64-bit fixed point on a per-tile grid of 2^-48 of the tile's magnitude",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "z_laps_per_iter": T, "z_lap_size": m, "z_entries": E,
                   "warm_start": "previous-iteration Z duals", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (374 MB z array), no flush"},
        "laps_per_s": {"warm": whole_job_rate(world, steps * T, warm_ms),
                       "cold": whole_job_rate(world, steps * T, cold_ms),
                       "z_stage_only_warm": T / (avg_lz * 1e-3)},
        "plain_cold": {"value": whole_job_rate(world, steps, cold_ms), "unit": "iters/s",
                       "ms_per_step": cold_ms / steps, "lb_last": cold["lb"],
                       "z_aug_per_lap": cold["stats"][1] / (steps * T), "cpu_oracle_cold": cpu_cold},
        "warm": {"lb_last": warm["lb"], "z_aug_per_lap": warm["stats"][1] / (steps * T),
                 "same_bound_as_cold": bool(warm["lb"] == cold["lb"]),
                 "same_bound_as_cold_rel": abs(warm["lb"] - cold["lb"]) / abs(cold["lb"])},
        "ms_per_iteration_windows": {
            "first_50_after_warmup": warm["windows"][0][1] / warm["windows"][0][0],
            "last_50": warm["windows"][-1][1] / warm["windows"][-1][0],
            "cold_first_50_after_warmup": cold["windows"][0][1] / cold["windows"][0][0],
            "cold_last_50": cold["windows"][-1][1] / cold["windows"][-1][0]},
        "kernels_ms_per_iteration": {k: v[0] / steps for k, v in warm["kt"].items() if v[1] > 0},
        "kernel_launches_per_iteration": {k: v[1] / steps for k, v in warm["kt"].items() if v[1] > 0},
        "kernel_times_run": {"iters_per_s": whole_job_rate(world, steps, warm_k_ms),
                             "note": "per-kernel times (and the rooflines) from a second run of the same warm "
                                     "workload with CUDA events around every launch, launched kernel by kernel; "
                                     "value and ms_per_step from graph replay without them"},
        "roofline_lap_z": {"bound": "alu", "kernel": "lap_z", "achieved": ach_lz, "peak": int64_peak,
                     "unit": INT64_UNIT, "frac": ach_lz / int64_peak, "traffic": traffic,
                     "algorithmic_ops_per_launch": fl_lz, "avg_launch_ms": avg_lz,
                     "arithmetic": "exact 64-bit fixed point (canonical duals, dual_mode 1)",
                     "peak_source": "measured in this run: add.s64 lane throughput of the device "
                                    "(rlt2_probe_rates, CUDA events); nominal 64 lanes/clk/SM x 152 x 2.07 GHz = "
                                    f"{INT64_PEAK_GOPS:.0f}",
                     "limiter": "the ALU pipe's compares, selects and warp reductions of the sequential "
                                "Dijkstra steps and instruction issue (ncu: ALU pipe 78 %, issue 81 % busy), "
                                "not the additions",
                     # the same additions counted as FP64 ops against the FP64 pipe (the roofline of
                     # an FP64 solve): above 1 means faster than an FP64 solve could be
                     "frac_of_fp64_add_peak": ach_lz / rates["dadd"]},
        "pipelined": {"cold": whole_job_rate(world, steps, pcold_ms), "warm": whole_job_rate(world, steps, pwarm_ms),
                      "unit": "iters/s", "same_bounds": bool(pcold["lb"] == cold["lb"] and pwarm["lb"] == warm["lb"]),
                      "note": "z move and next Z-LAPs in one persistent launch (rlt2_params.pipeline = 1)"},
        "fp64_canonical": {"value": whole_job_rate(world, steps, f64_ms), "unit": "iters/s",
                           "ms_per_step": f64_ms / steps, "lb_last": f64["lb"],
                           "lb_rel_diff_vs_fixed_point": abs(f64["lb"] - warm["lb"]) / abs(warm["lb"]),
                           "lap_z_ms": avg_lz64,
                           "roofline_lap_z": {"bound": "alu", "achieved": ach_lz64, "peak": rates["dadd"],
                                              "unit": FP64_UNIT, "frac": ach_lz64 / rates["dadd"],
                                              "peak_source": "measured add.rn.f64 lane throughput"}},
        "roofline_move_z": {"bound": "alu", "kernel": "move_z", "achieved": mz_ops / (mz_ms * 1e-3) / 1e9,
                            "peak": fp64_move_peak, "unit": FP64_UNIT,
                            "frac": mz_ops / (mz_ms * 1e-3) / 1e9 / fp64_move_peak, "traffic": traffic_mz,
                            "algorithmic_ops_per_launch": mz_ops,
                            "peak_source": "measured in this run: the kernel's FP64 mix (2 5/6 add/sub, 2 fma per "
                                           "entry) at the probed add.rn.f64 and fma.rn.f64 lane rates",
                            "frac_of_nominal": mz_ops / (mz_ms * 1e-3) / 1e9 / FP64_PEAK_GOPS,
                            "hbm_gbs": mz_bytes / (mz_ms * 1e-3) / 1e9,
                            "hbm_frac_of_measured": (mz_bytes / (mz_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                            "avg_launch_ms": mz_ms},
        "cpu_baseline": cpu,
        "cpu_oracle_detail": cpu_detail,
        "e2e": {"value": whole_job_rate(world, got, e2e_s * 1000.0), "unit": "iters/s",
                "h2d_bytes_per_step": 3 * 20 * 20 * 8 / steps, "d2h_bytes_per_step": 8,
                "note": "rlt2_create from host F,D,B + rlt2_iterate(K) with host bound history + destroy"},
        "measured_rates_gops": {k: v for k, v in rates.items() if k != "sm_clock_ghz"},
        "gpu_launches": int(launches),
        "gpu_kernel_ms_total": total_kernel_ms,
        "clocks": clk,
    }
    # the roofline of the kernel that takes the larger share of an iteration
    share = {k: warm["kt"][k][0] for k in ("lap_z", "move_z")}
    dominant = max(share, key=share.get)
    line["roofline"] = dict(line["roofline_" + dominant], share_of_step=share[dominant] / warm_ms)
    if world == 1 and not args.no_extra:
        line["extra"] = extra_workloads(R, torch)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
