"""Benchmark of the implicit EMHD zone step on B300.

Workload: the 2-D special-relativistic extended-MHD box, 1024 x 1024
periodic zones (gamma = 4/3, tau_R = 1, phi = psi = 1, MC reconstruction,
seeded Gaussian velocity field, dt = 0.5/1024).  One step is grim_step: the
half and full semi-implicit stages, each an explicit kernel (reconstruction,
LLF fluxes, flux-CT, closure constants) and a per-zone Newton solve to
max|r| <= 1e-10.

Default arm: prints one JSON line with zone-updates/s of the mixed-precision
path (float32 Jacobian and LU, float64 residual, update and test), the
float64 path beside it, the roofline of the dominant kernel, the end-to-end
rate through the C ABI with host buffers, the clocks seen during the timed
region, and the CPU oracle timed on a bounded sample.
`--impl reference`: the oracle alone on the host cores (the reference arm).
Under torchrun (N > 1) every rank steps its own independent box (weak
scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-updates/s at |R|\u22641e-10 (mixed+learned vs FP64 plain, 1 B300); % roofline"
N_SIDE = 1024
# bfloat16 MACs per zone of the learned-start network (32x128, 2 x 128x128,
# 128x80), 2 flops each.
MLP_FLOPS_PER_ZONE = 2 * (32 * 128 + 2 * 128 * 128 + 128 * 80)
MLP_TRAIN_STEPS = 24000   # Adam steps of the learned start (untimed, about 20 s)
MLP_SAMPLE_STRIDE = 6     # training stages from every 6th of the first 48 steps (the timed stretch)
# DRAM bytes read + written per launch at 1024^2 (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of each kernel on this workload;
# newton32 captured on the learned arm, the metric's, its in-order kernel;
# mlp the tcgen05 inference kernel; None while a kernel has changed since
# its capture).
NCU_TRAFFIC_BYTES = {"faces": 296.6e6, "zone_const": None, "newton64": 428.1e6, "newton32": 472.3e6,
                     "mlp": 162.5e6}
TOL = 1e-10
KERR_OUTLIER_LIMIT = 10.0  # training rows of the torus kept within this many central-99.8% spans of each median

# The mixed solver's explicit kernels evaluate in float-float on the float32
# pipes (the zone kernel keeps its conserved terms in float64); their limit
# is the issue rate, not a float64 peak.  ncu figures per launch on the
# 1024^2 box: issue slots busy (and, for the zone kernel, the FP64 pipe) in
# the half and the full stage.
NCU_FLOATFLOAT = {
    "faces": {"precision": "float-float", "bound": "issue", "issue_frac": 0.46},
    "zone_const": {"precision": "float-float sources, float64 conserved terms", "bound": "latency",
                   "issue_frac": [0.26, 0.35], "fp64_pipe_frac": [0.50, 0.40]},
}


def read_flop_counts():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "flop_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


# bf16 multiply-add flops of one Adam step per training row: the forward
# contractions (2 x 47 104), the weight gradients (the same) and the input
# gradients of the three upper layers (2 x 43 008).
MLP_STEP_FLOPS_PER_ROW = 2 * (2 * 47104 + 43008)


def training_rate(X, Y, peaks, steps=400, batch=4096):
    """Adam steps of a fresh network on the training rows, timed with CUDA
    events on the stream they run on (the default stream): ms per step and
    the bf16 rate of their contractions against the measured burst peak."""
    import torch
    from paper_1702_01106_b300.grim import MLP
    m = MLP(seed=5)
    m.fit_norm(X, Y)
    m.train(X, Y, steps=20, batch=batch, lr=1e-3, seed=3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    m.train(X, Y, steps=steps, batch=batch, lr=1e-3, seed=4)
    e1.record()
    torch.cuda.synchronize()
    m.close()
    ms = e0.elapsed_time(e1) / steps
    tf = MLP_STEP_FLOPS_PER_ROW * batch / (ms * 1e-3) / 1e12
    return {"ms_per_step": ms, "batch": batch, "launches_per_step": 33, "bf16_tflops": tf,
            "bf16_frac_of_burst": tf / peaks.get("bf16_tflops", 1800.0)}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(prob, P, dt, target_s=12.0, threads=0, max_side=512):
    """The oracle as it stands on the host cores, on a bounded sample of the
    same workload: a contiguous square block of zones of the 1024^2 box,
    stepped once (half step on the block plus a 4-zone margin, full step on
    the block).  threads = 0: all cores.  Returns (zone-updates/s, cores,
    sample description, seconds)."""
    import numpy as np
    from oracle import oracle
    cores = threads if threads > 0 else oracle.max_threads()
    side, elapsed = 16, 0.0
    while True:
        zs = np.array([(j * N_SIDE + i) for j in range(side) for i in range(side)], dtype=np.int64)
        t0 = time.perf_counter()
        out, it, st, _ = oracle.step_sampled(prob, P, dt, zs, threads=threads)
        elapsed = time.perf_counter() - t0
        if elapsed >= target_s / 4 or side >= max_side:
            break
        side *= 2
    rate = side * side / elapsed
    sample = (f"one oracle step of a {side}x{side}-zone block of the {N_SIDE}^2 box "
              f"(half step on the block plus a 4-zone margin), {elapsed:.1f} s on {cores} threads")
    return rate, cores, sample, elapsed


def cpu_baseline_torus(prob, P, dt, target_s=10.0, threads=0):
    """The oracle on the host cores on a bounded sample of the Kerr torus: a
    contiguous block of zones around the pressure maximum (r = 12, the
    equator; 16 of the 128 zones along X^3, doubling in X^1 and X^2 until
    the step takes a quarter of target_s), stepped once (half step on the
    block plus a 4-zone margin, full step on the block).  Returns
    (zone-updates/s, cores, sample description, seconds)."""
    import math
    import numpy as np
    from oracle import oracle
    cores = threads if threads > 0 else oracle.max_threads()
    n1, n2, n3 = prob.n
    i0 = int((math.log(12.0) - prob.x_start[0]) / prob.dx[0])
    j0 = n2 // 2
    side, elapsed = 8, 0.0
    while True:
        ii = range(max(0, i0 - side // 2), min(n1, i0 + side // 2))
        jj = range(max(0, j0 - side // 2), min(n2, j0 + side // 2))
        zs = np.array([(k * n2 + j) * n1 + i for k in range(16) for j in jj for i in ii], dtype=np.int64)
        t0 = time.perf_counter()
        oracle.step_sampled(prob, P, dt, zs, threads=threads)
        elapsed = time.perf_counter() - t0
        if elapsed >= target_s / 4 or side >= 64:
            break
        side *= 2
    rate = zs.size / elapsed
    sample = (f"one oracle step of a {len(ii)}x{len(jj)}x16-zone block of the {n1}x{n2}x{n3} torus around the "
              f"pressure maximum (half step on the block plus a 4-zone margin), {elapsed:.1f} s on {cores} threads")
    return rate, cores, sample, elapsed


def dist_setup(args):
    """Rank, world size and local rank from the torchrun environment; one
    process group for the barrier and the max-over-ranks timing (NCCL on GPU
    ranks, gloo for the CPU reference arm or without CUDA).  No collective
    touches the data path: every rank steps its own box (weak scaling)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        gpu = torch.cuda.is_available() and args.impl != "reference"
        if gpu:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if gpu else "gloo")
    return world, rank, local


def aggregate_rate(units_per_rank, seconds, world):
    """Whole-job throughput: every rank processed units_per_rank in the
    (max-over-ranks) time."""
    return world * units_per_rank / seconds


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    on_gpu = torch.cuda.is_available() and dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host cores."""
    if rank != 0:
        return
    from paper_1702_01106_b300 import inputs
    prob = inputs.turbulent_box_problem(N_SIDE, tol=TOL)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / N_SIDE
    budget = max(20.0, 120.0 / max(1, args.steps + args.warmup))
    rate, cores, sample, el = cpu_baseline(prob, P, dt, target_s=min(budget, 12.0))
    # warm-up / timed repetitions of the same bounded sample
    import numpy as np
    from oracle import oracle
    side = int(round((rate * el) ** 0.5))
    zs = np.array([(j * N_SIDE + i) for j in range(side) for i in range(side)], dtype=np.int64)
    for _ in range(max(0, args.warmup - 1)):
        oracle.step_sampled(prob, P, dt, zs)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step_sampled(prob, P, dt, zs)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = side * side / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"2-D SR extended-MHD turbulent box {N_SIDE}x{N_SIDE}, tol 1e-10 "
                                   f"(sampled {side}x{side} block per step)", "grid": [N_SIDE, N_SIDE],
                       "precision": "fp64"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{side}x{side}-zone block of the {N_SIDE}^2 box per step"},
            "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def nvtx_push(torch, name):
    """Mark the timed region (ncu --nvtx --nvtx-include "timed/" profiles only it)."""
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop(torch):
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def profile_case(args, dev, torch):
    """--case-only: the float64 and mixed steps of one workload alone
    (autotuned, warmed up, then `--steps` steps in the NVTX range "timed"),
    for ncu captures of single kernels; prints one JSON line of timings.
    --case box: the turbulent box of side --side; --case box-learned: its
    mixed arm with a learned start; --case torus: the Kerr torus on a --side x
    --side x --side/3 grid; --case train: Adam steps of the learned start's
    network at batch 4096 on 2^20 seeded rows (--steps steps inside the NVTX
    range "timed")."""
    from paper_1702_01106_b300 import inputs
    from paper_1702_01106_b300.grim import Grim, GRIM_FP64, GRIM_MIXED
    if args.case == "train":
        gen = torch.Generator(device=dev).manual_seed(7)
        X = torch.randn((1 << 20, 32), device=dev, generator=gen)
        Y = torch.randn((1 << 20, 16), device=dev, generator=gen)
        peaks, _ = read_peaks()
        training_rate(X, Y, peaks, steps=max(3, args.warmup))
        torch.cuda.nvtx.range_push("timed")
        rate = training_rate(X, Y, peaks, steps=args.steps)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": "MLP training, batch 4096", "steps": args.steps, "step": rate}))
        return
    if args.case == "torus":
        prob = inputs.torus_problem(args.side, args.side, max(1, args.side // 3))
        P = inputs.torus_state(prob)
        dt = inputs.torus_dt(prob)
        name = f"Kerr torus {args.side}x{args.side}x{max(1, args.side // 3)}"
    else:
        prob = inputs.turbulent_box_problem(args.side, tol=TOL)
        P = inputs.turbulent_box_state(prob)
        dt = 0.5 / args.side
        name = f"turbulent box {args.side}x{args.side}"
    out = {"case": name, "steps": args.steps}
    arms = [("fp64", GRIM_FP64), ("mixed", GRIM_MIXED)]
    mlp = None
    if args.case == "box-learned":
        # the learned start's inference costs the same whatever the weights:
        # an untrained network (its starts lose to P_n and fall back)
        from paper_1702_01106_b300.grim import MLP
        mlp = MLP(seed=1)
        arms = [("learned", GRIM_MIXED)]
    for nm, prec in arms:
        g = Grim(prob, precision=prec)
        if mlp is not None:
            g.set_guess(mlp, accept=1e-3)
        a = torch.from_numpy(P).to(dev)
        b = torch.empty_like(a)
        out[nm + "_tuning"] = g.autotune(a, dt)[0]
        ms, st, kt, _ = time_device(g, a, b, dt, args.steps, args.warmup, 1, torch)
        out[nm] = {"ms_per_step": ms,
                   "kernel_ms_per_stage": {k: v[0] / (2 * min(args.steps, 10)) for k, v in kt.items()},
                   "iters_per_zone_stage": st["iters"] / max(1, st["zones"]), "failed": st["failed"]}
        g.close()
    print(json.dumps(out))


def iters_p99(hist):
    """99th percentile of the per-zone Newton update counts (histogram)."""
    tot = sum(hist)
    acc = 0
    for k, n in enumerate(hist):
        acc += n
        if acc >= 0.99 * tot:
            return k
    return len(hist) - 1


def time_device(g, a, b, dt, steps, warmup, world, torch):
    """Timed steps as a user runs them: CUDA graphs on, no per-kernel events
    (the first warm-up step runs eagerly, the next two capture the graphs of
    the two ping-pong directions).  Then a separate pass of eager steps with
    per-kernel events gives the split between kernels; it is not the timed
    number."""
    g.use_graphs(True)
    for _ in range(max(warmup, 3)):
        g.step(a, b, dt)
        a, b = b, a
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    g.reset_stats()
    launches0 = g.stats()["launches"]
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nvtx_push(torch, "timed")
    e0.record(st)
    for _ in range(steps):
        g.step(a, b, dt)
        a, b = b, a
    e1.record(st)
    nvtx_pop(torch)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / steps
    stats = g.stats()
    stats["launches_timed"] = stats["launches"] - launches0
    # per-kernel split (eager launches with events around each kernel), with
    # the counters of the same pass for the kernels' algorithmic flops
    g.kernel_times()
    g.reset_stats()
    g.profile(True)
    for _ in range(min(steps, 10)):
        g.step(a, b, dt)
        a, b = b, a
    torch.cuda.synchronize()
    g.profile(False)
    kt = g.kernel_times()
    stats["profile_pass"] = g.stats()
    return ms, stats, kt, a


def bench_batched(dev, mlp, torch, world, steps=3):
    """64 independent linear-mode boxes of sides drawn from {128, 256, 512,
    1024} (seeded), stepped together through grim_batch_step (one graph
    launch per step after capture): zone-updates/s per arm."""
    from paper_1702_01106_b300 import inputs
    from paper_1702_01106_b300.grim import Batch, GRIM_FP64, GRIM_MIXED
    boxes = inputs.batched_boxes()
    probs = [b[0] for b in boxes]
    dts = [b[2] for b in boxes]
    zones = sum(p.zones for p in probs)
    host = [torch.from_numpy(b[1]) for b in boxes]
    out = {"boxes": len(boxes), "zones": zones, "sides": [p.n[0] for p in probs], "steps": steps,
           "timing": "2 untimed steps (eager, graph capture), then CUDA events around the timed steps"}
    for name, prec, learned in (("fp64", GRIM_FP64, False), ("mixed", GRIM_MIXED, False),
                                ("mixed_learned", GRIM_MIXED, True)):
        bt = Batch(probs, precision=prec)
        if learned:
            bt.set_guess(mlp, accept=1e-3)
        A = [h.to(dev) for h in host]
        B = [torch.empty_like(a) for a in A]
        for _ in range(2):
            bt.step(A, B, dts)
            A, B = B, A
        torch.cuda.synchronize()
        bt.reset_stats()
        l0 = bt.stats()["launches"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            bt.step(A, B, dts)
            A, B = B, A
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
        s = bt.stats()
        out[name] = {"value": aggregate_rate(zones, ms * 1e-3, world), "ms_per_step": ms,
                     "newton_iters_per_zone_stage": s["iters"] / max(1, s["zones"]), "failed": s["failed"],
                     "max_res": s["max_res"], "kernels_per_step": (s["launches"] - l0) / steps}
        bt.close()
        del A, B
        torch.cuda.empty_cache()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["speedup_mixed_learned_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed_learned"]["ms_per_step"]
    return out


def bench_kerr(dev, torch, world, steps=10, warmup=3, cpu=False, mixed_tol=1e-11):
    """3-D Fishbone-Moncrief torus around a Kerr black hole (a = 0.9375,
    modified Kerr-Schild, 192 x 192 x 128, floors on), dt fixed at CFL 0.5 of
    the light-speed bound: zone-updates/s of the float64 and mixed arms, and
    of the mixed arm with a learned start trained (untimed) on both stages
    of the first four float64 steps (8 stages of 4.7 M zones).  Every arm
    meets max |R| <= 1e-10; the mixed arms run to 1e-11 (mixed_tol), where
    their primitives agree with the float64 arm's to 1e-9 (at 1e-10 the
    linearly converging mixed solver stops just under the tolerance, and a
    torus conditioning of ~1e2 leaves ~1e-8)."""
    import numpy as np
    from paper_1702_01106_b300 import inputs, guess
    from paper_1702_01106_b300.grim import Grim, GRIM_FP64, GRIM_MIXED
    prob = inputs.torus_problem(192, 192, 128)
    P = torch.from_numpy(inputs.torus_state(prob))
    dt = inputs.torus_dt(prob)
    out = {"workload": "3-D Kerr torus a=0.9375 MKS 192x192x128, FM r_in=6 r_max=12, beta=100, floors, tol 1e-10",
           "zones": prob.zones, "dt": dt, "steps": steps, "tol_fp64": prob.tol,
           "tol_mixed": prob.tol if mixed_tol is None else mixed_tol}
    t0 = time.perf_counter()
    X, Y, _ = guess.collect(prob, P.numpy(), dt, 4, dev)
    n_all = int(X.shape[0])
    X, Y = guess.drop_outliers(X, Y, KERR_OUTLIER_LIMIT)
    mlp, losses = guess.train(X, Y, steps=MLP_TRAIN_STEPS)
    torch.cuda.synchronize()
    out["learned_training"] = {"samples": int(X.shape[0]), "samples_before_outliers": n_all,
                               "outlier_limit_spans": KERR_OUTLIER_LIMIT, "adam_steps": MLP_TRAIN_STEPS,
                               "loss_per_quarter": losses, "seconds": time.perf_counter() - t0}
    del X, Y
    torch.cuda.empty_cache()
    one = {}
    for name, prec, learned in (("fp64", GRIM_FP64, False), ("mixed", GRIM_MIXED, False),
                                ("mixed_learned", GRIM_MIXED, True)):
        g = Grim(prob if prec == GRIM_FP64 or mixed_tol is None else prob.with_(tol=mixed_tol), precision=prec)
        if learned:
            g.set_guess(mlp, accept=1e-3)
        a = P.to(dev)
        b = torch.empty_like(a)
        tuning = g.autotune(a, dt)[0]   # launch shapes, untimed
        ms, s, kt, _ = time_device(g, a, b, dt, steps, warmup, world, torch)
        ms = max_over_ranks(ms, world)
        # one step from the initial state, untimed: the arms' agreement with float64
        a1 = P.to(dev)
        b1 = torch.empty_like(a1)
        g.step(a1, b1, dt)
        one[name] = b1.cpu().numpy().reshape(10, -1)
        del a1, b1
        out[name] = {"value": aggregate_rate(prob.zones, ms * 1e-3, world), "ms_per_step": ms,
                     "newton_iters_per_zone_stage": s["iters"] / max(1, s["zones"]),
                     "fp64_residuals_per_zone_stage": s["evals64"] / max(1, s["zones"]),
                     "failed": s["failed"], "rescued": s["rescued"],
                     "max_res": s["max_res"], "fallbacks": s["fallbacks"], "tuning": tuning,
                     # per stage, from the profile pass (zone_const: derived + sources +
                     # stage constants, and the floors)
                     "kernel_ms_per_stage": {k: v[0] / (2 * min(steps, 10)) for k, v in kt.items()}}
        g.close()
        del a, b
        torch.cuda.empty_cache()
    ref = one["fp64"]
    scale = np.abs(ref) + np.abs(ref).max(axis=1, keepdims=True)
    scale[2:] += 1.0
    bulk = ref[0] > 0.05 * ref[0].max()   # inside the torus, away from its surface and the atmosphere
    for name in ("mixed", "mixed_learned"):
        d = np.abs(one[name] - ref) / scale
        out[name]["one_step_max_rel_diff_vs_fp64"] = float(d.max())
        out[name]["one_step_max_rel_diff_vs_fp64_bulk"] = float(d[:, bulk].max())
    del one, ref, scale, bulk
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["speedup_mixed_learned_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed_learned"]["ms_per_step"]
    if cpu:
        rate, cores, sample, _ = cpu_baseline_torus(prob, P.numpy(), dt)
        out["cpu_baseline"] = {"value": rate, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                               "sample": sample}
    mlp.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batched", action="store_true", help="skip the 64-box batched measurement")
    ap.add_argument("--skip-kerr", action="store_true", help="skip the 3-D Kerr torus measurement")
    ap.add_argument("--kerr-mixed-tol", type=float, default=1e-11,
                    help="convergence tolerance of the torus's mixed arms (the float64 arm runs at 1e-10)")
    ap.add_argument("--case-only", action="store_true",
                    help="only the float64 and mixed steps of a --side box (for ncu captures)")
    ap.add_argument("--side", type=int, default=N_SIDE, help="grid side for --case-only")
    ap.add_argument("--case", default="box", choices=["box", "box-learned", "torus", "train"],
                    help="workload of --case-only")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch
    from paper_1702_01106_b300 import inputs
    from paper_1702_01106_b300.grim import Grim, GRIM_FP64, GRIM_MIXED, peak_flops

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.case_only:
        profile_case(args, dev, torch)
        return
    prob = inputs.turbulent_box_problem(N_SIDE, tol=TOL)
    P = inputs.turbulent_box_state(prob)
    dt = 0.5 / N_SIDE
    N = prob.zones
    fl = read_flop_counts()
    peaks, peak_kind = read_peaks()
    p64, p32 = peak_flops()

    # Learned initial guess: trained (untimed) on 2^24 converged zone states of
    # this workload (both stages of 8 float64 steps, one in every 6 of the first
    # 48, at tol 1e-12), the stretch of the evolution the timed steps cover.
    from paper_1702_01106_b300 import guess
    t0 = time.perf_counter()
    Xtr, Ytr, _ = guess.collect(prob, P, dt, 8, dev, stride=MLP_SAMPLE_STRIDE)
    mlp, losses = guess.train(Xtr, Ytr, steps=MLP_TRAIN_STEPS)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_samples = int(Xtr.shape[0])
    train_rate = training_rate(Xtr, Ytr, peaks)
    del Xtr, Ytr
    torch.cuda.empty_cache()

    results, tunings = {}, {}
    with ClockSampler(local) as clk:
        for name, prec, learned in (("fp64", GRIM_FP64, False), ("mixed", GRIM_MIXED, False),
                                    ("learned", GRIM_MIXED, True)):
            g = Grim(prob, precision=prec)
            if learned:
                g.set_guess(mlp, accept=1e-3)
            a = torch.from_numpy(P).to(dev)
            b = torch.empty_like(a)
            tunings[name] = g.autotune(a, dt)[0]   # launch shapes, untimed
            ms, st, kt, last = time_device(g, a, b, dt, args.steps, args.warmup, world, torch)
            ms = max_over_ranks(ms, world)
            results[name] = (ms, st, kt, g)
    clocks = clk.summary()

    # accuracy of the learned path: one step from the initial state against the float64 path
    one = {}
    for name in ("fp64", "learned"):
        g = results[name][3]
        a = torch.from_numpy(P).to(dev)
        b = torch.empty_like(a)
        g.step(a, b, dt)
        one[name] = b.cpu().numpy().reshape(10, -1)
    ref = one["fp64"]
    scale = np.abs(ref) + np.abs(ref).max(axis=1, keepdims=True)
    scale[2:] += np.array([1, 1, 1, 1, 1, 1, 1, 1])[:, None]
    learned_err = float((np.abs(one["learned"] - ref) / scale).max())

    ms_l, st_l, kt_l, g_l = results["learned"]
    ms_m, st_m, kt_m, g_m = results["mixed"]
    ms_d, st_d, kt_d, g_d = results["fp64"]
    # the headline arm: mixed precision with the learned start
    ms_m, st_m, kt_m, g_m, ms_mp, st_mp = ms_l, st_l, kt_l, g_l, ms_m, st_m
    for nm, (ms, st, _, _) in results.items():
        if st["failed"] or st["max_res"] > TOL:
            print(f"warning: {nm} path: {st['failed']} zone solves failed, max|r| {st['max_res']:.2e}", file=sys.stderr)
    value = aggregate_rate(N, ms_m * 1e-3, world)
    fp64_value = aggregate_rate(N, ms_d * 1e-3, world)
    mixed_plain_value = aggregate_rate(N, ms_mp * 1e-3, world)

    # Roofline of the dominant kernel of the headline (mixed) path: FP64 pipe bound.
    # Algorithmic flops per launch (tests/golden/flop_counts.txt per unit):
    #   faces:      2 LLF face fluxes per zone (the flux-CT ring of boundary
    #               faces is overhead, not counted)
    #   zone_const: the per-zone explicit remainder
    #   newton:     residual evaluations, LU solves and update bookkeeping,
    #               split by precision from the kernel's own counters
    steps = args.steps

    def newton_flops(st):
        # the kernels solve the 7x7 non-magnetic block (7 Jacobian columns)
        f64 = st["evals64"] * fl["residual"] + st["lu64"] * fl["lu_solve_7x7"]
        f64 += st["iters"] * (fl["newton_update_bookkeeping_7x7"] if st["lu64"] else 60)
        f32 = st["evals32"] * fl["residual"] + st["lu32"] * fl["lu_solve_7x7"]
        f32 += st["iters"] * 154 if st["lu32"] else 0
        return f64, f32

    def class_flops(cls, st, launches):
        if cls == "faces":
            return 2 * N * fl["face_flux"], 0
        if cls == "zone_const":
            return N * fl["zone_explicit_remainder_2d"], 0
        if cls == "explicit":
            return N * (2 * fl["face_flux"] + fl["zone_explicit_remainder_2d"]), 0
        if cls == "mlp":
            return 0, 0
        f64, f32 = newton_flops(st)
        return f64 / launches, f32 / launches

    def rooflines(kt, st, floatfloat=False):
        out = {}
        for cls, (tot, n) in kt.items():
            f64, f32 = class_flops(cls, st, n)
            t = tot / n * 1e-3
            if floatfloat and cls in NCU_FLOATFLOAT:
                # the float64 algorithm's flops evaluated in float-float on the
                # float32 pipes: no FP64 fraction; what bounds the kernel is
                # the issue rate (ncu figures of the profiles)
                out[cls] = {"ms_per_launch": tot / n, "share": None, "algorithmic_tflops": f64 / t / 1e12,
                            **NCU_FLOATFLOAT[cls]}
                continue
            out[cls] = {"ms_per_launch": tot / n, "share": None, "fp64_tflops": f64 / t / 1e12,
                        "fp64_frac": f64 / t / 1e12 / p64, "fp32_tflops": f32 / t / 1e12}
            if cls == "mlp":    # bfloat16 tensor-core MACs of the network, 2 flops each
                bf = N * MLP_FLOPS_PER_ZONE / t / 1e12
                out[cls].update({"bf16_tflops": bf, "bf16_frac": bf / peaks.get("bf16_tflops_sustained", 1400.0)})
        total = sum(v[0] for v in kt.values())
        for cls, (tot, n) in kt.items():
            out[cls]["share"] = tot / total
        return out

    roof_m = rooflines(kt_m, st_m["profile_pass"], floatfloat=True)
    roof_d = rooflines(kt_d, st_d["profile_pass"])
    kern = {k: v["ms_per_launch"] for k, v in roof_m.items()}
    dom = max(kt_m.items(), key=lambda kv: kv[1][0])[0]
    names = {"faces": "face_flux_2d", "zone_const": "zone_const_2d", "newton32": "newton_dense<mixed>",
             "newton64": "newton_dense<fp64>", "explicit": "explicit_stage_2d"}
    ach = roof_m[dom]["fp64_tflops"]
    roof = {"bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s", "frac": ach / p64,
            "traffic": NCU_TRAFFIC_BYTES.get(dom), "kernel": names.get(dom, dom),
            "peak_source": "FP64 FMA-chain microbenchmark on this GPU (grim_peak_flops), of measured",
            "flops_convention": "oracle flop counter: +,-,*,/,sqrt = 1, FMA = 2 (tests/golden/flop_counts.txt)",
            "per_kernel": roof_m}
    f64_d, _ = newton_flops(st_d)     # over the timed steps
    exp_flops_launch = N * (2 * fl["face_flux"] + fl["zone_explicit_remainder_2d"])
    whole_fp64 = (f64_d / steps + 2 * exp_flops_launch) / (ms_d * 1e-3) / 1e12
    roof_fp64 = {"kernel": "newton_dense<fp64>", "achieved": roof_d["newton64"]["fp64_tflops"], "peak": p64,
                 "unit": "TFLOP/s", "frac": roof_d["newton64"]["fp64_frac"], "whole_step_frac": whole_fp64 / p64,
                 "per_kernel": roof_d}

    # End to end through the C ABI with host buffers (pinned), copies inside the timed region.
    g_m.profile(False)
    hin = torch.from_numpy(P).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    g_m.step_host(hin, hout, dt)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        g_m.step_host(hin, hout, dt)
        hin, hout = hout, hin
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / steps, world)
    e2e = {"value": aggregate_rate(N, e2e_s, world), "unit": "zone-updates/s", "h2d_bytes_per_step": int(P.nbytes),
           "d2h_bytes_per_step": int(P.nbytes)}

    batched = None if args.skip_batched else bench_batched(dev, mlp, torch, world)
    kerr = None if args.skip_kerr else bench_kerr(dev, torch, world,
                                                  cpu=rank == 0 and world == 1 and not args.no_cpu_baseline,
                                                  mixed_tol=args.kerr_mixed_tol)

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample, _ = cpu_baseline(prob, P, dt)
        cpu = {"value": rate, "unit": "zone-updates/s", "cores": cores, "kind": "oracle", "sample": sample}
        rate1, _, sample1, _ = cpu_baseline(prob, P, dt, target_s=8.0, threads=1, max_side=128)
        cpu1 = {"value": rate1, "unit": "zone-updates/s", "cores": 1, "kind": "oracle", "sample": sample1}

    launches_timed = int(st_m["launches_timed"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_m, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"2-D SR extended-MHD turbulent box {N_SIDE}x{N_SIDE} periodic, MC, "
                                   f"dt=0.5/{N_SIDE}, tol 1e-10, mixed precision (FP32 Jacobian/LU, FP64 residual) "
                                   f"with the learned Newton start",
                       "grid": [N_SIDE, N_SIDE], "zones_per_gpu": N, "precision": "mixed",
                       "l2": "no flush: per-step working set ~0.6 GB (states, stage constants) > 126 MB L2"},
            "fp64_plain": {"value": fp64_value, "ms_per_step": ms_d, "dtype": "f64",
                           "newton_iters_per_zone_stage": st_d["iters"] / max(1, st_d["zones"]),
                           "fp64_residuals_per_zone_stage": st_d["evals64"] / max(1, st_d["zones"]),
                           "fp32_residuals_per_zone_stage": st_d["evals32"] / max(1, st_d["zones"]),
                           "newton_iters_p99": iters_p99(st_d["hist"]),
                           "failed": st_d["failed"], "max_res": st_d["max_res"]},
            "mixed_plain_start": {"value": mixed_plain_value, "ms_per_step": ms_mp,
                                  "newton_iters_per_zone_stage": st_mp["iters"] / max(1, st_mp["zones"]),
                                  "fp64_residuals_per_zone_stage": st_mp["evals64"] / max(1, st_mp["zones"]),
                                  "fp32_residuals_per_zone_stage": st_mp["evals32"] / max(1, st_mp["zones"]),
                                  "newton_iters_p99": iters_p99(st_mp["hist"]),
                                  "failed": st_mp["failed"], "max_res": st_mp["max_res"]},
            "mixed_learned": {"newton_iters_per_zone_stage": st_m["iters"] / max(1, st_m["zones"]),
                              "fp64_residuals_per_zone_stage": st_m["evals64"] / max(1, st_m["zones"]),
                              "fp32_residuals_per_zone_stage": st_m["evals32"] / max(1, st_m["zones"]),
                              "newton_iters_p99": iters_p99(st_m["hist"]),
                              "failed": st_m["failed"], "max_res": st_m["max_res"],
                              "fallback_rate": st_m["fallbacks"] / max(1, st_m["zones"]),
                              "one_step_max_rel_diff_vs_fp64": learned_err,
                              "training": {"samples": n_samples, "adam_steps": MLP_TRAIN_STEPS, "batch": 4096,
                                           "loss_per_quarter": losses, "seconds_with_sampling": train_s,
                                           "step": train_rate}},
            "tuning": tunings,
            "speedup_mixed_learned_vs_fp64": ms_d / ms_m,
            "speedup_mixed_plain_vs_fp64": ms_d / ms_mp,
            "kernel_ms_per_launch": {"mixed": kern, "fp64": {k: v[0] / v[1] for k, v in kt_d.items()}},
            "roofline": roof, "roofline_fp64_newton": roof_fp64,
            "peaks": {"fp64_tflops": p64, "fp32_tflops": p32, "hbm_gbs": peaks.get("hbm_gbs"),
                      "hbm_source": peak_kind},
            "paper_context": {"value": 138000.0, "unit": "zone-updates/s",
                              "what": "grim's whole-step throughput per GPU, NVIDIA K20, FP64, 3-D 64^3 "
                                      "zones per GPU (Section 6); another machine and workload: context "
                                      "only"},
            "batched_64_boxes": batched,
            "kerr_torus_3d": kerr,
            "cpu_baseline": cpu, "cpu_baseline_1core": cpu1, "e2e": e2e, "gpu_launches": launches_timed,
            "clocks": clocks,
        }
        print(json.dumps(line))
    for _, (_, _, _, g) in results.items():
        g.close()
    mlp.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
