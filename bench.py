#!/usr/bin/env python3
"""Benchmark of the B300-native CTU-PPM hydro step: prints ONE JSON line.

Workload: the 3-D Sedov blast on a single 128^3 FP64 box (unit cube, 4 ghost
zones, outflow boundaries, gamma = 1.4, ambient rho = 1, p = 1e-5, E = 1
deposited as pressure in the zones within 4 dx of the centre, CFL 0.5) — the
pure-hydro Sedov problem of the paper's Castro scaling runs (Sec. 4, Fig. 3
left; Fig. 4 left), at the size one box of such a run holds.  A step is one
CTU-PPM advance of the whole box (primitive state, tracing, 12 Riemann solves
per zone, update, CFL reduction) through the library's C ABI with the state
resident in HBM; the next step uses the CFL step the library returns.  The
timed run is the whole 200-step problem from the initial state (--steps);
the warm-up steps run on a copy that is then reset.  Beside it: the 2-D Sod
tube (64^2, 50 steps), the batched level, serving, the 512^3 stratified box
and the other entry points' legs.

--impl ours (default): the CUDA library.  --impl reference: the CPU oracle
(test infrastructure, not the product) on the same workload, timed on the
host cores.  Under torchrun each rank advances its own box (weak scaling, no
collective on the data path); rank 0 prints the line.
"""
import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Algorithmic FP64 operations (+ - * / sqrt, each counted once) per unit of
# each stage, tallied by the counting build of the CPU oracle on this
# workload (Sedov 128^3 after 20 steps; python -m oracle.count_ops).  Units: grown-box zone (prim),
# zone-direction (trace), Riemann solve (flux1, flux2, flux3), interior zone
# (update).
FLOPS_PER_UNIT = {"prim": 20.0, "trace": 225.94, "flux1": 60.0, "flux2": 120.0, "flux3": 154.0, "update": 58.0}
LAUNCHES_PER_STEP_3D = {"prim": 2, "trace": 3, "flux1": 1, "flux2": 1, "flux3": 1, "update": 2}
# FP64 peak derived from B300's unit counts and clock: 148 SMs x 2 FP64 FMA
# lanes per SM per clock x 2 flops x 2032 MHz.  (A dependent-free DFMA stream
# measured 476 G lane-FMA/s = 0.95 TFLOP/s on the B300s.)
FP64_PEAK_GFLOPS = 148 * 2 * 2 * 2.032
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per unit of the dominant stage from one ncu
# capture of the current kernel (k_flux2, all six sets in one launch, Sedov
# 96^3: 921.2 MB for 5,475,456 solves), scaled to a launch by its units.
DRAM_BYTES_PER_UNIT = {"flux2": 168.2}


def units_per_step(n):
    return {
        "prim": (n + 8) ** 3,
        "trace": 3 * (n + 2) ** 3,
        "flux1": 3 * (n + 1) * (n + 2) ** 2,
        "flux2": 6 * (n + 1) * n * (n + 2),
        "flux3": 3 * (n + 1) * n * n,
        "update": n ** 3,
    }


def algorithmic_bytes_per_step(n):
    # read the 5 fields of the grown box once, write the 5 interior fields once
    return 40 * ((n + 8) ** 3 + n ** 3)


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs.

    Sampling starts before the timed region (start(), which waits for the
    first sample), every 50 ms; stop(t0, t1) keeps the samples whose
    timestamps fall inside the timed region's wall-clock window [t0, t1]
    (time.time() values), widened by one interval on each side."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_id):
        self.proc = None
        self.path = os.path.join("/tmp", f"hydro_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout_s=5.0):
        """Block until nvidia-smi has written its first sample (or timeout)."""
        t_end = time.perf_counter() + timeout_s
        while self.proc and time.perf_counter() < t_end:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    @staticmethod
    def _when(stamp):
        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.INTERVAL_MS / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((self._when(parts[0]), float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        pad = self.INTERVAL_MS / 1e3
        inside = [r for r in rows if t0 is not None and r[0] is not None and t0 - pad <= r[0] <= t1 + pad]
        window = "timed region" if inside else "whole run (no sample fell inside the timed region)"
        use = inside or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in use:
            for name, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm = [r[1] for r in use]
        mx = [r[2] for r in use]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window,
                "interval_ms": self.INTERVAL_MS}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, steps, total_ms):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def cpu_oracle_rate(U, n, steps, budget_s=25.0):
    """Oracle zone-updates/s on the host cores: up to `steps` full 128^3 steps
    from U, stopping once budget_s is spent (at least one step)."""
    import oracle
    P = oracle.params(3, (n, n, n), bc=oracle.BC_OUTFLOW, gamma=1.4, cfl=0.5)
    done, t_total = 0, 0.0
    for _ in range(steps):
        d, rc = oracle.dt(U, P)
        t0 = time.perf_counter()
        U, rc = oracle.step(U, P, d)
        t_total += time.perf_counter() - t0
        done += 1
        if t_total > budget_s:
            break
    return n ** 3 * done / t_total, done, t_total, U


def cpu_oracle_rate_one_core(n=64):
    """Oracle zone-updates/s on one host core: one n^3 Sedov step with the
    oracle's OpenMP runtime limited to one thread (restored afterwards)."""
    import ctypes

    import oracle
    from paper_1711_06203_b300 import inputs
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None
    before = gomp.omp_get_max_threads()
    U, _ = inputs.sedov(n)
    P = oracle.params(3, (n, n, n), bc=oracle.BC_OUTFLOW, gamma=1.4, cfl=0.5)
    d, _ = oracle.dt(U, P)
    gomp.omp_set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.step(U, P, d)
        sec = time.perf_counter() - t0
    finally:
        gomp.omp_set_num_threads(before)
    return {"value": n ** 3 / sec, "unit": "zone-updates/s", "cores": 1,
            "sample": f"one {n}^3 Sedov oracle step on one thread"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_1711_06203_b300 import inputs
    n = args.n
    U, _ = inputs.sedov(n)
    # warm-up steps from the initial state, then the timed run from the
    # initial state again, bounded so that it ends in minutes: the oracle's
    # cost per step barely depends on the state, so the first steps of the
    # run stand for all of them
    cpu_oracle_rate(U, n, args.warmup, budget_s=60.0)
    rate, done, t, _ = cpu_oracle_rate(U, n, args.steps, budget_s=150.0)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "3D PPM zone-updates/s", "value": rate, "unit": "zone-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "steps_done": done,
        "config": {"workload": f"sedov3d_{n}^3_{args.steps}steps", "n": n, "gamma": 1.4, "cfl": 0.5,
                   "bc": "outflow", "steps_from_initial_state": args.steps},
        "cpu_baseline": {"value": rate, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"the first {done} of the {args.steps} {n}^3 oracle steps from the initial "
                                   f"state, after {args.warmup} warm-up steps"},
        "e2e": {"value": rate, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_moving(args, dev, stream, n=128, steps=20):
    """The step on data in which every zone moves: a periodic 128^3 box of
    the random state of the batched level (rho, p lognormal, velocities
    N(0, 0.1), gamma 5/3, seed 1711), so no zone is at rest and the kernels'
    at-rest paths never apply.  Steps at a fixed dt of half the initial CFL
    step, timed with events after 3 warm-up steps."""
    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    U0 = inputs.random_box(np.random.default_rng(1711), (n, n, n), 3)
    ctx = hb.Context(dev.index)
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5)
    a = torch.from_numpy(U0).to(dev)
    b = torch.empty_like(a)
    box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_PERIODIC)
    dt = 0.5 * ctx.hydro_dt(box(a), p, stream)
    for _ in range(3):
        ctx.hydro_advance_box(box(a), box(b), p, dt, stream=stream)
    ctx.hydro_ctx_set_profiling(True)  # per-stage events, as in the Sedov run
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        ctx.hydro_advance_box(box(a), box(b), p, dt, stream=stream)
        a, b = b, a
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    stage_ms, calls = ctx.hydro_ctx_stage_times()
    physical = ctx.hydro_ctx_check() == hb.HYDRO_OK  # no zone met a non-physical state
    ctx.close()
    return {"workload": f"random-state {n}^3 periodic box (every zone moving), fixed dt", "steps": steps,
            "ms_per_step": ms, "zone_updates_per_s": n ** 3 / (ms * 1e-3), "physical": physical,
            "stages_ms_per_step": {k: v / calls for k, v in stage_ms.items()} if calls else None,
            "note": "no zone at rest: the tracing and final-solve shortcuts for gas at rest never apply"}


def bench_sod(args, dev, stream, steps=50):
    """2-D Sod shock tube along x on one 64x64 box (4 ghost zones, outflow,
    gamma 1.4, CFL 0.5): 50 steps from the initial state, each taking the CFL
    step the library returns, timed with events around the whole run.  The
    run is repeated: the first pass warms up, the second is reported."""
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    n = 64
    U0 = inputs.sod(n, 2, 0)
    ctx = hb.Context(dev.index)
    p = hb.params(2, gamma=1.4, cfl=0.5)
    a0 = torch.from_numpy(U0).to(dev)
    b = torch.empty_like(a0)
    box = lambda t: hb.box(t, (n, n, 1), (1.0 / n,) * 3, hb.BC_OUTFLOW)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        a = a0.clone()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        dt, t = ctx.hydro_dt(box(a), p, stream), 0.0
        for _ in range(steps):
            t += dt
            dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    # the same run as a device-resident time loop (hydro_advance_box_steps:
    # the CFL step stays on the device, two captured one-box graphs)
    dt_dev = torch.zeros(2, dtype=torch.float64, device=dev)
    t_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    a = torch.empty_like(a0)
    for _ in range(2):  # the same buffers both passes: the second replays the captured step graphs
        a.copy_(a0)
        t_dev.zero_()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        dt_dev[0] = ctx.hydro_dt(box(a), p, stream)
        ctx.hydro_advance_box_steps(box(a), box(b), p, steps, dt_dev, t_dev, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms_loop = e0.elapsed_time(e1) / steps
    t_loop = t_dev.item()
    ctx.close()
    return {"workload": "sod2d_64^2_50steps: Sod along x, 64x64, outflow, gamma 1.4, CFL 0.5", "steps": steps,
            "t_final": t, "ms_per_step": ms, "zone_updates_per_s": n * n / (ms * 1e-3),
            "note": "hydro_advance_box per step: launch- and host-sync-bound (each step returns its CFL step "
                    "to the host)",
            "device_loop": {"ms_per_step": ms_loop, "zone_updates_per_s": n * n / (ms_loop * 1e-3),
                            "t_final": t_loop, "call": "hydro_advance_box_steps"}}


def bench_batch(args, dev, stream, cpu_sample=False):
    """Batched level: 512 boxes, sides drawn from {16,24,32,48,64} per axis
    (seed 1711), random prefilled states, gamma = 5/3, dx = 1/64, one step at
    the level dt (min over boxes).  The batched step (one launch per stage over
    all boxes, graph-replayed, autotuned sweeps) against 512 per-box launches."""
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    sizes, Us = inputs.level_boxes(512, seed=1711)
    zones = sum(a * b * c for a, b, c in sizes)
    dx = (1.0 / 64,) * 3
    a = [torch.from_numpy(U).to(dev) for U in Us]
    del Us
    out = [torch.empty_like(x) for x in a]
    bin_ = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(a, sizes)]
    bout = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(out, sizes)]
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5)
    ctx = hb.Context(dev.index)
    level_dt = min(ctx.hydro_dt(bx, p, stream) for bx in bin_)
    dt_dev = torch.full((len(sizes),), level_dt, dtype=torch.float64, device=dev)
    dt_next = torch.empty_like(dt_dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ctx.hydro_advance_batch(bin_, bout, p, dt_dev, dt_next, stream=stream)  # plan, tuning, graph
    torch.cuda.synchronize(dev)
    plan_ms = 1e3 * (time.perf_counter() - t0)
    reps = max(3, min(args.steps, 10))

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    l0 = ctx.hydro_ctx_launches()
    ms_batch = timed(lambda: ctx.hydro_advance_batch(bin_, bout, p, dt_dev, dt_next, stream=stream), reps)
    launches_batch = (ctx.hydro_ctx_launches() - l0) // (reps + 2)

    def per_box():
        for bi, bo in zip(bin_, bout):
            ctx.hydro_advance_box(bi, bo, p, level_dt, stream=stream)

    l0 = ctx.hydro_ctx_launches()
    ms_plain = timed(per_box, max(2, reps // 3))
    launches_plain = (ctx.hydro_ctx_launches() - l0) // (max(2, reps // 3) + 2)
    # the same 512 per-box steps captured once into a CUDA graph and replayed
    ms_graph, graph_error = None, None
    try:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            for bi, bo in zip(bin_, bout):
                ctx.hydro_advance_box(bi, bo, p, level_dt, stream=side)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            ms_graph = timed(graph.replay, max(2, reps // 3))
        del graph
    except Exception as e:  # reported, not fatal: the other figures stand
        graph_error = f"{type(e).__name__}: {e}"[:200]
    tuning = ctx.hydro_batch_tuning()
    ctx.close()
    cpu = None
    if cpu_sample:
        # the CPU oracle on the level's boxes in order, one step each, until
        # about 8 s of host time are spent
        import oracle
        done_zones, t_cpu, nb = 0, 0.0, 0
        for x, sz in zip(a, sizes):
            U = x.cpu().numpy()
            P = oracle.params(3, sz, dx=dx, bc=oracle.BC_PREFILLED, gamma=5.0 / 3.0, cfl=0.5)
            t0 = time.perf_counter()
            oracle.step(U, P, level_dt)
            t_cpu += time.perf_counter() - t0
            done_zones += sz[0] * sz[1] * sz[2]
            nb += 1
            if t_cpu > 8.0:
                break
        cpu = {"zone_updates_per_s": done_zones / t_cpu, "cores": os.cpu_count(),
               "sample": f"one oracle step of each of the first {nb} boxes ({done_zones} zones)"}
    return {"workload": "level of 512 boxes, sides from {16,24,32,48,64} (seed 1711), prefilled, gamma 5/3",
            "interior_zones": zones, "zone_updates_per_s": zones / (ms_batch * 1e-3), "ms_per_step": ms_batch,
            "per_box_zone_updates_per_s": zones / (ms_plain * 1e-3), "per_box_ms_per_step": ms_plain,
            "speedup_vs_per_box": ms_plain / ms_batch, "launches_per_step": launches_batch,
            "per_box_graph_ms_per_step": ms_graph,
            "per_box_graph_zone_updates_per_s": zones / (ms_graph * 1e-3) if ms_graph else None,
            "speedup_vs_per_box_graph": ms_graph / ms_batch if ms_graph else None, "per_box_graph_error": graph_error,
            "per_box_launches_per_step": launches_plain, "plan_build_ms": plan_ms,
            "tracing_by_axis_extent": {f"{'xyz'[a]}{e}": (f"sweep {v}" if v else "rows/tiles")
                                       for (a, e), v in sorted(tuning.items())},
            "l2": "working set 3.7 GB of state + scratch, larger than L2", "cpu_oracle": cpu,
            "gpu_over_cpu_oracle": (zones / (ms_batch * 1e-3)) / cpu["zone_updates_per_s"] if cpu else None}


def batch_profile(args):
    """Batched steps of the first NBOX boxes of the 512-box level (same seed
    and shapes), one plan build then args.steps graph replays; prints the
    per-step time.  No per-box runs, so a profiler capture stays small."""
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    dev = torch.device("cuda", 0)
    sizes, Us = inputs.level_boxes(512, seed=1711)
    sizes, Us = sizes[:args.batch_profile], Us[:args.batch_profile]
    dx = (1.0 / 64,) * 3
    a = [torch.from_numpy(U).to(dev) for U in Us]
    out = [torch.empty_like(x) for x in a]
    bin_ = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(a, sizes)]
    bout = [hb.box(x, s, dx, hb.BC_PREFILLED) for x, s in zip(out, sizes)]
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5)
    ctx = hb.Context(0)
    dt_dev = torch.full((len(sizes),), 1e-4, dtype=torch.float64, device=dev)
    ctx.hydro_advance_batch(bin_, bout, p, dt_dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.hydro_advance_batch(bin_, bout, p, dt_dev)
    e1.record()
    torch.cuda.synchronize(dev)
    zones = sum(x * y * z for x, y, z in sizes)
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"boxes": len(sizes), "interior_zones": zones, "ms_per_step": ms,
                      "zone_updates_per_s": zones / (ms * 1e-3)}), flush=True)
    ctx.close()
    return 0


def stratified_device(n, dev, H=0.1, g=1.0, gamma=5.0 / 3.0, perturb=1e-3, seed=1711):
    """Isothermal atmosphere rho = exp(-z/H), p = rho g H (1 + perturb N(0,1)),
    at rest, built directly on the device (the recipe of inputs.stratified; a
    520^3 grown box is 5.6 GB per state, too large to stage through host numpy)."""
    import torch
    gsz = n + 8
    z = ((torch.arange(gsz, dtype=torch.float64, device=dev) - 4 + 0.5) / n).view(gsz, 1, 1)
    rho = torch.exp(-z / H).expand(gsz, gsz, gsz)
    p = rho * g * H
    if perturb:
        gen = torch.Generator(device=dev).manual_seed(seed)
        p = p * (1.0 + perturb * torch.randn((gsz, gsz, gsz), generator=gen, dtype=torch.float64, device=dev))
    U = torch.zeros((5, gsz, gsz, gsz), dtype=torch.float64, device=dev)
    U[0] = rho
    U[4] = p / (gamma - 1.0)
    return U


def bench_large(args, dev, stream):
    """Large box: 512^3 stratified atmosphere under g = -1 in z, seeded 1e-3
    pressure perturbations, periodic x/y, reflecting z, gamma 5/3, CFL 0.5;
    zone-updates/s and the step's algorithmic HBM traffic against the peak."""
    import torch

    from paper_1711_06203_b300 import binding as hb

    n = 512
    torch.cuda.empty_cache()
    a0 = stratified_device(n, dev)
    bc = ((hb.BC_PERIODIC,) * 2, (hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT,) * 2)
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5, grav=(0.0, 0.0, -1.0))

    def box(t):
        return hb.box(t, (n, n, n), (1.0 / n,) * 3, bc)

    steps = max(3, min(args.steps, 10))
    runs = {}
    # the default context (slab-by-slab step under the 16 GiB scratch
    # limit), then the whole-box step (137 GB of scratch) for comparison
    for name, limit in (("slabs", None), ("whole_box", 0)):
        a, b = a0.clone(), torch.empty_like(a0)
        ctx = hb.Context(dev.index)
        if limit is not None:
            ctx.hydro_ctx_set_scratch_limit(limit)
        dt = ctx.hydro_dt(box(a), p, stream)
        for _ in range(3):
            dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        torch.cuda.synchronize(dev)
        used = torch.cuda.mem_get_info(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        ctx.close()
        del a, b
        torch.cuda.empty_cache()
        free_after = torch.cuda.mem_get_info(dev)[0]
        # device memory the context held: what closing it and dropping the
        # two state buffers gave back, less the two states
        state_bytes = a0.numel() * a0.element_size()
        runs[name] = {"ms_per_step": ms, "zone_updates_per_s": n ** 3 / (ms * 1e-3),
                      "scratch_gb": (free_after - used[0] - 2 * state_bytes) / 1e9}
    del a0
    torch.cuda.empty_cache()
    ms = runs["slabs"]["ms_per_step"]
    hbm = algorithmic_bytes_per_step(n) / (ms * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6400.0)
    return {"workload": "512^3 stratified atmosphere, g = -1 in z, 1e-3 pressure perturbations, periodic x/y, "
                        "reflecting z", "steps_timed": steps, "ms_per_step": ms,
            "zone_updates_per_s": n ** 3 / (ms * 1e-3), "scratch_gb": runs["slabs"]["scratch_gb"],
            "whole_box": runs["whole_box"],
            "slab_over_whole_time": ms / runs["whole_box"]["ms_per_step"],
            "hbm_algorithmic_gbs": hbm, "hbm_peak_gbs": peak,
            "hbm_frac": hbm / peak, "l2": "inputs far larger than L2 (5.6 GB per state)"}


def bench_level(args, dev, stream):
    """Multi-step level advance: a 192^3 domain (periodic x, reflecting y,
    outflow z) tiled by uneven boxes (sides from {16,24,32,48,64}, seed 1711),
    random initial state; every step is a device ghost fill, a batched
    graph-replayed step and the level dt reduction, with no host
    synchronisation.  Compared with the single box covering the domain."""
    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    domain = (192, 192, 192)
    lo, sizes = inputs.level_tiling(domain, seed=1711)
    U = inputs.random_box(np.random.default_rng(1711), domain, 3)
    bc = ((hb.BC_PERIODIC,) * 2, (hb.BC_REFLECT,) * 2, (hb.BC_OUTFLOW,) * 2)
    dx = (1.0 / 192,) * 3
    p = hb.params(3, gamma=5.0 / 3.0, cfl=0.5)
    ctx = hb.Context(dev.index)
    a = []
    for c, s in zip(lo, sizes):
        B = np.zeros((5, s[2] + 8, s[1] + 8, s[0] + 8))
        B[:, 4:-4, 4:-4, 4:-4] = U[:, 4 + c[2]:4 + c[2] + s[2], 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        a.append(torch.from_numpy(B).to(dev))
    b = [torch.empty_like(x) for x in a]
    da = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(a, sizes)]
    db = [hb.box(t, s, dx, hb.BC_PREFILLED) for t, s in zip(b, sizes)]
    big = torch.from_numpy(U).to(dev)
    big2 = torch.empty_like(big)
    dt0 = ctx.hydro_dt(hb.box(big, domain, dx, bc), p, stream)
    dt_dev = torch.full((len(sizes),), dt0, dtype=torch.float64, device=dev)
    dt_next = torch.empty_like(dt_dev)

    def level_step():
        nonlocal da, db
        ctx.hydro_fill_boundary(da, lo, 3, domain, bc, stream=stream)
        ctx.hydro_advance_batch(da, db, p, dt_dev, dt_next, stream=stream)
        ctx.hydro_level_min_dt(dt_next, dt_dev, stream=stream)
        da, db = db, da

    steps = max(4, min(args.steps, 10))
    for _ in range(4):  # plans for both parities, tuning, graphs
        level_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        level_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_level = e0.elapsed_time(e1) / steps
    dt = dt0
    for _ in range(2):
        dt = ctx.hydro_advance_box(hb.box(big, domain, dx, bc), hb.box(big2, domain, dx, bc), p, dt,
                                   want_dt_next=True, stream=stream)
        big, big2 = big2, big
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        dt = ctx.hydro_advance_box(hb.box(big, domain, dx, bc), hb.box(big2, domain, dx, bc), p, dt,
                                   want_dt_next=True, stream=stream)
        big, big2 = big2, big
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_single = e0.elapsed_time(e1) / steps
    ctx.close()
    zones = domain[0] * domain[1] * domain[2]
    return {"workload": f"192^3 domain tiled by {len(sizes)} uneven boxes (sides from {{16,24,32,48,64}}), "
                        "periodic x / reflecting y / outflow z, random state",
            "boxes": len(sizes), "steps_timed": steps, "ms_per_step": ms_level,
            "zone_updates_per_s": zones / (ms_level * 1e-3), "single_box_ms_per_step": ms_single,
            "single_box_zone_updates_per_s": zones / (ms_single * 1e-3),
            "host_syncs_per_step": 0}


def bench_options(args, dev, stream):
    """Cost of the step's options on the bench workload (Sedov 128^3): Einfeldt
    wave speeds, and the flux-form gravity energy source (with g = -1 in z)."""
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    n = 128
    U0, _ = inputs.sedov(n)
    ctx = hb.Context(dev.index)
    out = {}
    for name, kw in (("davis", {}), ("einfeldt", dict(einfeldt=True)),
                     ("gravity_cell", dict(grav=(0.0, 0.0, -1.0))),
                     ("gravity_flux", dict(grav=(0.0, 0.0, -1.0), flux_grav_energy=True))):
        p = hb.params(3, gamma=1.4, cfl=0.5, **kw)
        a = torch.from_numpy(U0).to(dev)
        b = torch.empty_like(a)
        box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_OUTFLOW)
        dt = ctx.hydro_dt(box(a), p, stream)
        for _ in range(3):
            dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k = 5
        for _ in range(k):
            dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / k
        out[name] = {"ms_per_step": ms, "zone_updates_per_s": n ** 3 / (ms * 1e-3)}
    ctx.close()
    return out


def bench_amr(args, dev, stream):
    """Two-level subcycled advance (refinement ratio 2): a 128^3 periodic
    coarse level in eight 64^3 boxes with a Gaussian pressure bump at the
    centre (smooth periodic background), refined over the central 64^3 coarse
    zones by eight 64^3 fine boxes (128^3 fine zones).  One coarse step =
    coarse fill + step, two fine fills + steps of dt/2, flux registers,
    reflux, average down and the two-level dt, with no host synchronisation.
    Zone-updates count 128^3 coarse + 2 x 128^3 fine per coarse step.  Also
    timed: the same three batched steps without the synchronisation, giving
    the cost of the AMR machinery on top of the hydro steps."""
    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    domain = (128, 128, 128)
    clo = [(x, y, z) for z in (0, 64) for y in (0, 64) for x in (0, 64)]
    csz = [(64, 64, 64)] * 8
    flo = [(x, y, z) for z in (64, 128) for y in (64, 128) for x in (64, 128)]
    fsz = [(64, 64, 64)] * 8
    Uc, Uf, dx = inputs.amr_two_level(domain, 3, flo, fsz, gamma=1.4, p_amp=20.0, r0=0.08)
    dxf = tuple(v / 2 for v in dx)
    ca = []
    for c, s in zip(clo, csz):
        B = np.zeros((5, s[2] + 8, s[1] + 8, s[0] + 8))
        B[:, 4:-4, 4:-4, 4:-4] = Uc[:, 4 + c[2]:4 + c[2] + s[2], 4 + c[1]:4 + c[1] + s[1], 4 + c[0]:4 + c[0] + s[0]]
        ca.append(torch.from_numpy(B).to(dev))
    cb = [torch.empty_like(t) for t in ca]
    fa = [torch.from_numpy(U).to(dev) for U in Uf]
    fb = [torch.empty_like(t) for t in fa]
    del Uc, Uf
    bc = ((hb.BC_PERIODIC,) * 2,) * 3
    p = hb.params(3, gamma=1.4, cfl=0.5)
    ctx = hb.Context(dev.index)
    dt = torch.full((1,), 0.3 * dx[0] / 8.0, dtype=torch.float64, device=dev)
    dt_next = torch.empty_like(dt)

    def amr_step():
        nonlocal ca, cb, fa, fb
        ctx.hydro_amr_advance([hb.box(t, s, dx) for t, s in zip(ca, csz)], [hb.box(t, s, dx) for t, s in zip(cb, csz)],
                              clo, [hb.box(t, s, dxf) for t, s in zip(fa, fsz)],
                              [hb.box(t, s, dxf) for t, s in zip(fb, fsz)], flo, 3, domain, bc, p, dt, dt_next,
                              stream=stream)
        dt.copy_(dt_next)
        ca, cb, fa, fb = cb, ca, fb, fa

    steps = max(4, min(args.steps, 10))
    for _ in range(4):  # tables, batch plans for both parities, tuning, graphs
        amr_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        amr_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_amr = e0.elapsed_time(e1) / steps

    # the three batched steps alone (ghosts as they are: timing only)
    dtc = torch.full((8,), dt.item(), dtype=torch.float64, device=dev)
    dtf = dtc * 0.5
    dn = torch.empty_like(dtc)
    ft = [torch.empty_like(t) for t in fa]
    pre = hb.BC_PREFILLED

    def hydro_only():
        ctx.hydro_advance_batch([hb.box(t, s, dx, pre) for t, s in zip(ca, csz)],
                                [hb.box(t, s, dx, pre) for t, s in zip(cb, csz)], p, dtc, dn, stream=stream)
        ctx.hydro_advance_batch([hb.box(t, s, dxf, pre) for t, s in zip(fa, fsz)],
                                [hb.box(t, s, dxf, pre) for t, s in zip(ft, fsz)], p, dtf, dn, stream=stream)
        ctx.hydro_advance_batch([hb.box(t, s, dxf, pre) for t, s in zip(ft, fsz)],
                                [hb.box(t, s, dxf, pre) for t, s in zip(fb, fsz)], p, dtf, dn, stream=stream)

    for _ in range(2):
        hydro_only()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        hydro_only()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_hydro = e0.elapsed_time(e1) / steps
    ctx.close()
    zu = 128 ** 3 + 2 * 128 ** 3
    return {"workload": "two-level 128^3 coarse (8 x 64^3) + 128^3 fine (8 x 64^3) over the central 64^3 coarse "
                        "zones, periodic, Gaussian pressure bump",
            "steps_timed": steps, "ms_per_coarse_step": ms_amr, "zone_updates_per_coarse_step": zu,
            "zone_updates_per_s": zu / (ms_amr * 1e-3), "hydro_steps_only_ms": ms_hydro,
            "sync_overhead_frac": (ms_amr - ms_hydro) / ms_amr}


def bench_mol(args, dev, stream, cpu_sample=True):
    """Method-of-lines step with passive species, the configuration of the
    paper's GPU proxy (Sedov, 13 advected species): Sedov 128^3 (gamma 1.4,
    outflow) with 13 species of seeded Dirichlet mass fractions, SSP-RK2,
    CFL 0.4.  Also the same step without species, and the CPU oracle's
    method-of-lines rate on a 64^3 sample with 13 species."""
    import time

    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    n = args.n
    U0, _ = inputs.sedov(n)
    X = inputs.species_fractions(np.random.default_rng(1711), U0.shape[1:], 13)
    ctx = hb.Context(dev.index)
    p = hb.params(3, gamma=1.4, cfl=0.4)
    out = {"workload": f"sedov3d_{n}^3 + 13 passive species, SSP-RK2 method of lines, outflow"}
    for nspec in (13, 0):
        U = inputs.with_species(U0, X[:nspec])
        a = torch.from_numpy(U).to(dev)
        b = torch.empty_like(a)
        box = lambda t: hb.box(t, (n, n, n), (1.0 / n,) * 3, hb.BC_OUTFLOW)
        dt = ctx.hydro_dt(box(a), p, stream)
        for _ in range(3):
            dt = ctx.hydro_mol_advance_box(box(a), box(b), p, nspec, dt, want_dt_next=True, stream=stream)
            a, b = b, a
        torch.cuda.synchronize(dev)
        k = max(3, min(args.steps, 10))
        l0 = ctx.hydro_ctx_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            ctx.hydro_mol_advance_box(box(a), box(b), p, nspec, dt, stream=stream)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / k
        key = "species_13" if nspec else "hydro_only"
        out[key] = {"ms_per_step": ms, "zone_updates_per_s": n ** 3 / (ms * 1e-3), "steps_timed": k,
                    "launches_per_step": (ctx.hydro_ctx_launches() - l0) / k,
                    "state_gb": a.numel() * 8 / 1e9}
        del a, b
    ctx.close()
    torch.cuda.empty_cache()
    if cpu_sample:
        import oracle

        m = 64
        Us, _ = inputs.sedov(m)
        Us = inputs.with_species(Us, inputs.species_fractions(np.random.default_rng(1711), Us.shape[1:], 13))
        P = oracle.params(3, (m, m, m), gamma=1.4, cfl=0.4)
        d, _ = oracle.dt(Us, P)
        t0 = time.perf_counter()
        oracle.mol_step(Us, P, d)
        sec = time.perf_counter() - t0
        out["cpu_oracle"] = {"zone_updates_per_s": m ** 3 / sec, "cores": os.cpu_count(),
                             "sample": f"one {m}^3 method-of-lines oracle step with 13 species"}
        out["gpu_over_cpu_oracle"] = out["species_13"]["zone_updates_per_s"] / out["cpu_oracle"]["zone_updates_per_s"]
    return out


def bench_serve(args, dev, zone_rate):
    """Serving stream: a seeded prefix of independent 3-D problems (Sod,
    Sedov, two-state; sides 32..256; 10-100 steps) arriving as a Poisson
    process at 0.7 x the measured plain capacity (requests/s), served by the
    continuous-batching server with state resident on the device, under the
    scheduling policy --serve-policy (default: response ratio, 2.5 ms
    quantum).  Beside the latency percentiles: the slowdown of each request
    (its latency over its own steps' cost alone on the GPU, at the server's
    measured cost per zone), and the host time spent choosing sets and
    enqueueing."""
    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    reqs = inputs.serve_requests(args.serve_requests, seed=1711)
    mean_work = np.mean([r["steps"] * r["n"] ** 3 for r in reqs])
    expected_work = np.mean([s ** 3 for s in inputs.SERVE_SIDES]) * 55.0
    capacity = zone_rate / expected_work  # requests per second the plain step sustains
    rate = 0.7 * capacity
    arrivals = inputs.poisson_arrivals(len(reqs), rate, seed=1711)
    torch.cuda.empty_cache()
    srv = hb.Server(dev.index, max_slots=64)
    policy = hb.SERVE_ALL if args.serve_policy == "all" else hb.SERVE_RESPONSE_RATIO
    srv.serve_set_policy(policy, args.serve_quantum_ms)
    t0 = time.perf_counter()
    ids = []
    for r, ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        ids.append(srv.serve_submit(**r))
    res = [srv.serve_poll(i, timeout_ms=-1) for i in ids]
    wall = time.perf_counter() - t0
    st = srv.serve_stats()
    srv.close()
    lat = np.array([r["latency_ms"] for r in res])
    alone = np.array([q["steps"] * st["ms_per_unit"] * (q["n"] + 3) ** 3 for q in reqs])
    slow = lat / alone
    work = sum(r["zone_updates"] for r in res)
    ok = sum(1 for r in res if r["status"] == 0)
    return {"workload": "prefix of a seeded stream of 3-D Sod/Sedov/two-state requests, sides {32..256}, "
                        "10-100 steps, Poisson arrivals at 0.7 x plain capacity",
            "policy": args.serve_policy, "quantum_ms": args.serve_quantum_ms if policy else None,
            "requests": len(reqs), "completed_ok": ok, "arrival_rate_per_s": rate,
            "plain_capacity_requests_per_s": capacity, "mean_work_zone_updates": float(mean_work),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "slowdown_p50": float(np.percentile(slow, 50)), "slowdown_p99": float(np.percentile(slow, 99)),
            "alone_p50_ms": float(np.percentile(alone, 50)), "alone_p99_ms": float(np.percentile(alone, 99)),
            "mean_queue_ms": float(np.mean([r["queue_ms"] for r in res])),
            "zone_updates_per_s": work / wall, "busy_zone_updates_per_s": st["zone_updates"] / (st["busy_ms"] * 1e-3),
            "iterations": st["iterations"], "box_steps": st["box_steps"],
            "enqueue_ms_per_iteration": st["enqueue_ms"] / max(1, st["iterations"]),
            "busy_ms_per_iteration": st["busy_ms"] / max(1, st["iterations"]), "wall_s": wall,
            "hbm_budget_gb": st["hbm_budget"] / 1e9, "scratch_pool_gb": st["hbm_scratch_pool"] / 1e9}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1711_06203_b300 import binding as hb
    from paper_1711_06203_b300 import inputs

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    n = args.n
    dx = (1.0 / n,) * 3
    U0, ndep = inputs.sedov(n)
    ctx = hb.Context(local_rank)
    p = hb.params(3, gamma=1.4, cfl=0.5)
    a0 = torch.from_numpy(U0).to(dev)  # the initial state, kept for the timed and e2e runs
    a = a0.clone()
    b = torch.empty_like(a)
    stream = torch.cuda.current_stream(dev)

    def box(t):
        return hb.box(t, (n, n, n), dx, hb.BC_OUTFLOW)

    # warm-up: W untimed steps on a copy of the initial state (library
    # scratch, caches, clocks); the timed run then starts again from t = 0
    dt = ctx.hydro_dt(box(a), p, stream)
    for _ in range(args.warmup):
        dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
        a, b = b, a
    a.copy_(a0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.hydro_ctx_set_profiling(True)
    launches0 = ctx.hydro_ctx_launches()
    gpu_id = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None else str(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if sampler:
        sampler.wait_first()
    t_wall0 = time.time()
    wall0 = time.perf_counter()
    t_sim = 0.0
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        if k == 0:
            dt = ctx.hydro_dt(box(a), p, stream)  # the run's first CFL step, from the initial state
        t_sim += dt
        dt = ctx.hydro_advance_box(box(a), box(b), p, dt, want_dt_next=True, stream=stream)
        ev[k][1].record(stream)
        a, b = b, a
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    t_wall1 = time.time()
    clocks = sampler.stop(t_wall0, t_wall1) if sampler else None
    if dist:
        dist.barrier()
    launches = ctx.hydro_ctx_launches() - launches0
    stage_ms, calls = ctx.hydro_ctx_stage_times()
    ctx.hydro_ctx_set_profiling(False)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    zones = n ** 3
    value = whole_job_rate(zones, world, args.steps, total_ms)
    # the same run's steps 6-25: the early blast, when most of the box is at rest
    early = step_ms[5:25]
    early_window = ({"steps": "6-25", "ms_per_step": sum(early) / len(early),
                     "zone_updates_per_s": zones * len(early) / (sum(early) * 1e-3)} if len(early) == 20 else None)

    # end to end through the public host-buffer call: the same run from the
    # initial state, every step copying the pinned host state in and the
    # result out, inside the events
    h_in = torch.empty(a.shape, dtype=a.dtype, pin_memory=True)
    h_in.copy_(a)
    h_out = torch.empty_like(h_in, pin_memory=True)
    ctx.hydro_advance_box_host(box(h_in), box(h_out), p, dt, stream=stream)  # sizes the staging buffers
    h_in.copy_(a0)
    e2e_steps = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    dt = ctx.hydro_dt(box(a0), p, stream)
    for _ in range(e2e_steps):
        dt = ctx.hydro_advance_box_host(box(h_in), box(h_out), p, dt, want_dt_next=True, stream=stream)
        h_in, h_out = h_out, h_in
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    # outflow faces derive their ghost zones, so only the interior rows of
    # each field's interior z-planes cross the host link, in both directions
    nbytes = 5 * n * n * (n + 8) * a.element_size()
    sod = bench_sod(args, dev, stream) if world == 1 and not args.no_batch else None
    moving = bench_moving(args, dev, stream) if world == 1 else None

    # roofline of the dominant stage (FP64 ALU bound: every stage is)
    units = units_per_step(n)
    per_step = {k: v / calls for k, v in stage_ms.items()}
    dom = max(per_step, key=per_step.get)
    flops = FLOPS_PER_UNIT[dom] * units[dom]
    achieved = flops / (per_step[dom] * 1e-3) / 1e9
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    step_gbs = algorithmic_bytes_per_step(n) / (total_ms / args.steps * 1e-3) / 1e9
    step_gflops = sum(FLOPS_PER_UNIT[k] * units[k] for k in units) / (total_ms / args.steps * 1e-3) / 1e9

    # the device's FP64 rate, measured now (eight independent multiply-add
    # chains per thread over a resident grid): the issue ceiling that the
    # derived peak (unit counts x clock) overstates
    fp64_measured = hb.hydro_selftest_fp64_rate(stream=stream)

    batch = None
    if world == 1 and not args.no_batch:
        batch = bench_batch(args, dev, stream, cpu_sample=not args.no_cpu_baseline)
    serve = None
    if world == 1 and args.serve_requests > 0:
        serve = bench_serve(args, dev, value)
    level = None
    options = None
    amr = None
    mol = None
    if world == 1 and not args.no_batch:
        level = bench_level(args, dev, stream)
        options = bench_options(args, dev, stream)
        amr = bench_amr(args, dev, stream)
        mol = bench_mol(args, dev, stream, cpu_sample=not args.no_cpu_baseline)
    large = None
    if world == 1 and not args.no_large:
        large = bench_large(args, dev, stream)

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, done, t, _ = cpu_oracle_rate(U0, n, 50, budget_s=20.0)
        cpu = {"value": rate, "unit": "zone-updates/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} full {n}^3 oracle steps from the initial Sedov state",
               "cpu_model": cpu_model(), "one_core": cpu_oracle_rate_one_core()}
    line = {
        "metric": "3D PPM zone-updates/s", "value": value, "unit": "zone-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": statistics.median(step_ms), "ms_per_step_range": [min(step_ms), max(step_ms)],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"sedov3d_{n}^3_{args.steps}steps", "n": n, "gamma": 1.4, "cfl": 0.5,
                   "bc": "outflow", "steps_from_initial_state": args.steps, "t_final": t_sim,
                   "deposit_zones": ndep, "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"replica x{world}"},
        "early_window": early_window,
        "sod2d": sod,
        "moving_state": moving,
        "at_rest_note": ("every zone is traced and every face solved each step; in zones at rest (the ambient gas "
                         "around the blast) the kernels skip arithmetic whose terms are exactly zero (flat "
                         "parabolas, vanishing slopes, equal fluxes), with bit-identical results; moving_state "
                         "is the rate where no zone is at rest"),
        "roofline": {"bound": "alu", "kernel": f"{dom} stage ({LAUNCHES_PER_STEP_3D[dom]} launches/step)",
                     "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                     "frac": achieved / FP64_PEAK_GFLOPS,
                     "traffic": (DRAM_BYTES_PER_UNIT[dom] * units[dom] / LAUNCHES_PER_STEP_3D[dom]
                                 if dom in DRAM_BYTES_PER_UNIT else None),
                     "traffic_note": "bytes per launch: ncu dram read+write of a 96^3 capture, scaled by units",
                     "peak_note": "FP64 derived: 148 SMs x 2 FMA lanes x 2 flop x 2.032 GHz",
                     "peak_measured": fp64_measured, "frac_of_measured": achieved / fp64_measured,
                     "peak_measured_note": "hydro_selftest_fp64_rate in this run: dependency-free DFMA chains, "
                                           "2 flops per FMA",
                     "flop_note": "algorithmic flops (the oracle's +, -, *, /, sqrt, each counted once), not "
                                  "the hardware's issued operations: an FMA counts 2, a divide or square root 1 "
                                  "although it issues 4-9 FP64 instructions"},
        "step_fp64": {"algorithmic_gflops": step_gflops, "frac_of_derived": step_gflops / FP64_PEAK_GFLOPS,
                      "frac_of_measured": step_gflops / fp64_measured,
                      "note": "the oracle's operation count per unit, which forms every slope, interface value and "
                              "swept-volume integral; the tracing kernels skip those of zones at rest (flat data, "
                              "bit-identical results), so on a blast in a quiescent box this rate counts work the "
                              "GPU does not issue.  The roofline's dominant stage (intermediate solves) skips "
                              "nothing."},
        "hbm": {"achieved_gbs": step_gbs, "peak_gbs": hbm_peak, "frac": step_gbs / hbm_peak,
                "nominal_peak_gbs": 7700.0, "frac_of_nominal": step_gbs / 7700.0,
                "note": "algorithmic bytes of the whole step (read grown box, write interior) / step time, of measured"},
        "step_gflops": step_gflops,
        "stages_ms_per_step": per_step,
        "cpu_baseline": cpu,
        "e2e": {"value": zones / (e2e_ms * 1e-3) * world, "unit": "zone-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "batched_level": batch,
        "serve": serve,
        "large_box": large,
        "level_multistep": level,
        "options": options,
        "amr_two_level": amr,
        "mol_species": mol,
        "gpu_launches": launches,
        "wall_s_timed": wall,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed steps from the initial state (the workload is 200)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=128, help="box side (the workload is 128)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-level leg")
    ap.add_argument("--serve-requests", type=int, default=200, help="served request prefix (0 skips the leg)")
    ap.add_argument("--serve-policy", choices=("ratio", "all"), default="ratio",
                    help="serving policy: response ratio within a quantum (default) or every request every iteration")
    ap.add_argument("--serve-quantum-ms", type=float, default=2.5)
    ap.add_argument("--serve-plain-rate", type=float, default=5.6e8,
                    help="--serve-only: plain zone-updates/s that sets the arrival rate (0.7 x capacity)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving leg (at the plain rate measured by a short Sedov run) and print it")
    ap.add_argument("--no-large", action="store_true", help="skip the 512^3 large-box leg")
    ap.add_argument("--mol-only", action="store_true",
                    help="run only the method-of-lines leg at --n and print its JSON (for profiling)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched-level leg and print its JSON (for profiling)")
    ap.add_argument("--sod-only", action="store_true",
                    help="run only the 2-D Sod 64^2 leg and print its JSON (for profiling)")
    ap.add_argument("--moving-only", action="store_true",
                    help="run only the every-zone-moving 128^3 leg and print its JSON (for profiling)")
    ap.add_argument("--batch-profile", type=int, default=0, metavar="NBOX",
                    help="only batched steps of the first NBOX boxes of the level, no per-box comparison "
                         "(a small case for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_profile:
        return batch_profile(args)
    if args.serve_only:
        import torch

        dev = torch.device("cuda", 0)
        with torch.cuda.device(dev):
            print(json.dumps(bench_serve(args, dev, args.serve_plain_rate)), flush=True)
        return 0
    if args.mol_only or args.batch_only or args.moving_only or args.sod_only:
        import torch

        dev = torch.device("cuda", 0)
        with torch.cuda.device(dev):
            stream = torch.cuda.current_stream(dev)
            if args.mol_only:
                leg = bench_mol(args, dev, stream, cpu_sample=False)
            elif args.batch_only:
                leg = bench_batch(args, dev, stream)
            elif args.sod_only:
                leg = bench_sod(args, dev, stream)
            else:
                leg = bench_moving(args, dev, stream)
            print(json.dumps(leg), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
