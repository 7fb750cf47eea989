"""Benchmarks of the 2DSW and UFLES time steps.

Default workload (the headline line): the 2DSW time step on the 4096 x 4096
wet/dry grid, FP32.  Other workloads (--workload): ``ensemble`` (512
instances, persistent kernel vs separate launches), ``les`` (256x256x128
UFLES step at 1e-6 residual) and ``les-nn`` (the same, learned warm start
vs previous-pressure warm start on the same states).

One benchmark step = 900 model time steps of the 4096^2 grid (the fused
momentum / continuity / Shapiro / update kernel, temporally blocked: 300
launches of 3 fused steps) plus the FP64 volume reduction, i.e. every 2DSW
row of the hot path.  The state (268 MB of eta, u, v, H) is larger than the
129 MB L2, so no L2 flush is needed between steps.

The same line carries an ``les`` object: the UFLES 256x256x128 step at a
1e-6 FP64 residual over steps 21..200, the previous-pressure warm start and
the learned (U-Net) warm start compared on the same 10 states spread evenly
over those steps, with device times, SOR iterations, end-to-end wall time
through les_step and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbsw|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an
independent replica (the workload has no exchange step), the timed region
is bracketed by barriers and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_SIDE = 4096
STEPS_PER_BENCH_STEP = 900  # a multiple of every fusion depth 1..6: each launch fuses T whole steps
BYTES_PER_CELL_UPDATE = 28  # read eta, u, v, H; write eta, u, v (FP32)
METRIC = "cell-updates/s"
WORKLOAD = "2DSW 4096x4096 wet/dry (15% dry), FP32, 900 time steps + FP64 volume per step"
CSRC = os.path.join(ROOT, "paper_1711_04471_gb300", "csrc")

# DRAM bytes (read + write) per unit from ncu captures of the kernels below,
# with the SHA-256 (first 16 hex digits) of the kernel's source files at the
# time of the capture.  When a source changes the figure is stale: the
# bench then reports traffic as null until the kernel is captured again.
NCU_TRAFFIC = {
    # one sw_stream_kernel<3> launch on the 4096^2 grid
    "sw_stream_kernel<3>": ((297.057536 + 163.139072) * 1e6, ("sw_stream.cuh", "sw_kernels.cuh"), "fdc57507af7e9c15"),
    # one SOR iteration (red + black half-sweep) on 256x256x128, L2 warm (a single-pass capture of
    # the two DRAM counters, so that no replay changes what the L2 holds)
    "sor_iteration_256x256x128": ((2.642944 + 1.674496 + 2.863872 + 3.123200) * 1e6, ("poisson.cu", "poisson.cuh"),
                                  "ca5a6546772cd4c6"),
}


def source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """(bytes per unit, None) if the capture matches today's source, else (None, why)."""
    val, files, digest = NCU_TRAFFIC[key]
    try:
        now = source_hash(files)
    except OSError:
        return None, "kernel source not found"
    if now != digest:
        return None, f"stale: {'/'.join(files)} changed since the ncu capture"
    return val, None


def host_info() -> dict:
    """Host cores and CPU model (the oracle's timing platform)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:
        usable = os.cpu_count()
    return {"nproc": os.cpu_count(), "usable_cores": usable, "cpu_model": model or "unknown"}


def _l2_mb():
    """L2 size of the current device in MB (0 if unknown)."""
    try:
        import torch
        return getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 0) / 1e6
    except Exception:
        return 0.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampler run during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda_ok() else "gloo")
    return rank, world, local


def _cuda_ok():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda_ok() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sw(nsteps_serial=20, nsteps_omp=60, side=N_CELLS_SIDE):
    """The FP64 oracle on a bounded sample of the same workload (time steps
    of the full 4096^2 grid): its serial build on one thread and its OpenMP
    build on all host cores.  Returns the cpu_baseline object."""
    import oracle
    from paper_1711_04471_gb300 import inputs
    inp = inputs.sw_wetdry(n=side, seed=1001)
    res = {}
    for omp, n in ((False, nsteps_serial), (True, nsteps_omp)):
        oracle.use_openmp(omp)
        try:
            s = oracle.SWState(inp.params(), inp.H, inp.eta0)
            s.run(1)
            t0 = time.perf_counter()
            s.run(n)
            dt = time.perf_counter() - t0
        finally:
            oracle.use_openmp(False)
        res[omp] = (side * side * n / dt, dt, n)
    threads = oracle.threads()
    v, dt, n = res[True]
    v1, dt1, n1 = res[False]
    return {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{n} time steps of the full 4096^2 grid, FP64 oracle (OpenMP build, {threads} threads, "
                      f"{dt:.1f} s)",
            "single_thread": {"value": v1, "unit": METRIC, "cores": 1,
                              "sample": f"{n1} time steps of the full 4096^2 grid, serial build ({dt1:.1f} s)"},
            "host": host_info()}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1711_04471_gb300 import inputs
    inp = inputs.sw_wetdry(n=N_CELLS_SIDE, seed=1001)
    oracle.use_openmp(True)       # the oracle's OpenMP build: all host cores, results bitwise equal to the serial one
    threads = oracle.threads()
    s = oracle.SWState(inp.params(), inp.H, inp.eta0)
    for _ in range(args.warmup):
        s.run(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.run(1)
    dt = time.perf_counter() - t0
    oracle.use_openmp(False)
    cells = N_CELLS_SIDE ** 2 * args.steps
    value = cells / dt
    sample = (f"{args.steps} time steps of the full 4096^2 grid (1 model step per bench step), FP64, "
              f"{threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [N_CELLS_SIDE, N_CELLS_SIDE]},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gbsw(args, rank, world, local):
    import numpy as np
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.sw import SW

    P.build()
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    inp = inputs.sw_wetdry(n=N_CELLS_SIDE, seed=1001)
    cells = N_CELLS_SIDE * N_CELLS_SIDE
    sw = SW(inp.params(), inp.H, inp.eta0, stream=stream)
    if args.blocking:
        sw.set_blocking(args.blocking)
    T = args.blocking or 3
    fused_launches = math.ceil(STEPS_PER_BENCH_STEP / T)
    whole = STEPS_PER_BENCH_STEP % T == 0       # every launch of the timed step fuses T time steps
    launches_per_step = fused_launches + 2      # + the two volume-reduction kernels

    # ---- device-resident throughput (value) ----
    for _ in range(args.warmup):
        sw.step(STEPS_PER_BENCH_STEP)
        sw.volume()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    vols = []
    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        sw.step(STEPS_PER_BENCH_STEP)
        ev[k][1].record(stream)
        vols.append(sw.volume())  # synchronises: the step's result is read back
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_ms = start.elapsed_time(end)
    t_ms = max_over_ranks(t_ms, world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    fused_launch_ms = sum(step_ms) / (args.steps * fused_launches)
    value = cells * STEPS_PER_BENCH_STEP * args.steps * world / (t_ms * 1e-3)

    # ---- end to end through the public API with host buffers ----
    ny = nx = N_CELLS_SIDE
    eta_h = torch.empty((ny, nx), dtype=torch.float32).pin_memory().numpy()
    u_h = torch.empty((ny, nx + 1), dtype=torch.float32).pin_memory().numpy()
    v_h = torch.empty((ny + 1, nx), dtype=torch.float32).pin_memory().numpy()
    sw.get_state(eta=eta_h, u=u_h, v=v_h, want=("eta", "u", "v"))
    e2e_steps = max(3, args.steps // 3)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sw.set_state(eta_h, u_h, v_h)
        sw.step(STEPS_PER_BENCH_STEP)
        sw.volume()
        sw.get_state(eta=eta_h, u=u_h, v=v_h, want=("eta", "u", "v"))
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    h2d = eta_h.nbytes + u_h.nbytes + v_h.nbytes
    d2h = h2d + 3 * 8
    e2e_value = cells * STEPS_PER_BENCH_STEP * e2e_steps * world / t_e2e
    sw.close()

    if rank != 0:
        return
    peak, peak_kind = _peaks()
    achieved_gbs = BYTES_PER_CELL_UPDATE * cells * T / (fused_launch_ms * 1e-3) / 1e9
    compulsory_gbs = BYTES_PER_CELL_UPDATE * cells / (fused_launch_ms * 1e-3) / 1e9
    traffic, traffic_note = (args.traffic, "given on the command line") if args.traffic is not None else \
        (ncu_traffic("sw_stream_kernel<3>") if T == 3 else (None, f"no ncu capture of T = {T}"))
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sw()
    les = None
    if world == 1 and not args.no_les:
        les = les_object(args, local)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [nx, ny], "time_steps_per_step": STEPS_PER_BENCH_STEP,
                   "steps_per_launch": T, "l2": "state 268 MB > 129 MB L2, no flush needed",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak, "traffic": traffic, "traffic_note": traffic_note,
                     "peak_kind": peak_kind, "kernel": f"sw_stream_kernel<{T}>",
                     "per_unit": f"{BYTES_PER_CELL_UPDATE} B/cell-update x {T} steps x {cells} cells per launch",
                     "compulsory_gbs": compulsory_gbs, "compulsory_frac": compulsory_gbs / peak,
                     "launch_ms": fused_launch_ms,
                     "launch_ms_from": f"{fused_launches} launches per step, each fusing {T} time steps" if whole
                     else f"{fused_launches} launches per step, the last one fusing {STEPS_PER_BENCH_STEP % T}"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "volume_drift": (vols[-1][0] - vols[0][0]) / vols[0][0],
        "les": les,
    }
    print(json.dumps(line), flush=True)


def _timed_region(fn, world):
    """Barrier + synchronize on both sides of fn(); returns seconds (max over ranks)."""
    import torch
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(time.perf_counter() - t0, world)


def run_ensemble(args, rank, world, local):
    """512 2DSW instances (sides log-uniform in [64, 1024]), STEPS_PER_BENCH_STEP
    time steps per bench step: one persistent cooperative kernel per call
    (CUDA graph) vs one launch per instance and fused level."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.sw import SWBatch
    P.build()
    torch.cuda.set_device(local)
    sizes = inputs.sw_ensemble_sizes(512, seed=1002)[:args.members]
    members = [inputs.sw_ensemble_member(int(n), 1002, k) for k, n in enumerate(sizes)]
    cells = int(sum(int(n) * int(n) for n in sizes))
    stream = torch.cuda.current_stream()
    b = SWBatch(members, stream=stream)
    T, rows = b.autotune(trial_steps=60, cache_path=os.environ.get("GBSW_TUNE_CACHE"))  # ~25 ms per candidate
    per = STEPS_PER_BENCH_STEP
    for _ in range(args.warmup):
        b.step(per)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_graph = _timed_region(lambda: [b.step(per) for _ in range(args.steps)], world)
    clk = clocks.stop()
    vols, _ = b.volumes()
    for _ in range(max(1, args.warmup // 2)):
        b.step_separate(per)
    t_sep = _timed_region(lambda: [b.step_separate(per) for _ in range(args.steps)], world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.step(per)
        b.volumes()          # per-step FP64 volumes read back to the host
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    b.close()
    if rank != 0:
        return
    value = cells * per * args.steps * world / t_graph
    peak, peak_kind = _peaks()
    levels = per // T + (1 if per % T else 0)
    level_s = t_graph / (args.steps * levels)
    ach = BYTES_PER_CELL_UPDATE * cells * T / level_s / 1e9
    line = {"metric": "ensemble cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_graph / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"2DSW ensemble: {len(sizes)} instances, sides log-uniform 64..1024, "
                                   f"{cells} cells, {per} time steps + FP64 volumes per step",
                       "tiling": {"steps_per_level": T, "rows_per_item": rows}},
            "separate_launches": {"value": cells * per * args.steps * world / t_sep, "unit": "cell-updates/s",
                                  "ms_per_step": t_sep / args.steps * 1e3},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "peak_kind": peak_kind, "kernel": "sw_batch_kernel",
                         "per_unit": f"{BYTES_PER_CELL_UPDATE} B/cell-update x {T} steps x {cells} cells per level"},
            "e2e": {"value": cells * per * args.steps / t_e2e, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 8 * 3 * 512},
            "gpu_launches": args.steps, "clocks": clk, "volume_min": float(min(vols))}
    print(json.dumps(line), flush=True)


def _les_cpu_sample(shape, solid, sor_iters=20, openmp=False):
    """Oracle (FP64; its serial build on one thread, or its OpenMP build on
    all host cores) on the full grid: one predictor pass and sor_iters SOR
    iterations, timed separately."""
    import oracle
    oracle.use_openmp(openmp)
    try:
        return _les_cpu_sample_run(shape, solid, sor_iters)
    finally:
        oracle.use_openmp(False)


def _les_cpu_sample_run(shape, solid, sor_iters):
    from oracle import les as ol
    nx, ny, nz = shape
    Pm = ol.make_params(nx, ny, nz)
    st = ol.LESState(Pm, solid)
    t0 = time.perf_counter()
    ol.velnw(Pm, st.p, st.u, st.v, st.w)
    ol.bondv1(Pm, st.u, st.v, st.w)
    fu, fv, fw = ol.velfg(Pm, st.u, st.v, st.w)
    ol.feedbf(Pm, solid, st.u, st.v, st.w, st.gu, st.gv, st.gw, fu, fv, fw)
    nt = ol.nut(Pm, st.u, st.v, st.w)
    ol.visc(Pm, st.u, st.v, st.w, nt, fu, fv, fw)
    ol.adam(Pm, True, st.u, st.v, st.w, fu, fv, fw, st.fuo, st.fvo, st.fwo)
    b = ol.rhs(Pm, st.u, st.v, st.w)
    t_pred = time.perf_counter() - t0
    t0 = time.perf_counter()
    ol.sor(Pm, b, st.p, tol=0.0, max_iter=sor_iters)
    t_iter = (time.perf_counter() - t0) / sor_iters
    return t_pred, t_iter


LES_SHAPE = (256, 256, 128)


def l2_copy_gbs(mb=32.0, passes=64):
    """Copy bandwidth (read + write bytes) of two buffers that fit in L2
    together (2 x 32 MB): the ceiling of a kernel whose working set stays in
    L2 between launches.  The library's probe copies `passes` times inside
    one launch, so launch gaps do not count; best of five launches."""
    import ctypes as C

    from paper_1711_04471_gb300 import _native as N
    g = C.c_double()
    N.check(N.lib().gbsw_measure_l2_copy(int(mb * 1e6) // 16 * 16, passes, C.byref(g)), "gbsw_measure_l2_copy")
    return g.value


def les_compare(args, solid, shape=LES_SHAPE, log=lambda *a: None):
    """The UFLES step at the solver tolerance over steps spinup+1 ..
    spinup+horizon: one run advances with the learned (U-Net) warm start,
    and at `compared` evenly spaced steps its checkpoint is restored into a
    second context with the previous-pressure warm start, so that both take
    that step from the same state, to the same tolerance (device times from
    the step's own CUDA events).  Both solves reach the same 1e-6 residual,
    so the run's states are those of a previous-pressure run to within the
    solver tolerance.  The compared steps are the middle ones of `compared`
    equal blocks of the horizon (a stratified sample: the first steps, the
    most expensive, are represented like the rest).  Each compared step is
    also timed end to end on the host: les_step plus the read-back of the
    FP64 pressure to host memory."""
    import numpy as np

    from paper_1711_04471_gb300.les import LES
    from paper_1711_04471_gb300.unet import UNet
    kw = dict(check_every=args.check_every, max_iter=400000)
    horizon, compared = args.les_horizon, args.les_steps
    stride = max(1, horizon // max(1, compared))
    rows = []
    wall = {"plain": [], "learned": []}
    with UNet(seed=0) as net, LES(*shape, solid, **kw) as run, LES(*shape, solid, **kw) as plain:
        net.set_params(np.load(args.weights))
        run.set_warm_start(net)
        run.step(args.les_spinup, stats=False)
        for k in range(1, horizon + 1):
            if (k - 1) % stride == stride // 2 and len(rows) < compared:   # the middle step of each block
                state = run.get_state()          # the same state for both warm starts
                plain.set_state(state)
                t0 = time.perf_counter()
                a = plain.step(1)[0]
                plain.get("p")                   # end to end: the step and its pressure on the host
                t1 = time.perf_counter()
                b = run.step(1)[0]
                run.get("p")
                t2 = time.perf_counter()
                wall["plain"].append(t1 - t0)
                wall["learned"].append(t2 - t1)
                rows.append(dict(step=state["step"] + 1, plain_iters=a["iters"], nn_iters=b["iters"],
                                 plain_ms=a["ms_predictor"] + a["ms_solve"], plain_pred_ms=a["ms_predictor"],
                                 plain_solve_ms=a["ms_solve"], plain_res=a["rel_res"], plain_status=a["status"],
                                 nn_ms=b["ms_predictor"] + b["ms_guess"] + b["ms_solve"], nn_guess_ms=b["ms_guess"],
                                 nn_solve_ms=b["ms_solve"], nn_res=b["rel_res"], nn_status=b["status"]))
                log(rows[-1])
            else:
                run.step(1, stats=False)
        nbytes = int(np.prod([n + 2 for n in shape])) * 8    # the FP64 pressure with its ghost layer
        e2e = {name: {"value": sum(w) / len(w) * 1e3, "unit": "ms/step", "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": nbytes,
                      "what": f"wall time of les_step (stats read back) + the FP64 pressure to host memory, "
                              f"on the {len(w)} compared steps"}
               for name, w in wall.items()}
    return rows, e2e


def les_object(args, local):
    """The second half of the metric: UFLES step time at a 1e-6 residual,
    learned vs previous-pressure warm start (see les_compare), with the SOR
    sweep against the L2 copy bandwidth and the FP64 oracle on the host."""
    import torch

    from paper_1711_04471_gb300 import inputs
    shape = LES_SHAPE
    solid = inputs.les_buildings(*shape, dx=4.0, seed=args.les_seed)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_wall = time.perf_counter()
    rows, e2e = les_compare(args, solid, shape)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    l2 = l2_copy_gbs()
    n = len(rows)
    mean = lambda k: sum(r[k] for r in rows) / n
    cells = shape[0] * shape[1] * shape[2]
    it_plain = mean("plain_iters")
    per_iter_s = mean("plain_solve_ms") * 1e-3 / max(it_plain, 1)
    ach = 12.0 * cells / per_iter_s / 1e9      # 12 B/cell/iteration: correction in + out, residual in
    traffic, note = ncu_traffic("sor_iteration_256x256x128")
    out = {
        "workload": f"UFLES 256x256x128, dx 4 m, dt 0.025 s, 20 % building cover (building seed {args.les_seed}), "
                    f"SOR omega 1.8 to a 1e-6 relative FP64 residual checked every {args.check_every} iterations; "
                    f"{args.les_spinup} spin-up steps, then {n} of the steps "
                    f"{args.les_spinup + 1}..{args.les_spinup + args.les_horizon} compared"
                    + (" (every step)" if n == args.les_horizon else " (one per equal block)"),
        "metric": "LES step time at 1e-6 residual, learned vs previous-pressure warm start",
        "unit": "ms/step", "higher_is_better": False, "dtype": "f32 sweeps, f64 pressure and norms",
        "plain": {"ms_per_step": mean("plain_ms"), "sor_iters_per_step": it_plain,
                  "predictor_ms": mean("plain_pred_ms"), "solve_ms": mean("plain_solve_ms"),
                  "max_rel_res": max(r["plain_res"] for r in rows),
                  "all_converged": all(r["plain_status"] == 0 for r in rows)},
        "learned": {"ms_per_step": mean("nn_ms"), "sor_iters_per_step": mean("nn_iters"),
                    "guess_ms": mean("nn_guess_ms"), "solve_ms": mean("nn_solve_ms"),
                    "max_rel_res": max(r["nn_res"] for r in rows),
                    "all_converged": all(r["nn_status"] == 0 for r in rows)},
        "e2e": e2e, "wall_s": t_wall, "clocks": clk,
        "roofline": {"bound": "l2", "kernel": "SOR iteration (red + black half-sweep) inside the solve graph",
                     "achieved": ach, "peak": l2, "unit": "GB/s", "frac": ach / l2,
                     "peak_kind": "measured in this run: L2-resident copy (gbsw_measure_l2_copy, 2 x 32 MB buffers, "
                                  "64 passes per launch, best of 5)",
                     "per_unit": f"12 B/cell/iteration x {cells} cells (solve time / iterations, checks included)",
                     "traffic": traffic, "traffic_note": note or "DRAM bytes per iteration, warm L2",
                     "hbm_frac": ach / _peaks()[0]},
        "per_step": {k: [r[k] for r in rows] for k in ("step", "plain_iters", "nn_iters")}
                    | {k: [round(r[k], 2) for r in rows] for k in ("plain_ms", "nn_ms")},
    }
    out["learned"]["speedup"] = out["plain"]["ms_per_step"] / out["learned"]["ms_per_step"]
    if not args.no_cpu_baseline:
        cpu = {}
        for omp in (False, True):
            t_pred, t_iter = _les_cpu_sample(shape, solid, openmp=omp)
            cpu[omp] = (t_pred + it_plain * t_iter) * 1e3
        import oracle
        th = oracle.threads()
        out["cpu_baseline"] = {
            "value": cpu[True], "unit": "ms/step", "cores": th, "kind": "oracle",
            "sample": f"one predictor pass + 20 SOR iterations on the full grid (FP64, OpenMP build, {th} threads), "
                      f"step time extrapolated to the plain run's {it_plain:.0f} iterations",
            "single_thread": {"value": cpu[False], "unit": "ms/step", "cores": 1}, "host": host_info()}
    return out



def run_les(args, rank, world, local, learned):
    """UFLES 256x256x128 on its own line: the les object of the default line
    with args.steps compared states; value = the learned (les-nn) or the
    previous-pressure (les) warm start's device ms per step."""
    import torch

    import paper_1711_04471_gb300 as P
    P.build()
    torch.cuda.set_device(local)
    args.les_steps = args.steps
    args.les_spinup = args.spinup
    args.les_horizon = max(args.les_horizon, args.steps)
    obj = les_object(args, local)
    if rank != 0:
        return
    key = "learned" if learned else "plain"
    line = {"metric": "LES step time at 1e-6 residual" + (" (learned warm start)" if learned else ""),
            "value": obj[key]["ms_per_step"], "unit": "ms/step", "n_gpus": world, "steps": args.steps,
            "warmup": args.spinup, "ms_per_step": obj[key]["ms_per_step"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": obj["dtype"], "data": "synthetic",
            "config": {"workload": obj["workload"], "l2": f"e and r (71 MB) stay in the {_l2_mb():.0f} MB L2 "
                                                          "between sweeps; that reuse is the method's own"},
            "clocks": obj["clocks"], "sor_iters_per_step": obj[key]["sor_iters_per_step"],
            "roofline": obj["roofline"], "cpu_baseline": obj.get("cpu_baseline"), "e2e": obj["e2e"][key],
            "plain": obj["plain"], "learned": obj["learned"], "per_step": obj["per_step"]}
    print(json.dumps(line), flush=True)


def run_sw_paper(args, rank, world, local):
    """The paper's 2DSW sizes (Sec. 6.2): 500^2, 1000^2, 2000^2 cells, dx = 1 m,
    dt = 0.01 s, 10 000 steps; flat 10 m basin with a Gaussian hump (the
    textbook basin itself is not available)."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.sw import SW
    P.build()
    torch.cuda.set_device(local)
    res = []
    for n in (500, 1000, 2000):
        inp = inputs.sw_hump(n=n, dx=1.0, dt=0.01, sigma_cells=n / 20.0)
        with SW(inp.params(), inp.H, inp.eta0, stream=torch.cuda.current_stream()) as g:
            tiling = g.autotune(trial_steps=120)
            g.step(300)
            g.volume()
            t = _timed_region(lambda: (g.step(10000), g.volume()), world)
        cpu = {}
        if not args.no_cpu_baseline:
            import oracle
            for omp in (False, True):
                oracle.use_openmp(omp)
                o = oracle.SWState(inp.params(), inp.H, inp.eta0)
                steps = max(1, int((8e7 if omp else 2e7) // (n * n)))
                t0 = time.perf_counter()
                o.run(steps)
                cpu[omp] = n * n * steps / (time.perf_counter() - t0)
                oracle.use_openmp(False)
            cpu["threads"] = oracle.threads()
        res.append({"n": n, "seconds_10000_steps": t, "cell_updates_per_s": n * n * 10000 / t,
                    "tiling": {"steps_per_launch": tiling[0], "rows_per_block": tiling[1],
                               "kernel": ("tile, %d rows per tile" % (32 if tiling[1] == -1 else -tiling[1])
                                          if tiling[1] < 0 else "streaming")},
                    "oracle_cell_updates_per_s_1thread": cpu.get(False),
                    "oracle_cell_updates_per_s_all_cores": cpu.get(True), "oracle_threads": cpu.get("threads")})
    if rank != 0:
        return
    big = res[-1]
    print(json.dumps({"metric": "cell-updates/s (paper 2DSW sizes)", "value": big["cell_updates_per_s"],
                      "unit": "cell-updates/s", "n_gpus": world, "steps": 10000, "warmup": 300,
                      "ms_per_step": big["seconds_10000_steps"] / 10, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "2DSW at the paper's sizes, dx 1 m, dt 0.01 s, 10000 steps"},
                      "sizes": res}), flush=True)


def run_sw64(args, rank, world, local):
    """The FP64 variant of the 2DSW step (three kernels per step, every
    operation rounded as written) on the 4096^2 wet/dry grid:
    STEPS_PER_BENCH_STEP time steps plus the FP64 volume per bench step."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.sw import SW64
    P.build()
    torch.cuda.set_device(local)
    inp = inputs.sw_wetdry(n=N_CELLS_SIDE, seed=1001)
    cells = N_CELLS_SIDE * N_CELLS_SIDE
    with SW64(inp.params(), inp.H, inp.eta0, stream=torch.cuda.current_stream()) as g:
        for _ in range(args.warmup):
            g.step(STEPS_PER_BENCH_STEP)
            g.volume()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        t = _timed_region(lambda: [(g.step(STEPS_PER_BENCH_STEP), g.volume()) for _ in range(args.steps)], world)
        clk = clocks.stop()
    if rank != 0:
        return
    value = cells * STEPS_PER_BENCH_STEP * args.steps * world / t
    peak, peak_kind = _peaks()
    ach = 120.0 * cells * STEPS_PER_BENCH_STEP * args.steps / t / 1e9
    print(json.dumps({"metric": "cell-updates/s (FP64 2DSW)", "value": value, "unit": "cell-updates/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": "2DSW 4096x4096 wet/dry, FP64 end to end (3 kernels per time step), "
                                             f"{STEPS_PER_BENCH_STEP} time steps + FP64 volume per step"},
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                   "traffic": None, "peak_kind": peak_kind, "kernel": "sw64 momentum/continuity/shapiro",
                                   "per_unit": "120 B per cell-update (48 + 40 + 32 B over the three kernels)"},
                      "clocks": clk}), flush=True)


def run_les_paper(args, rank, world, local):
    """The paper's UFLES setup (Sec. 6.3.2): 300x300x90 cells, 50 SOR
    iterations per step, dt = 0.025 s over 1.2 km; per-phase device times."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.les import LES
    P.build()
    torch.cuda.set_device(local)
    shape = (300, 300, 90)
    solid = inputs.les_buildings(*shape, dx=4.0, seed=1004)
    with LES(*shape, solid) as g:
        g.set_fixed_iterations(50)
        g.step(args.spinup, stats=False)
        st = g.step(args.steps)
    pred = sum(a["ms_predictor"] for a in st) / len(st)
    solve = sum(a["ms_solve"] for a in st) / len(st)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        t_pred, t_iter = _les_cpu_sample(shape, solid, openmp=True)
        s_pred, s_iter = _les_cpu_sample(shape, solid, openmp=False)
        th = oracle.threads()
        cpu = {"value": (t_pred + 50 * t_iter) * 1e3, "unit": "ms/step", "cores": th, "kind": "oracle",
               "sample": f"one predictor pass + 20 SOR iterations on the full 300x300x90 grid (FP64, OpenMP build, "
                         f"{th} threads), step time for 50 iterations", "predictor_ms": t_pred * 1e3,
               "sor_iteration_ms": t_iter * 1e3,
               "single_thread": {"value": (s_pred + 50 * s_iter) * 1e3, "unit": "ms/step", "cores": 1},
               "host": host_info()}
    print(json.dumps({"metric": "LES step time, 50 SOR iterations (paper setup)", "value": pred + solve,
                      "unit": "ms/step", "n_gpus": world, "steps": args.steps, "warmup": args.spinup,
                      "ms_per_step": pred + solve, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f32 sweeps, f64 pressure", "data": "synthetic",
                      "config": {"workload": "UFLES 300x300x90, dx 4 m, dt 0.025 s, fixed 50 SOR iterations"},
                      "breakdown_ms": {"velnw..adam+rhs": pred, "press": solve},
                      "press_share": solve / (pred + solve), "cpu_baseline": cpu,
                      "final_rel_res": sum(a["rel_res"] for a in st) / len(st)}), flush=True)


def run_poisson(args, rank, world, local):
    """The pressure solve alone (poisson_solve) on a seeded random right-hand
    side of the --grid size: --iters iterations of the paper's fixed-count
    SOR launched directly (--mode fixed, the form an ncu launch list
    resolves per half-sweep), or the tolerance-driven conditional graph with
    a check every 50 iterations and an unreachable tolerance (--mode graph).
    Prints the time per iteration, setup included."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300.les import poisson_solve
    P.build()
    torch.cuda.set_device(local)
    nx, ny, nz = args.grid
    gen = torch.Generator(device="cuda").manual_seed(0)
    b = torch.randn((nz, ny, nx), device="cuda", generator=gen) * 1e-3
    p = torch.zeros_like(b)
    tol = -1.0 if args.mode == "fixed" else 1e-30
    poisson_solve(p.clone(), b, 4.0, tol=tol, max_iter=min(args.iters, 50), check_every=50)    # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, it, rr = poisson_solve(p, b, 4.0, tol=tol, max_iter=args.iters, check_every=50)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps({"metric": "SOR iteration time (poisson_solve alone)", "value": dt / max(it, 1) * 1e6,
                          "unit": "us/iteration", "higher_is_better": False, "grid": [nx, ny, nz],
                          "mode": args.mode, "iterations": it, "rel_res": rr, "status": st}), flush=True)


def run_unet(args, rank, world, local):
    """U-Net inference alone (unet_forward) on a random (1, D, H, W, 2)
    input of the --grid size (given as W H D), --iters repetitions."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300.unet import UNet
    P.build()
    torch.cuda.set_device(local)
    W, H, D = args.grid
    x = torch.randn((1, D, H, W, 2), device="cuda")
    with UNet(seed=0) as net:
        net.forward(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.iters):
            net.forward(x)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.iters
    if rank == 0:
        print(json.dumps({"metric": "U-Net forward time", "value": dt * 1e3, "unit": "ms", "higher_is_better": False,
                          "input": [1, D, H, W, 2], "reps": args.iters}), flush=True)


def run_unet_train(args, rank, world, local):
    """U-Net training alone (unet_train_step: forward, backward with the
    tcgen05 weight gradients, Adam) on the warm-start training batch: 32
    samples of the coarse grid (--grid W H D, default 16 16 8), --iters
    steps after 5 warm-up steps."""
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300.unet import UNet
    P.build()
    torch.cuda.set_device(local)
    W, H, D = args.grid if args.grid != [256, 256, 128] else (16, 16, 8)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((32, D, H, W, 2), device="cuda", generator=gen)
    t = torch.randn((32, D, H, W), device="cuda", generator=gen) * 0.1
    with UNet(seed=0) as net:
        for _ in range(5):
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.iters):
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.iters
    if rank == 0:
        print(json.dumps({"metric": "U-Net training step time", "value": dt * 1e3, "unit": "ms",
                          "higher_is_better": False, "batch": [32, D, H, W, 2], "steps": args.iters,
                          "note": "host-timed, loss read back every step"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sw4096", choices=["sw4096", "sw64", "ensemble", "les", "les-nn", "sw-paper",
                                                                 "les-paper", "poisson", "unet", "unet-train"])
    ap.add_argument("--grid", type=int, nargs=3, default=[256, 256, 128],
                    help="poisson / unet workloads: NX NY NZ")
    ap.add_argument("--iters", type=int, default=200, help="poisson: SOR iterations; unet: repetitions")
    ap.add_argument("--mode", default="fixed", choices=["fixed", "graph"], help="poisson workload")
    ap.add_argument("--spinup", type=int, default=20)
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1711_04471_gb300", "data", "unet_warmstart.npy"))
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbsw", choices=["gbsw", "reference"])
    ap.add_argument("--blocking", type=int, default=0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per fused launch, if captured for this kernel version")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-les", action="store_true", help="default workload: leave out the UFLES object")
    ap.add_argument("--les-spinup", type=int, default=20, help="UFLES object: spin-up steps before the comparison")
    ap.add_argument("--les-steps", type=int, default=180,
                    help="UFLES object: compared states (180: every step of the horizon)")
    ap.add_argument("--les-horizon", type=int, default=180,
                    help="UFLES object: steps after the spin-up over which the compared states are spread")
    ap.add_argument("--les-e2e-steps", type=int, default=3,
                    help="accepted for older command lines; the UFLES end-to-end figure is timed on the compared steps")
    ap.add_argument("--check-every", type=int, default=500,
                    help="les workloads: SOR iterations between FP64 residual checks")
    ap.add_argument("--les-seed", type=int, default=1003,
                    help="les workloads: building layout seed (1003: the benchmark layout)")
    ap.add_argument("--members", type=int, default=512,
                    help="ensemble workload: the first N of the 512 instances (smaller cases for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "ensemble":
        run_ensemble(args, rank, world, local)
    elif args.workload == "sw64":
        run_sw64(args, rank, world, local)
    elif args.workload == "sw-paper":
        run_sw_paper(args, rank, world, local)
    elif args.workload == "les-paper":
        run_les_paper(args, rank, world, local)
    elif args.workload == "poisson":
        run_poisson(args, rank, world, local)
    elif args.workload == "unet":
        run_unet(args, rank, world, local)
    elif args.workload == "unet-train":
        run_unet_train(args, rank, world, local)
    elif args.workload in ("les", "les-nn"):
        run_les(args, rank, world, local, learned=args.workload == "les-nn")
    else:
        run_gbsw(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
