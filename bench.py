"""Benchmarks of the 2DSW and UFLES time steps.

Default workload (the headline line): the 2DSW time step on the 4096 x 4096
wet/dry grid, FP32.  Other workloads (--workload): ``ensemble`` (512
instances, persistent kernel vs separate launches), ``les`` (256x256x128
UFLES step at 1e-6 residual) and ``les-nn`` (the same, learned warm start
vs previous-pressure warm start on the same states).

One benchmark step = 100 model time steps of the 4096^2 grid (the fused
momentum / continuity / Shapiro / update kernel, temporally blocked) plus
the FP64 volume reduction, i.e. every 2DSW row of the hot path.  The state
(268 MB of eta, u, v, H) is larger than the 129 MB L2, so no L2 flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbsw|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an
independent replica (the workload has no exchange step), the timed region
is bracketed by barriers and the slowest rank's time is reported.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_SIDE = 4096
STEPS_PER_BENCH_STEP = 100
BYTES_PER_CELL_UPDATE = 28  # read eta, u, v, H; write eta, u, v (FP32)
METRIC = "cell-updates/s"
# DRAM bytes (read + write) of one sw_stream_kernel<3> launch on the 4096^2
# grid, from the ncu capture summarised in profiles/sw_stream_kernel_4096.md;
# set to None whenever that kernel changes until it is captured again.
TRAFFIC_SW_STREAM_T3 = 458.705664e6
WORKLOAD = "2DSW 4096x4096 wet/dry (15% dry), FP32, 100 time steps + FP64 volume per step"
# DRAM bytes (read + write) of one SOR iteration (red + black half-sweep) on
# the 256x256x128 grid with the L2 warm, from the ncu capture summarised in
# profiles/sor_sweep_kernel_256x256x128.md; None whenever that kernel changes
# until it is captured again.
TRAFFIC_SOR_ITER_256 = (1.734144 + 0.464896 + 2.585344 + 0.501504) * 1e6


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


def cpu_oracle_rate(nsteps=10, side=N_CELLS_SIDE):
    """Time the FP64 oracle (single thread) on a bounded sample: nsteps time
    steps of the full 4096^2 grid (the same synthetic input)."""
    import oracle
    from paper_1711_04471_gb300 import inputs
    inp = inputs.sw_wetdry(n=side, seed=1001)
    s = oracle.SWState(inp.params(), inp.H, inp.eta0)
    t0 = time.perf_counter()
    s.run(nsteps)
    dt = time.perf_counter() - t0
    return side * side * nsteps / dt, dt


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1711_04471_gb300 import inputs
    inp = inputs.sw_wetdry(n=N_CELLS_SIDE, seed=1001)
    s = oracle.SWState(inp.params(), inp.H, inp.eta0)
    for _ in range(args.warmup):
        s.run(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.run(1)
    dt = time.perf_counter() - t0
    cells = N_CELLS_SIDE ** 2 * args.steps
    value = cells / dt
    sample = f"{args.steps} time steps of the full 4096^2 grid (1 model step per bench step), FP64, 1 thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [N_CELLS_SIDE, N_CELLS_SIDE]},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
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
    launches_per_step = math.ceil(STEPS_PER_BENCH_STEP / T) + 2

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
    fused_launch_ms = sum(step_ms) / (args.steps * math.ceil(STEPS_PER_BENCH_STEP / T))
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
    cpu_value, cpu_s = (None, None)
    if world == 1 and not args.no_cpu_baseline:
        cpu_value, cpu_s = cpu_oracle_rate()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [nx, ny], "time_steps_per_step": STEPS_PER_BENCH_STEP,
                   "steps_per_launch": T, "l2": "state 268 MB > 129 MB L2, no flush needed",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak,
                     "traffic": args.traffic if args.traffic is not None else
                     (TRAFFIC_SW_STREAM_T3 if T == 3 else None),
                     "peak_kind": peak_kind, "kernel": "sw_stream_kernel",
                     "per_unit": f"{BYTES_PER_CELL_UPDATE} B/cell-update x {T} steps x {cells} cells per launch",
                     "compulsory_gbs": compulsory_gbs, "compulsory_frac": compulsory_gbs / peak,
                     "launch_ms": fused_launch_ms},
        "cpu_baseline": None if cpu_value is None else {
            "value": cpu_value, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"10 time steps of the full 4096^2 grid, FP64 oracle, 1 thread ({cpu_s:.1f} s)"},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "volume_drift": (vols[-1][0] - vols[0][0]) / vols[0][0],
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
    """512 2DSW instances (sides log-uniform in [64, 1024]), 100 time steps per
    bench step: one persistent cooperative kernel per call (CUDA graph) vs one
    launch per instance and fused level."""
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
    T, rows = b.autotune(trial_steps=12, cache_path=os.environ.get("GBSW_TUNE_CACHE"))
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
                                   f"{cells} cells, 100 time steps + FP64 volumes per step",
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


def _les_cpu_sample(shape, solid, sor_iters=20):
    """Oracle (FP64, one thread) on the full grid: one predictor pass and
    sor_iters SOR iterations, timed separately."""
    import ctypes as C

    import oracle
    from oracle import les as ol
    nx, ny, nz = shape
    Pm = ol.make_params(nx, ny, nz)
    st = ol.LESState(Pm, solid)
    L = oracle.lib()
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


def run_les(args, rank, world, local, learned):
    """UFLES 256x256x128 (20 % building cover), SOR omega 1.8 to a 1e-6
    relative FP64 residual, 20 spin-up steps excluded.  With learned=True each
    timed state is stepped twice: previous-pressure warm start and the U-Net."""
    import numpy as np
    import torch

    import paper_1711_04471_gb300 as P
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.les import LES
    P.build()
    torch.cuda.set_device(local)
    shape = (256, 256, 128)
    solid = inputs.les_buildings(*shape, dx=4.0, seed=args.les_seed)
    kw = dict(check_every=args.check_every, max_iter=400000)
    rows = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if learned:
        from paper_1711_04471_gb300 import train_unet
        from paper_1711_04471_gb300.unet import UNet
        net = UNet(seed=0)
        net.set_params(np.load(args.weights))
        rows = train_unet.compare_warm_starts(net, shape=shape, seed=args.les_seed, spinup=args.spinup,
                                              steps=args.steps, log=lambda *a: None, **kw)
        net.close()
        t_plain = sum(r["plain_ms"] for r in rows) / len(rows)
        t_nn = sum(r["nn_ms"] for r in rows) / len(rows)
    else:
        with LES(*shape, solid, **kw) as g:
            g.step(args.spinup, stats=False)
            st = g.step(args.steps)
        rows = [dict(plain_iters=a["iters"], plain_ms=a["ms_predictor"] + a["ms_solve"],
                     pred_ms=a["ms_predictor"], solve_ms=a["ms_solve"], res=a["rel_res"]) for a in st]
        t_plain = sum(r["plain_ms"] for r in rows) / len(rows)
    clk = clocks.stop()
    if rank != 0:
        return
    cells = shape[0] * shape[1] * shape[2]
    iters = sum(r["plain_iters"] for r in rows) / len(rows)
    peak, peak_kind = _peaks()
    solve_ms = (sum(r.get("solve_ms", r["plain_ms"]) for r in rows) / len(rows))
    per_iter_s = solve_ms * 1e-3 / max(iters, 1)
    ach = 12.0 * cells / per_iter_s / 1e9      # 12 B/cell/iteration: correction in+out, residual in
    t_pred, t_iter = _les_cpu_sample(shape, solid) if (world == 1 and not args.no_cpu_baseline) else (None, None)
    line = {"metric": "LES step time at 1e-6 residual" + (" (learned warm start)" if learned else ""),
            "value": t_nn if learned else t_plain, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
            "warmup": args.spinup, "ms_per_step": t_nn if learned else t_plain, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweeps, f64 pressure and norms",
            "data": "synthetic",
            "config": {"workload": f"UFLES 256x256x128, dx 4 m, dt 0.025 s, 20 % building cover (building seed "
                                   f"{args.les_seed}), SOR omega 1.8, "
                                   "tol 1e-6 (FP64), warm start " + ("U-Net vs previous pressure" if learned
                                                                     else "previous pressure"),
                       "spinup_steps": args.spinup, "check_every": args.check_every,
                       "l2": f"e and r (71 MB) stay in the {_l2_mb():.0f} MB L2 between sweeps; that reuse is the "
                             "method's own"},
            "clocks": clk,
            "sor_iters_per_step": iters,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": TRAFFIC_SOR_ITER_256 if shape == (256, 256, 128) else None,
                         "traffic_unit": "bytes per SOR iteration (two half-sweeps), warm L2",
                         "peak_kind": peak_kind, "kernel": "sor_sweep_kernel",
                         "per_unit": "12 B/cell/iteration x 8388608 cells (solve time / iterations)"},
            "cpu_baseline": None if t_pred is None else {
                "value": (t_pred + iters * t_iter) * 1e3, "unit": "ms/step", "cores": 1, "kind": "oracle",
                "sample": f"one predictor pass + 20 SOR iterations on the full grid (FP64, 1 thread), "
                          f"step time extrapolated to {iters:.0f} iterations"},
            "rows": rows}
    if learned:
        line["plain"] = {"ms_per_step": t_plain, "sor_iters_per_step": iters}
        line["learned"] = {"ms_per_step": t_nn, "sor_iters_per_step": sum(r["nn_iters"] for r in rows) / len(rows),
                           "guess_ms": sum(r["nn_guess_ms"] for r in rows) / len(rows)}
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
            g.step(300)
            g.volume()
            t = _timed_region(lambda: (g.step(10000), g.volume()), world)
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            o = oracle.SWState(inp.params(), inp.H, inp.eta0)
            steps = max(1, int(2e7 // (n * n)))
            t0 = time.perf_counter()
            o.run(steps)
            cpu = n * n * steps / (time.perf_counter() - t0)
        res.append({"n": n, "seconds_10000_steps": t, "cell_updates_per_s": n * n * 10000 / t,
                    "oracle_cell_updates_per_s_1thread": cpu})
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
    operation rounded as written) on the 4096^2 wet/dry grid: 100 time
    steps plus the FP64 volume per bench step."""
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
                                             "100 time steps + FP64 volume per step"},
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
        t_pred, t_iter = _les_cpu_sample(shape, solid)
        cpu = {"value": (t_pred + 50 * t_iter) * 1e3, "unit": "ms/step", "cores": 1, "kind": "oracle",
               "sample": "one predictor pass + 20 SOR iterations on the full 300x300x90 grid (FP64, 1 thread), "
                         "step time for 50 iterations", "predictor_ms": t_pred * 1e3, "sor_iteration_ms": t_iter * 1e3}
    print(json.dumps({"metric": "LES step time, 50 SOR iterations (paper setup)", "value": pred + solve,
                      "unit": "ms/step", "n_gpus": world, "steps": args.steps, "warmup": args.spinup,
                      "ms_per_step": pred + solve, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f32 sweeps, f64 pressure", "data": "synthetic",
                      "config": {"workload": "UFLES 300x300x90, dx 4 m, dt 0.025 s, fixed 50 SOR iterations"},
                      "breakdown_ms": {"velnw..adam+rhs": pred, "press": solve},
                      "press_share": solve / (pred + solve), "cpu_baseline": cpu,
                      "final_rel_res": sum(a["rel_res"] for a in st) / len(st)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sw4096", choices=["sw4096", "sw64", "ensemble", "les", "les-nn", "sw-paper",
                                                                 "les-paper"])
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
    elif args.workload in ("les", "les-nn"):
        run_les(args, rank, world, local, learned=args.workload == "les-nn")
    else:
        run_gbsw(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
