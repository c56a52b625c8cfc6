#!/usr/bin/env python
"""Throughput of the PPV forward hot path: cell-channel updates per second.

Workload: a 256^3 FP32 field set (lognormal density, turbulent velocity plus
rotation), 13CO(2-1) in LTE, 256 channels of 1 km/s with f = 1; one step
renders the z view and the (theta, phi) = (30, 45) deg oblique trilinear view
with smooth (TR + BDF2) integration and runs the adjoint of the z view (the
gradient of a cube loss against a render of another snapshot).  Units of one
render or adjoint: sum over rays of (samples on the ray) x (channels).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl irt|reference]

N > 1 runs under torchrun, one rank per GPU, each rank rendering its own
snapshot (weak scaling, no collective on the data path).  Prints one JSON line
on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PPV cell-channel updates/s (fwd and adjoint) at stated error vs FP64 oracle"
UNIT = "cell-channel updates/s"
#: algorithmic FP32 / MUFU lane-operations of the smooth integrator: per
#: (sample, 32-velocity block) pair where the line is evaluated, per pair
#: integrated without the line, per sample (records and the three continuum
#: basis recurrences)
OPS_LINE = (10, 2)
OPS_DUST = (5, 0)
OPS_SAMPLE = (165, 9)
#: adjoint: the forward once more (each 32-sample segment recomputed from the
#: checkpoint the forward render saved, keeping its pre-ReLU values) plus the
#: reverse step (about 12 FP32 per block pair, 30 FP32 + 3 MUFU per line slot)
#: and the per-sample chain rule
ADJ_FWD = 1.0
OPS_ADJ_LINE = (ADJ_FWD * 10 + 12 + 30, ADJ_FWD * 2 + 3)
OPS_ADJ_DUST = (ADJ_FWD * 5 + 12, 0)
OPS_ADJ_SAMPLE = (ADJ_FWD * 165 + 60, ADJ_FWD * 9 + 6)
# Thin transfer modes (Sec. 4.6, 4.7), smooth integration: FP32 operations per
# (sample, channel) pair of the recurrences alone (dust source 2; selectively
# thin: continuum and total BDF2 steps with their ReLU 2 x 5; optically thin:
# the two Simpson sums 3).  The erf channel averages of the pairs the line
# reaches are not counted, so the rate derived from these is a lower bound.
OPS_THIN_PAIR = {"selectively_thin": 12, "thin": 5, "density_tracing": 2}
#: kernel sources whose DRAM traffic the committed step profile records
KERNEL_SOURCES = ("irt_adjoint.cu", "irt_forward.cuh", "irt_forward_impl.cuh",
                  "irt_internal.h", "irt_fwd_f32_smooth.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["irt", "reference"], default="irt")
    ap.add_argument("--integration", default="smooth")
    ap.add_argument("--n", type=int, default=256, help="grid side (default: the 256^3 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-thin", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank):
    """Each rank renders its own snapshot (weak scaling, no data-path collective)."""
    return 1000 + 17 * rank


def max_over_ranks(x, ws, device=None):
    """The slowest replica sets the whole job's time (all_reduce MAX)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Units of all ranks per second of the slowest rank."""
    return units_per_rank * ws / seconds


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        rows = [s for t, s in self.samples if t0 <= t <= t1]
        note = "during timed region"
        if len(rows) < 2:
            rows = [s for t, s in self.samples if t0 - 1.0 <= t <= t1 + 1.0]
            note = "within 1 s of the timed region (region shorter than the sampling period)"
        sm, smax, reasons = [], 0.0, set()
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "nvidia-smi unavailable"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "note": note}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload_inputs(n, seed):
    from synth import make_fields, to_storage, workload
    w = workload(1, n=n)
    fs = make_fields(w.n, seed)
    f32, deq = to_storage(fs, np.float32)
    return w, f32, deq


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0, "fallback": True}


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(w, deq, target_s=10.0, integration="smooth", seed=0):
    """Oracle throughput on a seeded sample of rays of both views, sized to
    about target_s seconds of CPU work.  Returns (units/s, cores, sample text,
    seconds)."""
    import oracle
    mode = oracle.SMOOTH if integration == "smooth" else oracle.FORMAL
    fields = deq.as_tuple()
    rng = np.random.default_rng(seed)
    cores = oracle.num_threads()

    def run(nrays):
        units = 0
        t = time.perf_counter()
        for view in w.views:
            pix = np.stack([rng.integers(0, view.npx, nrays), rng.integers(0, view.npy, nrays)],
                           axis=1)
            oracle.render(fields, w.cell_cm, w.line, w.dust, view, w.vaxis, pix,
                          integration=mode)
            for px, py in pix:
                smp, h = oracle.ray_samples(fields, w.cell_cm, view, int(px), int(py))
                units += len(smp) * w.vaxis.nchan
        return units, time.perf_counter() - t

    nr = max(cores, 4)
    units, dt = run(nr)
    for _ in range(3):   # grow the sample until it takes about target_s
        if dt >= target_s / 2:
            break
        nr = max(nr + 1, int(nr * target_s / max(dt, 1e-3)))
        units, dt = run(nr)
    sample = (f"{nr} seeded rays per view of the {w.n}^3 workload (z and oblique), "
              f"all {w.vaxis.nchan} channels, full depth")
    return units / dt, cores, sample, dt


def oracle_adjoint_rate(w, deq, target_s=4.0, seed=0):
    """Oracle dual-number gradient throughput on seeded z-view rays (units of
    the adjoint: samples x channels per ray).  Returns (units/s, nrays)."""
    import oracle
    fields = deq.as_tuple()
    rng = np.random.default_rng(seed + 99)
    view = w.views[0]
    tgt = np.zeros((w.vaxis.nchan, view.npy, view.npx))

    def run(nrays):
        pix = np.stack([rng.integers(0, view.npx, nrays), rng.integers(0, view.npy, nrays)],
                       axis=1)
        t = time.perf_counter()
        oracle.loss_grad_zview(fields, w.cell_cm, w.line, w.dust, w.vaxis, tgt, pixels=pix)
        return nrays * w.n * w.vaxis.nchan, time.perf_counter() - t

    nr = max(oracle.num_threads(), 2)
    units, dt = run(nr)
    for _ in range(3):
        if dt >= target_s / 2:
            break
        nr = max(nr + 1, int(nr * target_s / max(dt, 1e-3)))
        units, dt = run(nr)
    return units / dt, nr, dt


def combined_rate(r_fwd, r_adj, units_fwd, units_adj):
    """Rate of a step made of units_fwd forward and units_adj adjoint units."""
    return (units_fwd + units_adj) / (units_fwd / r_fwd + units_adj / r_adj)


def reference_arm(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    w, f32, deq = workload_inputs(args.n, 1000)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rate(w, deq, target_s=per_step / 4, integration=args.integration)
    rates, times = [], []
    cores, sample = 1, ""
    n = w.n
    units_fwd = n ** 3 * w.vaxis.nchan * 2      # z + oblique, about equal
    units_adj = n ** 3 * w.vaxis.nchan
    for s in range(args.steps):
        r, cores, sample, dt = oracle_rate(w, deq, target_s=per_step * 0.7,
                                           integration=args.integration, seed=s)
        ra, na, dta = oracle_adjoint_rate(w, deq, target_s=per_step * 0.3, seed=s)
        rates.append(combined_rate(r, ra, units_fwd, units_adj))
        times.append(dt + dta)
        sample += f"; adjoint: dual-number gradient of {na} seeded z-view rays"
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name} z + oblique(30,45) deg", "grid": w.n,
                       "nchan": w.vaxis.nchan, "f": w.vaxis.subsample_f,
                       "integration": args.integration},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_arm(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B

    seed = replica_seed(rank)
    w, f32, deq = workload_inputs(args.n, seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    fields_d = [torch.from_numpy(a).to(dev) for a in f32.as_tuple()]
    grid = irt.Grid(*fields_d, w.cell_cm)
    outs = [irt.alloc_cubes(v, w.vaxis) for v in w.views]
    stream = torch.cuda.current_stream()
    # loss = mean over the z-view [L] cube of (L - L_target)^2, the target
    # rendered from another snapshot; its cotangent feeds the adjoint
    from synth import make_fields, to_storage
    tfs, _ = to_storage(make_fields(w.n, seed + 7), np.float32)
    tgrid = irt.Grid(*[torch.from_numpy(a).to(dev) for a in tfs.as_tuple()], w.cell_cm)
    l_target = irt.forward(tgrid, w.views[0], w.vaxis, w.line, w.dust,
                           integration=args.integration, components=("L",))["L"]
    tgrid.close()
    irt.forward(grid, w.views[0], w.vaxis, w.line, w.dust, integration=args.integration,
                out=outs[0])
    cot = {"L": 2.0 * (outs[0]["L"] - l_target) / outs[0]["L"].numel()}
    grads = tuple(torch.empty((w.n, w.n, w.n), dtype=torch.float32, device=dev)
                  for _ in range(3))

    # the z-view render keeps its transfer checkpoints for the adjoint that
    # follows it (smooth integration), as the autograd function does
    save = B.IRT_FLAG_SAVE_CHECKPOINTS if args.integration == "smooth" else 0
    vflags = [save if vi == 0 else 0 for vi in range(len(w.views))]

    def step(flags=0):
        for view, out, vf in zip(w.views, outs, vflags):
            irt.forward(grid, view, w.vaxis, w.line, w.dust, integration=args.integration,
                        out=out, flags=flags | vf)
        irt.adjoint(grid, w.views[0], w.vaxis, w.line, w.dust, cot,
                    integration=args.integration, grads=grads)

    # units and work counters from one counted pass
    B.irt_grid_stats(grid.handle, reset=True)
    per_view = []
    for view, out in zip(w.views, outs):
        irt.forward(grid, view, w.vaxis, w.line, w.dust, integration=args.integration, out=out,
                    flags=B.IRT_FLAG_STATS)
        per_view.append(B.irt_grid_stats(grid.handle, reset=True))
    units_view = [st["samples"] * w.vaxis.nchan for st in per_view]
    units_adj = units_view[0]
    units_step = sum(units_view) + units_adj

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pipe_peaks = B.irt_measure_pipe_peaks(int(torch.cuda.current_stream().cuda_stream))

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    nk = len(w.views) + 1
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(nk * args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    irt.irt_launch_count()
    wall0 = time.time()
    t_start.record(stream)
    i = 0
    for _ in range(args.steps):
        for view, out, vf in zip(w.views, outs, vflags):
            ev[i][0].record(stream)
            irt.forward(grid, view, w.vaxis, w.line, w.dust, integration=args.integration,
                        out=out, flags=vf)
            ev[i][1].record(stream)
            i += 1
        ev[i][0].record(stream)
        irt.adjoint(grid, w.views[0], w.vaxis, w.line, w.dust, cot,
                    integration=args.integration, grads=grads)
        ev[i][1].record(stream)
        i += 1
    t_end.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    launches = irt.irt_launch_count()
    if ws > 1:
        torch.distributed.barrier()
    time.sleep(0.2)
    clocks.stop()
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), ws, dev)
    ms_step = elapsed_ms / args.steps
    value = whole_job_rate(units_step, ws, elapsed_ms / 1e3 / args.steps)
    launch_ms = [[] for _ in range(nk)]
    for j, (a, b) in enumerate(ev):
        launch_ms[j % nk].append(a.elapsed_time(b))
    kern_ms = [float(np.mean(x)) for x in launch_ms]
    view_ms = kern_ms[:len(w.views)]
    adj_ms = kern_ms[-1]

    # ---- roofline of the dominant kernel (the launch with the most time)
    pk = peaks()
    dom = int(np.argmax(kern_ms))
    is_adj = dom == nk - 1
    st = per_view[0] if is_adj else per_view[dom]
    ol, od, os_ = (OPS_ADJ_LINE, OPS_ADJ_DUST, OPS_ADJ_SAMPLE) if is_adj else \
        (OPS_LINE, OPS_DUST, OPS_SAMPLE)
    fp32 = 32 * (ol[0] * st["line_block_samples"]
                 + od[0] * (st["hull_block_samples"] - st["line_block_samples"])) \
        + os_[0] * st["samples"]
    mufu = 32 * ol[1] * st["line_block_samples"] + os_[1] * st["samples"]
    fclk = float(pk.get("sm_max_mhz", 2032.0)) * 1e6
    nom_fp32 = 148 * 128 * fclk / 1e12          # Top/s, lane count x clock
    nom_mufu = 148 * 16 * fclk / 1e12
    # denominators: the pipes measured by the library's microbenchmark on
    # this GPU at its present clock
    peak_fp32 = pipe_peaks["fp32_ops_per_s"] / 1e12
    peak_mufu = pipe_peaks["mufu_ops_per_s"] / 1e12
    t_dom = kern_ms[dom] / 1e3
    a_fp32 = fp32 / t_dom / 1e12
    a_mufu = mufu / t_dom / 1e12
    if a_fp32 / peak_fp32 >= a_mufu / peak_mufu:
        ach, peak, pipe = a_fp32, peak_fp32, "fp32"
    else:
        ach, peak, pipe = a_mufu, peak_mufu, "mufu"
    nx = w.n
    vw = w.views[0 if is_adj else dom]
    hbm_bytes = nx ** 3 * 32 + 5 * 4 * w.vaxis.nchan * vw.npx * vw.npy
    kname = ("adjoint (z view): adj_kernel<4,F32>, then the wider hulls in adj_kernel<9,F32> "
             "and adj_kernel<17,F32>, then adj_dense_kernel for explicit-channel rays"
             if is_adj else f"fwd_kernel<float,17,F32,smooth> ({['z', 'oblique'][dom]} view)")
    # DRAM bytes per launch of the dominant kernel from the committed ncu
    # summary of this workload, only while the kernel sources it was captured
    # from are unchanged; other sizes have no capture
    traffic = None
    tp = traffic_from_profile() if nx == 256 else None
    if tp:
        key = "adjoint_dram_bytes_per_launch" if is_adj else \
            ("z_view_dram_bytes_per_launch" if dom == 0 else "oblique_view_dram_bytes_per_launch")
        traffic = tp.get(key)
    roofline = {"bound": "alu", "pipe": pipe, "achieved": ach, "peak": peak, "unit": "Top/s",
                "frac": ach / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "kernel": kname,
                "launch_ms": kern_ms[dom],
                "peak_source": "measured: irt_measure_pipe_peaks (FP32 FMA and ex2 chains on "
                               "every SM) in this run",
                "peak_fp32_top_s": peak_fp32, "peak_mufu_top_s": peak_mufu,
                "nominal_fp32_top_s": nom_fp32, "nominal_mufu_top_s": nom_mufu,
                "fp32_top_s": a_fp32, "mufu_top_s": a_mufu,
                "hbm_gbs": hbm_bytes / t_dom / 1e9, "hbm_peak_gbs": pk.get("hbm_gbs"),
                "hbm_frac": hbm_bytes / t_dom / 1e9 / float(pk.get("hbm_gbs", 6400.0)),
                "dense_fine_updates_per_launch": st["dense_fine_updates"],
                "work_per_launch": st}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_in = [torch.from_numpy(a).pin_memory() for a in f32.as_tuple()]
        host_out = [{k: torch.empty(o[k].shape, dtype=o[k].dtype).pin_memory() for k in o}
                    for o in outs]
        host_tgt = l_target.cpu().pin_memory()
        host_grads = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in grads]
        host_loss = torch.empty((), dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host_in) + \
            host_tgt.numel() * host_tgt.element_size()
        d2h = sum(t.numel() * t.element_size() for o in host_out for t in o.values()) + \
            sum(t.numel() * t.element_size() for t in host_grads) + 4
        # double-buffered device inputs and results: step i computes on the
        # compute stream while the inputs of step i + 1 go up on one copy
        # stream and the results of step i come down on another
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        dev_in = [[torch.empty_like(t, device=dev) for t in host_in] for _ in range(2)]
        dev_tgt = [torch.empty_like(host_tgt, device=dev) for _ in range(2)]
        outs2 = [outs, [irt.alloc_cubes(v, w.vaxis) for v in w.views]]
        grads2 = [grads, tuple(torch.empty_like(x) for x in grads)]

        def run_steps(n):
            ms = torch.cuda.current_stream()
            ev = lambda: torch.cuda.Event()  # noqa: E731
            inputs_free = [None, None]     # the step that used buffer b has read its inputs
            results_free = [None, None]    # its cubes and gradients have come down
            grids = []

            def upload(i):
                b = i % 2
                with torch.cuda.stream(up):
                    if inputs_free[b] is not None:
                        up.wait_event(inputs_free[b])
                    for d, h in zip(dev_in[b], host_in):
                        d.copy_(h, non_blocking=True)
                    dev_tgt[b].copy_(host_tgt, non_blocking=True)
                    e = ev()
                    e.record(up)
                return e

            ready = upload(0)
            for i in range(n):
                b = i % 2
                nxt = upload(i + 1) if i + 1 < n else None
                ms.wait_event(ready)
                if results_free[b] is not None:
                    ms.wait_event(results_free[b])
                g = irt.Grid(*dev_in[b], w.cell_cm)
                grids.append(g)
                for view, out, ho, vf in zip(w.views, outs2[b], host_out, vflags):
                    irt.forward(g, view, w.vaxis, w.line, w.dust, integration=args.integration,
                                out=out, flags=vf)
                    done = ev()
                    done.record(ms)
                    with torch.cuda.stream(down):
                        down.wait_event(done)
                        for k in out:
                            ho[k].copy_(out[k], non_blocking=True)
                resid = outs2[b][0]["L"] - dev_tgt[b]
                inputs_free[b] = ev()
                inputs_free[b].record(ms)
                loss_d = torch.mean(resid * resid)
                irt.adjoint(g, w.views[0], w.vaxis, w.line, w.dust,
                            {"L": 2.0 * resid / resid.numel()}, integration=args.integration,
                            grads=grads2[b])
                done = ev()
                done.record(ms)
                # every read-back goes through the copy stream: a device-to-host
                # copy queued on the compute stream would wait behind the
                # cube copies in the copy engine and hold the adjoint back
                loss_d.record_stream(down)
                with torch.cuda.stream(down):
                    down.wait_event(done)
                    host_loss.copy_(loss_d, non_blocking=True)
                    for hg, dg in zip(host_grads, grads2[b]):
                        hg.copy_(dg, non_blocking=True)
                    results_free[b] = ev()
                    results_free[b].record(down)
                ready = nxt
            torch.cuda.synchronize()
            return grids

        for g in run_steps(2):
            g.close()
        e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grids_e2e = run_steps(e_steps)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / e_steps, ws, dev)
        for g in grids_e2e:
            g.close()
        e2e_v = whole_job_rate(units_step, ws, dt)
        e2e = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
               "path": "pinned host fields and target -> device, irt_create_grid, "
                       "irt_forward_ppv x2, loss, irt_adjoint_ppv, cubes + gradients + loss -> "
                       "pinned host; pipelined over steps: the next step's upload and this "
                       "step's read-back run on two copy streams beside the renders and the "
                       "adjoint (double-buffered device inputs and results; the grids are "
                       "released after the timed steps)"}

    clk = clocks.summary(wall0, wall1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, cores, sample, dt = oracle_rate(w, deq, target_s=10.0, integration=args.integration)
        ra, na, dta = oracle_adjoint_rate(w, deq, target_s=8.0)
        cpu = {"value": combined_rate(r, ra, sum(units_view), units_adj), "unit": UNIT,
               "cores": cores, "kind": "oracle",
               "sample": sample + f"; adjoint: dual-number gradient of {na} seeded z-view rays",
               "forward_rate": r, "adjoint_rate": ra, "seconds": dt + dta}

    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        accuracy = accuracy_measure(w, deq, outs, grads, l_target)
    extra = {}
    if rank == 0 and not args.no_thin:
        extra["ot"] = ot_measure(grid, w)
        extra["lines"] = lines_measure(grid, w)
    reduce_ = beam = None
    if rank == 0 and not args.no_thin:
        reduce_ = reduce_measure(outs[0])
        beam = beam_measure(outs[0])
    thin = None
    if not args.no_thin and rank == 0:
        thin = thin_measure(grid, w, deq, outs, units_view, pipe_peaks,
                            cpu=ws == 1 and not args.no_cpu_baseline)
    grid.close()
    for t in list(outs) + [grads]:
        del t
    torch.cuda.empty_cache()
    batch = None
    if not args.no_batch and args.n == 256:
        batch = batch_measure(args)
    large = None
    if not args.no_large and args.n == 256:
        torch.cuda.empty_cache()
        large = large_measure()
    adj128 = None
    if not args.no_large and rank == 0:
        torch.cuda.empty_cache()
        adj128 = adjoint128_measure()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{w.name}: z view + oblique (30,45) deg trilinear "
                                       f"forward, z-view adjoint, {args.integration} integration",
                           "grid": w.n, "nchan": w.vaxis.nchan, "f": w.vaxis.subsample_f,
                           "units_per_step": units_step, "units_per_view": units_view,
                           "l2": "inputs larger than L2 (packed fields 32 B/cell = "
                                 f"{w.n ** 3 * 32 / 1e6:.0f} MB > 126 MB)",
                           "parallelism": f"replicas x{ws}", "per_view_ms": view_ms,
                           "adjoint_ms": adj_ms, "units_adjoint": units_adj},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "accuracy": accuracy,
                "batch": batch, "large": large, "adjoint_128cube": adj128,
                "thin": thin, "latitude_mean": reduce_, "beam": beam, **extra,
                "clocks": clk, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# batched workload: 64 uneven snapshots, BF16 storage, Kahan formal transfer
# ---------------------------------------------------------------------------
def reduce_measure(cubes, reps=4):
    """The latitude-mean reduction (Sec. 6.1, the l-v image u) of the z-view
    cubes of the step: the five [nchan][npy][npx] float cubes in turn (5 x
    67 MB > L2, so each launch reads its cube from HBM), replayed as one CUDA
    graph with CUDA events around it.  Roofline: bytes read + written per launch against
    the measured HBM copy bandwidth."""
    import torch
    import paper_2607_01338_b300 as irt
    xs = [cubes[k] for k in ("T", "C", "D", "L", "B")]
    # the launches are captured in a CUDA graph so that the host's per-call
    # overhead (tens of microseconds against a kernel of about ten) does not
    # leave the GPU idle between them
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for x in xs:
            irt.latitude_mean(x)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        keep = [irt.latitude_mean(x) for _ in range(reps) for x in xs]
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    del keep
    ms = e0.elapsed_time(e1) / (reps * len(xs))
    A, B, C = xs[0].shape
    nbytes = 4 * (A * B * C + A * C)
    pk = peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": f"mean over b of a {A} x {B} x {C} float PPV cube (l-v image)",
            "launch_ms": ms, "bytes_per_launch": nbytes,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": float(pk["hbm_gbs"]),
                         "unit": "GB/s", "frac": gbs / float(pk["hbm_gbs"]),
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" +
                                        (" (fallback)" if pk.get("fallback") else "")}}


def beam_measure(cubes, fwhm_px=3.0, reps=2):
    """Gaussian beam convolution (Sec. 4.11) of the five z-view cubes in turn
    (FWHM 3 pixels), replayed as one CUDA graph.  Algorithmic bytes per call:
    two passes, each reading and writing the cube once."""
    import torch
    import paper_2607_01338_b300 as irt
    xs = [cubes[k] for k in ("T", "C", "D", "L", "B")]
    outs = [torch.empty_like(x) for x in xs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for x, o in zip(xs, outs):
            irt.beam_convolve(x, fwhm_px, out=o)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(reps):
            for x, o in zip(xs, outs):
                irt.beam_convolve(x, fwhm_px, out=o)
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * len(xs))
    nbytes = 4 * 4 * xs[0].numel()
    pk = peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": f"FWHM {fwhm_px} px Gaussian beam on a {tuple(xs[0].shape)} float cube",
            "call_ms": ms, "bytes_per_call": nbytes,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": float(pk["hbm_gbs"]),
                         "unit": "GB/s", "frac": gbs / float(pk["hbm_gbs"])}}


def thin_measure(grid, w, deq, outs, units_view, pipe_peaks, cpu=True, reps=5):
    """Selectively thin and optically thin transfer (Sec. 4.6, 4.7) and the
    density-tracing cube (Sec. 5.10), smooth integration, on both views of the
    step's grid: each view timed with CUDA
    events on the launching stream over ``reps`` warm launches (inputs larger
    than L2).  Units as the thick step (samples x channels); the oracle's rate
    in the same mode on a seeded sample of rays beside it."""
    import torch
    import oracle
    import paper_2607_01338_b300 as irt
    res = {"workload": f"{w.name}: z view + oblique (30,45) deg, smooth integration, "
                       "no velocity subsampling (channel-averaged profile)"}
    units = float(sum(units_view))
    for tr in ("selectively_thin", "thin", "density_tracing"):
        ms = []
        for view, out in zip(w.views, outs):
            for _ in range(2):
                irt.forward(grid, view, w.vaxis, w.line, w.dust, out=out, transfer=tr)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                irt.forward(grid, view, w.vaxis, w.line, w.dust, out=out, transfer=tr)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1) / reps)
        t = sum(ms) / 1e3
        fp32 = OPS_THIN_PAIR[tr] * units / t / 1e12
        r = {"per_view_ms": ms, "value": units / t, "unit": UNIT,
             "fp32_lower_bound_top_s": fp32,
             "frac_of_measured_fp32_lower_bound": fp32 / (pipe_peaks["fp32_ops_per_s"] / 1e12)}
        if cpu:
            rng = np.random.default_rng(5)
            mode = {"selectively_thin": oracle.SELECTIVELY_THIN, "thin": oracle.THIN,
                    "density_tracing": oracle.DENSITY_TRACING}[tr]
            nr, done, t0 = 64, 0.0, time.perf_counter()
            for view in w.views:
                pix = np.stack([rng.integers(0, view.npx, nr), rng.integers(0, view.npy, nr)],
                               axis=1)
                oracle.render(deq.as_tuple(), w.cell_cm, w.line, w.dust, view, w.vaxis, pix,
                              integration=oracle.SMOOTH, transfer=mode)
                for px, py in pix:
                    smp, _ = oracle.ray_samples(deq.as_tuple(), w.cell_cm, view, int(px), int(py))
                    done += len(smp) * w.vaxis.nchan
            r["oracle_rate"] = done / (time.perf_counter() - t0)
            r["oracle_sample"] = f"{nr} seeded rays per view, all channels, full depth, " \
                                 f"{oracle.num_threads()} threads"
        res[tr] = r
    return res


def accuracy_measure(w, deq, outs, grads, l_target, seed=11):
    """Error of every output of the timed step against the FP64 oracle on the
    same stored inputs, measured in the run: the five cubes of both views on
    an 8 x 8 pixel window at a seeded offset (all channels, rays at full
    depth), and the three gradients on two z-view columns (the oracle's
    dual-number gradient of the same loss).  Per output: the largest error
    over its allowance (FP32 rule: 1e-5 relative or 1e-6 of the cube peak;
    gradients: 1e-3 relative or 1e-7 of the largest) and the largest error
    over the peak."""
    import oracle
    mode = oracle.SMOOTH
    rng = np.random.default_rng(seed)
    res = {}
    for vi, (view, out) in enumerate(zip(w.views, outs)):
        x0 = int(rng.integers(0, view.npx - 8))
        y0 = int(rng.integers(0, view.npy - 8))
        py, px = np.meshgrid(np.arange(y0, y0 + 8), np.arange(x0, x0 + 8), indexing="ij")
        pix = np.stack([px.ravel(), py.ravel()], axis=1)
        orc = oracle.render(deq.as_tuple(), w.cell_cm, w.line, w.dust, view, w.vaxis, pix,
                            integration=mode)
        peak = float(np.abs(orc["T"]).max())
        comp = {}
        for k in "TCDLB":
            g = out[k][:, y0:y0 + 8, x0:x0 + 8].double().cpu().numpy()
            g = g.reshape(g.shape[0], -1).T
            err = np.abs(g - orc[k])
            allow = np.maximum(1e-5 * np.abs(orc[k]), 1e-6 * peak)
            comp[k] = {"worst_error_over_allowance": float((err / allow).max()),
                       "max_error_over_peak": float(err.max() / peak)}
        res[["z_view", "oblique_view"][vi]] = {"window": [x0, y0, 8, 8], "cubes": comp}
    cols = np.stack([rng.integers(0, w.n, 2), rng.integers(0, w.n, 2)], axis=1)
    tgt = l_target.double().cpu().numpy()
    loss, on, ot, ov = oracle.loss_grad_zview(deq.as_tuple(), w.cell_cm, w.line, w.dust,
                                              w.vaxis, tgt, pixels=cols)
    gres = {}
    for name, gg, oo in (("n_h2", grads[0], on), ("t_gas", grads[1], ot),
                         ("v_los", grads[2], ov)):
        gh = gg.double().cpu().numpy()
        a = np.stack([gh[:, y, x] for x, y in cols])
        b = np.stack([oo[:, y, x] for x, y in cols])
        err = np.abs(a - b)
        allow = 1e-3 * np.abs(b) + 1e-7 * np.abs(b).max()
        gres[name] = {"worst_error_over_allowance": float((err / allow).max()),
                      "max_error_over_max": float(err.max() / np.abs(b).max())}
    res["adjoint_columns"] = {"columns": cols.tolist(), "gradients": gres}
    res["rule"] = ("cubes: |gpu - oracle| <= max(1e-5 |oracle|, 1e-6 peak[T]); gradients: "
                   "<= 1e-3 |oracle| + 1e-7 max|oracle|; values <= 1 pass")
    return res


def traffic_from_profile():
    """DRAM bytes per launch of the step's kernels from the committed ncu
    summary, valid only while the kernel sources it was captured from are
    unchanged (their SHA-256 is recorded beside the numbers); else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_256cube_launches_and_dram.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        line = line.strip().strip("`")
        if ":" in line and line.split(":", 1)[0].strip() in (
                "kernel_sources_sha256", "adjoint_dram_bytes_per_launch",
                "z_view_dram_bytes_per_launch", "oblique_view_dram_bytes_per_launch"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if "kernel_sources_sha256" not in vals:
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2607_01338_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != vals["kernel_sources_sha256"]:
        return None
    try:
        return {k: float(v) for k, v in vals.items() if k != "kernel_sources_sha256"}
    except ValueError:
        return None


def adjoint128_measure(reps=5):
    """The 128^3 / 128-channel / f = 2 adjoint workload (smooth): the z-view
    forward keeping its checkpoints, the adjoint of a squared-error loss on
    [L]; and the same grid's (30, 45) deg oblique view's adjoint (its own
    forward sweep, gradients scattered to the trilinear cells).  Units:
    samples x channels of the adjoint's rays."""
    import torch
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    from synth import make_fields, to_storage, workload
    w = workload(3)
    f32, _ = to_storage(make_fields(w.n, w.seed), np.float32)
    t32, _ = to_storage(make_fields(w.n, w.seed + 7), np.float32)
    dev = torch.device("cuda", torch.cuda.current_device())
    g = irt.Grid(*[torch.from_numpy(a).to(dev) for a in f32.as_tuple()], w.cell_cm)
    tg = irt.Grid(*[torch.from_numpy(a).to(dev) for a in t32.as_tuple()], w.cell_cm)
    view = w.views[0]
    tgt = irt.forward(tg, view, w.vaxis, w.line, w.dust, components=("L",))["L"]
    tg.close()
    out = irt.alloc_cubes(view, w.vaxis)
    grads = tuple(torch.empty((w.n,) * 3, device=dev) for _ in range(3))
    from synth import View
    obl = View(math.radians(30), math.radians(45), w.n, w.n, w.cell_cm, 1)
    oout = irt.alloc_cubes(obl, w.vaxis)
    B.irt_grid_stats(g.handle, reset=True)
    irt.forward(g, obl, w.vaxis, w.line, w.dust, out=oout, flags=B.IRT_FLAG_STATS)
    units_obl = B.irt_grid_stats(g.handle, reset=True)["samples"] * w.vaxis.nchan

    def z_step():
        irt.forward(g, view, w.vaxis, w.line, w.dust, out=out,
                    flags=B.IRT_FLAG_SAVE_CHECKPOINTS)
        cot = {"L": 2.0 * (out["L"] - tgt) / out["L"].numel()}
        return cot

    cot = z_step()
    ocot = {"L": 2.0 * (oout["L"] - oout["L"].mean()) / oout["L"].numel()}
    for _ in range(2):
        irt.adjoint(g, view, w.vaxis, w.line, w.dust, cot, grads=grads)
        irt.adjoint(g, obl, w.vaxis, w.line, w.dust, ocot, grads=grads)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record()
    for _ in range(reps):
        z_step()
    ev[1].record()
    for _ in range(reps):
        irt.adjoint(g, view, w.vaxis, w.line, w.dust, cot, grads=grads)
    ev[2].record()
    for _ in range(reps):
        irt.adjoint(g, obl, w.vaxis, w.line, w.dust, ocot, grads=grads)
    ev[3].record()
    torch.cuda.synchronize()
    t_f = ev[0].elapsed_time(ev[1]) / reps
    t_a = ev[1].elapsed_time(ev[2]) / reps
    t_o = ev[2].elapsed_time(ev[3]) / reps
    units = w.n ** 3 * w.vaxis.nchan
    g.close()
    return {"workload": f"{w.name}: z view, smooth; forward keeping checkpoints, adjoint of "
                        "mean(([L] - target)^2); and the (30, 45) deg oblique view's adjoint "
                        "(fast sweep, gradients scattered to the trilinear cells)",
            "forward_ms": t_f, "adjoint_ms": t_a, "forward_value": units / (t_f / 1e3),
            "adjoint_value": units / (t_a / 1e3), "unit": UNIT,
            "oblique_adjoint_ms": t_o, "oblique_adjoint_value": units_obl / (t_o / 1e3),
            "accuracy": "gradients vs FP64 central differences on 200 cells and the oracle "
                        "gradient (tests/test_gpu_adjoint.py, tests/test_gpu_adjoint_general.py)"}


def ot_measure(grid, w, reps=5):
    """The optically thin level balance (Sec. 4.2, 4.3): the paper's
    128 x 64 x 64 grid built on the GPU for a 41-level rotor model (FP64
    solves, timed with CUDA events on the stream), and the z- and oblique-view
    renders of the step's grid with the 13CO 2-1 line's coefficients from that
    grid, against the LTE renders of the same line (units of the step)."""
    import torch
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    from synth.levels import OT_AXES, rotor_model
    model = rotor_model(nlev=41, seed=2)
    line = dict(w.line, nu_ul_hz=float(model["nu_hz"][1]))
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    irt.LevelTable(model, dict(OT_AXES, n_n=8, n_chi=4, n_t=8), [1]).close()   # warm-up
    torch.cuda.synchronize()
    e[0].record()
    tab = irt.LevelTable(model, OT_AXES, [0, 1, 2])
    e[1].record()
    torch.cuda.synchronize()
    build_ms = e[0].elapsed_time(e[1])
    res = {"grid": [OT_AXES["n_n"], OT_AXES["n_chi"], OT_AXES["n_t"]], "levels": 41,
           "lines": 3, "build_ms": build_ms,
           "model": "synthetic rigid rotor (13CO B0, 0.11 D dipole, invented collision rates "
                    "for p-H2, o-H2, H, He): no LAMDA file is available"}
    for vi, view in enumerate(w.views):
        out = irt.alloc_cubes(view, w.vaxis)
        B.irt_grid_stats(grid.handle, reset=True)
        irt.forward(grid, view, w.vaxis, line, w.dust, out=out, flags=B.IRT_FLAG_STATS)
        units = B.irt_grid_stats(grid.handle, reset=True)["samples"] * w.vaxis.nchan
        t = {}
        for kind in ("lte", "ot"):
            kw = dict(levels=tab, line_index=1) if kind == "ot" else {}
            for _ in range(2):
                irt.forward(grid, view, w.vaxis, line, w.dust, out=out, **kw)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(reps):
                irt.forward(grid, view, w.vaxis, line, w.dust, out=out, **kw)
            ev[1].record()
            torch.cuda.synchronize()
            t[kind] = ev[0].elapsed_time(ev[1]) / reps
        res[["z_view", "oblique_view"][vi]] = {
            "lte_ms": t["lte"], "ot_ms": t["ot"], "ot_value": units / (t["ot"] / 1e3),
            "unit": UNIT}
    res["accuracy"] = ("grid vs the oracle's grid to 1e-10 and renders vs the oracle with the "
                       "same grid at the FP32 rule (tests/test_gpu_ot.py)")
    tab.close()
    return res


def lines_measure(grid, w, reps=5):
    """Three lines (13CO 1-0, 2-1, 3-2 of a rigid rotor, each with its own
    dust opacity) rendered in one launch that samples each ray's fields once,
    against three single-line launches, on both views of the step's grid."""
    import torch
    import paper_2607_01338_b300 as irt
    from synth.levels import rotor_model
    model = rotor_model(nlev=8)
    b0 = float(model["nu_hz"][0]) / 2.0
    lines = []
    for r in (0, 1, 2):
        u, l = int(model["rad_up"][r]), int(model["rad_lo"][r])
        lines.append(dict(w.line, nu_ul_hz=float(model["nu_hz"][r]),
                          a_ul_s=float(model["a_ul_s"][r]), e_u_k=float(model["energy_k"][u]),
                          b0_hz=b0, g_u=float(model["g"][u]), g_l=float(model["g"][l])))
    dusts = [dict(w.dust, kappa_cm2_per_g_gas=k) for k in (0.004, 0.01, 0.02)]
    res = {"lines": "13CO 1-0, 2-1, 3-2 (rotor constants), kappa 0.004 / 0.01 / 0.02 cm^2/g"}
    for vi, view in enumerate(w.views):
        outs = [irt.alloc_cubes(view, w.vaxis) for _ in lines]
        t = {}
        for kind in ("one_launch", "three_launches"):
            def run():
                if kind == "one_launch":
                    irt.forward_lines(grid, view, w.vaxis, lines, dusts, outs=outs)
                else:
                    for ln, du, o in zip(lines, dusts, outs):
                        irt.forward(grid, view, w.vaxis, ln, du, out=o)
            for _ in range(2):
                run()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(reps):
                run()
            ev[1].record()
            torch.cuda.synchronize()
            t[kind] = ev[0].elapsed_time(ev[1]) / reps
        res[["z_view", "oblique_view"][vi]] = {
            "one_launch_ms": t["one_launch"], "three_launches_ms": t["three_launches"],
            "speedup": t["three_launches"] / t["one_launch"]}
        del outs
    res["accuracy"] = ("each line equals its single-line render to 1e-6 of the peak and the "
                       "oracle at the FP32 rule (tests/test_gpu_lines.py)")
    return res


def batch_measure(args, njobs=64, steps=3):
    """The 64-job batch (N in 64..256, 128..512 channels, random directions,
    BF16 fields with an FP16 velocity, Kahan-compensated formal transfer) as
    one autotuned persistent launch in a CUDA graph, against the same jobs
    rendered one launch per job from FP32 fields."""
    import torch
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    from synth import DUST, LINE_13CO_21, batch_jobs, make_fields_torch
    dev = torch.device("cuda", torch.cuda.current_device())
    jobs = batch_jobs(njobs, seed=2000)
    grids16, grids32, specs = [], [], []
    for bj in jobs:
        f = make_fields_torch(bj.n, bj.seed, n_mean=bj.n_mean, device=dev)
        t16 = [f[0].to(torch.bfloat16), f[1].to(torch.bfloat16), f[2].to(torch.bfloat16),
               f[3].to(torch.float16), f[4].to(torch.bfloat16)]
        t32 = [x.float() for x in f]
        grids16.append(irt.Grid(*t16, bj.cell_cm))
        grids32.append(irt.Grid(*t32, bj.cell_cm))
        specs.append((bj.view(), bj.vaxis))
        del f, t16, t32
    torch.cuda.synchronize()
    integ = "formal_kahan"
    # units: samples of every ray times its channel count
    units = 0
    outs = [irt.alloc_cubes(v, va) for v, va in specs]
    for g, (v, va), o in zip(grids16, specs, outs):
        B.irt_grid_stats(g.handle, reset=True)
        irt.forward(g, v, va, LINE_13CO_21, DUST, integration=integ, out=o,
                    flags=B.IRT_FLAG_STATS)
        units += B.irt_grid_stats(g.handle, reset=True)["samples"] * va.nchan
    stream = torch.cuda.current_stream()
    # batched BF16: autotune, capture, time graph launches
    bjobs = [(g, v, va) for g, (v, va) in zip(grids16, specs)]
    irt.forward_batch(bjobs, LINE_13CO_21, DUST, integration=integ, outs=outs, autotune=True)
    graph = irt.ForwardGraph(bjobs, LINE_13CO_21, DUST, integration=integ, outs=outs)
    graph.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / steps / 1e3
    plan = graph.plan()
    graph.close()
    # FP32 single-cube launches of the same jobs
    for g, (v, va), o in zip(grids32, specs, outs):
        irt.forward(g, v, va, LINE_13CO_21, DUST, integration=integ, out=o)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for g, (v, va), o in zip(grids32, specs, outs):
            irt.forward(g, v, va, LINE_13CO_21, DUST, integration=integ, out=o)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / steps / 1e3
    for g in grids16 + grids32:
        g.close()
    return {"workload": f"{njobs} snapshots, N 64..256, 128..512 channels at 1 km/s, f = 1, "
                        "random directions (trilinear), BF16 fields + FP16 v_los, "
                        "Kahan-compensated formal transfer",
            "units": units, "value": units / t_batch, "unit": UNIT, "ms": t_batch * 1e3,
            "plan": {"NI": plan[0], "tile": [plan[1], plan[2]]},
            "fp32_single_cube": {"value": units / t_single, "ms": t_single * 1e3,
                                 "launches": njobs},
            "speedup_vs_fp32_single_cube": t_single / t_batch,
            "accuracy": "FP32 parity rule vs the FP64 oracle on the stored values "
                        "(tests/test_gpu_batch.py)"}


# ---------------------------------------------------------------------------
# large single render: 512^3, FP16 storage, 500 channels, forward + adjoint
# ---------------------------------------------------------------------------
def large_measure(steps=3):
    """The 512^3 grid with five FP16-stored fields (per-field scales), 500
    channels from -250 to +250 km/s, z view, smooth integration: forward and
    the adjoint of mean(L^2), against the same fields stored as FP32."""
    import torch
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    from synth import DUST, LINE_13CO_21, make_fields_torch, workload
    w = workload(4)
    view, va = w.views[0], w.vaxis
    scales = (1.0e4, 1.0, 1.0, 1.0, 1.0e-6)
    f = make_fields_torch(w.n, w.seed)
    h = [(f[q] / scales[q]).to(torch.float16) for q in range(5)]
    f32 = [x.float() for x in f]
    del f
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    res = {}
    for name, grid in (("fp16", irt.Grid(*h, w.cell_cm, scales=scales)),
                       ("fp32", irt.Grid(*f32, w.cell_cm))):
        out = irt.alloc_cubes(view, va)
        B.irt_grid_stats(grid.handle, reset=True)
        irt.forward(grid, view, va, LINE_13CO_21, DUST, out=out, flags=B.IRT_FLAG_STATS)
        st = B.irt_grid_stats(grid.handle, reset=True)
        units = st["samples"] * va.nchan
        cot = {"L": 2.0 * out["L"] / out["L"].numel()}
        grads = tuple(torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
                      for _ in range(3))
        irt.adjoint(grid, view, va, LINE_13CO_21, DUST, cot, grads=grads)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = ta = 0.0
        for _ in range(steps):
            ev[0].record(stream)
            irt.forward(grid, view, va, LINE_13CO_21, DUST, out=out,
                        flags=B.IRT_FLAG_SAVE_CHECKPOINTS)
            ev[1].record(stream)
            irt.adjoint(grid, view, va, LINE_13CO_21, DUST, cot, grads=grads)
            ev[2].record(stream)
            torch.cuda.synchronize()
            tf += ev[0].elapsed_time(ev[1]) / steps
            ta += ev[1].elapsed_time(ev[2]) / steps
        fwd_fp32 = 32 * (OPS_LINE[0] * st["line_block_samples"]
                         + OPS_DUST[0] * (st["hull_block_samples"] - st["line_block_samples"])) \
            + OPS_SAMPLE[0] * st["samples"]
        res[name] = {"forward_ms": tf, "adjoint_ms": ta,
                     "value": 2 * units / ((tf + ta) / 1e3), "unit": UNIT,
                     "forward_fp32_top_s": fwd_fp32 / (tf / 1e3) / 1e12,
                     "forward_hbm_gbs": (grid_bytes(w.n, name) + 5 * 4 * va.nchan * w.n ** 2)
                     / (tf / 1e3) / 1e9}
        grid.close()
        del out, cot, grads
        torch.cuda.empty_cache()
    return {"workload": f"{w.name}: 512^3, five FP16 fields with per-field scales, 500 channels "
                        "-250..+250 km/s, z view, smooth; forward (keeping its checkpoints) + "
                        "adjoint of mean(L^2)",
            "fp16_storage": res["fp16"], "fp32_storage": res["fp32"],
            "speedup_fp16_vs_fp32": (res["fp32"]["forward_ms"] + res["fp32"]["adjoint_ms"])
            / (res["fp16"]["forward_ms"] + res["fp16"]["adjoint_ms"]),
            "accuracy": "FP32 parity rule on the stored values (tests/test_gpu_large.py)"}


def grid_bytes(n, storage):
    return n ** 3 * (16 if storage == "fp16" else 32)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
