#!/usr/bin/env python
"""Benchmark of the gDRR projection path on GB300.

Workload: the 2 mm ellipsoid torso (256x256x128 voxels, uint8 material +
FP32 density), 120 kVp Kramers spectrum with 2.5 mm Al, aluminium bowtie
0-30 mm, 512x384 detector of 0.776 mm pixels, CsI-like response, 1e8 photon
histories per projection.  One step = one whole projection, Steps 1-4:
ray-traced primary, Monte Carlo primary + scatter, tally finalisation,
4x4 scatter binning, Poisson denoising (Eq. 5), upsampling, noise scaling.

Metric: photon histories per second (and seconds per projection).
Multi-GPU (torchrun): each rank simulates its own projection angle of a scan
(independent work, no data-path collective): weak scaling.

--impl reference runs the CPU oracle on the host cores instead (bounded
samples of the same workload).
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

METRIC = "MC photon histories/s and s/projection, 2 mm torso 120 kVp; batched vs plain"
UNIT = "histories/s"
WORKLOAD = "torso-256x256x128-2mm, 120kVp Kramers+2.5mmAl, Al bowtie 0-30mm, 512x384 det 0.776mm, CsI response, 1e8 histories"
BYTES_PER_STEP_ALGO = 8 * 5          # 8 corner voxels x (1 B material + 4 B density) per Woodcock step
RECORD_BYTES_PER_STEP = 8 * 8        # the 8 corner records the kernel loads, 8 bytes each
FLOPS_PER_STEP_ALGO = 40             # trilinear weights, 8-corner mixture, free path: ~40 FP32 flops


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--histories", type=float, default=1e8)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU-oracle sample time")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scan", action="store_true", help="skip the 64-angle batched-scan comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1 mm / 4 mm voxel-size timings")
    ap.add_argument("--no-learned", action="store_true", help="skip training / evaluating the learned estimator")
    ap.add_argument("--no-variants", action="store_true", help="skip the nearest-voxel / Siddon / filter timings")
    ap.add_argument("--no-fdk", action="store_true", help="skip the 360-view FDK reconstruction timing")
    ap.add_argument("--mc-config", default=None, metavar="BLOCK,BATCH_MIN,HIST_PER_THREAD",
                    help="fix the transport's launch configuration (lane form) instead of autotuning it")
    ap.add_argument("--local-majorant", type=int, default=None, metavar="CELL_SHIFT",
                    help="run the transport with the local-majorant option (cells of 2^CELL_SHIFT voxels) "
                         "instead of the paper's global Woodcock majorant, to profile the option")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json (measured on the GB300s),
    else the fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except (OSError, ValueError, KeyError):
        return fallback


def profile_record(name, cell_shift=None):
    """Counters of the transport kernel from a committed ncu summary
    (profiles/<name>): its "key value" lines as a dict, with its "config ..."
    lines (one per launch configuration measured) as a list under "configs";
    None when the kernel source changed since those counters were taken, or
    they were taken with other macro cells (cell_shift given)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    vals, configs = {}, []
    try:
        for l in open(path):
            f = l.split()
            if not f or l.startswith("#"):
                continue
            if f[0] == "config":
                configs.append(f[1:])
            elif len(f) == 2:
                vals[f[0]] = f[1]
            else:
                return None
    except OSError:
        return None
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1204_6367_gb300", "csrc", "mc_transport.cu"), "rb").read())
    if h.hexdigest()[:16] != vals.get("source_sha256_16"):
        return None
    if cell_shift is not None and str(cell_shift) != vals.get("cell_shift"):
        return None
    vals["configs"] = configs
    return vals


def kernel_traffic(cell_shift=None):
    """DRAM bytes per transport launch (ncu), or None for another kernel source
    or other macro cells."""
    v = profile_record("mc_kernel_torso2mm_traffic.txt", cell_shift)
    return int(v["bytes_per_launch"]) if v else None


# The instruction count per flight depends on batch_min (how often the warp
# serves its waiting lanes) and is keyed to the block size as well; the
# histories a lane claims at a time (hist_per_thread) leave it unchanged
# (measured: 266.14 and 266.12 per flight at 1 and 8), so a line's third
# field is informational.
ISSUE_CONFIG_KEYS = ("block_size", "batch_min")


def kernel_inst_per_step(cell_shift=None, config=None):
    """Thread instructions the transport executes per Woodcock free flight
    (ncu smsp__thread_inst_executed.sum / free flights of the same launch)
    from the record's line for the launch configuration given (block_size
    and batch_min; config None: the first line), or None for another kernel
    source, other macro cells or an unmeasured configuration."""
    v = profile_record("mc_kernel_torso2mm_issue.txt", cell_shift)
    if not v:
        return None
    for c in v["configs"]:
        if config is None or [str(config.get(k)) for k in ISSUE_CONFIG_KEYS] == c[:2]:
            return float(c[3])
    return None


def transport_roofline(steps, mc_s, hbm_peak, traffic, inst_per_step=None, n_sm=152, sm_max_mhz=2070.0,
                       context=None):
    """The transport's roofline entry on its algorithmic unit: 40 B of voxel
    data (8 corners x (1 B material + 4 B density)) per Woodcock free flight x
    the free flights counted live in the timed launches, over their mean
    CUDA-event time, against the measured HBM copy peak.  The issue rate
    (thread instructions per flight from an ncu record of this kernel source
    and launch configuration, against SMs x 4 schedulers x 32 lanes x the
    maximum SM clock) and the other ceilings ride along as context."""
    achieved = steps * BYTES_PER_STEP_ALGO / mc_s / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
         "traffic": traffic, "kernel": "mc_kernel",
         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
         "algorithmic": f"{BYTES_PER_STEP_ALGO} B of voxel data per Woodcock step x {steps} steps per launch",
         "mc_ms": 1e3 * mc_s, "woodcock_steps": steps}
    issue_peak = n_sm * 4 * 32 * sm_max_mhz * 1e6 / 1e12
    if inst_per_step:
        issue = inst_per_step * steps / mc_s / 1e12
        r.update(issue_tinst_s=issue, issue_peak_tinst_s=issue_peak, issue_frac=issue / issue_peak,
                 inst_per_step=inst_per_step)
    else:
        r.update(issue_frac=None, inst_per_step=None)
    r.update(context or {})
    return r


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_angle(rank, world):
    """Gantry angle of a rank's projection: the ranks split one scan's orbit,
    one angle each (independent histories, no data-path exchange)."""
    return 2.0 * math.pi * rank / max(world, 1)


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values: the job's time is its slowest rank's."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_hist, world, steps, tot_ms):
    """Whole-job histories/s: every rank's histories over the slowest rank's time."""
    return n_hist * world * steps / (tot_ms / 1e3)


def cpu_oracle_rate(prob, target_s, threads, seed=1, first=400000):
    """Histories/s of the CPU oracle (FP32 transport, the parity reference) on
    a bounded sample of the same workload: first history ids of the stream."""
    import oracle
    oracle.build()
    n = first
    t0 = time.perf_counter()
    oracle.mc_run(prob, n, seed=seed, threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(max(n, min(1e8, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.mc_run(prob, n2, seed=seed, threads=threads)
    dt2 = time.perf_counter() - t0
    return n2 / dt2, n2, dt2


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1204_6367_gb300 import inputs
    import oracle
    oracle.build()
    prob = inputs.torso_problem()
    threads = os.cpu_count() or 1
    # each step: a bounded sample of the projection's histories, sized so the
    # whole --steps/--warmup run stays within a few minutes
    probe = 400000
    t0 = time.perf_counter()
    oracle.mc_run(prob, probe, seed=1, threads=threads)
    rate0 = probe / (time.perf_counter() - t0)
    per_step = int(max(probe, min(2e7, rate0 * 150.0 / max(1, args.steps + args.warmup))))
    for w in range(args.warmup):
        oracle.mc_run(prob, per_step, seed=1, history_offset=w * per_step, threads=threads)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.mc_run(prob, per_step, seed=1, history_offset=(args.warmup + k) * per_step, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * args.steps / tot
    sample = f"{per_step} histories per step of the 1e8-history projection (history ids in order), FP32 oracle"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "s_per_projection": args.histories / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "histories_per_projection": int(args.histories),
                   "l2": "oracle runs on host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1204_6367_gb300 import gdrr, inputs
    gdrr.lib()
    prob = inputs.torso_problem()
    n_hist = int(args.histories)
    angle = rank_angle(rank, world)                  # one projection angle per rank
    seed = 1
    stream = torch.cuda.current_stream()
    ctx = gdrr.Context(prob, stream)
    npix = prob.nu * prob.nv
    iters = 300
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    stats = torch.zeros(gdrr.GDRR_NSTATS, dtype=torch.int64, device="cuda")

    # one step = one gdrr_project call (Steps 1-4, every scalar on the device)
    # into preallocated outputs; the library times the transport launch with
    # CUDA events on the stream it runs on
    out = {}

    def step():
        return gdrr.project(ctx, n_hist, seed, angle, bin_factor=4, beta=0.02, iters=iters, stats=stats, out=out)

    if args.local_majorant is not None:
        gdrr.gdrr_set_options(ctx, local_majorant=1, cell_shift=args.local_majorant)
    # launch configuration from the project's autotuner, or the one given
    # (tallies do not depend on it)
    if args.mc_config:
        b, m, h = (int(x) for x in args.mc_config.split(","))
        gdrr.gdrr_set_options(ctx, block_size=b, batch_min=m, hist_per_thread=h, blocks_per_sm=0, photon_pool=-1)
        tuned = gdrr.gdrr_get_options(ctx)
    else:
        tuned = gdrr.gdrr_autotune(ctx, angle, 20_000_000, seed)

    for _ in range(max(args.warmup, 3)):
        res = step()
    torch.cuda.synchronize()
    st = gdrr.stats_dict(stats)
    steps_per_proj = st["steps"]
    skips_per_proj = gdrr.cell_skips(stats)            # virtual collisions decided without corner gathers
    gathers_per_proj = steps_per_proj - skips_per_proj
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    mc_ms, dn_ms = [], []

    # memory ceiling for the transport's access pattern: the same corner
    # gathers at as many random cells as the projection gathers (free flights
    # less those the macro-cell bound decided)
    gdrr.gdrr_gather_roofline(ctx, min(gathers_per_proj, 10**9))
    probe_s = gdrr.gdrr_gather_roofline(ctx, gathers_per_proj)
    # machine ceilings measured on this GPU: random 8-byte L2 gathers, FP32 FMA
    l2_probe_gbs = gdrr.gdrr_probe_l2_gather(32 << 20)
    fp32_probe_tflops = gdrr.gdrr_probe_fp32()
    # kernels per step: ray trace, 3 finalisations, binning, the scalars,
    # upsampling, noise (8); the transport (the pool form: one launch; the
    # lane form: a source pass and a transport launch per 2^27 histories);
    # the denoiser (one cooperative launch, else one per iteration + 2)
    transport_launches = 1 if tuned["photon_pool"] > 0 else 2 * -(-n_hist // (1 << 27))
    launches_per_step = 8 + transport_launches + (1 if res["denoise_fused"] else iters + 2)

    clocks = ClockSampler(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                     # evict L2 between timed iterations
        ev[k][0].record(stream)
        r = step()
        ev[k][1].record(stream)
        mc_ms.append(r["transport_ms"])
        dn_ms.append(r["denoise_ms"])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), world)

    # end to end through the public API: inputs from pinned host memory
    # (gdrr_create stages phantom and tables), one projection, results read
    # back to host (P, P^, S^, S, N)
    e2e = None
    if not args.no_e2e:
        pinned = {}
        for name in ("material", "density", "mu_hat", "spec_e", "spec_w", "fluence", "response"):
            a = np.ascontiguousarray(getattr(prob, name))
            t_pin = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t_pin.numpy()[...] = a
            pinned[name] = t_pin
        import copy
        hp = copy.copy(prob)
        for name, t_pin in pinned.items():
            setattr(hp, name, t_pin.numpy())
        h2d = sum(t_pin.numel() * t_pin.element_size() for t_pin in pinned.values())
        host_out = [torch.empty((prob.nv, prob.nu), dtype=torch.float64, pin_memory=True) for _ in range(5)]
        d2h = sum(h.numel() * h.element_size() for h in host_out)
        e2e_steps = max(1, min(args.steps, 3))

        def e2e_step():
            with gdrr.Context(hp, stream) as c2:
                gdrr.gdrr_set_options(c2, **tuned)
                o = gdrr.project(c2, n_hist, seed, angle, beta=0.02, iters=iters)
                for h, key in zip(host_out, ("P", "P_hat", "S_hat", "S", "N")):
                    h.copy_(o[key], non_blocking=True)
                torch.cuda.synchronize()

        e2e_step()                                   # untimed: the library's memory pool grows once
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)   # the slowest rank's
        e2e = {"value": job_rate(n_hist, world, 1, 1e3 * e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "s_per_projection": e2e_s}

    # multi-angle scan: 64 angles over 360 degrees with per-angle budgets
    # drawn from U(1e7, 5e7), one persistent launch replayed from a CUDA
    # graph, against 64 plain per-angle launches of the same histories
    batched = None
    if not args.no_scan:
        angles, budgets = inputs.batched_budgets(64, 1e7, 5e7, seed=1)
        angles = angles + angle
        tot_hist = int(budgets.sum())
        sp, ss = gdrr.new_tallies(ctx, angles.size)
        scan = gdrr.gdrr_scan_create(ctx, angles, budgets, seed, sp, ss, zero_tallies=True)
        scan.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        scan.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        graph_s = e0.elapsed_time(e1) / 1e3
        pp, ps = gdrr.new_tallies(ctx, angles.size)
        scan_stats = torch.zeros(gdrr.GDRR_NSTATS, dtype=torch.int64, device="cuda")
        e0.record(stream)
        for a in range(angles.size):
            gdrr.gdrr_mc_project(ctx, int(budgets[a]), seed, float(angles[a]), a, prim=pp[a], scat=ps[a],
                                 stats=scan_stats)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_s = e0.elapsed_time(e1) / 1e3
        same = bool(torch.equal(sp, pp) and torch.equal(ss, ps))
        scan.close()
        del sp, ss, pp, ps
        # the same histories' free flights (identical tallies, so identical
        # flights): algorithmic bytes against the HBM peak and the gather probe
        scan_steps = gdrr.stats_dict(scan_stats)["steps"]
        scan_probe_s = gdrr.gdrr_gather_roofline(ctx, scan_steps - gdrr.cell_skips(scan_stats))
        batched = {"angles": int(angles.size), "histories": tot_hist,
                   "graph_s": graph_s, "plain_64_launches_s": plain_s,
                   "graph_histories_per_s": tot_hist / graph_s, "plain_histories_per_s": tot_hist / plain_s,
                   "speedup": plain_s / graph_s, "tallies_identical": same,
                   "woodcock_steps": scan_steps,
                   "graph_algorithmic_gbs": scan_steps * BYTES_PER_STEP_ALGO / graph_s / 1e9,
                   "graph_frac_of_hbm_peak": scan_steps * BYTES_PER_STEP_ALGO / graph_s / 1e9
                   / measured_peak("hbm_gbs", 6800.0),
                   "graph_frac_of_gather_roof": scan_probe_s / graph_s}

    # voxel-size sweep: the same torso at 1 mm (512x512x256, 537 MB of
    # records: beyond L2) and 4 mm (128x128x64), transport only, 1e8 histories
    voxel_sweep = None
    if not args.no_sweep:
        voxel_sweep = {}
        for vox in (1.0, 4.0):
            pv = inputs.torso_problem(vox=vox)
            with gdrr.Context(pv, stream) as cv:
                vstats = torch.zeros(gdrr.GDRR_NSTATS, dtype=torch.int64, device="cuda")
                vp, vs = gdrr.gdrr_mc_project(cv, n_hist, seed, angle, stats=vstats)
                torch.cuda.synchronize()
                vstats.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(1.0)
                e0.record(stream)
                gdrr.gdrr_mc_project(cv, n_hist, seed, angle, prim=vp, scat=vs, stats=vstats)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_v = e0.elapsed_time(e1)
                sv = gdrr.stats_dict(vstats)
                probe_v = gdrr.gdrr_gather_roofline(cv, sv["steps"] - gdrr.cell_skips(vstats))
                voxel_sweep[f"{vox:g}mm"] = {
                    "shape_zyx": list(pv.material.shape), "mc_ms": ms_v, "histories_per_s": n_hist / ms_v * 1e3,
                    "free_flights": sv["steps"], "algorithmic_gbs": sv["steps"] * BYTES_PER_STEP_ALGO / ms_v / 1e6,
                    "gather_roof_frac": (probe_v * 1e3) / ms_v}
            del pv

    # the paper's speed variants (appendix): transport without density
    # interpolation, and Siddon ray tracing, against the defaults
    variants = None
    if not args.no_variants:
        variants = {}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for name, fn in (("rt_trilinear_ms", lambda: gdrr.gdrr_raytrace_primary(ctx, angle)),
                         ("rt_siddon_ms", lambda: gdrr.gdrr_raytrace_primary_siddon(ctx, angle))):
            fn()
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            variants[name] = e0.elapsed_time(e1)
        opts = gdrr.gdrr_get_options(ctx)
        for name, kw in (("mc_nearest_voxel_ms", dict(nearest_voxel=1)),
                         ("mc_first_order_compton_ms", dict(scatter_filter=1)),
                         ("mc_rayleigh_form_factor_ms", dict(rayleigh_form_factor=1)),
                         # the macro-cell test of virtual collisions: off, and cells of 8 and 16 mm
                         # (4 and 8 voxels; the default is 4 mm, 2 voxels); tallies are identical
                         # in every case
                         ("mc_no_cell_bound_ms", dict(cell_shift=-1)),
                         ("mc_cells_8mm_ms", dict(cell_shift=2)),
                         ("mc_cells_16mm_ms", dict(cell_shift=3)),
                         # delta tracking with local majorants (an option beside the paper's
                         # global one): the cell bounds of 32 mm (default) or 16 mm cells as
                         # the flights' majorant, lane form, batch_min 24; same expected images
                         ("mc_local_majorant_32mm_ms", dict(local_majorant=1, cell_shift=4, batch_min=24,
                                                            photon_pool=-1)),
                         ("mc_local_majorant_16mm_ms", dict(local_majorant=1, cell_shift=3, batch_min=24,
                                                            photon_pool=-1))):
            gdrr.gdrr_set_options(ctx, **kw)
            vp, vs = gdrr.gdrr_mc_project(ctx, n_hist, seed, angle)
            torch.cuda.synchronize()
            flush.fill_(2.0)
            e0.record(stream)
            gdrr.gdrr_mc_project(ctx, n_hist, seed, angle, prim=vp, scat=vs)
            e1.record(stream)
            torch.cuda.synchronize()
            variants[name] = e0.elapsed_time(e1)
            gdrr.gdrr_set_options(ctx, **opts)
        variants["mc_trilinear_ms"] = statistics.mean(mc_ms)
        # per-column spectra behind the bowtie (energy-dependent hardening)
        ph = inputs.torso_problem(vox=2.0, hardened_bowtie=True)
        with gdrr.Context(ph, stream=stream) as ch:
            gdrr.gdrr_set_options(ch, **{k: v for k, v in opts.items() if k != "rayleigh_form_factor"})
            gdrr.gdrr_mc_project(ch, n_hist, seed, angle, prim=vp, scat=vs)
            torch.cuda.synchronize()
            flush.fill_(2.0)
            e0.record(stream)
            gdrr.gdrr_mc_project(ch, n_hist, seed, angle, prim=vp, scat=vs)
            e1.record(stream)
            torch.cuda.synchronize()
            variants["mc_hardened_bowtie_ms"] = e0.elapsed_time(e1)
        del vp, vs, ph

    # reconstruction of a simulated scan (Section 3.5): 360 ray-traced views
    # of the torso, line integrals, FDK filter and backprojection onto the
    # phantom's own 2 mm grid
    recon = None
    if not args.no_fdk:
        n_views = 360
        angles_r = np.arange(n_views) * (2.0 * math.pi / n_views)
        sig = torch.empty((n_views, prob.nv, prob.nu), dtype=torch.float64, device="cuda")
        e_p0, e_p1, e_f0, e_f1, e_b1 = (torch.cuda.Event(enable_timing=True) for _ in range(5))
        e_p0.record(stream)
        for i, a in enumerate(angles_r):
            gdrr.gdrr_raytrace_primary(ctx, float(a), out=sig[i])
        I0 = gdrr.gdrr_air_scan(ctx)
        g = gdrr.gdrr_line_integrals(sig, I0.expand_as(sig).contiguous())
        e_p1.record(stream)
        geo = gdrr.fdk_geometry(prob.sad, prob.sdd, prob.nu, prob.nv, prob.du, prob.dv, prob.material.shape,
                                prob.voxel)
        for _ in range(2):                                 # the second pass is timed
            flush.fill_(3.0)
            e_f0.record(stream)
            qf = gdrr.gdrr_fdk_filter(geo, g)
            e_f1.record(stream)
            vol = gdrr.gdrr_fdk_backproject(geo, qf, angles_r)
            e_b1.record(stream)
            torch.cuda.synchronize()
        nz_, ny_, nx_ = prob.material.shape
        bp_ms = e_f1.elapsed_time(e_b1)
        recon = {"views": n_views, "grid_zyx": [nz_, ny_, nx_], "voxel_mm": list(prob.voxel),
                 "ray_traced_views_ms": e_p0.elapsed_time(e_p1),
                 "filter_ms": e_f0.elapsed_time(e_f1), "backproject_ms": bp_ms,
                 "voxel_views_per_s": nz_ * ny_ * nx_ * n_views / bp_ms * 1e3}
        del sig, g, qf, vol, I0

    # learned scatter estimator against the plain method: train on pairs the
    # method generates (256 torsos, one random angle each: denoised 1e6-history
    # scatter + ray-traced primary -> denoised 1e8-history scatter), evaluate on
    # held-out torsos against a denoised 2e9-history reference, next to the
    # plain method at 1e6 ... 1e8 histories; the photon count the plain method
    # needs for the learned error gives the saving at matched error
    learned = None
    if not args.no_learned:
        from paper_1204_6367_gb300 import scatter_net as sn
        t_data = time.perf_counter()
        LX, LY = sn.make_dataset(range(100, 356), 1, 10**6, 10**8, rng_seed=1)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t_data
        net = gdrr.Cnn(64, sn.H, sn.W, 32, seed=1)
        t_train = time.perf_counter()
        n_train = 4000
        losses = sn.train(net, LX, LY, n_train, 16, 1e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t_train
        rng_l = np.random.default_rng(7)
        plain_counts = (10**6, 3 * 10**6, 10**7, 10**8)
        e_net, e_plain, cost = [], {n: [] for n in plain_counts}, {}
        for sd in (900, 901):
            with gdrr.Context(sn.coarse_problem(sd)) as cl:
                for a in range(2):
                    ang = float(rng_l.uniform(0, 2 * math.pi))
                    ref = sn.estimate(cl, 2 * 10**9, 91 + 10 * sd + a, ang, a, 1.5)[0].cpu().numpy()
                    xl = torch.empty((1, 2, sn.H, sn.W), dtype=torch.float32, device="cuda")
                    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                    e0.record(stream)
                    sn.low_input(cl, 10**6, 31 + 10 * sd + a, ang, a, xl[0])
                    pred = sn.predict(net, xl)
                    e1.record(stream)
                    plain8, _ = sn.estimate(cl, 10**8, 57 + 10 * sd + a, ang, a, sn.HIGH_LENGTH)
                    e2.record(stream)
                    torch.cuda.synchronize()
                    cost.setdefault("learned_ms", []).append(e0.elapsed_time(e1))
                    cost.setdefault("plain_1e8_ms", []).append(e1.elapsed_time(e2))
                    e_net.append(sn.rel_l2(pred.cpu().numpy()[0], ref))
                    e_plain[10**8].append(sn.rel_l2(plain8.cpu().numpy(), ref))
                    for n in plain_counts[:-1]:
                        sp_, _ = sn.estimate(cl, n, 31 + 10 * sd + a, ang, a, sn.plain_length(n))
                        e_plain[n].append(sn.rel_l2(sp_.cpu().numpy(), ref))
        err_plain = {n: float(np.mean(v)) for n, v in e_plain.items()}
        err_net = float(np.mean(e_net))
        # photons the plain method needs for the learned error (log-log interpolation)
        lx = np.log(np.array(plain_counts, np.float64))
        ly = np.log(np.array([err_plain[n] for n in plain_counts]))
        order = np.argsort(ly)
        matched = float(np.exp(np.interp(math.log(err_net), ly[order], lx[order])))
        xb = LX[:64]
        net.forward(xb)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.forward(xb)
        e1.record(stream)
        torch.cuda.synchronize()
        # the network's building block against the measured BF16 tensor peak:
        # one 8192^3 GEMM through the library's tcgen05 kernel
        ga = torch.randn((8192, 8192), dtype=torch.bfloat16, device="cuda")
        gb = torch.randn((8192, 8192), dtype=torch.bfloat16, device="cuda")
        gc = torch.empty((8192, 8192), dtype=torch.float32, device="cuda")
        gdrr.gdrr_gemm_bf16(ga, gb, out=gc)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gdrr.gdrr_gemm_bf16(ga, gb, out=gc)
        g1.record(stream)
        torch.cuda.synchronize()
        gemm_ms = g0.elapsed_time(g1)
        bf16_peak = measured_peak("bf16_tflops", 1900.0)
        gemm = {"m_n_k": 8192, "ms": gemm_ms, "tflops": 2 * 8192**3 / gemm_ms / 1e9,
                "frac_of_measured_bf16_peak": 2 * 8192**3 / gemm_ms / 1e9 / bf16_peak}
        del ga, gb, gc
        # the network's own convolution flops (2 x pixels x Cin x Cout x taps
        # per layer) against the measured BF16 peak
        fwd_flops = sn.network_flops(32)
        inf_ms = e0.elapsed_time(e1)
        inf_tflops = 64 * fwd_flops / inf_ms / 1e9
        train_tflops = n_train * 16 * 3 * fwd_flops / t_train / 1e12
        net_roof = {"bound": "tensor", "achieved": inf_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                    "frac": inf_tflops / bf16_peak, "kernel": "network forward, batch 64",
                    "algorithmic": f"{fwd_flops / 1e9:.3f} GFLOP per 96x128 image (conv layers) x 64",
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)",
                    "training_tflops": train_tflops, "training_frac": train_tflops / bf16_peak,
                    "training_what": "3 x forward flops per image (forward, data and weight gradients) x 16 x steps "
                                     "over the training wall time"}
        learned = {"train_pairs": int(LX.shape[0]), "data_s": t_data, "train_steps": n_train, "train_s": t_train,
                   "gemm_bf16": gemm, "roofline": net_roof,
                   "final_loss": float(np.mean(losses[-50:])),
                   "rel_l2_vs_2e9_reference": {"learned_1e6": err_net,
                                               **{f"plain_denoised_{n:.0e}": err_plain[n] for n in plain_counts}},
                   "plain_histories_at_learned_error": matched,
                   "photon_saving_at_matched_error": matched / 1e6,
                   "ms_per_projection": {"learned_1e6_plus_inference": float(np.mean(cost["learned_ms"])),
                                         "plain_1e8_plus_denoise": float(np.mean(cost["plain_1e8_ms"]))},
                   "inference_batch64_ms": inf_ms}
        net.close()
        del LX, LY

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    mc_avg_s = statistics.mean(mc_ms) / 1e3
    n_mat = prob.mu_hat.shape[0]
    cell_bytes = 4 * (2 if n_mat <= 2 else (4 if n_mat <= 4 else 8))
    loaded_bytes = gathers_per_proj * RECORD_BYTES_PER_STEP + steps_per_proj * cell_bytes
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    value = job_rate(n_hist, world, args.steps, tot_ms)
    traffic = kernel_traffic(tuned["cell_shift"])

    # The transport on its algorithmic unit (40 B of voxel data per free
    # flight) against the HBM copy peak; the phantom is L2-resident and most
    # flights skip the gathers, so the issue rate and the L2 gather probe are
    # the binding ceilings, reported beside it.
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    inst_per_step = kernel_inst_per_step(tuned["cell_shift"], tuned)
    l2_achieved = loaded_bytes / mc_avg_s / 1e9
    context = {
        "l2_gather_probe_gbs": l2_probe_gbs, "l2_gather_achieved_gbs": l2_achieved,
        "l2_gather_frac": l2_achieved / l2_probe_gbs,
        "l2_gather_what": "random 8-byte loads over a 32 MiB L2-resident set vs the bytes the transport loads: "
                          f"8 x 8-byte voxel records per gathering flight, one {cell_bytes}-byte macro-cell record "
                          "per flight",
        "gather_probe_ms": 1e3 * probe_s, "gather_probe_frac": probe_s / mc_avg_s,
        "fp32_probe_tflops": fp32_probe_tflops,
        "fp32_frac": steps_per_proj * FLOPS_PER_STEP_ALGO / mc_avg_s / 1e12 / fp32_probe_tflops,
        "cell_skips_per_projection": skips_per_proj,
        "denoise_ms": statistics.mean(dn_ms), "denoise_fused": bool(res["denoise_fused"]),
    }
    roofline = transport_roofline(steps_per_proj, mc_avg_s, hbm_peak, traffic, inst_per_step, n_sm, sm_max_mhz,
                                  context)

    cpu = None
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, n_s, dt = cpu_oracle_rate(prob, args.cpu_seconds, threads)
        rate1, n_1, dt1 = cpu_oracle_rate(prob, args.cpu_seconds / 2, 1, first=20000)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {n_s} histories of the 1e8-history projection, FP32 oracle, {dt:.1f} s on "
                         f"{threads} threads; single thread: first {n_1} histories, {dt1:.1f} s",
               "single_thread_value": rate1}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "s_per_projection": tot_ms / args.steps / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "histories_per_projection": n_hist, "angle_rad": angle,
                   "woodcock_steps_per_projection": steps_per_proj, "l2": "256 MB buffer written between timed steps",
                   "tracking": "global majorant (Woodcock, Section 2.4)" if not tuned.get("local_majorant")
                               else f"local majorants, cells of 2^{tuned['cell_shift']} voxels (option)",
                   "parallelism": f"one projection angle per GPU x{world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batched,
        "voxel_sweep": voxel_sweep,
        "variants": variants,
        "reconstruction": recon,
        "learned": learned,
        "autotuned": tuned,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
