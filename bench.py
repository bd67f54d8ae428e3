"""Benchmark of the two-body macro-ion PIC step on GB300.

Workload (default): the 3D neutral medium -- 512 x 256 x 256 cells,
dx = lambda/16, 8 two-body ions per cell over x cells [4, 508) (y, z
periodic, x open), thermal momenta sigma = 1e-3, omega_b = 3, n_b = 0.02 n_c,
a0 = 1e-3 Gaussian pulse with waist 6 lambda: 264,241,152 ions.  A step is the
whole hot path: re-sort check, B half step, gather + internal force + Boris
+ drift + Esirkepov deposit (sorted mode: into the 64-bit fixed-point
current), the antenna sheet, B half step, E step (J formed from the
fixed-point current) with Mur faces.  Also reported: the end-to-end rate
through the C ABI from pinned host arrays, the 2D Bragg crystal, the 1D
medium and the adjoint's cost on the 2D adjoint workload.

Metric: two-body ion pushes per second (ions x steps / time), whole job.
One JSON line on rank 0.  Multi-GPU: independent replicas (the step is not
sharded across GPUs), weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "two-body ion pushes/s (gather+push+deposit+Yee) FP32 vs FP64; adjoint/fwd ratio"
# Algorithmic bytes of the push per unit (3D two-body ion, FP32 state: cell,
# 3 offsets, r, u1, u2 = 52 B): a fully pushed ion reads and writes its whole
# state; a quiet ion (moved by the quiet-tile pass: a co-moving neutral pair
# ahead of the field, which carries no current) reads it and writes its cell
# and offsets; per cell, E and B are read once and J written once.
BYTES_FULL_ION = 104
BYTES_QUIET_ION = 68
BYTES_CELL = 36
# FP32 operations of one fully pushed 3D two-body ion (gather of six
# components at both bodies, internal field, two Boris rotations, drift,
# three-node Esirkepov deposit of both bodies in fixed point), counted by
# ncu's executed-instruction classes on the small 3D case with a field in
# every tile: FFMA2 x 4 + FMUL2 x 2 + FADD2 x 2 + FFMA x 2 + FMUL + FADD.
FLOPS_FULL_ION = 2371
# DRAM bytes (read + write) per ion, from ncu on the small 3D case
# (128x64x64 cells, 3,932,160 ions; one launch each): k_push with a field in
# every tile (the field and current bytes included, so per ion at this
# workload's 8 ions per cell) and k_push_quiet ahead of the field.
TRAFFIC_FULL_ION = 108.1
TRAFFIC_QUIET_ION = 54.7
# the late window starts here: the field has crossed most of the medium
LATE_START = 450
UNIT = "ion-pushes/s"


def whole_job(ms_local, units_local, dist=None, device="cpu"):
    """The job's figures over the ranks: the longest timed span in ms (every
    rank's timed region is bracketed by barriers) and the total units
    processed (each replica runs its own copy of the workload)."""
    if dist is None:
        return float(ms_local), float(units_local)
    import torch
    m = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(m.item()), float(u.item())


def workload_neutral_3d(size="full"):
    from paper_2208_08038_gb300 import synth
    n = (512, 256, 256) if size == "full" else (128, 64, 64)
    wl = synth.neutral_3d(n=n, build_particles=False)
    m = wl.meta
    n_ion = m["ppc"] * (m["hi"][0] - m["lo"][0]) * (m["hi"][1] - m["lo"][1]) * (m["hi"][2] - m["lo"][2])
    return wl, n_ion


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
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
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi's CSV lines (ClockSampler.FIELDS, no header, no units)."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(nm)
    sm.sort()
    med = sm[len(sm) // 2] if sm else None
    return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_neutral_3d(seconds_target: float = 10.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: a
    32^3-cell periodic box with the workload's dx, dt, ppc, momenta and
    omega_b (262,144 ions), timed over whole steps."""
    import oracle as O
    from paper_2208_08038_gb300 import synth
    n = (32, 32, 32)
    wl = synth.neutral_3d(n=n, margin=0)
    wl.bc = (0, 0, 0)
    sp = wl.species[0]
    s = O.Sim(3, n, wl.dx, wl.dt, wl.bc)
    sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    s.load(sid, sp.x, sp.u)
    t0 = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t0
    k = max(1, min(20, int(seconds_target / max(one, 1e-3))))
    t0 = time.perf_counter()
    s.step(k)
    el = time.perf_counter() - t0
    s.close()
    threads = 1  # the particle loop is serial; field loops use OpenMP only above 65,536 cells
    return {"value": len(sp.x) * k / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"32^3-cell periodic box of the 3D workload ({len(sp.x)} ions, 8/cell), {k} steps, FP64"}


def run_e2e(wl, n_ion, mode, steps, rank, world, dist=None):
    import numpy as np
    import torch
    from paper_2208_08038_gb300 import binding as B
    from paper_2208_08038_gb300 import synth
    m = wl.meta
    x, u = synth.medium(m["seed"] + rank, 3, wl.dx, m["lo"], m["hi"], m["ppc"], m["sigma_u"])
    xh = torch.from_numpy(x).pin_memory()
    uh = torch.from_numpy(u).pin_memory()
    del x, u
    nx, ny, nz = wl.n
    out = torch.empty(nx * ny * nz, dtype=torch.float32, pin_memory=True)
    sp = wl.species[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=mode, tile=wl.tile)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    rc = B.lib().bp_load_particles(ctx._h, sid, B._ptr(xh.data_ptr()), B._ptr(uh.data_ptr()), None, n_ion)
    ctx._check(rc, "bp_load_particles")
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    for _ in range(steps):
        ctx.step(1)
        # the step's E_y to pinned host memory: a device snapshot, then the copy
        # on a side stream while the next steps run (valid after sync)
        ctx._check(B.lib().bp_read_field_async(ctx._h, B.EY, B._ptr(out.data_ptr())), "bp_read_field_async")
    ctx.sync()
    el = time.perf_counter() - t0
    ctx.close()
    if dist:
        dist.barrier()
    ms, units = whole_job(el * 1e3, n_ion * steps, dist, "cuda")
    h2d = n_ion * (3 + 3) * 8
    return {"value": units / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": nx * ny * nz * 4, "steps": steps,
            "note": "initial ion state uploaded once from pinned host memory, amortised over the steps; "
                    "E_y read back to pinned host memory every step (bp_read_field_async: device snapshot, "
                    "copy overlapping the next steps); context creation included"}


BRAGG_BYTES_CELL = 168  # per cell and step: 2 B half steps (36 B), E step (72 B), clearing the current (24 B)


def updated_cells(act_tiles, act_steps, ncell, ntiles, steps):
    """Cells the field kernels updated over `steps` steps: the device's count
    of active tiles (summed over the steps it flagged) times the cells of a
    tile, or every cell every step on a grid that keeps no flags (fewer than
    1,024 tiles: act_steps = 0)."""
    return act_tiles * (ncell // ntiles) if act_steps else ncell * steps


def run_bragg(steps, warmup):
    """The 2D Bragg crystal (2048^2 cells, dx = lambda/32, 40 x 40 sites of
    4 two-body ions, 30-degree p-polarised beam): grid cells advanced per
    second, the cells the field kernels updated per second (they skip tiles
    the beam has not reached, whose fields stay exactly zero), and the HBM
    fraction of the field kernels' algorithmic bytes over the updated cells
    (E, B, J and the fixed-point current, 251 MB, exceed L2)."""
    import torch
    from paper_2208_08038_gb300 import binding as B
    from paper_2208_08038_gb300 import synth
    wl = synth.bragg_2d()
    sp = wl.species[0]
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=B.BP_DEPOSIT_SORTED, tile=wl.tile)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    ctx.load_particles(sid, sp.x, sp.u)
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    ctx.step(warmup)
    ctx.sync()
    stream = torch.cuda.current_stream()
    # the steps as a user runs them (graph replays), then as many with the
    # push timed (launched directly) for the push's own time; the field
    # kernels' work counted over the first window (they skip the tiles the
    # beam has not reached)
    ctx.field_work()
    ms, _, _, _, _, launches = timed_window(ctx, steps, stream, time_push=False)
    act_tiles, act_steps = ctx.field_work()
    ms_direct, push_ms, push_n, _, _, _ = timed_window(ctx, steps, stream)
    ctx.close()
    ncell = wl.n[0] * wl.n[1]
    ntiles = ncell // (wl.tile[0] * wl.tile[1])
    cells = updated_cells(act_tiles, act_steps, ncell, ntiles, steps)
    hbm, src = peaks()
    gbs = BRAGG_BYTES_CELL * cells / (ms * 1e-3) / 1e9
    return {"workload": "bragg_2d: 2048x2048 cells, dx=lambda/32, 6400 two-body ions on a 40x40 lattice, "
                        "p-polarised beam at 30 degrees, sorted deposit",
            "steps": f"{warmup}..{warmup + steps}", "ms_per_step": ms / steps,
            "grid_cells_per_s": ncell * steps / (ms * 1e-3), "cell_updates_per_s": cells / (ms * 1e-3),
            "ion_pushes_per_s": len(sp.x) * steps / (ms * 1e-3),
            "push_ms_per_launch": push_ms / max(push_n, 1), "gpu_launches": launches,
            "ms_per_step_launched_directly": ms_direct / steps,
            "field_tiles_updated_fraction": cells / (ncell * steps),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes_per_cell": BRAGG_BYTES_CELL, "peak_source": src,
                         "scope": "whole step: the field kernels' algorithmic bytes over the cells of the "
                                  "tiles they updated (the others, never reached by the beam, stay zero "
                                  "and are skipped)"}}


def run_neutral_1d(steps, warmup):
    """The 1D neutral medium (2048 cells, dx = lambda/64, 16,384 two-body ions
    in the 16-lambda slab, 10-cycle pulse): a few microseconds of work per
    kernel, so the step is bound by kernel launches; reported as time per
    step and launches per step."""
    import torch
    from paper_2208_08038_gb300 import binding as B
    from paper_2208_08038_gb300 import synth
    wl = synth.neutral_1d()
    sp = wl.species[0]
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=B.BP_DEPOSIT_SORTED, tile=wl.tile)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    ctx.load_particles(sid, sp.x, sp.u)
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    ctx.step(warmup)
    ctx.sync()
    stream = torch.cuda.current_stream()
    ms, _, _, _, _, launches = timed_window(ctx, steps, stream, time_push=False)
    ms_direct, push_ms, push_n, _, _, _ = timed_window(ctx, steps, stream)
    ctx.close()
    return {"workload": "neutral_1d: 2048 cells, dx=lambda/64, 16384 two-body ions, sorted deposit",
            "steps": f"{warmup}..{warmup + steps}", "ms_per_step": ms / steps,
            "ion_pushes_per_s": len(sp.x) * steps / (ms * 1e-3), "push_ms_per_launch": push_ms / max(push_n, 1),
            "gpu_launches_per_step": launches / steps, "ms_per_step_launched_directly": ms_direct / steps,
            "bound": "kernel launches (a few microseconds of work per kernel): each step is one graph "
                     "launch (the conditional re-sort, then the step's kernels)"}


def run_adjoint_ratio(steps=400, K=20, reps=3):
    """Adjoint cost on the 2D adjoint workload (1024^2 cells, dx = lambda/32,
    524,288 ions in the bound slab on 4096 sites, per-column omega_b, 400
    steps, checkpoints every 20): (checkpointed forward + backward) / plain
    forward, each timed with CUDA events on the context stream."""
    import numpy as np
    import torch
    from paper_2208_08038_gb300 import binding as B
    from paper_2208_08038_gb300 import synth
    from paper_2208_08038_gb300.adjoint import SiteProblem
    wl = synth.adjoint_2d(steps=steps)
    sp = wl.species[0]
    m = wl.meta
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=B.BP_DEPOSIT_SORTED)
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    pid = ctx.add_probe(wl.probe_comp, wl.probe_nodes, steps)
    prob = SiteProblem(ctx, sid, pid, m["site_of_ion"], m["off"], m["column"], steps, K)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sites = m["sites"]
    x0 = sites[m["site_of_ion"]] + m["off"]

    def plain():
        ctx.reset()
        ctx.load_particles(sid, x0, None, m["column"])
        ctx.step(steps)
        ctx.sync()

    plain()  # warm-up
    probe = prob.run(sp.omega_b, sites)  # warm-up of the checkpointed path
    dl = (2.0 * probe).astype(np.float32)
    prob.gradients(dl, len(sp.omega_b))
    # each phase `reps` times, interleaved; the medians (a single repetition
    # is exposed to host-side delays in the set-up calls)
    tp, tf, tb = [], [], []
    for _ in range(reps):
        tp.append(timed(plain))
        tf.append(timed(lambda: prob.run(sp.omega_b, sites)))
        tb.append(timed(lambda: prob.gradients(dl, len(sp.omega_b))))
    t_plain, t_fwd, t_bwd = (sorted(v)[len(v) // 2] for v in (tp, tf, tb))
    ctx.close()
    return {"workload": "adjoint_2d: 1024x1024 cells, dx=lambda/32, 524288 ions on 4096 sites, "
                        "1024 per-column omega_b, 400 steps, checkpoint every 20",
            "plain_forward_ms": t_plain, "ckpt_forward_ms": t_fwd, "backward_ms": t_bwd,
            "repetitions_ms": {"plain": tp, "ckpt_forward": tf, "backward": tb},
            "ratio": (t_fwd + t_bwd) / t_plain,
            "backward_over_forward": t_bwd / t_plain,
            "definitions": "ratio = (checkpointed forward + backward) / plain forward; backward_over_forward = "
                           "backward (segment recompute + reverse steps) / plain forward"}


def our_config(n_ion, mode, world, warmup, steps, n=(512, 256, 256)):
    return {"workload": f"neutral_3d: {n[0]}x{n[1]}x{n[2]} cells, dx=lambda/16, 8 two-body ions/cell "
                        f"({n_ion} ions), thermal sigma=1e-3, omega_b=3, a0=1e-3 pulse, {mode} deposit",
            "timed": f"steps {warmup}..{warmup + steps} of the 500-step run from t=0: the quiet start (the "
                     "field has reached only the tiles near the antenna; the co-moving neutral ions ahead of "
                     "it are drifted by the quiet-tile pass without gather or deposit); the field-covered "
                     f"regime is timed separately from step {LATE_START} (key 'late')",
            "l2": f"inputs larger than L2 (particles {n_ion * 52 / 1e9:.3g} GB)", "parallelism": f"replicas x{world}"}


def fp32_peak_tflops(sm_mhz, sms=None):
    """FP32 non-tensor peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms


def push_roofline(full, quiet, launches, push_ms, ncell, hbm, hbm_src, sm_max, sms=None):
    """Roofline of the push launch (k_push_quiet + k_push + k_records) over a
    timed window: `full` and `quiet` are the device-counted full pushes and
    quiet drifts of the window's `launches` push launches, `push_ms` their
    summed CUDA-event time.  FP32 operations (the binding roof) from the full
    pushes only; algorithmic bytes from both kinds of work plus the per-cell
    field and current bytes; traffic from ncu's DRAM bytes per ion of each
    kernel (small 3D case)."""
    per = max(launches, 1)
    avg_ms = push_ms / per
    alg = (full * BYTES_FULL_ION + quiet * BYTES_QUIET_ION) / per + ncell * BYTES_CELL
    flops = full * FLOPS_FULL_ION / per
    achieved_gbs = alg / (avg_ms * 1e-3) / 1e9
    achieved_tf = flops / (avg_ms * 1e-3) / 1e12
    fp32_peak, sms = fp32_peak_tflops(sm_max, sms)
    traffic = None
    if TRAFFIC_FULL_ION is not None and TRAFFIC_QUIET_ION is not None:
        traffic = (full * TRAFFIC_FULL_ION + quiet * TRAFFIC_QUIET_ION) / per
    return {"bound": "alu", "achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved_tf / fp32_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "window": "late", "kernel": "push launch: k_push_quiet<3> + k_push<3,sorted> + k_records<3>",
            "peak_source": f"FP32 lanes: {sms} SMs x 128 x 2 flops x {sm_max:.0f} MHz (max SM clock)",
            "flops_per_full_push": FLOPS_FULL_ION,
            "limiter": "instruction issue (ncu on the small 3D case with a field in every tile)",
            "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                    "bytes_per_launch": alg, "peak_source": hbm_src}}


def timed_window(ctx, steps, stream, time_push=True):
    """CUDA-event time of `steps` steps, with the push launches timed and
    their work counted on the device (time_push); without push timing the
    steps replay the library's graph of a step."""
    import torch
    ctx.time_push(time_push)
    launches0 = ctx.kernel_launches()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(steps)
    e1.record(stream)
    ctx.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    push_ms, push_n = ctx.push_time()
    full, quiet = ctx.push_work()
    launches = ctx.kernel_launches() - launches0
    ctx.time_push(False)
    return ms, push_ms, push_n, full, quiet, launches


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: W untimed and K timed
    steps of a bounded sample of the 3D workload (a 16^3-cell periodic box
    with the workload's dx, dt, 8 ions per cell, thermal momenta, omega_b),
    on rank 0 only."""
    if rank != 0:
        return
    import oracle as O
    from paper_2208_08038_gb300 import synth
    # box side sized so that the K timed steps take about a minute at the
    # oracle's ~1.7e5 ion-pushes/s
    side = int(max(8, min(16, round((60.0 * 1.7e5 / max(args.steps, 1) / 8) ** (1.0 / 3.0)))))
    n = (side, side, side)
    wl = synth.neutral_3d(n=n, margin=0)
    wl.bc = (0, 0, 0)
    sp = wl.species[0]
    s = O.Sim(3, n, wl.dx, wl.dt, wl.bc)
    sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    s.load(sid, sp.x, sp.u)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    el = time.perf_counter() - t0
    s.close()
    value = len(sp.x) * args.steps / el
    wl_full, n_ion = workload_neutral_3d()
    sample = f"{side}^3-cell periodic box of the 3D workload ({len(sp.x)} ions, 8/cell), FP64, {args.steps} timed steps"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(our_config(n_ion, "oracle", world, args.warmup, args.steps), sample=sample,
                                                          timed=f"{args.steps} steps of the sample after "
                                                                f"{args.warmup} untimed ones (every ion "
                                                                "takes the oracle's full step)"),
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed steps from t = 0 (after the warm-up)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="sorted", choices=["sorted", "atomic"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="end-to-end steps (default: --steps)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-bragg", action="store_true", help="skip the 2D Bragg crystal and 1D medium legs")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="STEPS",
                    help="only the adjoint/forward ratio of the 2D adjoint workload over STEPS steps")
    ap.add_argument("--late-start", type=int, default=LATE_START,
                    help="step at which the late (field-covered) window starts")
    ap.add_argument("--adjoint-reps", type=int, default=3, help="timed repetitions of each adjoint phase")
    ap.add_argument("--small-legs-only", action="store_true",
                    help="only the 2D Bragg crystal and 1D medium legs (one JSON line with their keys)")
    ap.add_argument("--size", default="full", choices=["full", "small"],
                    help="small: the 3D workload on 128x64x64 cells (profiling)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.small_legs_only:
        import torch
        torch.cuda.set_device(local)
        if rank == 0:
            print(json.dumps({"bragg_2d": run_bragg(max(args.steps, 100), max(args.warmup, 3)),
                              "neutral_1d": run_neutral_1d(1000, 5)}), flush=True)
        return

    if args.adjoint_only:
        import torch
        torch.cuda.set_device(local)
        if rank == 0:
            print(json.dumps({"adjoint": run_adjoint_ratio(steps=args.adjoint_only, reps=args.adjoint_reps)}),
                  flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_

    from paper_2208_08038_gb300 import binding as B
    from paper_2208_08038_gb300 import build_lib
    if not os.path.exists(B.LIB_PATH):
        build_lib.build()

    wl, n_ion = workload_neutral_3d(args.size)
    mode = B.BP_DEPOSIT_SORTED if args.mode == "sorted" else B.BP_DEPOSIT_ATOMIC
    stream = torch.cuda.current_stream()
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=mode, tile=wl.tile)
    sp = wl.species[0]
    m = wl.meta
    sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    ctx.set_medium(sid, m["lo"], m["hi"], m["ppc"], m["seed"] + rank, m["sigma_u"])
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    ctx.step(args.warmup)
    ctx.sync()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    # the driver's window: K steps right after the warm-up, from t = 0
    ms, push_ms, push_n, full0, quiet0, launches = timed_window(ctx, args.steps, stream)
    if dist:
        dist.barrier()
    ms, units = whole_job(ms, n_ion * args.steps, dist, "cuda")
    # the field-covered regime: advance (untimed) to LATE_START, then time a
    # second window there; the roofline describes this window
    done = args.warmup + args.steps
    if done < args.late_start:
        ctx.step(args.late_start - done)
        ctx.sync()
        done = args.late_start
    late_steps = max(args.steps, 20)
    lms, lpush_ms, lpush_n, lfull, lquiet, llaunch = timed_window(ctx, late_steps, stream)
    clocks = sampler.stop()
    lms_job, lunits = whole_job(lms, n_ion * late_steps, dist, "cuda")
    ctx.close()
    # end to end through the C ABI with host buffers: a fresh context loads
    # the ions' FP64 positions and momenta from pinned host memory
    # (bp_load_particles: copy, device-side conversion, sort), runs the steps
    # and reads every step's E_y field back to pinned host memory
    e2e = None
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps
    if e2e_steps > 0:
        e2e = run_e2e(wl, n_ion, mode, e2e_steps, rank, world, dist)
    hbm, src = peaks()
    ncell = wl.n[0] * wl.n[1] * wl.n[2]
    # per push launch of the late window: algorithmic bytes from the work the
    # device counted (full pushes and quiet drifts), FP32 operations of the
    # full pushes
    per = max(lpush_n, 1)
    lpush_avg = lpush_ms / per
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    roofline = push_roofline(lfull, lquiet, lpush_n, lpush_ms, ncell, hbm, src, sm_max)
    push_avg0 = push_ms / max(push_n, 1)
    value = units / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": our_config(n_ion, args.mode, world, args.warmup, args.steps, wl.n),
        "push_ms_per_launch": push_avg0,
        "push_work_per_launch": {"full": full0 / max(push_n, 1), "quiet": quiet0 / max(push_n, 1)},
        "late": {"steps": f"{done}..{done + late_steps}", "ms_per_step": lms_job / late_steps,
                 "value": lunits / (lms_job * 1e-3), "unit": UNIT, "push_ms_per_launch": lpush_avg,
                 "full_pushes_per_launch": lfull / per, "quiet_per_launch": lquiet / per,
                 "full_fraction": lfull / max(lfull + lquiet, 1), "gpu_launches": llaunch},
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_neutral_3d()
    if rank == 0 and not args.no_adjoint:
        line["adjoint"] = run_adjoint_ratio()
    if rank == 0 and not args.no_bragg:
        line["bragg_2d"] = run_bragg(max(args.steps, 100), max(args.warmup, 3))
        line["neutral_1d"] = run_neutral_1d(1000, max(args.warmup, 3))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
