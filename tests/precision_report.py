"""FP32 error of the GPU path against the FP64 oracle, per configuration.

Run on a machine with a GB300 (python tests/precision_report.py); prints a
markdown table.  Each configuration runs on both sides from the same seeded
inputs:

  neutral_1d          full size and length (2048 cells, 16 ions/cell, 3000 steps)
  bragg_2d            full grid (2048^2 cells, 6,400 ions), 1 and 120 steps
  neutral_3d          the workload's dx, ppc, momenta and pulse on 64x32x32
                      cells (the oracle cannot run 264 M ions), 1 and 10
                      steps; plus sampled ions of the full-size medium pushed
                      one step in the GPU's own full-grid fields
  adjoint_2d          full grid and ions (1024^2 cells, 524,288 ions), 1 and 3
                      steps; gradients on the small problems of the adjoint pin
  ionized_crystal_2d  256x64 cells of the configuration (a0 = 0.3), 1 and 60
                      steps; plus sampled particles of the full size (25 M
                      free electrons) pushed one step

Field error: relative L2 over E and B; J separately; particle errors: the
largest position difference in cells and the relative L2 of the momenta.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_2208_08038_gb300 import synth  # noqa: E402
from _common import field_rel_l2, gpu_from_workload, oracle_from_workload, rel_l2  # noqa: E402


def fields_at(wl, checks):
    ora, osid, _ = oracle_from_workload(wl, probe_cap=1)
    gpu, gsid, _ = gpu_from_workload(wl, probe_cap=1)
    out, done = [], 0
    for s in checks:
        ora.step(s - done)
        gpu.step(s - done)
        gpu.sync()
        done = s
        g, o = gpu.fields(), ora.fields()
        out.append((s, field_rel_l2(g, o), rel_l2(g[6:9], o[6:9])))
    x1o, _, u1o, _ = ora.bodies(osid[0])
    x1g, _, u1g, _ = gpu.read_particles(gsid[0], len(x1o))
    L = np.array([wl.n[a] * wl.dx[a] if a < wl.D else 1.0 for a in range(3)])
    d = (x1g - x1o + 0.5 * L) % L - 0.5 * L
    dpos = float(np.abs(d[:, :wl.D]).max() / min(wl.dx[:wl.D]))
    du = rel_l2(u1g, u1o)
    gpu.close()
    ora.close()
    return out, dpos, du


def row(name, size, out, dpos=None, du=None, extra=""):
    cells = []
    for s, f, j in out:
        cells.append(f"step {s}: E,B {f:.2e}, J {j:.2e}")
    p = "" if dpos is None else f"{dpos:.1e} cells, u {du:.1e}"
    return f"| {name} | {size} | {'; '.join(cells)} | {p} | {extra} |"


def main():
    import torch
    assert torch.cuda.is_available()
    rows = []
    t0 = time.time()

    wl = synth.neutral_1d()
    ora, osid, opid = oracle_from_workload(wl)
    gpu, gsid, gpid = gpu_from_workload(wl)
    out, done = [], 0
    for s in (1, wl.steps):
        ora.step(s - done)
        gpu.step(s - done)
        gpu.sync()
        done = s
        g, o = gpu.fields(), ora.fields()
        out.append((s, field_rel_l2(g, o), rel_l2(g[6:9], o[6:9])))
    pr = rel_l2(gpu.read_probe(gpid), ora.probe(opid, 1))
    gpu.close()
    ora.close()
    rows.append(row("neutral_1d (config 0)", "full: 2048 cells, 16,384 ions, 3000 steps", out,
                    extra=f"probe trace {pr:.2e}"))

    wl = synth.bragg_2d()
    out, dpos, du = fields_at(wl, (1, 120))
    rows.append(row("bragg_2d (config 1)", "full grid: 2048^2 cells, 6,400 ions", out, dpos, du))

    wl = synth.neutral_3d(n=(64, 32, 32), margin=4, steps=10)
    wl.lasers[0].waist = 2 * synth.LAMBDA0
    wl.lasers[0].yc, wl.lasers[0].zc = 0.5 * 32 * wl.dx[1], 0.5 * 32 * wl.dx[2]
    wl.lasers[0].a0 = 0.02
    out, dpos, du = fields_at(wl, (1, 10))
    from test_gpu_fullsize import neutral_3d_context, sampled_step
    full = synth.neutral_3d(build_particles=False)
    ctx, sid, n_ion = neutral_3d_context(full)
    ctx.step(40)
    ctx.sync()
    rng = np.random.default_rng(5)
    ids = np.unique(rng.choice(n_ion, 3000, replace=False))
    (g, o, n), = sampled_step(full, ctx, [sid], [ids])
    ctx.close()
    L = np.array([full.n[a] * full.dx[a] for a in range(3)])
    d = (g[0] - o[0] + 0.5 * L) % L - 0.5 * L
    rows.append(row("neutral_3d (config 2)", "64x32x32 cells at the workload's dx, ppc, momenta", out, dpos, du,
                    extra=f"full size, {n} sampled ions, one step at step 40: position {np.abs(d).max() / full.dx[0]:.1e}"
                          f" cells, u1 {rel_l2(g[2], o[2]):.1e}, u2 {rel_l2(g[3], o[3]):.1e}"))

    wl = synth.adjoint_2d()
    out, dpos, du = fields_at(wl, (1, 3))
    from test_gpu_adjoint import gpu_problem, oracle_gradients
    ge = []
    for D in (1, 2):
        w2, steps, groups, target, probe_o, g_om, g_site = oracle_gradients(D)
        prob = gpu_problem(w2, steps, K=20)
        prob.run(w2.species[0].omega_b, np.zeros((groups, D)))
        go, gs = prob.gradients((2.0 * (probe_o - target)).astype(np.float32), groups)
        ge.append(f"{D}D: d/d omega_b {np.abs(go - g_om).max() / np.abs(g_om).max():.1e}, "
                  f"d/d site {np.abs(gs - g_site).max() / np.abs(g_site).max():.1e}")
        prob.ctx.close()
    rows.append(row("adjoint_2d (config 3)", "full: 1024^2 cells, 524,288 ions", out, dpos, du,
                    extra="gradients vs the oracle's adjoint (FD-pinned problems): " + "; ".join(ge)))

    wl = synth.ionized_crystal_2d(n=(256, 64), span=(2.0, 6.0), steps=60, a0=0.3)
    wl.lasers[0].fwhm = 2 * synth.T0
    wl.lasers[0].t0 = 1.5 * wl.lasers[0].fwhm
    out, dpos, du = fields_at(wl, (1, 60))
    full = synth.ionized_crystal_2d()
    gpu, gsid, _ = gpu_from_workload(full, probe_cap=1)
    gpu.step(30)
    gpu.sync()
    ids = [np.unique(rng.choice(len(sp.x), min(2000, len(sp.x)), replace=False)) for sp in full.species]
    res = sampled_step(full, gpu, gsid, ids)
    gpu.close()
    ge, go_, n = res[1]
    Lf = np.array([full.n[a] * full.dx[a] if a < full.D else 1.0 for a in range(3)])
    d = (ge[0][:, :2] - go_[0][:, :2] + 0.5 * Lf[:2]) % Lf[:2] - 0.5 * Lf[:2]
    rows.append(row("ionized_crystal_2d (config 4)", "256x64 cells of the configuration, a0 = 0.3", out, dpos, du,
                    extra=f"full size, {n} sampled free electrons, one step at step 30: position "
                          f"{np.abs(d).max() / full.dx[0]:.1e} cells, u {rel_l2(ge[2], go_[2]):.1e}"))

    print("| configuration | size compared | fields, relative L2 against FP64 | ions after the run "
          "(max position error, momentum rel. L2) | also |")
    print("|---|---|---|---|---|")
    for r in rows:
        print(r)
    print(f"\n({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
