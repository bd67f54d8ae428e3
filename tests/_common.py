"""Shared helpers of the tests: build the oracle and the CUDA path from the
same seeded workload description, and compare them."""
import numpy as np

import oracle as O
from paper_2208_08038_gb300 import synth


def oracle_from_workload(wl: synth.Workload, probe_cap=None):
    s = O.Sim(wl.D, wl.n, wl.dx, wl.dt, wl.bc)
    sids = []
    for sp in wl.species:
        if isinstance(sp, synth.TwoBody):
            sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
            s.load(sid, sp.x, sp.u, sp.pidx)
        else:
            sid = s.add_free(sp.q, sp.m, sp.w)
            s.load(sid, sp.x, sp.u)
        sids.append(sid)
    for L in wl.lasers:
        s.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    lo = [2.0 if (a < wl.D and wl.bc[a] == 1) else -1e300 for a in range(3)]
    hi = [wl.n[a] - 2.0 if (a < wl.D and wl.bc[a] == 1) else 1e300 for a in range(3)]
    s.set_free_bounds(lo, hi)
    pid = None
    if wl.probe_nodes is not None:
        pid = s.add_probe(wl.probe_comp, wl.probe_nodes, probe_cap or wl.steps)
    return s, sids, pid


def gpu_from_workload(wl: synth.Workload, deposit_mode=1, tile=None, probe_cap=None):
    from paper_2208_08038_gb300 import binding as B
    ctx = B.Context(wl.D, wl.n, wl.dx, wl.dt, wl.bc, deposit_mode=deposit_mode, tile=tile or wl.tile)
    sids = []
    for sp in wl.species:
        if isinstance(sp, synth.TwoBody):
            sid = ctx.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
            ctx.load_particles(sid, sp.x, sp.u, sp.pidx)
        else:
            sid = ctx.add_free(sp.q, sp.m, sp.w)
            ctx.load_particles(sid, sp.x, sp.u)
        sids.append(sid)
    for L in wl.lasers:
        ctx.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    pid = None
    if wl.probe_nodes is not None:
        pid = ctx.add_probe(wl.probe_comp, wl.probe_nodes, probe_cap or wl.steps)
    return ctx, sids, pid


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.sqrt((a * a).sum()))


def field_rel_l2(gpu_fields, ora_fields, comps=range(6)):
    """Relative L2 over the E and B components together."""
    g = np.concatenate([np.asarray(gpu_fields[c], dtype=np.float64).ravel() for c in comps])
    o = np.concatenate([np.asarray(ora_fields[c], dtype=np.float64).ravel() for c in comps])
    return rel_l2(g, o)
