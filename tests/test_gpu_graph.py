"""The step graph: a call of two or more steps replays one captured graph of
a step's launches (the laser time and the probe slots read from the device
step clock); single steps, and steps with the push timed, launch the kernels
directly.  In the sorted deposit mode both paths must give the same bits:
fields, probe traces (including a probe that fills up) and particles.
"""
import numpy as np
import pytest

from paper_2208_08038_gb300 import synth
from _common import gpu_from_workload

pytestmark = pytest.mark.gpu


def _state(ctx, sids, pid, n_probe):
    out = {"fields": ctx.fields()}
    if pid is not None:
        out["probe"] = ctx.read_probe(pid)
    for s, n in zip(sids, n_probe):
        out[f"parts{s}"] = np.concatenate(ctx.read_particles(s, n), axis=1)
    return out


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].shape == b[k].shape, k
        assert np.array_equal(a[k], b[k]), f"{k}: {np.abs(a[k] - b[k]).max()}"


def _hot_3d():
    """Fast thermal ions that cross tile margins: the conditional re-sort at
    the head of the step graph runs."""
    wl = synth.neutral_3d(seed=2, steps=30, n=(48, 16, 16), ppc=4, sigma_u=0.15, margin=2)
    wl.bc = (0, 0, 0)
    wl.lasers[0].waist = 0.5 * synth.LAMBDA0
    wl.lasers[0].yc, wl.lasers[0].zc = 0.5 * 16 * wl.dx[1], 0.5 * 16 * wl.dx[2]
    wl.lasers[0].a0 = 0.05
    return wl


def _workloads():
    w1 = synth.neutral_1d(steps=60)
    w2 = synth.refraction_2d(n=(64, 48), steps=40)
    return [("1d", w1, 60, 60), ("2d", w2, 40, 25), ("3d", _hot_3d(), 30, 30)]


@pytest.mark.parametrize("name,wl,steps,cap", _workloads(), ids=["1d", "2d", "3d-resorting"])
def test_graph_steps_match_direct_steps(name, wl, steps, cap):
    """step(n) (graph replays) against n x step(1) (direct launches), with
    the probe's capacity below the step count in 2D."""
    n_probe = [len(sp.x) for sp in wl.species]
    a, sa, pa = gpu_from_workload(wl, probe_cap=cap)
    b, sb, pb = gpu_from_workload(wl, probe_cap=cap)
    if pa is None:  # a line of E_z nodes across the box
        nodes = np.array([20 + wl.n[0] * j for j in range(wl.n[1])], dtype=np.int64)
        pa, pb = a.add_probe(2, nodes, cap), b.add_probe(2, nodes, cap)
    a.step(steps)
    for _ in range(steps):
        b.step(1)
    a.sync()
    b.sync()
    sa_, sb_ = _state(a, sa, pa, n_probe), _state(b, sb, pb, n_probe)
    assert sa_["probe"].shape[0] == min(steps, cap)
    _same(sa_, sb_)
    # both paths count the same kernels, re-sorts that ran included (the
    # single-step path has one more clock set per call)
    assert a.kernel_launches() + (steps - 1) == b.kernel_launches()
    a.close()
    b.close()


def test_graph_rebuilt_when_arguments_change():
    """A probe and a laser added between calls (the captured arguments
    change), and calls with the push timed (direct launches) between graph
    calls: the same bits as direct steps throughout."""
    wl = synth.refraction_2d(n=(64, 48), steps=40)
    n_probe = [len(sp.x) for sp in wl.species]
    a, sa, pa = gpu_from_workload(wl)
    b, sb, pb = gpu_from_workload(wl)
    nodes = np.arange(10, 10 + 64 * 48, 64, dtype=np.int64)[:40]
    L = wl.lasers[0]

    def schedule(ctx, direct):
        def run(n):
            if direct:
                for _ in range(n):
                    ctx.step(1)
            else:
                ctx.step(n)
        run(7)
        extra = ctx.add_probe(1, nodes, 30)
        run(6)
        ctx.add_laser(L.comp, 0.5 * L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0 + 3.0, L.ramp, L.phase,
                      L.ia + 2, L.yc, L.zc)
        ctx.time_push(True)
        run(3)
        ctx.time_push(False)
        run(9)
        ctx.sync()
        return extra

    ea = schedule(a, direct=False)
    eb = schedule(b, direct=True)
    st_a, st_b = _state(a, sa, pa, n_probe), _state(b, sb, pb, n_probe)
    _same(st_a, st_b)
    assert np.array_equal(a.read_probe(ea), b.read_probe(eb))
    assert a.read_probe(ea).shape[0] == 18
    a.close()
    b.close()
