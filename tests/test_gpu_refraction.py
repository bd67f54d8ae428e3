"""GPU run of the oblique refraction benchmark (Sec. 3.1: gold at 56 nm,
Z_b = 20, incidence pi/6) against the FP64 oracle: E_z every step (relative
L2 of the final fields <= 1e-3, and of the w0 amplitude over the run), the
refracted angle that the library's diagnostics measure, against the
oracle's measurement (0.02 deg) and the discrete Snell prediction (the
oracle pin's 0.3 deg)."""
import math

import numpy as np
import pytest

from paper_2208_08038_gb300 import diagnostics as Dg
from paper_2208_08038_gb300 import synth
from _common import field_rel_l2, gpu_from_workload, oracle_from_workload, rel_l2
import _refraction as F
import _resonance as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def test_refraction_matches_oracle_and_snell():
    wl = synth.refraction_2d()
    ora, _, _ = oracle_from_workload(wl)
    gpu, _, _ = gpu_from_workload(wl, deposit_mode=1)
    frames_o = []
    lock = Dg.LockIn(wl.dt)
    for s in range(wl.steps):
        ora.step(1)
        gpu.step(1)
        frames_o.append(ora.field(2)[0].copy())
        lock.add(gpu.read_field(2)[0])
        if s == 0:
            assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-5
    gpu.sync()
    assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-3
    A_o = F.lockin(frames_o, wl.dt)
    assert rel_l2(np.abs(lock.amplitude), np.abs(A_o)) < 1e-3
    lo, dx = wl.meta["surface"], wl.dx[0]
    x0, x1 = lo + 16, wl.n[0] - 8
    th_g = Dg.refraction_angle(lock.amplitude, dx, x0, x1)
    kx, ky = F.wavevector(A_o, dx, x0, x1)
    th_o = math.atan2(ky, kx)
    assert abs(math.degrees(th_g - th_o)) < 0.02, (math.degrees(th_g), math.degrees(th_o))
    sp = wl.species[0]
    n = wl.meta["n_ion"]
    eps = lambda w: R.eps_r(w, n, sp.Zb, sp.qc, sp.mc, wl.meta["omega_b"], n)
    disc = F.yee_refraction_angle(wl.meta["theta"], dx, wl.dt, lambda w: eps(w) - 1.0)
    assert abs(math.degrees(th_g - disc)) < 0.3
    ora.close()
    gpu.close()
