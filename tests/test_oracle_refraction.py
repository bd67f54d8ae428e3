"""Pin of the oblique refraction run (Sec. 3.1: gold at 56 nm with Z_b = 20,
a beam incident at pi/6; the code must give the refraction angle the
model's permittivity predicts).

  * Snell's law with sqrt(eps_r) against the discrete dispersion solver in
    the limit of a fine grid, and the vacuum case (no refraction);
  * the oracle's refracted wave vector, from the phase gradient of the
    w0 component of E_z inside the medium: within 0.3 deg of the discrete
    prediction (2D Yee grid, leapfrog frequency, shape factor) and 0.6 deg
    of the continuum Snell angle (the grid's own anisotropy at lambda/16
    moves the angle by 0.26 deg);
  * the paper's own reading, the 2D Fourier transform of the field in the
    medium: its peak lies within one FFT bin of Snell's wave vector.
"""
import math

import numpy as np
import pytest

from paper_2208_08038_gb300 import synth
from _common import oracle_from_workload
import _refraction as F
import _resonance as R


def medium_eps(wl):
    sp = wl.species[0]
    n = wl.meta["n_ion"]
    return lambda w: R.eps_r(w, n, sp.Zb, sp.qc, sp.mc, wl.meta["omega_b"], n)


def test_snell_against_discrete_solver_and_vacuum():
    th = math.pi / 6
    chi = lambda w: 0.94 - 0.1 / (w * w)
    fine = F.yee_refraction_angle(th, 1e-4, 0.5e-4, chi)
    assert abs(fine - F.snell_angle(th, 1.0 + chi(1.0))) < 1e-6
    assert abs(F.yee_refraction_angle(th, 0.05, 0.03, lambda w: 0.0) - th) < 2e-3
    assert abs(F.snell_angle(th, 1.0) - th) < 1e-12


@pytest.fixture(scope="module")
def run():
    wl = synth.refraction_2d()
    s, _, _ = oracle_from_workload(wl)
    frames = []
    for _ in range(wl.steps):
        s.step(1)
        frames.append(s.field(2)[0].copy())
    s.close()
    return wl, frames


def test_refraction_angle(run):
    wl, frames = run
    A = F.lockin(frames, wl.dt)
    lo, dx = wl.meta["surface"], wl.dx[0]
    kx, ky = F.wavevector(A, dx, lo + 16, wl.n[0] - 8)
    meas = math.atan2(ky, kx)
    eps = medium_eps(wl)
    disc = F.yee_refraction_angle(wl.meta["theta"], dx, wl.dt, lambda w: eps(w) - 1.0)
    cont = F.snell_angle(wl.meta["theta"], eps(1.0))
    assert eps(1.0) > 1.5  # the model's permittivity above one (Sec. 3.1): refraction towards the normal
    assert abs(math.degrees(meas - disc)) < 0.3, (math.degrees(meas), math.degrees(disc))
    assert abs(math.degrees(meas - cont)) < 0.6, (math.degrees(meas), math.degrees(cont))
    assert abs(ky - math.sin(wl.meta["theta"])) < 5e-3  # the incident k_y, conserved


def test_fourier_peak_within_one_bin_of_snell(run):
    wl, frames = run
    lo, dx = wl.meta["surface"], wl.dx[0]
    x0, x1 = lo + 8, wl.n[0]
    E = frames[-1][:, x0:x1]
    Fk = np.abs(np.fft.fft2(E))
    ny, nx = E.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, dx)
    Fk[:, kx <= 0] = 0.0  # the wave moves towards +x
    j, i = np.unravel_index(np.argmax(Fk), Fk.shape)
    th = wl.meta["theta"]
    n = math.sqrt(medium_eps(wl)(1.0))
    t = F.snell_angle(th, n * n)
    want = (n * math.cos(t), n * math.sin(t))
    # sign of k_y: fft2 over exp(-i k.r); the wave's phase grows along +y
    assert abs(abs(kx[i]) - want[0]) <= 2 * np.pi / (nx * dx) + 1e-9, (kx[i], want)
    assert abs(abs(ky[j]) - want[1]) <= 2 * np.pi / (ny * dx) + 1e-9, (ky[j], want)
