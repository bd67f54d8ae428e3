"""Pins of the oracle in the relativistic regime of the x-ray wakefield
application (Sec. 3.2: a0 = 3).

An electron that starts at rest in a vacuum plane wave E_y(t - x) keeps, in
the continuum, u_y = a (the transverse canonical momentum) and
gamma - u_x = 1 (the light-front invariant), so it reaches u_x = a0^2 / 2.
On the Yee grid with the leapfrog the invariant holds to second order in the
grid spacing (the wave's phase velocity falls below c by (k dx)^2/24):
  * at lambda/32: |gamma - u_x - 1| <= 1.5% of 1 + max u_x, max u_x within
    3% of a0^2/2 = 4.5, max |u_y| within 5% of a0;
  * at lambda/64 the largest deviation from the invariant is at least 3
    times smaller (second-order convergence; measured 3.9x).
A sign or factor error in the magnetic rotation, the relativistic gamma or
the drift breaks these by O(1).

A two-body ion of the wakefield's gold (Z_b = 49, q_c = +30) in the same
wave: the modified Coulomb field holds the bound electron with at most
q1 kappa / (1.5^{3/2} sqrt(2) a_c^2) ~ 0.43 (its maximum, at r = a_c / sqrt 2),
far below a0 = 3, so the wave tears the bound electron out (r >> a_c: the
Coulomb tail of V_M, not its harmonic core).  Released at a finite phase, it
keeps a drift (it does not end at u_x = a0^2/2), but once free it has an
electron's q/m in the wave alone, and the light-front invariant holds to 2%.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth


def plane_wave_run(cpl, species="free", a0=3.0):
    dx = synth.LAMBDA0 / cpl
    n = 64 * cpl
    s = O.Sim(1, (n,), (dx,), 0.95 * dx, (1,))
    x0 = np.array([[6 * synth.LAMBDA0]])
    if species == "free":
        sid = s.add_free(-1.0, 1.0, 1e-12)
        s.load(sid, x0, np.zeros((1, 3)))
    else:
        sid = s.add_two_body(49.0, 30.0, synth.M_AU, 1e-12, 0.26e-9, [4.0])
        s.load(sid, x0, np.zeros((1, 3)))
    fwhm = 4 * synth.T0
    s.add_laser(1, a0, 1.0, 0.0, 0.0, fwhm, 1.5 * fwhm, 0.0, 0.0, 8, 0.0, 0.0)
    s.set_free_bounds([2.0, -1e300, -1e300], [n - 2.0, 1e300, 1e300])
    worst, uy_max, ux_max, r_max = 0.0, 0.0, 0.0, 0.0
    for _ in range(int(round(40 * synth.T0 / (0.95 * dx)))):
        s.step(1)
        x1, x2, u1, u2 = s.bodies(sid)
        u = u1[0] if species == "free" else u2[0]
        g = math.sqrt(1 + u @ u)
        worst = max(worst, abs(g - u[0] - 1))
        uy_max = max(uy_max, abs(u[1]))
        ux_max = max(ux_max, u[0])
        if species != "free":
            r_max = max(r_max, float(np.linalg.norm(x1[0] - x2[0])))
    ac = s.ac(sid, 0) if species != "free" else 0.0
    s.close()
    return worst, uy_max, ux_max, r_max, ac


def test_free_electron_plane_wave_invariant():
    w32, uy, ux, _, _ = plane_wave_run(32)
    assert w32 <= 0.015 * (1 + ux), (w32, ux)
    assert abs(ux / 4.5 - 1) < 0.03, ux
    assert abs(uy / 3.0 - 1) < 0.05, uy
    w64, *_ = plane_wave_run(64)
    assert w32 / w64 >= 3.0, (w32, w64)


def test_bound_electron_leaves_the_harmonic_core():
    w, uy, ux, r_max, ac = plane_wave_run(32, species="two_body")
    kappa = O.RE * 2 * math.pi / 0.26e-9
    e_max = 79 * kappa / (1.5 ** 1.5 * math.sqrt(2) * ac * ac)
    assert e_max < 0.2 * 3.0, e_max
    assert r_max > 100 * ac, (r_max, ac)
    assert w <= 0.02 * (1 + ux), (w, ux)
    assert ux > 4.0, ux
