"""Pins of the resonance diagnostics (Sec. 3.1): the group velocity of the
x-ray pulse in gold and the phase shift of its reflection near the
bound-electron resonance w ~ w_c, scanned in a_c (here in the equivalent
natural frequency w_c, Sec. 3.1's w_c^2 = |q1 q2| / (4 pi eps0 m_r a_c^3)).

Closed forms first, each against an independent route:
  * the group velocity formula against 1 / (dk/dw) of the dispersion
    relation k = w sqrt(eps_r) (and the Drude limit, v_g = sqrt(eps_r));
  * the reflection phase on its atan2 branch against the argument of the
    Fresnel ratio (1 - beta) / (1 + beta), beta = i Gamma, in complex
    arithmetic, and its special values.
Then the oracle's own runs of the paper's case (Au at 12.4 nm, Z_b = 78, one
free electron per atom, 5.9e22 atoms/cm^3), measured from probe traces:
  * group velocity above (w_c = 3, 1.5) and below (w_c = 0.3) the
    reflecting band, against the discrete dispersion relation (Yee grid,
    leapfrog, quadratic shape factor): 0.1%, and 1.5% at w_c = 0.3, where
    v_g changes by 15% across the pulse's spectrum (the slab spreads the
    pulse, so the phase slope at w0 depends on the time window by ~0.7%);
    against the continuum formula of Sec. 3.1: 0.5% (2% at w_c = 0.3);
  * reflection phase inside the band (w_c = 0.7, 0.8, 0.9: eps_r < 0),
    against Sec. 3.1's formula with the leapfrog frequency (2/dt) sin(w dt/2)
    in eps_r, and against the continuum formula: 0.01 rad.
"""
import cmath
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth
from _common import oracle_from_workload
import _resonance as R


def ac_metres(omega_c, Zb=78.0, qc=1.0, mc=synth.M_AU, lambda0_m=12.4e-9):
    """a_c of a natural frequency w_c (units of omega0) through Sec. 3.1's
    w_c^2 = |q1 q2| kappa / (m_r a_c^3), kappa = r_e k0; returned in metres."""
    q2, m2 = -Zb, Zb
    q1, m1 = qc - q2, mc - m2
    mr = m1 * m2 / (m1 + m2)
    k0 = 2 * math.pi / lambda0_m
    ac = (abs(q1 * q2) * O.RE * k0 / (mr * omega_c ** 2)) ** (1.0 / 3.0)
    return ac / k0


def medium_eps(wl, omega_b):
    sp = wl.species[0]
    n = wl.meta["n_ion"]
    return lambda w: R.eps_r(w, n, sp.Zb, sp.qc, sp.mc, omega_b, n)


# ---------------------------------------------------------------------------
# closed forms

def test_group_velocity_formula_against_dispersion_relation():
    n = synth.N_AU_OVER_NC_12NM
    for wc in (3.0, 1.5, 0.3):
        eps = lambda w: R.eps_r(w, n, 78.0, 1.0, synth.M_AU, wc, n)
        k = lambda w: w * math.sqrt(eps(w))
        h = 1e-5
        vg_route = 2 * h / (k(1 + h) - k(1 - h))
        assert abs(R.group_velocity(1.0, eps) / vg_route - 1) < 1e-8, wc
    # Drude medium alone: v_g = c sqrt(1 - w_p^2 / w^2)
    drude = lambda w: 1.0 - 0.3 / (w * w)
    assert abs(R.group_velocity(1.0, drude) - math.sqrt(0.7)) < 1e-8


def test_reflection_phase_formula_branch_and_values():
    for G in (0.1, 0.5, 0.9, 1.0, 1.5, 4.0):
        ratio = (1 - 1j * G) / (1 + 1j * G)
        assert abs(R.reflection_phase(-G * G) - cmath.phase(ratio)) < 1e-12, G
    assert abs(R.reflection_phase(-1.0) + math.pi / 2) < 1e-12
    assert abs(R.reflection_phase(-1e-12)) < 1e-5
    assert abs(R.reflection_phase(-1e12) + math.pi) < 1e-5


def test_scan_brackets_the_resonance():
    """The scan's w_c values lie on both sides of w_c = w0 (a_c = 9.54e-11 m,
    the resonance radius of Sec. 3.1), and the reflecting band (eps_r < 0)
    is w_c in (0.600, 1)."""
    assert abs(ac_metres(1.0) / 9.54e-11 - 1) < 2e-3
    n = synth.N_AU_OVER_NC_12NM
    band = lambda wc: R.eps_r(1.0, n, 78.0, 1.0, synth.M_AU, wc, n) < 0
    assert [band(w) for w in (3.0, 1.5, 0.3)] == [False] * 3
    assert [band(w) for w in (0.7, 0.8, 0.9)] == [True] * 3
    assert band(0.61) and not band(0.59)


# ---------------------------------------------------------------------------
# the oracle's runs

def _trace(wl):
    s, _, pid = oracle_from_workload(wl)
    s.step(wl.steps)
    tr = s.probe(pid, 1)[:, 0]
    s.close()
    return tr


@pytest.fixture(scope="module")
def vacuum():
    """The vacuum reference trace of each geometry."""
    return {role: _trace(synth.resonance_1d(1.0, role=role, vacuum=True)) for role in ("transmit", "reflect")}


@pytest.mark.parametrize("wc,tol_disc,tol_cont", [(3.0, 1e-3, 5e-3), (1.5, 1e-3, 5e-3), (0.3, 1.5e-2, 2e-2)])
def test_group_velocity_scan(vacuum, wc, tol_disc, tol_cont):
    vac = vacuum["transmit"]
    wl = synth.resonance_1d(wc)
    tr = _trace(wl)
    lo, hi = wl.meta["slab"]
    dx = wl.dx[0]
    eps = medium_eps(wl, wc)
    meas = R.measured_group_velocity(tr, vac, wl.dt, (hi - lo) * dx, dx, 2.5 * wl.meta["fwhm"])
    disc = R.yee_group_velocity(1.0, dx, wl.dt, lambda w: eps(w) - 1.0)
    cont = R.group_velocity(1.0, eps)
    assert abs(meas / disc - 1) < tol_disc, (wc, ac_metres(wc), meas, disc, cont)
    assert abs(meas / cont - 1) < tol_cont, (wc, meas, disc, cont)


@pytest.mark.parametrize("wc", [0.7, 0.8, 0.9])
def test_reflection_phase_scan(vacuum, wc):
    vac = vacuum["reflect"]
    wl = synth.resonance_1d(wc, role="reflect")
    tr = _trace(wl)
    dx, dt = wl.dx[0], wl.dt
    dist = wl.meta["slab"][0] * dx - wl.meta["probe_x"]
    eps = medium_eps(wl, wc)
    meas = R.measured_reflection_phase(tr, vac, dt, dist, dx)
    W = 2.0 / dt * math.sin(dt / 2.0)
    assert abs(meas - R.reflection_phase(eps(W))) < 1e-2, (wc, ac_metres(wc), meas)
    assert abs(meas - R.reflection_phase(eps(1.0))) < 1e-2, (wc, meas)
