"""Diagnostics of the benchmarks of Sec. 3.1 from recorded fields: the group
velocity of a pulse through a slab and the phase shift of its reflection
from a slab (near the bound-electron resonance), and the wave vector of a
beam refracted at oblique incidence.

These functions post-process what bp_read_probe and bp_read_field return
(host arrays): they are analysis, not part of the step, and call nothing on
the device.  The slab diagnostics compare a run with the medium against a
run of the same geometry without it (the incident pulse), so the laser's own
shape and the probe's time origin drop out.

Time of sample s of a probe: (s + 1) dt (the probe records after each step).
Spectra use the exp(-i w t) convention: the amplitude of a component
A exp(-i w t) is the sum over samples of E(t) exp(+i w t), so a delay t_d
multiplies it by exp(+i w t_d).
"""
from __future__ import annotations

import math

import numpy as np


def yee_wavenumber(omega: float, dx: float, dt: float) -> float:
    """Vacuum wavenumber of frequency omega on the 1D Yee grid with the
    leapfrog step: sin(k dx / 2) / dx = sin(omega dt / 2) / dt."""
    return 2.0 / dx * math.asin(dx / dt * math.sin(0.5 * omega * dt))


def yee_group_velocity(omega: float, dx: float, dt: float) -> float:
    """d omega / dk of that relation: cos(k dx / 2) / cos(omega dt / 2)."""
    k = yee_wavenumber(omega, dx, dt)
    return math.cos(0.5 * k * dx) / math.cos(0.5 * omega * dt)


def _amplitude(samples: np.ndarray, dt: float, omega: float) -> complex:
    t = dt * np.arange(1, len(samples) + 1, dtype=np.float64)
    return complex(np.dot(np.asarray(samples, dtype=np.float64), np.exp(1j * omega * t)))


def _window(samples: np.ndarray, dt: float, half: float) -> np.ndarray:
    """The samples within `half` (time) of the largest |E|; zero elsewhere."""
    s = np.asarray(samples, dtype=np.float64)
    c = int(np.abs(s).argmax())
    h = int(round(half / dt))
    w = np.zeros_like(s)
    a, b = max(c - h, 0), min(c + h, len(s))
    w[a:b] = s[a:b]
    return w


def group_velocity(medium: np.ndarray, vacuum: np.ndarray, dt: float, length: float, dx: float,
                   window: float, omega: float = 1.0, domega: float = 0.02) -> float:
    """Group velocity in a slab of the given length, from the probe behind it.

    The transmitted spectrum over the vacuum one has the phase
    (k_slab(w) - k_vac(w)) length, whose slope in w is length (1/v_g -
    1/v_vac); the slope is taken between omega -+ domega, each trace kept
    within `window` of its peak (which drops the echoes of the slab's two
    surfaces), and v_vac is the Yee grid's own group velocity."""
    m = _window(medium, dt, window)
    v = _window(vacuum, dt, window)
    lo = _amplitude(m, dt, omega - domega) / _amplitude(v, dt, omega - domega)
    hi = _amplitude(m, dt, omega + domega) / _amplitude(v, dt, omega + domega)
    slope = np.angle(hi / lo) / (2.0 * domega)
    return 1.0 / (1.0 / yee_group_velocity(omega, dx, dt) + slope / length)


def reflection_phase(with_slab: np.ndarray, vacuum: np.ndarray, dt: float, distance: float, dx: float,
                     omega: float = 1.0) -> float:
    """Phase shift of the reflection at the slab surface, from a probe at
    `distance` in front of it: the reflected wave is the difference of the
    two runs; over the incident wave it is the reflection coefficient times
    the round trip probe -> surface -> probe (2 distance, Yee wavenumber),
    which is taken out.  Returns arg r in (-pi, pi]."""
    ref = np.asarray(with_slab, dtype=np.float64) - np.asarray(vacuum, dtype=np.float64)
    ratio = _amplitude(ref, dt, omega) / _amplitude(vacuum, dt, omega)
    k = yee_wavenumber(omega, dx, dt)
    return float(np.angle(ratio * np.exp(-2j * k * distance)))


class LockIn:
    """Running complex amplitude of one frequency at every cell of a field:
    after each step, add(field) accumulates field * exp(i omega t) with
    t = (number of steps added) * dt, the probe convention above.  The result
    is the exp(-i omega t) component's amplitude, whose phase gradient is the
    local wave vector (Sec. 3.1's refraction benchmark reads the refracted
    wave vector off the field's Fourier transform)."""

    def __init__(self, dt: float, omega: float = 1.0):
        self.dt = dt
        self.omega = omega
        self.steps = 0
        self.amplitude = None

    def add(self, field: np.ndarray) -> None:
        self.steps += 1
        f = np.asarray(field, dtype=np.float64)
        c = np.exp(1j * self.omega * self.steps * self.dt)
        if self.amplitude is None:
            self.amplitude = f * c
        else:
            self.amplitude += f * c


def wave_vector(amplitude: np.ndarray, dx: float, x0: int, x1: int, periodic_y: bool = True):
    """(k_x, k_y) of the wave in the columns [x0, x1) of a 2D amplitude
    [y][x]: the |A|^2-weighted mean of the phase advance between neighbouring
    cells along x and along y, divided by dx."""
    a = np.asarray(amplitude)[:, x0:x1]
    sx = np.vdot(a[:, :-1], a[:, 1:])  # sum conj(a_i) a_{i+1}
    if periodic_y:
        sy = np.vdot(a, np.roll(a, -1, axis=0))
    else:
        sy = np.vdot(a[:-1, :], a[1:, :])
    return float(np.angle(sx)) / dx, float(np.angle(sy)) / dx


def refraction_angle(amplitude: np.ndarray, dx: float, x0: int, x1: int) -> float:
    """Angle of the local wave vector to the x axis (radians)."""
    kx, ky = wave_vector(amplitude, dx, x0, x1)
    return math.atan2(ky, kx)
