"""Linear theory of Sec. 3.1 near the bound-electron resonance, written from
the paper (test infrastructure): the permittivity of a medium of two-body
ions plus free electrons, the group velocity and the reflection phase shift,
their discrete (Yee grid, leapfrog) forms, and the measurement of both from
probe traces of the oracle.  Units: c = 1, omega0 = 1, densities in n_c,
charges in e, masses in m_e."""
import cmath
import math

import numpy as np

from test_oracle_physics import two_body_chi


def eps_r(w, n_ion, Zb, qc, mc, omega_b, n_free=0.0):
    """eps / eps0 of Sec. 3.1: 1 + n (q1 r1 + q2 r2) / E for the two-body
    ions (the driven solution r1, r2) plus the free electrons' Drude term
    -n_e e^2 / (m_e w^2)."""
    return 1.0 + two_body_chi(n_ion, Zb, qc, mc, omega_b, w) - n_free / (w * w)


def group_velocity(w, eps_fn, h=1e-6):
    """v_g = (k/w + w^2/(2 c^2 k) d eps_r/dw)^-1 with k = w sqrt(eps_r) (the
    group-velocity formula of Sec. 3.1); d eps_r/dw by a central difference
    of eps_r itself."""
    e = eps_fn(w)
    k = w * math.sqrt(e)
    de = (eps_fn(w + h) - eps_fn(w - h)) / (2 * h)
    return 1.0 / (k / w + w * w / (2 * k) * de)


def reflection_phase(eps):
    """phi = arctan(-2 Gamma / (1 - Gamma^2)) for sqrt(eps_r) = i Gamma (the
    reflection formula of Sec. 3.1), on the atan2 branch."""
    G = math.sqrt(-eps)
    return math.atan2(-2.0 * G, 1.0 - G * G)


def yee_k(w, dx, dt, chi_fn=None, iters=60):
    """Real wavenumber of the discrete system at frequency w: the Yee
    dispersion (2/dx) sin(k dx/2) = W sqrt(1 + S_k^2 chi(W)), W = (2/dt)
    sin(w dt/2) (leapfrog), S_k = sinc^3(k dx/2) the quadratic shape's form
    factor (gather and deposit)."""
    W = 2.0 / dt * math.sin(w * dt / 2.0)
    k = 2.0 / dx * math.asin(dx / 2.0 * W)
    if chi_fn is None:
        return k
    for _ in range(iters):
        sk = (math.sin(k * dx / 2) / (k * dx / 2)) ** 3
        k = 2.0 / dx * math.asin(dx / 2.0 * W * math.sqrt(1.0 + sk * sk * chi_fn(W)))
    return k


def yee_group_velocity(w, dx, dt, chi_fn=None, h=1e-5):
    """dw/dk of the discrete dispersion relation, by a central difference."""
    return 2 * h / (yee_k(w + h, dx, dt, chi_fn) - yee_k(w - h, dx, dt, chi_fn))


def spectrum(trace, dt, w):
    """sum_t E(t) exp(i w t), t = (s + 1) dt for sample s (the probe records
    after each step): the complex amplitude of the exp(-i w t) component."""
    t = (np.arange(len(trace)) + 1) * dt
    return np.sum(np.asarray(trace) * np.exp(1j * w * t))


def gate(trace, dt, half_width):
    """The trace kept within half_width of its envelope peak (|E| maximum),
    zero elsewhere: keeps the pulse, drops late echoes."""
    tr = np.asarray(trace, dtype=np.float64)
    p = int(np.argmax(np.abs(tr)))
    m = int(round(half_width / dt))
    out = np.zeros_like(tr)
    out[max(0, p - m):p + m] = tr[max(0, p - m):p + m]
    return out


def measured_group_velocity(tr_med, tr_vac, dt, L, dx, half_width, w=1.0, dw=0.02):
    """v_g from the slope of the transmitted phase: arg(T(w)), T = spectrum of
    the medium trace / spectrum of the vacuum trace, grows by L (1/v_g -
    1/v_g,vac) per unit w; v_g,vac the Yee grid's."""
    a, b = gate(tr_med, dt, half_width), gate(tr_vac, dt, half_width)
    ph = [cmath.phase(spectrum(a, dt, x) / spectrum(b, dt, x)) for x in (w - dw, w + dw)]
    d = (ph[1] - ph[0] + math.pi) % (2 * math.pi) - math.pi
    inv = 1.0 / yee_group_velocity(w, dx, dx * 0.95) + d / (2 * dw) / L
    return 1.0 / inv


def measured_reflection_phase(tr_slab, tr_vac, dt, dist, dx, w=1.0):
    """arg r of the reflected wave: (slab trace - vacuum trace) over the
    vacuum trace at the probe, both as spectra at w, with the round trip
    probe -> surface -> probe (dist each way, Yee wavenumber) taken out."""
    R = spectrum(np.asarray(tr_slab) - np.asarray(tr_vac), dt, w) / spectrum(tr_vac, dt, w)
    r = R * cmath.exp(-2j * yee_k(w, dx, dt) * dist)
    return cmath.phase(r)
