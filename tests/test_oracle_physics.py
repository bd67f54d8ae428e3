"""Whole-step pins of the FP64 oracle: the paper's benchmark physics.

(b)  phase delay of a pulse through a neutral bound-electron slab against the
     Lorentz-oscillator index of Sec. 3.1 (continuum) and its Yee/leapfrog
     discrete form;
(b') the same with free electrons and charged two-body ions: the Drude term of
     Sec. 3.1 plus the two-body response with q_c != 0;
(f)  independence of the index from Z_b at fixed bound density and w_b;
(c)  Bragg scattering by a 2D lattice in the 2 theta_B direction (Sec. 3.2).

The predictions below are written from the paper's linear theory (the
equations of motion of the two bodies under a uniform field, their solution
r1, r2, the permittivity and the dispersion relation), not from the oracle.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth

KAPPA = lambda lam: O.RE * 2 * math.pi / lam


def two_body_chi(n_ion, Zb, qc, mc, omega_b, w):
    """Susceptibility of a medium of two-body ions at frequency w from the
    driven solution of Sec. 3.1:
      r1 = [-q_c/(m_c w^2) + m2/(m1+m2) q_r/(m_r (w_c^2 - w^2))] E
      r2 = [-q_c/(m_c w^2) - m1/(m1+m2) q_r/(m_r (w_c^2 - w^2))] E
      P  = n (q1 r1 + q2 r2)."""
    q2, m2 = -Zb, Zb
    q1, m1 = qc - q2, mc - m2
    mr = m1 * m2 / (m1 + m2)
    qr = (q1 * m2 - q2 * m1) / (m1 + m2)
    base = -qc / (mc * w * w) if qc else 0.0
    lor = qr / (mr * (omega_b ** 2 - w * w))
    r1 = base + m2 / (m1 + m2) * lor
    r2 = base - m1 / (m1 + m2) * lor
    return n_ion * (q1 * r1 + q2 * r2)


def predicted_delay(L, dx, dt, chi_fn, omega=1.0):
    """Phase delay (k_med - k_vac) L.  Continuum: k = w sqrt(1 + chi(w)).
    Discrete: the Yee dispersion (2/dx) sin(k dx/2) = W sqrt(1 + S_k^2 chi(W))
    with W = (2/dt) sin(w dt/2) for the leapfrog, and S_k = sinc^3(k dx/2)
    the quadratic shape's form factor, once for gather and once for deposit."""
    cont = omega * L * (math.sqrt(1 + chi_fn(omega)) - 1)
    W = 2 / dt * math.sin(omega * dt / 2)
    kv = 2 / dx * math.asin(dx / 2 * W)
    km = kv
    for _ in range(50):
        sk = (math.sin(km * dx / 2) / (km * dx / 2)) ** 3
        km = 2 / dx * math.asin(dx / 2 * W * math.sqrt(1 + sk * sk * chi_fn(W)))
    return cont, (km - kv) * L


def run_1d(wl: synth.Workload, steps: int, extra=None):
    s = O.Sim(1, wl.n, wl.dx, wl.dt, wl.bc)
    for sp in wl.species:
        if isinstance(sp, synth.TwoBody):
            sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
            s.load(sid, sp.x, sp.u)
        else:
            sid = s.add_free(sp.q, sp.m, sp.w)
            s.load(sid, sp.x, sp.u)
    for L in wl.lasers:
        s.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    pid = s.add_probe(wl.probe_comp, wl.probe_nodes, steps)
    s.step(steps)
    tr = s.probe(pid, 1)[:, 0]
    s.close()
    return tr


def measured_delay(tr_med, tr_vac, dt, omega=1.0):
    t = (np.arange(len(tr_vac)) + 1) * dt
    ph = np.exp(1j * omega * t)
    return float(np.angle(np.sum(tr_med * ph) / np.sum(tr_vac * ph)))


STEPS_B = 4500  # the whole 10-cycle pulse passes the probe at 26 lambda


@pytest.fixture(scope="module")
def vacuum_trace():
    wl = synth.neutral_1d(ppc=1, vacuum=True)
    return run_1d(wl, STEPS_B)


def test_lorentz_index_phase_delay(vacuum_trace):
    """Pin (b): the 1D neutral medium's geometry (16 lambda slab, n_b = 0.01, w_b = 3).
    n - 1 = 6.248e-4, so the delay is k0 L (n - 1) ~ 0.0628 rad."""
    wl = synth.neutral_1d(ppc=1)
    sp = wl.species[0]
    tr = run_1d(wl, STEPS_B)
    meas = measured_delay(tr, vacuum_trace, wl.dt)
    lo, hi = wl.meta["slab"]
    L = (hi - lo) * wl.dx[0]
    n_ion = sp.w * 1
    chi = lambda w: two_body_chi(n_ion, sp.Zb, sp.qc, sp.mc, 3.0, w)
    cont, disc = predicted_delay(L, wl.dx[0], wl.dt, chi)
    assert abs(cont - 0.0628) < 5e-4
    assert abs(meas / disc - 1) < 0.01, (meas, disc, cont)
    assert abs(meas / cont - 1) < 0.03, (meas, disc, cont)


def test_drude_plus_bound_index(vacuum_trace):
    """Pin (b'): free electrons (Drude term -n_e e^2/(m_e w^2), Sec. 3.1) plus
    charged two-body ions (q_c = +1, Z_b = 1) at the same positions, so the
    slab starts neutral; the phase advances by k0 L (n - 1) < 0."""
    base = synth.neutral_1d(ppc=1)
    sp = base.species[0]
    n_ion = 0.01
    ion = synth.TwoBody(Zb=1.0, qc=1.0, mc=sp.mc, w=n_ion, lambda0_m=sp.lambda0_m,
                        omega_b=np.array([3.0]), x=sp.x, u=sp.u)
    ele = synth.Free(q=-1.0, m=1.0, w=n_ion, x=sp.x.copy(), u=np.zeros_like(sp.u))
    base.species = [ion, ele]
    tr = run_1d(base, STEPS_B)
    meas = measured_delay(tr, vacuum_trace, base.dt)
    lo, hi = base.meta["slab"]
    L = (hi - lo) * base.dx[0]
    chi = lambda w: two_body_chi(n_ion, 1.0, 1.0, sp.mc, 3.0, w) - n_ion / (w * w)
    cont, disc = predicted_delay(L, base.dx[0], base.dt, chi)
    assert cont < -0.4
    assert abs(meas / disc - 1) < 0.01, (meas, disc, cont)
    assert abs(meas / cont - 1) < 0.03, (meas, disc, cont)


def test_zb_invariance(vacuum_trace):
    """Pin (f): at fixed bound density n_b = Z_b n_ion and w_b, the linear
    index depends on Z_b only through m2/m1 ~ 2e-4, so the delay is the same
    for Z_b = 1, 20, 78 to 1e-3."""
    vals = []
    for Zb in (1.0, 20.0, 78.0):
        wl = synth.neutral_1d(ppc=1, Zb=Zb)
        tr = run_1d(wl, STEPS_B)
        vals.append(measured_delay(tr, vacuum_trace, wl.dt))
    vals = np.array(vals)
    assert np.abs(vals / vals[0] - 1).max() < 1e-3, vals


def _bragg_run(theta_deg, steps=620):
    n = 384
    cpl = 16
    dx = synth.LAMBDA0 / cpl
    wl = synth.bragg_2d(seed=1, n=n, cells_per_lambda=cpl, sites=(8, 8), theta_deg=theta_deg,
                             waist_lambda=4.0, fwhm_lambda=4.0, nb=0.05)
    s = O.Sim(2, wl.n, wl.dx, wl.dt, wl.bc)
    sp = wl.species[0]
    sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, sp.omega_b)
    s.load(sid, sp.x, sp.u)
    for L in wl.lasers:
        s.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    s.step(steps)
    Bz = s.field(O.BZ)[0].copy()
    s.close()
    F = np.fft.fftshift(np.abs(np.fft.fft2(Bz)))
    k = np.fft.fftshift(np.fft.fftfreq(n, d=dx)) * 2 * np.pi
    KX, KY = np.meshgrid(k, k, indexing="xy")
    return F, KX, KY, wl


def _ring_peak(F, KX, KY, exclude_deg, half_width=20.0):
    kr = np.hypot(KX, KY)
    ang = np.degrees(np.arctan2(KY, KX))
    ring = (kr > 0.85) & (kr < 1.15) & (KX > 0)
    ring &= np.abs(ang - exclude_deg) > half_width
    i = np.argmax(np.where(ring, F, 0))
    return F.flat[i], ang.flat[i], kr.flat[i], KX.flat[i], KY.flat[i]


@pytest.mark.slow
def test_bragg_peak_direction():
    """Pin (c): a square lattice of period d = lambda, beam at theta_B = 30 deg
    to the lattice rows (Bragg's law 2 d sin(theta_B) = lambda, Sec. 3.2):
    besides the incident beam, the strongest forward component of the field
    spectrum lies at k_i + G, i.e. at 2 theta_B = 60 deg from the incident
    direction (-30 deg): the peak's wave vector lies within one FFT bin of
    k_s = k_i + G, G = (2 pi / d)(0, -1), in each component (the bins of the
    Cartesian FFT grid; |k_i| is the grid's own wavenumber at w0, 0.3% above
    k0 at lambda/16).  Control (lattice rows along the beam, Sec. 3.2 case
    (b)): nothing comparable at 60 deg from incidence."""
    F, KX, KY, wl = _bragg_run(30.0)
    peak, ang, kr, kx, ky = _ring_peak(F, KX, KY, exclude_deg=30.0)
    L = wl.n[0] * wl.dx[0]
    dk = 2 * math.pi / L
    d = wl.meta["d"]
    dx, dt = wl.dx[0], wl.dt
    th = math.radians(30.0)
    # the grid's wavenumber along the beam: the 2D Yee dispersion at w0,
    # sin^2(k cos(th) dx/2) + sin^2(k sin(th) dx/2) = (dx/dt)^2 sin^2(dt/2), by bisection
    f = lambda k: (math.sin(k * math.cos(th) * dx / 2) ** 2 + math.sin(k * math.sin(th) * dx / 2) ** 2
                   - (dx / dt * math.sin(dt / 2)) ** 2)
    lo, hi = 0.9, 1.1
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    k = 0.5 * (lo + hi)
    assert abs(k - 1.0) < 5e-3
    ks = (k * math.cos(th), k * math.sin(th) - 2 * math.pi / d)
    assert abs(kx - ks[0]) <= dk + 1e-9 and abs(ky - ks[1]) <= dk + 1e-9, ((kx, ky), ks, dk, ang)
    Fc, KXc, KYc, _ = _bragg_run(0.0)
    angc = np.degrees(np.arctan2(KYc, KXc))
    krc = np.hypot(KXc, KYc)
    cone = (krc > 0.85) & (krc < 1.15) & (np.abs(np.abs(angc) - 60.0) < 5.0)
    assert Fc[cone].max() < 0.2 * peak
