"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than the oracle
itself: closed forms, invariants, the paper's printed worked example, or
exact identities of the discrete scheme.  A plausible slip (a dropped factor
1/2, a wrong stagger, a sign, a transposed operand) fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


# ---------------------------------------------------------------------------
# shape: quadratic B-spline

def test_shape_moments():
    """Partition of unity, exact first moment, second central moment 1/4
    (three convolved unit boxes have variance 3/12)."""
    rng = np.random.default_rng(0)
    for X in rng.uniform(-3, 3, 200):
        nodes = np.arange(math.floor(X) - 3, math.floor(X) + 4)
        w = np.array([O.shape(X - i) for i in nodes])
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w * nodes).sum() - X) < 1e-13
        assert abs((w * (nodes - X) ** 2).sum() - 0.25) < 1e-13
    assert O.shape(0.0) == 0.75 and O.shape(1.5) == 0.0 and O.shape(-2.0) == 0.0


def test_shape_is_three_box_convolution():
    """S equals the box function convolved with itself three times,
    evaluated by numerical quadrature of the piecewise-linear hat * box."""
    def hat(t):  # box * box
        return max(0.0, 1.0 - abs(t))
    for x in np.linspace(-1.6, 1.6, 33):
        q = np.linspace(x - 0.5, x + 0.5, 20001)
        val = np.trapezoid([hat(t) for t in q], q)
        assert abs(val - O.shape(x)) < 1e-8


# ---------------------------------------------------------------------------
# gather: staggered interpolation reproduces linear fields exactly

@pytest.mark.parametrize("D", [1, 2, 3])
def test_gather_linear_field_exact(D):
    """With the quadratic B-spline, a field linear in position is reproduced
    exactly at any point, provided each component is sampled at its own Yee
    location.  A wrong stagger shifts the result by half a cell times the
    slope."""
    n = [16, 12, 10][:D]
    dx = [0.3, 0.25, 0.2][:D]
    s = O.Sim(D, n, dx, 0.1, [O.OPEN] * D)
    stag = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0.5, 0.5), 4: (0.5, 0, 0.5),
            5: (0.5, 0.5, 0)}
    rng = np.random.default_rng(D)
    coef = rng.normal(size=(6, 4))
    nn = s.n
    k, j, i = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    for c in range(6):
        st = stag[c]
        pos = [i + st[0], j + st[1] * (D >= 2), k + st[2] * (D >= 3)]
        f = coef[c, 0] + sum(coef[c, a + 1] * pos[a] for a in range(D))
        s.field(c)[...] = f
    for _ in range(30):
        X = [rng.uniform(3, n[a] - 4) for a in range(D)]
        for c in range(6):
            want = coef[c, 0] + sum(coef[c, a + 1] * X[a] for a in range(D))
            assert abs(s.interp(c, X) - want) < 1e-12 * (1 + abs(want))
    s.close()


# ---------------------------------------------------------------------------
# Boris push

def test_boris_pure_electric_kick():
    """B = 0: two half kicks give u' = u + (q/m) dt E exactly."""
    u0 = np.array([0.1, -0.2, 0.3])
    E = np.array([0.5, 0.25, -1.0])
    u = O.boris(-1.0, 1.0, 0.05, E, np.zeros(3), u0)
    assert np.allclose(u, u0 - 0.05 * E, rtol=0, atol=1e-15)


def test_boris_magnetic_rotation_angle():
    """E = 0: |u| is preserved and u turns about B by the Boris angle
    2 atan(|t|), t = q dt B / (2 m gamma)."""
    q, m, dt = -1.0, 1.0, 0.2
    B = np.array([0.0, 0.0, 3.0])
    u0 = np.array([0.6, 0.0, 0.4])
    g = math.sqrt(1 + u0 @ u0)
    u = O.boris(q, m, dt, np.zeros(3), B, u0)
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-15
    assert abs(u[2] - u0[2]) < 1e-16
    ang = math.atan2(u[1], u[0]) - math.atan2(u0[1], u0[0])
    t = q * dt * B[2] / (2 * m * g)
    # rotation is by -2 atan(t) about +z for the cross-product order u x t
    assert abs(ang - (-2 * math.atan(t))) < 1e-14


# ---------------------------------------------------------------------------
# internal force: the modified Coulomb interaction

def test_internal_force_is_gradient_of_modified_potential():
    """The force on body 1 equals -grad_r1 of V_M = q1 q2 kappa / sqrt(r^2 + ac^2)
    (Sec. 2), checked by central differences of V_M; body 2 gets the opposite
    force (Newton's third law)."""
    q1, q2, kappa, ac = 3.0, -2.0, 1.7e-3, 0.05
    V = lambda r: q1 * q2 * kappa / math.sqrt(r @ r + ac * ac)
    rng = np.random.default_rng(3)
    for _ in range(20):
        r = rng.normal(scale=0.04, size=3)
        F1 = q1 * O.internal_field(q2, kappa, ac, r)
        F2 = q2 * O.internal_field(q1, kappa, ac, -r)
        h = 1e-6
        grad = np.array([(V(r + h * e) - V(r - h * e)) / (2 * h) for e in np.eye(3)])
        assert np.allclose(F1, -grad, rtol=1e-7, atol=1e-12)
        assert np.abs(F1 + F2).max() <= 4e-16 * np.abs(F1).max()


def test_resonance_radius_golden():
    """Paper's worked example: 12.4 nm light in gold with Z_b = 78 and one
    free electron per atom resonates (w_c = w) at a_c ~ 9.5e-11 m."""
    g = read_golden("resonance_ac.txt")
    s = O.Sim(1, [8], [1.0], 0.1, [O.PERIODIC])
    sid = s.add_two_body(g["Zb"], g["qc"], synth.M_AU, 1.0, g["lambda_m"], [1.0])
    ac_m = s.ac(sid) / (2 * math.pi / g["lambda_m"])
    assert round(ac_m / 1e-11, 1) == g["ac_m"] / 1e-11
    s.close()


def test_species_split_invariants():
    """q1 + q2 = q_c, m1 + m2 = m_c, and the combined electron has the
    electron's charge-to-mass ratio (Sec. 2)."""
    s = O.Sim(1, [8], [1.0], 0.1, [O.PERIODIC])
    for Zb, qc in [(1, 0), (78, 1), (49, 30)]:
        sid = s.add_two_body(Zb, qc, synth.M_AU, 1.0, 12.4e-9, [3.0])
        info = s.species_info(sid)
        assert info["q1"] + info["q2"] == qc
        assert abs(info["m1"] + info["m2"] - synth.M_AU) < 1e-9
        assert info["q2"] / info["m2"] == -1.0
        assert info["q2"] == -Zb
    s.close()


def _isolated_ion(omega_b, Zb=1.0, qc=0.0, r0_over_ac=1e-5, steps=400, dt=0.05, lambda0_m=12.4e-9):
    s = O.Sim(1, [16], [1.0], dt, [O.PERIODIC])
    s.set_switches(fields_on=False, deposit_on=False)
    sid = s.add_two_body(Zb, qc, synth.M_AU, 1.0, lambda0_m, [omega_b])
    s.load(sid, np.zeros((1, 1)), np.zeros((1, 3)))
    info = s.species_info(sid)
    ac = s.ac(sid)
    r0 = r0_over_ac * ac
    m1, m2 = info["m1"], info["m2"]
    x1 = np.array([[r0 * m2 / (m1 + m2), 0, 0]])
    x2 = np.array([[-r0 * m1 / (m1 + m2), 0, 0]])
    s.set_bodies(sid, x1=x1, x2=x2)
    r, p = [], []
    for _ in range(steps):
        s.step(1)
        a, b, u1, u2 = s.bodies(sid)
        r.append(a[0, 0] - b[0, 0])
        p.append((m1 * u1[0, 0] + m2 * u2[0, 0], m2 * abs(u2[0, 0])))
    s.close()
    return np.array(r), np.array(p), ac


@pytest.mark.parametrize("omega_b,Zb,qc", [(3.0, 1.0, 0.0), (4.0, 49.0, 30.0), (1.5, 78.0, 1.0)])
def test_isolated_ion_natural_frequency(omega_b, Zb, qc):
    """Pin (a): with no external field, a small internal displacement
    oscillates at w_c of Sec. 3.1; under the leapfrog the discrete frequency
    obeys cos(W dt) = 1 - (w_c dt)^2 / 2, and every triple of successive
    displacements satisfies r+ + r- = 2 cos(W dt) r0."""
    dt = 0.05
    r, p, ac = _isolated_ion(omega_b, Zb, qc, dt=dt)
    big = np.abs(r[1:-1]) > 0.5 * np.abs(r).max()
    c = (r[2:] + r[:-2])[big] / (2 * r[1:-1][big])
    w2 = 2 * (1 - c) / dt ** 2
    assert np.all(np.abs(w2 / omega_b ** 2 - 1) < 1e-8)
    # equal and opposite internal kicks: total momentum stays zero
    assert np.abs(p[:, 0]).max() <= 1e-14 * p[:, 1].max()


def test_isolated_ion_anharmonic_period():
    """Large amplitude (r0 = a_c): the period follows the modified Coulomb
    potential, checked against the FP64 quadrature of the energy integral
    T = 2 * int dr / sqrt(2 (E - V(r)) / m_r) with V = -k / sqrt(r^2 + a^2)
    (small dt, so the leapfrog error is far below the tolerance; a long
    physical wavelength keeps the swing non-relativistic, v^2 ~ 1e-9)."""
    omega_b, dt = 3.0, 0.002
    r, _, ac = _isolated_ion(omega_b, r0_over_ac=1.0, steps=8000, dt=dt, lambda0_m=1e-4)
    # zero crossings with linear interpolation
    idx = np.where(np.sign(r[:-1]) != np.sign(r[1:]))[0]
    tc = [(i + r[i] / (r[i] - r[i + 1])) * dt for i in idx]
    T_sim = 2 * np.mean(np.diff(tc))
    # V(r) = -m_r w^2 a^3 / sqrt(r^2 + a^2) (spring constant m_r w^2 at r = 0)
    from scipy.integrate import quad
    V = lambda x: -(omega_b ** 2) * ac ** 3 / math.sqrt(x * x + ac * ac)
    E = V(ac)
    # substitution x = a sin(th) removes the endpoint singularity
    f = lambda th: ac * math.cos(th) / math.sqrt(2 * (E - V(ac * math.sin(th))))
    T_th = 4 * quad(f, 0, math.pi / 2, epsabs=1e-14, epsrel=1e-12)[0]
    assert abs(T_sim / T_th - 1) < 1e-5


def test_initial_conditions_neutral_and_charged():
    """Sec. 2 initial conditions: r1 = r2 = r_c, p1 + p2 = p_c, q1 v1 + q2 v2 = 0
    (non-relativistic split for charged ions), and a cold neutral medium has
    rho = 0 and carries no current."""
    s = O.Sim(1, [32], [0.5], 0.2, [O.PERIODIC])
    sid = s.add_two_body(1.0, 0.0, synth.M_AU, 0.1, 12.4e-9, [3.0])
    x, _ = synth.medium(5, 1, (0.5,), (4,), (28,), 3)
    uc = np.random.default_rng(1).normal(scale=1e-3, size=(len(x), 3))
    s.load(sid, x, uc)
    x1, x2, u1, u2 = s.bodies(sid)
    assert np.array_equal(x1, x2) and np.array_equal(u1, uc) and np.array_equal(u2, uc)
    assert np.abs(s.rho()).max() == 0.0
    sid2 = s.add_two_body(49.0, 30.0, synth.M_AU, 0.1, 0.26e-9, [4.0])
    s.load(sid2, x[:10], uc[:10])
    info = s.species_info(sid2)
    _, _, v1, v2 = s.bodies(sid2)
    mc = info["m1"] + info["m2"]
    assert np.allclose(info["m1"] * v1 + info["m2"] * v2, mc * uc[:10], rtol=1e-12, atol=0)
    assert np.allclose(info["q1"] * v1 + info["q2"] * v2, 0.0, atol=1e-15)
    s.close()


# ---------------------------------------------------------------------------
# Esirkepov deposit

@pytest.mark.parametrize("D", [1, 2, 3])
def test_deposit_total_current(D):
    """Summed over the grid, the Esirkepov current of one particle is
    q w (X1 - X0) dx / dt along simulated axes and q w v along invariant
    ones: the first moment of the quadratic shape is exact."""
    n = [20, 18, 16][:D]
    dx = [0.3, 0.25, 0.2]
    dt = 0.07
    rng = np.random.default_rng(10 + D)
    for _ in range(20):
        s = O.Sim(D, n, dx[:D], dt, [O.PERIODIC] * D)
        X0 = [rng.uniform(5, n[a] - 6) for a in range(D)]
        X1 = [X0[a] + rng.uniform(-0.9, 0.9) for a in range(D)]
        v = rng.uniform(-0.5, 0.5, 3)
        qw = -0.37
        s.deposit_one(qw, X0, X1, v)
        for a in range(3):
            tot = s.field(6 + a).sum()
            want = qw * (X1[a] - X0[a]) * dx[a] / dt if a < D else qw * v[a]
            assert abs(tot - want) < 1e-12 * (1 + abs(want))
        s.close()


@pytest.mark.parametrize("D", [1, 2, 3])
def test_deposit_continuity_single_particle(D):
    """Discrete continuity for one move: rho1 - rho0 + dt div J = 0 at every
    node, with rho the quadratic-shape charge on nodes."""
    n = [14, 12, 10][:D]
    dx = [0.3, 0.25, 0.2][:D]
    dt = 0.05
    rng = np.random.default_rng(20 + D)
    for _ in range(10):
        s = O.Sim(D, n, dx, dt, [O.PERIODIC] * D)
        sid = s.add_free(-1.0, 1.0, 0.3)
        X0 = np.array([rng.uniform(0, n[a]) for a in range(D)])
        X1 = X0 + rng.uniform(-0.9, 0.9, D)
        s.load(sid, (X0 * dx)[None, :], np.zeros((1, 3)))
        rho0 = s.rho()
        s.set_bodies(sid, x1=np.array([list(X1 * dx) + [0.0] * (3 - D)]))
        rho1 = s.rho()
        s.deposit_one(-0.3, X0, X1, np.zeros(3))
        div = np.zeros_like(rho0)
        for a in range(D):
            J = s.field(6 + a)
            div += (J - np.roll(J, 1, axis=2 - a)) / dx[a]
        assert np.abs(rho1 - rho0 + dt * div).max() < 1e-14
        s.close()


# ---------------------------------------------------------------------------
# Yee: vacuum dispersion

@pytest.mark.parametrize("D", [1, 2, 3])
def test_yee_vacuum_dispersion(D):
    """Pin (e): a single periodic mode oscillates at W with
    sin(W dt / 2) / dt = sqrt(sum_a sin^2(k_a dx_a / 2) / dx_a^2); every
    triple of successive samples obeys E+ + E- = 2 cos(W dt) E."""
    n = [32, 24, 16][:D]
    dx = [0.2, 0.25, 0.3][:D]
    dt = 0.9 / math.sqrt(sum(1 / d ** 2 for d in dx))
    s = O.Sim(D, n, dx, dt, [O.PERIODIC] * D)
    m = [3, 2, 1][:D]
    k = [2 * math.pi * m[a] / (n[a] * dx[a]) for a in range(D)]
    nn = s.n
    kk, jj, ii = np.meshgrid(np.arange(nn[2]), np.arange(nn[1]), np.arange(nn[0]), indexing="ij")
    # a transverse, divergence-free mode: E_z(x, y) in 1D/2D, E_x(y, z) in 3D
    if D < 3:
        comp = 2
        ph = k[0] * ii * dx[0] + (k[1] * jj * dx[1] if D == 2 else 0)
        K2 = sum((2 / dx[a] * math.sin(k[a] * dx[a] / 2)) ** 2 for a in range(D))
    else:
        comp = 0
        ph = k[1] * jj * dx[1] + k[2] * kk * dx[2]
        K2 = sum((2 / dx[a] * math.sin(k[a] * dx[a] / 2)) ** 2 for a in (1, 2))
    s.field(comp)[...] = np.cos(ph)
    probe = (0, 0, 0)
    vals = [s.field(comp)[probe]]
    for _ in range(200):
        s.step(1)
        vals.append(s.field(comp)[probe])
    v = np.array(vals)
    big = np.abs(v[1:-1]) > 0.3
    c = (v[2:] + v[:-2])[big] / (2 * v[1:-1][big])
    want = 1 - dt * dt * K2 / 2
    assert np.abs(c - want).max() < 1e-12
    s.close()


def test_mur_absorbs_and_antenna_amplitude():
    """A 1D pulse launched by the antenna has amplitude a0 and leaves through
    the Mur faces: afterwards the field energy left is a tiny fraction of
    the pulse's."""
    nx = 800
    dx = 2 * math.pi / 32
    s = O.Sim(1, [nx], [dx], 0.95 * dx, [O.OPEN])
    fwhm = 4 * 2 * math.pi
    s.add_laser(comp=1, a0=1e-3, fwhm=fwhm, t0=2 * fwhm, ia=200)
    pid = s.add_probe(O.EY, [500], 5000)
    peak_energy = 0.0
    for _ in range(10):
        s.step(100)
        e = (s.field(O.EY) ** 2).sum() + (s.field(O.BZ) ** 2).sum()
        peak_energy = max(peak_energy, e)
    tr = s.probe(pid, 1)[:, 0]
    assert abs(np.abs(tr).max() / 1e-3 - 1) < 0.02
    s.step(1200)
    e = (s.field(O.EY) ** 2).sum() + (s.field(O.BZ) ** 2).sum()
    assert e < 1e-5 * peak_energy
    s.close()


@pytest.mark.parametrize("D", [1, 2, 3])
def test_continuity_full_step(D):
    """Pin (d): with Esirkepov currents and Yee fields, div E - rho keeps its
    initial value to round-off over many full steps (moving free electrons
    and two-body ions with non-zero internal displacement, fields on)."""
    n = [40, 16, 12][:D]
    dx = [0.3, 0.3, 0.3][:D]
    dt = 0.9 * dx[0] / math.sqrt(D)
    s = O.Sim(D, n, dx, dt, [O.PERIODIC] * D)
    rng = np.random.default_rng(30 + D)
    N = 60
    X = rng.uniform(0, 1, (N, D)) * np.array(n) * np.array(dx)
    sid = s.add_free(-1.0, 1.0, 0.05)
    s.load(sid, X, rng.normal(scale=0.05, size=(N, 3)))
    sid2 = s.add_two_body(1.0, 0.0, synth.M_AU, 0.05, 12.4e-9, [3.0])
    s.load(sid2, X[:20], rng.normal(scale=0.02, size=(20, 3)))
    x1, x2, _, _ = s.bodies(sid2)
    s.set_bodies(sid2, x2=x2 + rng.normal(scale=0.05, size=x2.shape) * (np.arange(3) < 3))
    R0 = s.residual()
    rmax = np.abs(s.rho()).max()
    for _ in range(25):
        s.step(1)
    R = s.residual()
    assert np.abs(R - R0).max() < 1e-12 * rmax
    s.close()


# ---------------------------------------------------------------------------
# Pin (a'): a two-body ion driven by a uniform field E0 cos(w t).  Sec. 3.1
# gives the steady-state displacements of nucleus and bound electron,
#   r1 = [-qc/(mc w^2) + m2/(m1+m2) qr/(mr (wc^2 - w^2))] E,
#   r2 = [-qc/(mc w^2) - m1/(m1+m2) qr/(mr (wc^2 - w^2))] E,
# qr = (q1 m2 - q2 m1)/(m1+m2), mr = m1 m2/(m1+m2).  The leapfrog (x and E
# at t_n) has the same particular solution with w replaced by
# (2/dt) sin(w dt/2); the free oscillation at the discrete natural frequency
# and the centre of mass's uniform drift are fitted out.

@pytest.mark.parametrize("Zb,qc", [(1.0, 0.0), (10.0, 5.0)])
def test_driven_ion_steady_state_amplitudes(Zb, qc):
    # a light nucleus (mass 100 m_e) so that both bodies move by far more than the
    # rounding of their positions; the formula holds for any two masses
    dt, w, steps, wb = 0.05, 1.0, 2000, 3.0
    s = O.Sim(1, [16], [1.0], dt, [O.PERIODIC])
    s.set_switches(fields_on=False, deposit_on=False)
    sid = s.add_two_body(Zb, qc, 100.0, 1.0, 12.4e-9, [wb])
    s.load(sid, np.array([[0.5]]), np.zeros((1, 3)))
    info = s.species_info(sid)
    q1, m1, q2, m2 = info["q1"], info["m1"], info["q2"], info["m2"]
    mc, qcc = m1 + m2, q1 + q2
    mr, qr = m1 * m2 / mc, (q1 * m2 - q2 * m1) / mc
    # relative amplitude 1e-4 a_c: the internal force stays linear to 1e-8
    E0 = 1e-4 * s.ac(sid) * mr * (wb ** 2 - w ** 2) / abs(qr)
    x1s, x2s = [], []
    for n in range(steps):
        s.field(0)[...] = E0 * math.cos(w * n * dt)   # uniform E_x at t_n
        s.step(1)
        a, b, _, _ = s.bodies(sid)
        x1s.append(a[0, 0])
        x2s.append(b[0, 0])
    s.close()
    t = np.arange(1, steps + 1) * dt
    wd = 2.0 / dt * math.sin(w * dt / 2)                       # driving frequency seen by the leapfrog
    wn = math.acos(1.0 - (wb * dt) ** 2 / 2) / dt               # discrete free frequency
    A = np.stack([np.ones_like(t), t, np.cos(w * t), np.sin(w * t), np.cos(wn * t), np.sin(wn * t)], axis=1)
    want1 = (-qcc / (mc * wd ** 2) + m2 / mc * qr / (mr * (wb ** 2 - wd ** 2))) * E0
    want2 = (-qcc / (mc * wd ** 2) - m1 / mc * qr / (mr * (wb ** 2 - wd ** 2))) * E0
    for xs, want in ((x1s, want1), (x2s, want2)):
        coef, *_ = np.linalg.lstsq(A, np.array(xs), rcond=None)
        assert abs(coef[2] / want - 1) < 1e-6, (coef[2], want)
        assert abs(coef[3]) < 1e-6 * abs(want)        # in phase with the drive


# ---------------------------------------------------------------------------
# Pin (g): one whole step of the oracle against a second, hand-expanded FP64
# step written here with no stencil logic: every gather and deposit sums the
# quadratic B-spline over all nodes of a periodic 8^3 grid (minimum-image
# distances), the running sums of the current start outside the support.

def _S(xi):
    a = np.abs(xi)
    return np.where(a <= 0.5, 0.75 - xi * xi, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def _wrap(d, n):
    return (d + 0.5 * n) % n - 0.5 * n


def _weights(X, stag, n):
    """Per-axis weight vectors over all nodes (node a-index i sits at i + stag[a])."""
    return [_S(_wrap(X[a] - (np.arange(n[a]) + stag[a]), n[a])) for a in range(3)]


def _gather(F, X, stag, n):
    wx, wy, wz = _weights(X, stag, n)
    return float(np.einsum("k,j,i,kji->", wz, wy, wx, F))


def _curl_fwd(F, d):   # (dFz/dy - dFy/dz, ...) at the B locations, arrays [z][y][x]
    Fx, Fy, Fz = F
    dy = lambda A: (np.roll(A, -1, 1) - A) / d[1]
    dz = lambda A: (np.roll(A, -1, 0) - A) / d[2]
    dxx = lambda A: (np.roll(A, -1, 2) - A) / d[0]
    return [dy(Fz) - dz(Fy), dz(Fx) - dxx(Fz), dxx(Fy) - dy(Fx)]


def _curl_bwd(F, d):
    Fx, Fy, Fz = F
    dy = lambda A: (A - np.roll(A, 1, 1)) / d[1]
    dz = lambda A: (A - np.roll(A, 1, 0)) / d[2]
    dxx = lambda A: (A - np.roll(A, 1, 2)) / d[0]
    return [dy(Fz) - dz(Fy), dz(Fx) - dxx(Fz), dxx(Fy) - dy(Fx)]


def _boris(h, E, B, u):
    um = u + h * E
    g = math.sqrt(1.0 + um @ um)
    t = h * B / g
    s = 2.0 * t / (1.0 + t @ t)
    up = um + np.cross(um + np.cross(um, t), s)
    return up + h * E


def _reference_step(E, B, bodies, sp, d, dt, n):
    q1, m1, q2, m2, w, kappa, ac = sp
    B = [b - 0.5 * dt * c for b, c in zip(B, _curl_fwd(E, d))]
    stE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    stB = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    J = [np.zeros(E[0].shape) for _ in range(3)]
    out = []
    for x1, x2, u1, u2 in bodies:
        X1, X2 = x1 / d, x2 / d
        E1 = np.array([_gather(E[c], X1, stE[c], n) for c in range(3)])
        B1 = np.array([_gather(B[c], X1, stB[c], n) for c in range(3)])
        E2 = np.array([_gather(E[c], X2, stE[c], n) for c in range(3)])
        B2 = np.array([_gather(B[c], X2, stB[c], n) for c in range(3)])
        r = _wrap(x1 - x2, d * np.array(n))
        f = kappa * r / (r @ r + ac * ac) ** 1.5
        E1, E2 = E1 + q2 * f, E2 - q1 * f
        v1n = _boris(q1 * dt / (2 * m1), E1, B1, u1)
        v2n = _boris(q2 * dt / (2 * m2), E2, B2, u2)
        y1 = x1 + dt * v1n / math.sqrt(1.0 + v1n @ v1n)
        y2 = x2 + dt * v2n / math.sqrt(1.0 + v2n @ v2n)
        for q, X0, Y in ((q1, X1, y1 / d), (q2, X2, y2 / d)):
            S0 = _weights(X0, (0, 0, 0), n)
            S1 = _weights(Y, (0, 0, 0), n)
            DS = [S1[a] - S0[a] for a in range(3)]
            for a in range(3):
                b, c = [k for k in range(3) if k != a]
                fac = (np.outer(S0[c], S0[b]) + 0.5 * np.outer(DS[c], S0[b]) + 0.5 * np.outer(S0[c], DS[b])
                       + np.outer(DS[c], DS[b]) / 3.0)          # [axis c][axis b]
                Wa = DS[a]
                start = int((np.floor(X0[a] + 0.5) + 3) % n[a])  # a node outside the support
                run = np.roll(np.cumsum(np.roll(Wa, -start)), start)
                contrib = -q * w * (d[a] / dt) * run            # along axis a
                # assemble the 3D array [z][y][x] from (a, b, c)
                arr = np.einsum("m,cb->mcb", contrib, fac)      # [a][c][b]
                axes = {a: 0, c: 1, b: 2}
                J[a] += np.transpose(arr, [axes[2], axes[1], axes[0]])
        out.append((y1, y2, v1n, v2n))
    B = [b - 0.5 * dt * c for b, c in zip(B, _curl_fwd(E, d))]
    E = [e + dt * (c - j) for e, c, j in zip(E, _curl_bwd(B, d), J)]
    return E, B, J, out


def test_whole_step_against_hand_expanded_reference():
    n = (8, 8, 8)
    d = np.array([0.5, 0.6, 0.7])
    dt = 0.2
    rng = np.random.default_rng(8)
    s = O.Sim(3, n, d, dt, [O.PERIODIC] * 3)
    sid = s.add_two_body(3.0, 2.0, synth.M_AU, 0.7, 12.4e-9, [3.0])
    xs = rng.uniform(0, 1, (2, 3)) * d * np.array(n)
    s.load(sid, xs, np.zeros((2, 3)))
    info = s.species_info(sid)
    ac = s.ac(sid)
    r = rng.normal(0, 0.3, (2, 3)) * d
    x1, x2 = xs, (xs - r) % (d * np.array(n))
    u1 = rng.normal(0, 0.3, (2, 3))
    u2 = rng.normal(0, 0.5, (2, 3))
    s.set_bodies(sid, x1=x1, x2=x2, u1=u1, u2=u2)
    for c in range(6):
        s.field(c)[...] = rng.normal(0, 0.05, s.field(c).shape)
    F = s.fields()
    E, B = [F[c].copy() for c in range(3)], [F[3 + c].copy() for c in range(3)]
    bodies = [(x1[k].copy(), x2[k].copy(), u1[k].copy(), u2[k].copy()) for k in range(2)]
    sp = (info["q1"], info["m1"], info["q2"], info["m2"], info["w"], info["kappa"], ac)
    L = d * np.array(n)
    for _ in range(2):
        E, B, J, bodies = _reference_step(E, B, bodies, sp, d, dt, n)
        s.step(1)
        F = s.fields()
        scale = max(np.abs(F[c]).max() for c in range(9))
        for c in range(3):
            assert np.abs(F[c] - E[c]).max() <= 1e-12 * scale
            assert np.abs(F[3 + c] - B[c]).max() <= 1e-12 * scale
            assert np.abs(F[6 + c] - J[c]).max() <= 1e-12 * scale
        ox1, ox2, ou1, ou2 = s.bodies(sid)
        for k in range(2):
            assert np.abs(_wrap(ox1[k] - bodies[k][0], L)).max() <= 1e-12 * L.max()
            assert np.abs(_wrap(ox2[k] - bodies[k][1], L)).max() <= 1e-12 * L.max()
            assert np.abs(ou1[k] - bodies[k][2]).max() <= 1e-12
            assert np.abs(ou2[k] - bodies[k][3]).max() <= 1e-12
    s.close()
