"""Pins of the oracle's discrete adjoint.

Each reverse operator is checked against the forward operator it
transposes: linear operators by dot-product identities <A x, y> = <x, A^T y>,
non-linear ones (Boris, internal force, gather, Esirkepov) by central finite
differences of the forward function; the whole reverse pass by FP64 central
finite differences of the probe loss on the 1D neutral medium's grid (2048 cells).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_08038_gb300 import synth

RNG = np.random.default_rng(7)


def fd_grad(f, x, h):
    g = np.zeros_like(x)
    for i in range(x.size):
        e = np.zeros_like(x)
        e.flat[i] = h
        g.flat[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_boris_vjp_matches_finite_differences():
    q, m, dt = -1.0, 1.0, 0.1
    for _ in range(10):
        E, B, u = RNG.normal(size=3) * 0.5, RNG.normal(size=3) * 2.0, RNG.normal(size=3) * 0.8
        w = RNG.normal(size=3)
        ub0, Eb, Bb = O.boris_adj(q, m, dt, E, B, u, w)
        L = lambda uu, EE, BB: float(w @ O.boris(q, m, dt, EE, BB, uu))
        assert np.allclose(ub0, fd_grad(lambda x: L(x, E, B), u, 1e-6), rtol=1e-7, atol=1e-9)
        assert np.allclose(Eb, fd_grad(lambda x: L(u, x, B), E, 1e-6), rtol=1e-7, atol=1e-9)
        assert np.allclose(Bb, fd_grad(lambda x: L(u, E, x), B, 1e-6), rtol=1e-7, atol=1e-9)


def test_internal_field_vjp():
    for _ in range(10):
        q, kappa, ac = 2.0, 1.3e-3, 0.05
        d = RNG.normal(size=3) * 0.05
        w = RNG.normal(size=3)
        db, acb = O.internal_field_adj(q, kappa, ac, d, w)
        Ld = lambda x: float(w @ O.internal_field(q, kappa, ac, x))
        La = lambda a: float(w @ O.internal_field(q, kappa, a[0], d))
        assert np.allclose(db, fd_grad(Ld, d, 1e-7), rtol=1e-6, atol=1e-8)
        assert np.allclose(acb, fd_grad(La, np.array([ac]), 1e-8)[0], rtol=1e-6)


def test_dshape_is_derivative():
    for x in np.linspace(-1.7, 1.7, 69):
        assert abs(O.dshape(x) - (O.shape(x + 1e-6) - O.shape(x - 1e-6)) / 2e-6) < 1e-6


def _sim(D, bc, n=(12, 10, 8), dx=(0.3, 0.25, 0.2), dt=0.05):
    return O.Sim(D, n[:D], dx[:D], dt, bc[:D])


@pytest.mark.parametrize("D", [1, 2, 3])
def test_gather_adjoint(D):
    s = _sim(D, [O.OPEN, O.PERIODIC, O.PERIODIC])
    nn = s.n
    F = [RNG.normal(size=nn[::-1]) for _ in range(6)]
    for c in range(6):
        s.field(c)[...] = F[c]
    x = [RNG.uniform(3, s.n[a] - 4) * s.dx[a] for a in range(D)] + [0.0] * (3 - D)
    Eb, Bb = RNG.normal(size=3), RNG.normal(size=3)
    FE = [np.zeros(np.prod(nn)) for _ in range(3)]
    FB = [np.zeros(np.prod(nn)) for _ in range(3)]
    xb = O.gather_adj(s, x, Eb, Bb, FE, FB)

    def L(xx):
        X = [xx[a] / s.dx[a] for a in range(D)]
        return sum(Eb[c] * s.interp(c, X) + Bb[c] * s.interp(3 + c, X) for c in range(3))

    # field transpose: <G F, e> = <F, G^T e>
    lhs = L(np.array(x))
    rhs = sum((FE[c] * F[c].ravel()).sum() + (FB[c] * F[3 + c].ravel()).sum() for c in range(3))
    assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
    g = fd_grad(L, np.array(x), 1e-7)
    assert np.allclose(xb[:D], g[:D], rtol=1e-6, atol=1e-8)
    s.close()


@pytest.mark.parametrize("D", [1, 2, 3])
def test_deposit_adjoint(D):
    s = _sim(D, [O.PERIODIC] * 3, n=(14, 12, 10))
    nn = s.n
    lam = [RNG.normal(size=np.prod(nn)) for _ in range(3)]
    for _ in range(8):
        X0 = np.array([RNG.uniform(4, s.n[a] - 5) for a in range(D)])
        X1 = X0 + RNG.uniform(-0.6, 0.6, D)
        v = RNG.normal(size=3) * 0.3
        qw = -0.7

        def L(X0_, X1_, v_):
            for c in range(6, 9):
                s.field(c)[...] = 0
            s.deposit_one(qw, list(X0_), list(X1_), v_)
            return sum((s.field(6 + c).ravel() * lam[c]).sum() for c in range(3))

        X0b, X1b, vb = O.deposit_adj(s, qw, list(X0), list(X1), v, lam)
        assert np.allclose(X0b[:D], fd_grad(lambda x: L(x, X1, v), X0, 1e-7), rtol=1e-6, atol=1e-8)
        assert np.allclose(X1b[:D], fd_grad(lambda x: L(X0, x, v), X1, 1e-7), rtol=1e-6, atol=1e-8)
        assert np.allclose(vb, fd_grad(lambda x: L(X0, X1, x), v, 1e-6), rtol=1e-6, atol=1e-9)
    s.close()


@pytest.mark.parametrize("D,bc", [(1, [O.OPEN]), (2, [O.OPEN, O.OPEN]), (2, [O.OPEN, O.PERIODIC]),
                                  (3, [O.OPEN, O.PERIODIC, O.OPEN])])
def test_yee_adjoint_dot_products(D, bc):
    s = _sim(D, bc + [O.PERIODIC] * 2)
    nn = s.n
    N = int(np.prod(nn))
    E = [RNG.normal(size=N) for _ in range(3)]
    Bf = [RNG.normal(size=N) for _ in range(3)]
    J = [RNG.normal(size=N) for _ in range(3)]
    yE = [RNG.normal(size=N) for _ in range(3)]
    yB = [RNG.normal(size=N) for _ in range(3)]
    # B' = B - h curl E:  <B', yB> = <B, yB> + <E, (curl^T part)>
    for c in range(3):
        s.field(c).ravel()[:] = E[c]
        s.field(3 + c).ravel()[:] = Bf[c]
    h = 0.037
    s.yee_b(h)
    lhs = sum((s.field(3 + c).ravel() * yB[c]).sum() for c in range(3))
    Eb = O.yee_b_adj(s, h, [np.zeros(N)] * 3, yB)
    rhs = sum((Bf[c] * yB[c]).sum() + (E[c] * Eb[c]).sum() for c in range(3))
    assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    # E' = M(E, B, J) with Mur faces: <E', yE> = <E, Hn> + <B, Bb> + <J, Jb>
    for c in range(3):
        s.field(c).ravel()[:] = E[c]
        s.field(3 + c).ravel()[:] = Bf[c]
        s.field(6 + c).ravel()[:] = J[c]
    s.yee_e()
    lhs = sum((s.field(c).ravel() * yE[c]).sum() for c in range(3))
    Hn, Bb, Jb = O.yee_e_adj(s, yE, [np.zeros(N)] * 3)
    rhs = sum((E[c] * Hn[c]).sum() + (Bf[c] * Bb[c]).sum() + (J[c] * Jb[c]).sum() for c in range(3))
    assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    s.close()


# ---------------------------------------------------------------------------
# whole reverse pass against finite differences of the loss

def fd_problem(D=1):
    """The 1D neutral medium's grid (2048 cells, lambda/64), a short bound slab with
    8 parameter groups (per-group omega_b; the ions of a group form one
    'site' that moves rigidly), a short pulse and a probe behind the slab."""
    if D == 1:
        wl = synth.neutral_1d(ppc=2, slab=(6.0, 7.0), probe_x=8.0, nb=0.05)
        wl.lasers[0].fwhm = 2 * synth.T0
        wl.lasers[0].t0 = 2.0 * wl.lasers[0].fwhm
        steps = 900
    else:
        wl = synth.adjoint_2d(n=(128, 32), slab=(1.0, 1.5), probe_x=2.0, sites_x=2, nb=0.05)
        wl.lasers[0].ia = 8
        steps = 260
    sp = wl.species[0]
    n = len(sp.x)
    groups = 8
    sp.pidx = (np.arange(n) * groups // n).astype(np.int32)
    sp.omega_b = synth.uniform_params(3, groups, 2.5, 3.5)
    return wl, steps, groups


def build_oracle(wl, omega, shift=None):
    sp = wl.species[0]
    s = O.Sim(wl.D, wl.n, wl.dx, wl.dt, wl.bc)
    sid = s.add_two_body(sp.Zb, sp.qc, sp.mc, sp.w, sp.lambda0_m, omega)
    x = sp.x.copy()
    if shift is not None:
        x = x + shift
    s.load(sid, x, sp.u, sp.pidx)
    for L in wl.lasers:
        s.add_laser(L.comp, L.a0, L.omega, L.theta, L.waist, L.fwhm, L.t0, L.ramp, L.phase, L.ia, L.yc, L.zc)
    pid = s.add_probe(wl.probe_comp, wl.probe_nodes, 100000)
    return s, sid, pid


def run_loss(wl, steps, omega, target, shift=None):
    s, sid, pid = build_oracle(wl, omega, shift)
    a = O.Adjoint(s, sid)
    L, p = a.forward(steps, pid, target)
    a.close()
    s.close()
    return L, p


@pytest.mark.parametrize("D", [1, 2])
def test_adjoint_gradient_matches_finite_differences(D):
    wl, steps, groups = fd_problem(D)
    sp = wl.species[0]
    npts = len(wl.probe_nodes)
    om_true = synth.uniform_params(33, groups, 2.5, 3.5)
    _, target = run_loss(wl, steps, om_true, np.zeros((steps, npts)))
    om = sp.omega_b
    s, sid, pid = build_oracle(wl, om)
    a = O.Adjoint(s, sid)
    L0, _ = a.forward(steps, pid, target)
    g_om, g_x = a.backward(groups, len(sp.x))
    a.close()
    s.close()
    assert L0 > 0
    # omega_b per group
    for i in range(groups):
        h = 1e-6 * om[i]
        e = np.zeros(groups)
        e[i] = h
        Lp, _ = run_loss(wl, steps, om + e, target)
        Lm, _ = run_loss(wl, steps, om - e, target)
        fd = (Lp - Lm) / (2 * h)
        assert abs(g_om[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g_om).max()), (i, g_om[i], fd)
    # rigid shift of each group's ions (a 'site') along x
    for i in (0, groups // 2, groups - 1):
        sel = sp.pidx == i
        h = 1e-6 * np.abs(sp.x[sel, 0]).mean()  # 1e-6 of the site position
        d = np.zeros_like(sp.x)
        d[sel, 0] = h
        Lp, _ = run_loss(wl, steps, om, target, d)
        Lm, _ = run_loss(wl, steps, om, target, -d)
        fd = (Lp - Lm) / (2 * h)
        ad = g_x[sel, 0].sum()
        assert abs(ad - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(ad)), (i, ad, fd)
