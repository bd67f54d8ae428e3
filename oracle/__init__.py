"""FP64 CPU oracle for the two-body macro-ion PIC step (arXiv 2208.08038).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the
product path (``paper_2208_08038_gb300``) never imports it, and it imports
nothing from there.  The arithmetic lives in ``bp_oracle.c`` (plain C, FP64);
this module compiles it with gcc on first use and wraps it with ctypes.

Functions without an independent pin are listed in ``UNPINNED``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "bp_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# every oracle function is pinned by at least one -m "not gpu" test; see
# tests/test_oracle_pins.py and tests/test_oracle_adjoint.py
UNPINNED: tuple[str, ...] = ()

PERIODIC, OPEN = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP on independent per-cell loops)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_d, _i, _l, _p = C.c_double, C.c_int, C.c_long, C.c_void_p
_i64 = C.c_int64


def _declare(L: C.CDLL) -> None:
    sig = {
        "or_create": (_p, [_i, _p, _p, _d, _p]),
        "or_destroy": (None, [_p]),
        "or_field_ptr": (C.POINTER(_d), [_p, _i]),
        "or_ncell": (_l, [_p]),
        "or_step_index": (_i64, [_p]),
        "or_set_switches": (None, [_p, _i, _i]),
        "or_set_free_bounds": (None, [_p, _p, _p]),
        "or_omega_to_ac": (_d, [_d, _d, _d, _d, _d, _d]),
        "or_add_two_body": (_i, [_p, _d, _d, _d, _d, _d, _p, _i]),
        "or_add_free": (_i, [_p, _d, _d, _d]),
        "or_species_info": (None, [_p, _i, _p]),
        "or_species_ac": (_d, [_p, _i, _i]),
        "or_set_omega": (None, [_p, _i, _p, _i]),
        "or_load_ions": (_i, [_p, _i, _i64, _p, _p, _p]),
        "or_get_bodies": (None, [_p, _i, _p, _p, _p, _p]),
        "or_set_bodies": (None, [_p, _i, _p, _p, _p, _p]),
        "or_get_alive": (None, [_p, _i, _p]),
        "or_add_laser": (_i, [_p, _p]),
        "or_add_probe": (_i, [_p, _i, _i64, _p, _i64]),
        "or_probe_data": (_i64, [_p, _i, _p]),
        "or_shape": (_d, [_d]),
        "or_interp": (_d, [_p, _i, _p]),
        "or_internal_field": (None, [_d, _d, _d, _p, _p]),
        "or_boris": (None, [_d, _d, _d, _p, _p, _p]),
        "or_deposit_one": (None, [_p, _d, _p, _p, _p]),
        "or_yee_b": (None, [_p, _d]),
        "or_yee_e": (None, [_p]),
        "or_step": (None, [_p, _i]),
        "or_rho": (None, [_p, _p]),
        "or_residual": (None, [_p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    adj = {
        "or_dshape": (_d, [_d]),
        "or_boris_adj": (None, [_d, _d, _d, _p, _p, _p, _p, _p, _p, _p]),
        "or_internal_field_adj": (_d, [_d, _d, _d, _p, _p, _p]),
        "or_gather_adj": (None, [_p, _p, _p, _p, _p, _p, _p]),
        "or_deposit_adj": (None, [_p, _d, _p, _p, _p, _p, _p, _p, _p]),
        "or_yee_b_adj": (None, [_p, _d, _p, _p]),
        "or_yee_e_adj": (None, [_p, _p, _p, _p, _p]),
        "ora_create": (_p, [_p, _i]),
        "ora_destroy": (None, [_p]),
        "ora_forward": (_d, [_p, _i, _i, _p, _p, _i64]),
        "ora_backward": (None, [_p, _p, _p]),
    }
    for name, (res, args) in adj.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# thin functional wrappers of the single-operation entry points

def shape(xi: float) -> float:
    """Quadratic B-spline S(xi)."""
    return lib().or_shape(float(xi))


def omega_to_ac(q1, m1, q2, m2, kappa, omega) -> float:
    """a_c from the natural frequency w_c^2 = |q1 q2| kappa / (m_r a_c^3) (Sec. 3.1)."""
    return lib().or_omega_to_ac(q1, m1, q2, m2, kappa, omega)


def internal_field(q_other, kappa, ac, d) -> np.ndarray:
    d = f64(d)
    out = np.zeros(3)
    lib().or_internal_field(q_other, kappa, ac, _ptr(d), _ptr(out))
    return out


def boris(q, m, dt, E, B, u) -> np.ndarray:
    E, B, u = f64(E), f64(B), f64(u).copy()
    lib().or_boris(q, m, dt, _ptr(E), _ptr(B), _ptr(u))
    return u


RE = 2.8179403262e-15  # classical electron radius [m], CODATA 2018


class Sim:
    """FP64 PIC state: Yee fields, two-body ion and free-particle species."""

    def __init__(self, D: int, n, dx, dt: float, bc):
        self._L = lib()
        n3 = (C.c_long * 3)(*(list(n) + [1] * (3 - len(n))))
        dx3 = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
        bc3 = (C.c_int * 3)(*(list(bc) + [0] * (3 - len(bc))))
        self.D = D
        self.n = tuple(int(v) for v in n3)
        self.dx = tuple(float(v) for v in dx3)
        self.dt = dt
        self._s = self._L.or_create(D, n3, dx3, dt, bc3)
        if not self._s:
            raise ValueError("bad grid")
        self._keep = []

    def close(self):
        if self._s:
            self._L.or_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # fields ---------------------------------------------------------------
    def field(self, comp: int) -> np.ndarray:
        """View (nz, ny, nx) of field component comp (0..8: E, B, J)."""
        ptr = self._L.or_field_ptr(self._s, comp)
        nx, ny, nz = self.n
        return np.ctypeslib.as_array(ptr, shape=(nz * ny * nx,)).reshape(nz, ny, nx)

    def fields(self) -> np.ndarray:
        return np.stack([self.field(c).copy() for c in range(9)])

    def set_switches(self, fields_on=True, deposit_on=True):
        self._L.or_set_switches(self._s, int(fields_on), int(deposit_on))

    def set_free_bounds(self, lo, hi):
        lo3 = (C.c_double * 3)(*lo)
        hi3 = (C.c_double * 3)(*hi)
        self._L.or_set_free_bounds(self._s, lo3, hi3)

    # species --------------------------------------------------------------
    def add_two_body(self, Zb, qc, mc, w, lambda0_m, omega_b) -> int:
        om = f64(np.atleast_1d(omega_b))
        self._keep.append(om)
        sid = self._L.or_add_two_body(self._s, Zb, qc, mc, w, lambda0_m, _ptr(om), len(om))
        if sid < 0:
            raise ValueError("cannot add species")
        return sid

    def add_free(self, q, m, w) -> int:
        return self._L.or_add_free(self._s, q, m, w)

    def species_info(self, sid) -> dict:
        out = np.zeros(8)
        self._L.or_species_info(self._s, sid, _ptr(out))
        return dict(q1=out[0], m1=out[1], q2=out[2], m2=out[3], w=out[4], kappa=out[5],
                    nac=int(out[6]), n=int(out[7]))

    def ac(self, sid, i=0) -> float:
        return self._L.or_species_ac(self._s, sid, i)

    def set_omega(self, sid, omega_b):
        om = f64(np.atleast_1d(omega_b))
        self._L.or_set_omega(self._s, sid, _ptr(om), len(om))

    def load(self, sid, xc, uc=None, pidx=None):
        xc = f64(xc)
        n = xc.shape[0]
        uc = None if uc is None else f64(uc)
        pidx = None if pidx is None else np.ascontiguousarray(pidx, dtype=np.int32)
        rc = self._L.or_load_ions(self._s, sid, n, _ptr(xc), _ptr(uc), _ptr(pidx))
        if rc:
            raise ValueError("species already loaded")

    def bodies(self, sid):
        n = self.species_info(sid)["n"]
        x1, x2, u1, u2 = (np.zeros((n, 3)) for _ in range(4))
        self._L.or_get_bodies(self._s, sid, _ptr(x1), _ptr(x2), _ptr(u1), _ptr(u2))
        return x1, x2, u1, u2

    def set_bodies(self, sid, x1=None, x2=None, u1=None, u2=None):
        arrs = [None if a is None else f64(a) for a in (x1, x2, u1, u2)]
        self._L.or_set_bodies(self._s, sid, *[_ptr(a) for a in arrs])

    def alive(self, sid) -> np.ndarray:
        n = self.species_info(sid)["n"]
        out = np.zeros(n, dtype=np.uint8)
        self._L.or_get_alive(self._s, sid, _ptr(out))
        return out

    # lasers / probes ------------------------------------------------------
    def add_laser(self, comp, a0, omega=1.0, theta=0.0, waist=0.0, fwhm=0.0, t0=0.0, ramp=0.0,
                  phase=0.0, ia=2, yc=0.0, zc=0.0) -> int:
        p = f64([comp, a0, omega, theta, waist, fwhm, t0, ramp, phase, ia, yc, zc])
        return self._L.or_add_laser(self._s, _ptr(p))

    def add_probe(self, comp: int, idx, cap: int) -> int:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        return self._L.or_add_probe(self._s, comp, len(idx), _ptr(idx), cap)

    def probe(self, pid: int, npts: int) -> np.ndarray:
        cnt = self._L.or_probe_data(self._s, pid, None)
        out = np.zeros((cnt, npts))
        self._L.or_probe_data(self._s, pid, _ptr(out))
        return out

    # operations -----------------------------------------------------------
    def interp(self, comp: int, X) -> float:
        X = f64(list(X) + [0.0] * (3 - len(X)))
        return self._L.or_interp(self._s, comp, _ptr(X))

    def deposit_one(self, qw, X0, X1, v):
        X0 = f64(list(X0) + [0.0] * (3 - len(X0)))
        X1 = f64(list(X1) + [0.0] * (3 - len(X1)))
        v = f64(v)
        self._L.or_deposit_one(self._s, qw, _ptr(X0), _ptr(X1), _ptr(v))

    def yee_b(self, h: float):
        self._L.or_yee_b(self._s, h)

    def yee_e(self):
        self._L.or_yee_e(self._s)

    def step(self, n: int = 1):
        self._L.or_step(self._s, int(n))

    @property
    def step_index(self) -> int:
        return int(self._L.or_step_index(self._s))

    def rho(self) -> np.ndarray:
        nx, ny, nz = self.n
        out = np.zeros(nx * ny * nz)
        self._L.or_rho(self._s, _ptr(out))
        return out.reshape(nz, ny, nx)

    def residual(self) -> np.ndarray:
        nx, ny, nz = self.n
        out = np.zeros(nx * ny * nz)
        self._L.or_residual(self._s, _ptr(out))
        return out.reshape(nz, ny, nx)


# ---------------------------------------------------------------------------
# adjoint

def _ptrs3(arrs):
    """C array of three double* for a list of three float64 arrays."""
    P = (C.c_void_p * 3)(*[a.ctypes.data for a in arrs])
    return P


def boris_adj(q, m, dt, E, B, u0, ubn):
    E, B, u0, ubn = f64(E), f64(B), f64(u0), f64(ubn)
    ub0, Eb, Bb = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().or_boris_adj(q, m, dt, _ptr(E), _ptr(B), _ptr(u0), _ptr(ubn), _ptr(ub0), _ptr(Eb), _ptr(Bb))
    return ub0, Eb, Bb


def internal_field_adj(q_other, kappa, ac, d, Eb):
    d, Eb = f64(d), f64(Eb)
    db = np.zeros(3)
    acb = lib().or_internal_field_adj(q_other, kappa, ac, _ptr(d), _ptr(Eb), _ptr(db))
    return db, acb


def dshape(x: float) -> float:
    return lib().or_dshape(float(x))


class Adjoint:
    """Forward run with stored states, then the discrete reverse pass."""

    def __init__(self, sim: "Sim", sid: int):
        self.sim = sim
        self._o = lib().ora_create(sim._s, sid)

    def forward(self, nsteps: int, pid: int, target: np.ndarray) -> tuple:
        target = f64(target)
        npts = target.shape[1]
        out = np.zeros((nsteps, npts))
        L = lib().ora_forward(self._o, nsteps, pid, _ptr(target), _ptr(out), npts)
        return L, out

    def backward(self, nac: int, n: int):
        go = np.zeros(nac)
        gx = np.zeros((n, 3))
        lib().ora_backward(self._o, _ptr(go), _ptr(gx))
        return go, gx

    def close(self):
        if self._o:
            lib().ora_destroy(self._o)
            self._o = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather_adj(sim: "Sim", x, Eb, Bb, FEb=None, FBb=None):
    x, Eb, Bb = f64(list(x) + [0.0] * (3 - len(x))), f64(Eb), f64(Bb)
    xb = np.zeros(3)
    pe = _ptrs3(FEb) if FEb is not None else None
    pb = _ptrs3(FBb) if FBb is not None else None
    lib().or_gather_adj(sim._s, _ptr(x), _ptr(Eb), _ptr(Bb), pe, pb, _ptr(xb))
    return xb


def deposit_adj(sim: "Sim", qw, X0, X1, v, lam):
    X0 = f64(list(X0) + [0.0] * (3 - len(X0)))
    X1 = f64(list(X1) + [0.0] * (3 - len(X1)))
    v = f64(v)
    lam = [f64(l).ravel() for l in lam]
    X0b, X1b, vb = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().or_deposit_adj(sim._s, qw, _ptr(X0), _ptr(X1), _ptr(v), _ptrs3(lam), _ptr(X0b), _ptr(X1b), _ptr(vb))
    return X0b, X1b, vb


def yee_b_adj(sim: "Sim", h, Eb, Bb):
    Eb = [f64(a).ravel().copy() for a in Eb]
    Bb = [f64(a).ravel() for a in Bb]
    lib().or_yee_b_adj(sim._s, h, _ptrs3(Eb), _ptrs3(Bb))
    return Eb


def yee_e_adj(sim: "Sim", G, Bb):
    G = [f64(a).ravel().copy() for a in G]
    Bb = [f64(a).ravel().copy() for a in Bb]
    n = G[0].size
    Hn = [np.zeros(n) for _ in range(3)]
    Jb = [np.zeros(n) for _ in range(3)]
    lib().or_yee_e_adj(sim._s, _ptrs3(G), _ptrs3(Hn), _ptrs3(Bb), _ptrs3(Jb))
    return Hn, Bb, Jb
