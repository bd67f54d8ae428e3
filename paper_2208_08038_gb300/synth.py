"""Seeded synthetic inputs: the only module both the CUDA path's tests and the
FP64 oracle read.  It holds none of the PIC method's arithmetic (no species
split, no a_c mapping, no push or deposit): only random numbers, positions,
momenta and the workload descriptions.

Random numbers follow SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the finaliser is Stafford's
"Mix13" as published with it).  The generator is used counter-based: draw k of
stream (seed, s) is mix(key(seed, s) + (k + 1) * GOLDEN), so ion i's draws are
reproducible independently, by this module and by the library's device-side
generator, which implements the same published definition.

  uniform  u = (draw >> 11) * 2^-53            in [0, 1)
  normal   Box-Muller: sqrt(-2 ln(1 - u1)) cos(2 pi u2)

Units are normalised: c = 1, lengths in 1/k0 (lambda0 = 2 pi), times in
1/omega0 (T0 = 2 pi), fields in m_e c omega0 / e, densities in n_c.
"""
from __future__ import annotations

import dataclasses as dc
import math
from typing import Optional

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1

STREAM_POS, STREAM_JITTER, STREAM_MOM, STREAM_PARAM = 1, 2, 3, 4

TWO_PI = 2.0 * math.pi
LAMBDA0 = TWO_PI          # wavelength in normalised length units
T0 = TWO_PI               # laser period in normalised time units
M_AU = 197.0 * 1836.15267  # gold atom mass in m_e (reading of Sec. 3.1's Au example)


def _mix_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * MIX1) & MASK
    z = ((z ^ (z >> 27)) * MIX2) & MASK
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    """Key of one stream: mix(seed + stream * GOLDEN) folded with mix(seed)."""
    return _mix_int((_mix_int(seed & MASK) + (stream * GOLDEN)) & MASK)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def draws(key: int, counter: np.ndarray) -> np.ndarray:
    """64-bit draws number `counter` (uint64 array) of the stream `key`."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * np.uint64(GOLDEN)
    return _mix(z)


def uniform(key: int, counter: np.ndarray) -> np.ndarray:
    return (draws(key, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: int, counter_pair: np.ndarray) -> np.ndarray:
    """Box-Muller with uniforms number 2c and 2c+1."""
    c = np.asarray(counter_pair, dtype=np.uint64)
    u1 = uniform(key, c * np.uint64(2))
    u2 = uniform(key, c * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(TWO_PI * u2)


# ---------------------------------------------------------------------------
# particle loads

def medium(seed: int, D: int, dx, lo, hi, ppc: int, sigma_u: float = 0.0,
           first: int = 0, count: Optional[int] = None):
    """Ions at seeded uniform in-cell positions, ppc per cell, over the cell box
    [lo, hi) (x fastest).  Ion g (g = cell rank * ppc + p) takes uniforms
    3g + a for its position along axis a and normals 3g + a for its momentum.
    Returns (x [n, D], u [n, 3]) for ions first .. first + count."""
    ext = [hi[a] - lo[a] for a in range(D)]
    total = int(np.prod(ext)) * ppc
    if count is None:
        count = total - first
    g = np.arange(first, first + count, dtype=np.int64)
    cell = g // ppc
    x = np.empty((count, D))
    kp = stream_key(seed, STREAM_POS)
    rem = cell.copy()
    for a in range(D):
        c_a = rem % ext[a] + lo[a]
        rem //= ext[a]
        u = uniform(kp, (g * 3 + a).astype(np.uint64))
        x[:, a] = (c_a.astype(np.float64) + u) * dx[a]
    uc = np.zeros((count, 3))
    if sigma_u > 0:
        km = stream_key(seed, STREAM_MOM)
        for a in range(3):
            uc[:, a] = sigma_u * normal(km, (g * 3 + a).astype(np.uint64))
    return x, uc


def lattice(seed: int, sites: np.ndarray, per_site: int, jitter: float, sigma_u: float = 0.0):
    """per_site ions at every site (sites [ns, D]) with Gaussian jitter of
    standard deviation `jitter` per axis; ion g = site * per_site + p takes
    normals D*g + a."""
    sites = np.asarray(sites, dtype=np.float64)
    ns, D = sites.shape
    g = np.arange(ns * per_site, dtype=np.int64)
    x = np.repeat(sites, per_site, axis=0)
    if jitter > 0:
        kj = stream_key(seed, STREAM_JITTER)
        for a in range(D):
            x[:, a] += jitter * normal(kj, (g * D + a).astype(np.uint64))
    uc = np.zeros((len(g), 3))
    if sigma_u > 0:
        km = stream_key(seed, STREAM_MOM)
        for a in range(3):
            uc[:, a] = sigma_u * normal(km, (g * 3 + a).astype(np.uint64))
    return x, uc


def square_lattice(origin, d, counts):
    """Site (i, j) at origin + d (i + 1/2, j + 1/2), i fastest."""
    ii, jj = np.meshgrid(np.arange(counts[0]), np.arange(counts[1]), indexing="xy")
    return np.stack([origin[0] + d * (ii.ravel() + 0.5), origin[1] + d * (jj.ravel() + 0.5)], axis=1)


def uniform_params(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """n seeded values uniform in [lo, hi) (e.g. per-column omega_b)."""
    k = stream_key(seed, STREAM_PARAM)
    return lo + (hi - lo) * uniform(k, np.arange(n, dtype=np.uint64))


# ---------------------------------------------------------------------------
# workload descriptions

@dc.dataclass
class Laser:
    comp: int            # 1: current/field along y, 2: along z
    a0: float
    omega: float = 1.0
    theta: float = 0.0   # incidence angle in the x-y plane
    waist: float = 0.0   # 0: plane wave
    fwhm: float = 0.0    # intensity FWHM of the Gaussian envelope; 0: CW with sin^2 ramp
    t0: float = 0.0
    ramp: float = 0.0
    phase: float = 0.0
    ia: int = 2          # x node index of the antenna plane
    yc: float = 0.0
    zc: float = 0.0


@dc.dataclass
class TwoBody:
    Zb: float
    qc: float
    mc: float
    w: float                 # density weight per macro-ion [n_c]
    lambda0_m: float         # physical wavelength fixing kappa = r_e 2 pi / lambda0
    omega_b: np.ndarray      # bound-electron natural frequency per parameter index
    x: np.ndarray            # ion positions [n, D]
    u: np.ndarray            # ion momenta p_c/(m_c c) [n, 3]
    pidx: Optional[np.ndarray] = None


@dc.dataclass
class Free:
    q: float
    m: float
    w: float
    x: np.ndarray
    u: np.ndarray


@dc.dataclass
class Workload:
    name: str
    D: int
    n: tuple
    dx: tuple
    dt: float
    bc: tuple                # per axis: 0 periodic, 1 open
    steps: int
    species: list
    lasers: list
    tile: tuple
    probe_comp: int = 1
    probe_nodes: Optional[np.ndarray] = None   # linear node indices
    free_bounds: Optional[tuple] = None         # (lo[3], hi[3]) in cells
    meta: dict = dc.field(default_factory=dict)

    @property
    def n_ions(self) -> int:
        return sum(len(s.x) for s in self.species if isinstance(s, TwoBody))


def _lin(n, i, j=0, k=0):
    return i + n[0] * (j + n[1] * k)


def neutral_1d(ppc: int = 16, seed: int = 0, steps: int = 3000, nb: float = 0.01,
                    Zb: float = 1.0, omega_b: float = 3.0, slab=(8.0, 24.0), probe_x: float = 26.0,
                    vacuum: bool = False, nx: int = 2048, cells_per_lambda: int = 64) -> Workload:
    """1D neutral-medium propagation: 2048 cells, dx = lambda/64, dt = 0.95 dx,
    bound slab x in [8, 24) lambda, 16 ions/cell, cold, n_b = 0.01 n_c,
    omega_b = 3, a0 = 1e-3 Gaussian pulse of 10-cycle intensity FWHM."""
    dx = LAMBDA0 / cells_per_lambda
    lo, hi = int(slab[0] * cells_per_lambda), int(slab[1] * cells_per_lambda)
    x, u = medium(seed, 1, (dx,), (lo,), (hi,), ppc)
    sp = []
    if not vacuum:
        sp.append(TwoBody(Zb=Zb, qc=0.0, mc=M_AU, w=nb / Zb / ppc, lambda0_m=12.4e-9,
                          omega_b=np.array([omega_b]), x=x, u=u))
    fwhm = 10 * T0
    las = [Laser(comp=1, a0=1e-3, fwhm=fwhm, t0=1.5 * fwhm, ia=8)]
    n = (nx, 1, 1)
    probe = np.array([_lin(n, int(probe_x * cells_per_lambda))], dtype=np.int64)
    return Workload("neutral_1d", 1, (nx,), (dx,), 0.95 * dx, (1,), steps, sp, las,
                    tile=(16,), probe_comp=1, probe_nodes=probe,
                    meta=dict(slab=(lo, hi), ppc=ppc, nb=nb, omega_b=omega_b, Zb=Zb))


def bragg_2d(seed: int = 1, steps: int = 4000, n: int = 2048, cells_per_lambda: int = 32,
                  sites=(40, 40), theta_deg: float = 30.0, waist_lambda: float = 8.0,
                  fwhm_lambda: float = 19.0, nb: float = 0.01, omega_b: float = 4.0,
                  lattice_angle_deg: float = 0.0) -> Workload:
    """2D crystal Bragg scattering: 2048^2 cells, dx = lambda/32, square lattice
    of period d = lambda / (2 sin 30 deg) = lambda, 40x40 sites centred in the
    box, 4 ions per site, jitter 0.01 d, omega_b = 4, p-polarised Gaussian beam
    a0 = 1e-3, waist 8 lambda, incident at 30 deg."""
    dx = LAMBDA0 / cells_per_lambda
    L = n * dx
    d = LAMBDA0 / (2.0 * math.sin(math.radians(30.0)))
    origin = (0.5 * L - 0.5 * sites[0] * d, 0.5 * L - 0.5 * sites[1] * d)
    st = square_lattice(origin, d, sites)
    if lattice_angle_deg:
        a = math.radians(lattice_angle_deg)
        c0 = np.array([0.5 * L, 0.5 * L])
        R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        st = (st - c0) @ R.T + c0
    per_site = 4
    x, u = lattice(seed, st, per_site, 0.01 * d)
    w = nb * (d / dx) ** 2 / per_site
    sp = [TwoBody(Zb=1.0, qc=0.0, mc=M_AU, w=w, lambda0_m=0.26e-9, omega_b=np.array([omega_b]), x=x, u=u)]
    th = math.radians(theta_deg)
    ia = 8
    yc = 0.5 * L - (0.5 * L - ia * dx) * math.tan(th)
    fwhm = fwhm_lambda * T0
    las = [Laser(comp=1, a0=1e-3, theta=th, waist=waist_lambda * LAMBDA0, fwhm=fwhm, t0=1.5 * fwhm,
                 ia=ia, yc=yc)]
    dt = 0.95 * dx / math.sqrt(2.0)
    return Workload("bragg_2d", 2, (n, n), (dx, dx), dt, (1, 1), steps, sp, las, tile=(16, 16),
                    meta=dict(d=d, sites=sites, theta=th, origin=origin))


def neutral_3d(seed: int = 2, steps: int = 500, n=(512, 256, 256), cells_per_lambda: int = 16,
                    ppc: int = 8, nb: float = 0.02, omega_b: float = 3.0, sigma_u: float = 1e-3,
                    margin: int = 4, build_particles: bool = True) -> Workload:
    """3D neutral medium: 512x256x256 cells, dx = lambda/16, 8 ions per cell at
    seeded uniform positions (cells margin .. nx-margin along the open x
    axis; y, z periodic), thermal momenta sigma = 1e-3, omega_b = 3,
    n_b = 0.02 n_c, a0 = 1e-3 Gaussian pulse with waist 6 lambda."""
    dx = LAMBDA0 / cells_per_lambda
    lo, hi = (margin, 0, 0), (n[0] - margin, n[1], n[2])
    if build_particles:
        x, u = medium(seed, 3, (dx, dx, dx), lo, hi, ppc, sigma_u)
    else:
        x = np.zeros((0, 3)); u = np.zeros((0, 3))
    sp = [TwoBody(Zb=1.0, qc=0.0, mc=M_AU, w=nb / ppc, lambda0_m=12.4e-9, omega_b=np.array([omega_b]),
                  x=x, u=u)]
    fwhm = 10 * T0
    las = [Laser(comp=1, a0=1e-3, waist=6 * LAMBDA0, fwhm=fwhm, t0=1.5 * fwhm, ia=2,
                 yc=0.5 * n[1] * dx, zc=0.5 * n[2] * dx)]
    dt = 0.95 * dx / math.sqrt(3.0)
    return Workload("neutral_3d", 3, tuple(n), (dx, dx, dx), dt, (1, 0, 0), steps, sp, las,
                    tile=(8, 8, 8), meta=dict(seed=seed, lo=lo, hi=hi, ppc=ppc, sigma_u=sigma_u,
                                              nb=nb, omega_b=omega_b))


def adjoint_2d(seed: int = 3, target_seed: int = 33, steps: int = 400, n=(1024, 1024),
                    cells_per_lambda: int = 32, ppc: int = 8, nb: float = 0.01, slab=(2.0, 4.0),
                    sites_x: int = 4, probe_x: float = 6.0, target: bool = False) -> Workload:
    """2D adjoint workload: 1024^2 cells, dx = lambda/32, bound slab x in [2, 4)
    lambda, 8 ions per cell, per-column omega_b ~ U[2.5, 3.5] (1024 columns),
    ions grouped on 4 x 1024 lattice sites (each site's ions move rigidly with
    it), s-polarised CW wave, E_z probed on the line x = 6 lambda."""
    dx = LAMBDA0 / cells_per_lambda
    nx, ny = n
    lo, hi = int(slab[0] * cells_per_lambda), int(slab[1] * cells_per_lambda)
    wsite = (hi - lo) // sites_x
    per_site = ppc * wsite
    # site (a, j): centre of the wsite x 1 cell block
    a_idx, j_idx = np.meshgrid(np.arange(sites_x), np.arange(ny), indexing="xy")
    sites = np.stack([(lo + wsite * (a_idx.ravel() + 0.5)) * dx, (j_idx.ravel() + 0.5) * dx], axis=1)
    # ion offsets from their site: uniform over the site's block
    g = np.arange(len(sites) * per_site, dtype=np.int64)
    kp = stream_key(seed, STREAM_POS)
    off = np.stack([(uniform(kp, (g * 2).astype(np.uint64)) - 0.5) * wsite * dx,
                    (uniform(kp, (g * 2 + 1).astype(np.uint64)) - 0.5) * dx], axis=1)
    site_of_ion = g // per_site
    x = sites[site_of_ion] + off
    column = (site_of_ion // sites_x).astype(np.int32)
    omega = uniform_params(target_seed if target else seed, ny, 2.5, 3.5)
    sp = [TwoBody(Zb=1.0, qc=0.0, mc=M_AU, w=nb / ppc, lambda0_m=12.4e-9, omega_b=omega, x=x,
                  u=np.zeros((len(x), 3)), pidx=column)]
    las = [Laser(comp=2, a0=1e-3, ramp=2 * T0, ia=16)]
    dt = 0.95 * dx / math.sqrt(2.0)
    ip = int(probe_x * cells_per_lambda)
    probe = np.array([_lin((nx, ny, 1), ip, j) for j in range(ny)], dtype=np.int64)
    return Workload("adjoint_2d", 2, (nx, ny), (dx, dx), dt, (1, 0), steps, sp, las,
                    tile=(16, 16), probe_comp=2, probe_nodes=probe,
                    meta=dict(sites=sites, off=off, site_of_ion=site_of_ion, column=column,
                              per_site=per_site, omega=omega))


def ionized_crystal_2d(seed: int = 4, steps: int = 6000, n=(4096, 2048), cells_per_lambda: int = 32,
                            period_lambda: float = 0.6, span=(16.0, 112.0), e_ppc: int = 4,
                            ne: float = 0.1, Te_eV: float = 10.0, a0: float = 0.3,
                            build_particles: bool = True) -> Workload:
    """2D partially ionised crystal: 4096x2048 cells, dx = lambda/32, ion
    lattice of period 0.6 lambda (4 two-body ions per site, Z_b = 49,
    q_c = +30, omega_b = 4) plus free electrons, 4 per cell, n_e = 0.1 n_c,
    Maxwellian 10 eV, a0 = 0.3 pulse; both fill x in [16, 112) lambda."""
    dx = LAMBDA0 / cells_per_lambda
    nx, ny = n
    d = period_lambda * LAMBDA0
    Ly = ny * dx
    nsx = int(round((span[1] - span[0]) / period_lambda))
    nsy = int(Ly // d)
    st = square_lattice((span[0] * LAMBDA0, 0.0), d, (nsx, nsy))
    per_site = 4
    Zf = 30.0
    n_ion = ne / Zf
    w_ion = n_ion * (d / dx) ** 2 / per_site
    lo, hi = (int(span[0] * cells_per_lambda), 0), (int(span[1] * cells_per_lambda), ny)
    sigma = math.sqrt(Te_eV / 510998.95)
    if build_particles:
        xi, ui = lattice(seed, st, per_site, 0.0)
        xe, ue = medium(seed + 1000, 2, (dx, dx), lo, hi, e_ppc, sigma)
    else:
        xi = np.zeros((0, 2)); ui = np.zeros((0, 3)); xe = np.zeros((0, 2)); ue = np.zeros((0, 3))
    sp = [TwoBody(Zb=49.0, qc=Zf, mc=M_AU, w=w_ion, lambda0_m=0.26e-9, omega_b=np.array([4.0]), x=xi, u=ui),
          Free(q=-1.0, m=1.0, w=ne / e_ppc, x=xe, u=ue)]
    fwhm = 10 * T0
    las = [Laser(comp=1, a0=a0, fwhm=fwhm, t0=1.5 * fwhm, ia=8)]
    dt = 0.95 * dx / math.sqrt(2.0)
    return Workload("ionized_crystal_2d", 2, (nx, ny), (dx, dx), dt, (1, 0), steps, sp, las,
                    tile=(16, 16), free_bounds=((2.0, -1e300, -1e300), (nx - 2.0, 1e300, 1e300)),
                    meta=dict(sites=st, lo=lo, hi=hi, sigma=sigma))


# ---------------------------------------------------------------------------
# resonance scan (Sec. 3.1: group velocity and reflection phase against a_c)

N_AU_OVER_NC_12NM = 5.9e22 / (1.11485e21 / 0.0124 ** 2)  # Au atoms per n_c at 12.4 nm: 8.14e-3


def resonance_1d(omega_b: float, role: str = "transmit", seed: int = 6, ppc: int = 2,
                 cells_per_lambda: int = 64, nx: int = 2048, slab=None, probe_lambda: float = None,
                 fwhm_cycles: float = 5.0, a0: float = 1e-5, Zb: float = 78.0, steps: int = None,
                 vacuum: bool = False) -> Workload:
    """1D scan of Sec. 3.1's gold at 12.4 nm: two-body ions with Z_b = 78
    bound electrons and q_c = +1 (one free electron per atom, present as a
    free species at the same positions, so the slab starts neutral), atom
    density 5.9e22 cm^-3 = 8.14e-3 n_c, natural frequency omega_b (the a_c
    scan of Sec. 3.1 in the equivalent omega_b form).  Ions and electrons sit
    at regular sub-cell positions (ppc per cell, no jitter: a uniform medium).
    role "transmit": a 12 lambda slab from x = 4 lambda, the probe 4 lambda
    behind it (group velocity from the transmitted pulse); role "reflect": a
    4 lambda slab from x = 6 lambda, the probe 2 lambda in front of it
    (reflection phase from the reflected pulse).  vacuum: the same geometry
    without the medium (the reference trace).  An a0 = 1e-5 Gaussian pulse of
    fwhm_cycles intensity FWHM, E_y."""
    dx = LAMBDA0 / cells_per_lambda
    if slab is None:
        slab = (4.0, 16.0) if role == "transmit" else (6.0, 10.0)
    if probe_lambda is None:
        probe_lambda = slab[1] + 4.0 if role == "transmit" else slab[0] - 2.0
    lo, hi = int(round(slab[0] * cells_per_lambda)), int(round(slab[1] * cells_per_lambda))
    n_ion = N_AU_OVER_NC_12NM
    cells = np.arange(lo, hi)
    sub = (np.arange(ppc) + 0.5) / ppc
    x = ((cells[:, None] + sub[None, :]) * dx).reshape(-1, 1)
    u = np.zeros((len(x), 3))
    sp = []
    if not vacuum:
        sp.append(TwoBody(Zb=Zb, qc=1.0, mc=M_AU, w=n_ion / ppc, lambda0_m=12.4e-9,
                          omega_b=np.array([omega_b]), x=x, u=u))
        sp.append(Free(q=-1.0, m=1.0, w=n_ion / ppc, x=x.copy(), u=u.copy()))
    fwhm = fwhm_cycles * T0
    las = [Laser(comp=1, a0=a0, fwhm=fwhm, t0=1.5 * fwhm, ia=8)]
    dt = 0.95 * dx
    if steps is None:
        # the pulse has passed the probe even when the slab delays it by 2.5
        # times its length (group index up to 3.5)
        steps = int(round((1.5 * fwhm + probe_lambda * T0 + 3.0 * fwhm + 2.5 * (slab[1] - slab[0]) * T0) / dt))
    n = (nx, 1, 1)
    probe = np.array([_lin(n, int(round(probe_lambda * cells_per_lambda)))], dtype=np.int64)
    return Workload("resonance_1d", 1, (nx,), (dx,), dt, (1,), steps, sp, las, tile=(16,),
                    probe_comp=1, probe_nodes=probe,
                    free_bounds=((2.0, -1e300, -1e300), (nx - 2.0, 1e300, 1e300)),
                    meta=dict(slab=(lo, hi), n_ion=n_ion, omega_b=omega_b, Zb=Zb, role=role,
                              probe_x=probe[0] * dx, fwhm=fwhm, t0=1.5 * fwhm))


# ---------------------------------------------------------------------------
# oblique refraction (Sec. 3.1: gold at 56 nm, Z_b = 20, incidence pi/6)

N_AU_OVER_NC_56NM = 5.9e22 / (1.11485e21 / 0.056 ** 2)  # Au atoms per n_c at 56 nm: 0.166


def refraction_2d(omega_b: float = 2.0, n=(192, 160), cells_per_lambda: int = 16, surface_lambda: float = 3.0,
                  theta_deg: float = 30.0, waist_lambda: float = 2.0, fwhm_cycles: float = 3.0,
                  a0: float = 1e-5, Zb: float = 20.0, steps: int = None, vacuum: bool = False) -> Workload:
    """2D oblique refraction of Sec. 3.1's gold at 56 nm: two-body ions with
    Z_b = 20 and q_c = +1 plus one free electron per atom (at the same
    positions: the medium starts neutral), 5.9e22 atoms/cm^3 = 0.166 n_c,
    natural frequency omega_b, one ion (and one electron) per cell at the cell
    centre, filling x >= surface_lambda (to the open x face) over the
    periodic y extent.  An s-polarised (E_z) Gaussian pulse of intensity FWHM
    fwhm_cycles and waist waist_lambda, incident at theta_deg on the surface,
    aimed at the centre of the surface."""
    dx = LAMBDA0 / cells_per_lambda
    nx, ny = n
    lo = int(round(surface_lambda * cells_per_lambda))
    n_ion = N_AU_OVER_NC_56NM
    ii, jj = np.meshgrid(np.arange(lo, nx), np.arange(ny), indexing="xy")
    x = np.stack([(ii.ravel() + 0.5) * dx, (jj.ravel() + 0.5) * dx], axis=1)
    u = np.zeros((len(x), 3))
    sp = []
    if not vacuum:
        sp.append(TwoBody(Zb=Zb, qc=1.0, mc=M_AU, w=n_ion, lambda0_m=56e-9, omega_b=np.array([omega_b]),
                          x=x, u=u))
        sp.append(Free(q=-1.0, m=1.0, w=n_ion, x=x.copy(), u=u.copy()))
    th = math.radians(theta_deg)
    ia = 8
    Ly = ny * dx
    yc = 0.5 * Ly - (lo - ia) * dx * math.tan(th)
    fwhm = fwhm_cycles * T0
    las = [Laser(comp=2, a0=a0, theta=th, waist=waist_lambda * LAMBDA0, fwhm=fwhm, t0=1.5 * fwhm, ia=ia, yc=yc)]
    dt = 0.95 * dx / math.sqrt(2.0)
    if steps is None:
        # the pulse centre has gone some 7 lambda (vacuum path) past the surface
        steps = int(round((1.5 * fwhm + ((lo - ia) * dx / math.cos(th)) + 7.0 * LAMBDA0) / dt))
    return Workload("refraction_2d", 2, (nx, ny), (dx, dx), dt, (1, 0), steps, sp, las, tile=(16, 16),
                    free_bounds=((2.0, -1e300, -1e300), (nx - 2.0, 1e300, 1e300)),
                    meta=dict(surface=lo, n_ion=n_ion, omega_b=omega_b, Zb=Zb, theta=th))


def wakefield_2d(seed: int = 4, steps: int = 6000, n=(4096, 2048), span=(16.0, 112.0), a0: float = 3.0,
                 build_particles: bool = True) -> Workload:
    """The x-ray wakefield application of Sec. 3.2: the partially ionised
    crystal of ionized_crystal_2d (gold pre-ionised with 30 free electrons per
    ion, two-body ions with Z_b = 49 and q_c = +30 on a 0.6 lambda lattice,
    free electrons at 0.1 n_c, 10 eV) driven by an a0 = 3 pulse: the
    electrons' quiver is relativistic and the bound electrons are pulled far
    beyond a_c, so the whole modified Coulomb potential acts, not its
    harmonic core."""
    wl = ionized_crystal_2d(seed=seed, steps=steps, n=n, span=span, a0=a0, build_particles=build_particles)
    wl.name = "wakefield_2d"
    return wl
