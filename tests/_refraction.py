"""Refraction at an oblique incidence (Sec. 3.1), written from the paper
(test infrastructure): Snell's law with the model's sqrt(eps_r), its discrete
form on the 2D Yee grid, and the measurement of the refracted wave vector
from the oracle's fields.  Units: c = 1, omega0 = 1."""
import math

import numpy as np


def snell_angle(theta_i, eps):
    """sin(theta_t) = sin(theta_i) / sqrt(eps_r)."""
    return math.asin(math.sin(theta_i) / math.sqrt(eps))


def yee_refraction_angle(theta_i, dx, dt, chi_fn, w=1.0, iters=80):
    """The refracted wave vector's angle on the 2D Yee grid: k_y = w sin(theta_i)
    (the antenna's phase along y) is conserved; k_x solves
    (2/dx)^2 [sin^2(k_x dx/2) + sin^2(k_y dx/2)] = W^2 (1 + S^2 chi(W)),
    W = (2/dt) sin(w dt/2), S = sinc^3(k_x dx/2) sinc^3(k_y dx/2)."""
    W = 2.0 / dt * math.sin(w * dt / 2.0)
    ky = w * math.sin(theta_i)
    sinc = lambda z: math.sin(z) / z if z else 1.0
    sy = math.sin(ky * dx / 2) ** 2
    kx = w
    for _ in range(iters):
        S = (sinc(kx * dx / 2) * sinc(ky * dx / 2)) ** 3
        rhs = (dx / 2) ** 2 * W * W * (1 + S * S * chi_fn(W)) - sy
        kx = 2.0 / dx * math.asin(math.sqrt(rhs))
    return math.atan2(ky, kx)


def lockin(frames, dt, w=1.0):
    """sum_s E_s exp(i w t_s), t_s = (s + 1) dt: the complex amplitude of the
    exp(-i w t) component at every cell."""
    A = np.zeros(frames[0].shape, dtype=np.complex128)
    for s, f in enumerate(frames):
        A += np.asarray(f, dtype=np.float64) * np.exp(1j * w * (s + 1) * dt)
    return A


def wavevector(A, dx, x0, x1):
    """(k_x, k_y) of the wave in columns [x0, x1) of the amplitude A[y, x]:
    the phase differences between neighbouring cells, weighted by |A|^2."""
    B = A[:, x0:x1]
    gx = B[:, 1:] * np.conj(B[:, :-1])
    gy = np.roll(B, -1, axis=0) * np.conj(B)  # y is periodic
    kx = np.angle(gx.sum()) / dx
    ky = np.angle(gy.sum()) / dx
    return kx, ky
