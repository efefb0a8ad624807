"""Two-fluid conductivity and the diagonal (resistive + kinetic) terms (oracle).

Sec. II.A, Eq. 3:  sigma = sigma0 - j / (omega mu lambda^2)   (time factor e^{j omega t}).
App. A, Eq. 22-23: a = sigma0 (omega mu lambda^2)^2 / (1 + (sigma0 omega mu lambda^2)^2),
                   b = lambda^2 / (1 + (sigma0 omega mu lambda^2)^2),
so that 1/sigma = a + j omega mu b =: c.
Eq. 9 / Eq. 16-18: z^beta = c * s_beta / dx with s = (1, 1, 1, 1/6, 1/2) for
beta = x, y, z, 2D, 3D.
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi
S_BETA = np.array([1.0, 1.0, 1.0, 1.0 / 6.0, 0.5])


def sigma(omega, lam, sigma0, mu=MU0):
    """Eq. 3."""
    return sigma0 - 1j / (omega * mu * lam ** 2)


def ab(omega, lam, sigma0, mu=MU0):
    """Eq. 22-23: real a (ohm m) and b (m^2)."""
    t = sigma0 * omega * mu * lam ** 2
    den = 1.0 + t * t
    a = sigma0 * (omega * mu * lam ** 2) ** 2 / den
    b = lam ** 2 / den
    return a, b


def c_of(omega, lam, sigma0, mu=MU0):
    """c = a + j omega mu b (Eq. 9 text)."""
    a, b = ab(omega, lam, sigma0, mu)
    return a + 1j * omega * mu * b


def zdiag(omega, lam, sigma0, dx, mu=MU0):
    """z^beta per voxel -> [5, K] complex (Eq. 9)."""
    c = c_of(omega, np.asarray(lam, float), np.asarray(sigma0, float), mu)
    return S_BETA[:, None] * c[None, :] / dx


def dc_dlambda(omega, lam, sigma0, mu=MU0):
    """d c / d lambda with c = 1/sigma: -(1/sigma^2) d sigma/d lambda, d sigma/d lambda = 2j/(omega mu lambda^3)."""
    s = sigma(omega, lam, sigma0, mu)
    return -(2j / (omega * mu * lam ** 3)) / (s * s)
