"""Closed forms used to pin the oracle (test helper; not part of the oracle).

F(x, y, z) is a sixfold antiderivative of 1/r (d^2/dx^2 d^2/dy^2 d^2/dz^2 F = 1/r),
the function behind the published exact partial-inductance formula of a
rectangular bar (Hoer and Love, 1965; Ruehli, 1972). For two boxes the double
volume integral of 1/|r - r'| is a signed sum of F over the 64 differences of
their corner coordinates: along one axis,

    int_{a1}^{a2} int_{b1}^{b2} f(x - x') dx' dx = Phi(a2-b1) - Phi(a1-b1) - Phi(a2-b2) + Phi(a1-b2)

for any Phi with Phi'' = f. The unit cube's self integral also has the short
closed form 2 [(1 + sqrt2 - 2 sqrt3)/5 - pi/3 + ln((1 + sqrt2)(2 + sqrt3))].
"""
from __future__ import annotations

import itertools

import mpmath as mp
import numpy as np

CUBE_SELF = 2.0 * ((1 + np.sqrt(2.0) - 2 * np.sqrt(3.0)) / 5 - np.pi / 3
                   + np.log((1 + np.sqrt(2.0)) * (2 + np.sqrt(3.0))))


def cube_self_mp():
    return 2 * ((1 + mp.sqrt(2) - 2 * mp.sqrt(3)) / 5 - mp.pi / 3
                + mp.log((1 + mp.sqrt(2)) * (2 + mp.sqrt(3))))


def F(x, y, z):
    """Sixfold antiderivative of 1/r, float64, vectorised."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    r = np.sqrt(x * x + y * y + z * z)

    def L(a, b, c):
        rho = np.sqrt(b * b + c * c)
        coef = b * b * c * c / 4 - b ** 4 / 24 - c ** 4 / 24
        with np.errstate(divide="ignore", invalid="ignore"):
            v = coef * a * np.arcsinh(np.where(rho > 0, a / np.where(rho > 0, rho, 1), 0.0))
        return np.where(rho > 0, v, 0.0)

    def T(a, b, c):
        with np.errstate(divide="ignore", invalid="ignore"):
            v = a * b * c ** 3 / 6 * np.arctan(a * b / (c * r))
        return np.where((a != 0) & (b != 0) & (c != 0), v, 0.0)

    return (L(x, y, z) + L(y, x, z) + L(z, x, y)
            + (x ** 4 + y ** 4 + z ** 4 - 3 * x * x * y * y - 3 * y * y * z * z - 3 * x * x * z * z) * r / 60
            - T(x, y, z) - T(y, z, x) - T(z, x, y))


def F_mp(x, y, z):
    """Same antiderivative in mpmath (for offsets where float64 cancellation bites)."""
    x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
    r = mp.sqrt(x * x + y * y + z * z)

    def L(a, b, c):
        if b == 0 and c == 0:
            return mp.mpf(0)
        return (b * b * c * c / 4 - b ** 4 / 24 - c ** 4 / 24) * a * mp.asinh(a / mp.sqrt(b * b + c * c))

    def T(a, b, c):
        if a == 0 or b == 0 or c == 0:
            return mp.mpf(0)
        return a * b * c ** 3 / 6 * mp.atan(a * b / (c * r))

    return (L(x, y, z) + L(y, x, z) + L(z, x, y)
            + (x ** 4 + y ** 4 + z ** 4 - 3 * x * x * y * y - 3 * y * y * z * z - 3 * x * x * z * z) * r / 60
            - T(x, y, z) - T(y, z, x) - T(z, x, y))


def _axis_terms(a1, a2, b1, b2):
    return ((a2 - b1, 1.0), (a1 - b1, -1.0), (a2 - b2, -1.0), (a1 - b2, 1.0))


def box_box(obs, src, Ffun=F):
    """int_obs int_src 1/|r - r'| for boxes given as ((x1,x2),(y1,y2),(z1,z2)).

    Vectorised over array-valued endpoints when ``Ffun`` is the float64 F."""
    tx = _axis_terms(obs[0][0], obs[0][1], src[0][0], src[0][1])
    ty = _axis_terms(obs[1][0], obs[1][1], src[1][0], src[1][1])
    tz = _axis_terms(obs[2][0], obs[2][1], src[2][0], src[2][1])
    total = 0.0
    for (X, sx), (Y, sy), (Z, sz) in itertools.product(tx, ty, tz):
        total = total + sx * sy * sz * Ffun(X, Y, Z)
    return total


def unit_box(center):
    return tuple((c - 0.5, c + 0.5) for c in center)


def g00_closed(d, mpmode=False):
    """G00(d) = (1/4pi) int_{cube(d)} int_{cube(0)} 1/|r - r'|."""
    if mpmode:
        with mp.workdps(40):
            v = box_box(unit_box([mp.mpf(t) for t in d]), unit_box([mp.mpf(0)] * 3), F_mp)
            return float(v / (4 * mp.pi))
    return float(box_box(unit_box(d), unit_box((0.0, 0.0, 0.0))) / (4 * np.pi))


def tanh_sinh(h=1.0 / 16, tmax=3.2):
    """Double-exponential nodes/weights on [-1/2, 1/2] (robust to endpoint singularities)."""
    tau = np.arange(-tmax, tmax + h / 2, h)
    u = 0.5 * np.pi * np.sinh(tau)
    x = 0.5 * np.tanh(u)
    w = h * 0.5 * (0.5 * np.pi * np.cosh(tau)) / np.cosh(u) ** 2
    keep = np.abs(x) < 0.5
    return x[keep], w[keep]


def s_closed(d, axis):
    """S_axis(d) = int int xi'_a G(d + xi - xi'), written with xi' = int_{-1/2}^{1/2} (1[t < xi'] - 1/2) dt
    as a 1-D integral over t of closed-form box-box integrals."""
    t, w = tanh_sinh()
    obs = unit_box(d)
    full = unit_box((0.0, 0.0, 0.0))
    src = [list(full[0]), list(full[1]), list(full[2])]
    src[axis] = (t, np.full_like(t, 0.5))
    part = box_box(obs, src)
    whole = box_box(obs, full)
    return float(np.sum(w * (part - 0.5 * whole)) / (4 * np.pi))


def q_closed(d, axis):
    """Q_axis(d) = int int xi_a xi'_a G(d + xi - xi') via the same indicator form in both xi and xi'.

    The 2-D integrand over (s, t) is non-smooth on the diagonal s = t (the two
    restricted boxes share an endpoint there), so the square is split into its
    two triangles, each mapped to have that line on its boundary."""
    x, wx = tanh_sinh()
    v = x + 0.5
    total = 0.0
    for lower in (True, False):
        A, V = np.meshgrid(x, v, indexing="ij")
        W = wx[:, None] * wx[None, :] * (0.5 - A)
        B = A + (0.5 - A) * V
        S, T = (A, B) if lower else (B, A)
        total += np.sum(W * _q_integrand(d, axis, S, T))
    return float(total / (4 * np.pi))


def _q_integrand(d, axis, S, T):
    full_o = unit_box(d)
    full_s = unit_box((0.0, 0.0, 0.0))
    o = [full_o[0], full_o[1], full_o[2]]
    sr = [full_s[0], full_s[1], full_s[2]]
    o_r = list(o)
    o_r[axis] = (d[axis] + S, np.full_like(S, d[axis] + 0.5))
    s_r = list(sr)
    s_r[axis] = (T, np.full_like(T, 0.5))
    both = box_box(o_r, s_r)
    o_only = box_box(o_r, sr)
    s_only = box_box(o, s_r)
    whole = box_box(o, sr)
    return both - 0.5 * o_only - 0.5 * s_only + 0.25 * whole


def bar_self(a, b, c):
    """int int over an a x b x c box of 1/|r - r'| (exact)."""
    return float(box_box(((0, a), (0, b), (0, c)), ((0, a), (0, b), (0, c))))
