"""Unit Green's-function kernels between two voxels (oracle, float64).

Every inductive block of Z (Eq. 8) is mu * dx * (a signed sum of seven unit
kernels) evaluated at the lattice offset d = n_obs - n_src. With the voxel
scaled to the unit cube (App. B, Eq. 24-27) and the basis moments expressed in
local coordinates xi in [-1/2, 1/2]^3, each kernel is the 6-D integral

    T(d) = int_{cube} int_{cube} p(xi) q(xi') G(d + xi - xi') dxi dxi',
    G(r) = 1 / (4 pi |r|)                                  (Eq. 1, Eq. 25)

whose polynomial weights p, q depend on one axis only. Substituting
u = xi - xi' folds it to a 3-D integral over u in [-1, 1]^3 with the
product of 1-D overlap weights

    w0(t) = 1 - |t|                   constant observer, constant source
    w1(t) = -t (1 - |t|) / 2          constant observer, source weight xi'
    w2(t) = 1/12 - |t|/4 + |t|^3/6    observer weight xi, source weight xi'

(an observer-linear, source-constant pair gives -w1). The seven kernels are

    G00 = w0 w0 w0;   S_a = w1 on axis a;   Q_a = w2 on axis a  (w0 elsewhere).

The Eq. 19 self integral and the Eq. 20-21 moment integrals are G00(0),
Q_x(0) + Q_y(0) and Q_x(0) + Q_y(0) + 4 Q_z(0) in these units (the sign of
Eq. 19 is taken as + so that the inductive Gram operator is positive).

Quadrature: [-1,1]^3 is split into its 8 unit octant boxes, on each of which
the weight is a polynomial. The integrand's only singular point u = -d is a
lattice point, so it is either a vertex of a box (then a Duffy map from that
vertex into three pyramids removes the 1/|u| singularity) or at sup-distance
>= 1 from it (then a tensor Gauss-Legendre rule converges geometrically).
"""
from __future__ import annotations

import numpy as np

KERNELS = ("G00", "Sx", "Sy", "Sz", "Qx", "Qy", "Qz")
# 1-D weight used on each axis (0: w0, 1: w1, 2: w2), per kernel
AXIS_WEIGHTS = (
    (0, 0, 0),
    (1, 0, 0), (0, 1, 0), (0, 0, 1),
    (2, 0, 0), (0, 2, 0), (0, 0, 2),
)
FOUR_PI = 4.0 * np.pi


def w0(t):
    a = np.abs(t)
    return 1.0 - a


def w1(t):
    a = np.abs(t)
    return -t * (1.0 - a) / 2.0


def w2(t):
    a = np.abs(t)
    return 1.0 / 12.0 - a / 4.0 + a ** 3 / 6.0


_W = (w0, w1, w2)


def kernel_weights(u):
    """Product weights of the 7 kernels at points u[..., 3] -> [7, ...]."""
    vals = [[_W[j](u[..., a]) for j in range(3)] for a in range(3)]
    out = np.empty((7,) + u.shape[:-1])
    for k, (jx, jy, jz) in enumerate(AXIS_WEIGHTS):
        out[k] = vals[0][jx] * vals[1][jy] * vals[2][jz]
    return out


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _box_nodes(n):
    """Tensor Gauss-Legendre nodes/weights on all 8 octant boxes of [-1,1]^3."""
    t, w = _gl01(n)
    pts, wts = [], []
    for sx in (-1.0, 1.0):
        for sy in (-1.0, 1.0):
            for sz in (-1.0, 1.0):
                X, Y, Z = np.meshgrid(sx * t, sy * t, sz * t, indexing="ij")
                W = w[:, None, None] * w[None, :, None] * w[None, None, :]
                pts.append(np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1))
                wts.append(W.ravel())
    return np.concatenate(pts), np.concatenate(wts)


def _gl_order(rinf):
    """Gauss-Legendre points per axis and box for offsets at sup-distance rinf.

    Chosen so that the error stays below 1e-13 of G00(d) (checked against a
    20-point rule in the tests); beyond rinf ~ 40 the linear-linear kernels
    reach the float64 cancellation floor of direct quadrature anyway."""
    if rinf <= 2:
        return 12
    if rinf <= 4:
        return 8
    if rinf <= 10:
        return 6
    if rinf <= 40:
        return 5
    return 4


def unit_kernels_at(d, n_duffy=16, n_gl=None):
    """The 7 unit kernels at one integer offset d = (dx, dy, dz) -> array[7].

    Near offsets (|d|_inf <= 1) use Duffy on the boxes that have u = -d as a
    vertex and Gauss-Legendre on the others; far offsets use Gauss-Legendre
    of an order that falls with distance (override with ``n_gl``)."""
    d = np.asarray(d, float)
    rinf = np.max(np.abs(d))
    n = _gl_order(rinf) if n_gl is None else n_gl
    total = np.zeros(7)
    t, w = _gl01(n)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    Wq = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                sg = np.array([sx, sy, sz], float)
                # box = {u : sg * u in [0,1]^3}; its vertex at the origin is 0,
                # the opposite one is sg. -d is a vertex iff sg*(-d) in {0,1}^3.
                vloc = sg * (-d)
                if np.all((vloc == 0.0) | (vloc == 1.0)):
                    # reflect so the singular vertex sits at the local origin
                    flip = np.where(vloc == 1.0, -1.0, 1.0)
                    # points u = -d + flip*sg*v, v in [0,1]^3  (inside the box)
                    total += _duffy_box_shift(d, flip * sg, n_duffy)
                else:
                    u = base * sg
                    r = np.linalg.norm(d + u, axis=-1)
                    total += kernel_weights(u) @ (Wq / r) / FOUR_PI
    return total


def _duffy_box_shift(d, dirs, n):
    """Duffy integral over the box with vertex -d, spanned along ``dirs``."""
    x, w = _gl01(n)
    S, T1, T2 = np.meshgrid(x, x, x, indexing="ij")
    Wq = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    S, T1, T2 = S.ravel(), T1.ravel(), T2.ravel()
    total = np.zeros(7)
    for a in range(3):
        b, c = [i for i in range(3) if i != a]
        v = np.empty((S.size, 3))
        v[:, a] = S
        v[:, b] = S * T1
        v[:, c] = S * T2
        u = -np.asarray(d, float) + v * dirs
        jac_over_r = S / np.sqrt(1.0 + T1 * T1 + T2 * T2)
        total += kernel_weights(u) @ (Wq * jac_over_r)
    return total / FOUR_PI


def toeplitz_signed(Kx, Ky, Kz, n_duffy=16):
    """All 7 kernels at every signed offset d in (-K, K)^3 -> [7, 2Kz-1, 2Ky-1, 2Kx-1].

    Index [k, dz + Kz - 1, dy + Ky - 1, dx + Kx - 1] holds kernel k at
    offset d. No parity is assumed: every offset is integrated directly."""
    ox, oy, oz = Kx - 1, Ky - 1, Kz - 1
    dz, dy, dx = np.meshgrid(np.arange(-oz, oz + 1), np.arange(-oy, oy + 1),
                             np.arange(-ox, ox + 1), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], -1).astype(float)
    return _toeplitz_from_offsets(D, n_duffy).reshape(7, 2 * Kz - 1, 2 * Ky - 1, 2 * Kx - 1)


def toeplitz_octant(Kx, Ky, Kz, n_duffy=16, processes=1):
    """The 7 kernels at non-negative offsets 0 <= d < K -> [7, Kz, Ky, Kx].

    processes > 1 integrates the z planes in that many worker processes
    (spawned, so it is safe in a process that already uses a GPU). Every
    offset is integrated on its own, so the result is the same to the bit."""
    if processes > 1 and Kz > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(processes, Kz)) as pool:
            planes = pool.starmap(_octant_plane, [(Kx, Ky, z, n_duffy) for z in range(Kz)])
        return np.stack(planes, axis=1)
    dz, dy, dx = np.meshgrid(np.arange(Kz), np.arange(Ky), np.arange(Kx), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], -1).astype(float)
    return _toeplitz_from_offsets(D, n_duffy).reshape(7, Kz, Ky, Kx)


def _octant_plane(Kx, Ky, z, n_duffy):
    """The 7 kernels at the offsets (0 <= dx < Kx, 0 <= dy < Ky, dz = z) -> [7, Ky, Kx]."""
    dy, dx = np.meshgrid(np.arange(Ky), np.arange(Kx), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), np.full(dx.size, z)], -1).astype(float)
    return _toeplitz_from_offsets(D, n_duffy).reshape(7, Ky, Kx)


def signed_from_octant(T):
    """Extend octant kernels [7, Kz, Ky, Kx] to signed offsets by their parity.

    G00 and Q_a are even in every axis; S_a is odd along a and even along the
    others (tested on directly integrated signed offsets)."""
    _, Kz, Ky, Kx = T.shape
    out = np.empty((7, 2 * Kz - 1, 2 * Ky - 1, 2 * Kx - 1))
    for k in range(7):
        odd = AXIS_WEIGHTS[k].index(1) if 1 in AXIS_WEIGHTS[k] else -1
        a = T[k]
        for ax, K in ((2, Kx), (1, Ky), (0, Kz)):
            neg = np.flip(np.take(a, np.arange(1, K), axis=ax), axis=ax)
            if odd == 2 - ax:
                neg = -neg
            a = np.concatenate([neg, a], axis=ax)
        out[k] = a
    return out


def kernels_at_offsets(D, n_duffy=16):
    """The 7 unit kernels at arbitrary integer offsets D[n, 3] (x, y, z) -> [7, n]."""
    return _toeplitz_from_offsets(np.asarray(D, float), n_duffy)


def _toeplitz_from_offsets(D, n_duffy):
    """Kernels at many integer offsets D[n, 3] -> [7, n]."""
    out = np.zeros((7, D.shape[0]))
    rinf = np.max(np.abs(D), axis=1)
    near = rinf <= 1
    for i in np.flatnonzero(near):
        out[:, i] = unit_kernels_at(D[i], n_duffy=n_duffy)
    orders = np.array([_gl_order(r) for r in rinf])
    for n in np.unique(orders[~near]):
        sel = np.flatnonzero((~near) & (orders == n))
        pts, wts = _box_nodes(int(n))
        cw = kernel_weights(pts) * wts  # [7, q]
        Ds = D[sel]
        acc = np.zeros((7, sel.size))
        for q in range(pts.shape[0]):
            r = np.sqrt(((Ds + pts[q]) ** 2).sum(-1))
            inv = 1.0 / r
            acc += cw[:, q:q + 1] * inv[None, :]
        out[:, sel] = acc / FOUR_PI
    return out
