"""The Eq. 7 operator: dense Z (Eq. 8) and the FFT-accelerated product (Eq. 9), oracle.

Z_{(beta,l),(alpha,k)} = delta_{lk} delta_{beta alpha} z^beta_k
                         + j omega mu dx * sum_u BLOCKS[beta][alpha][u] T_u(n_l - n_k)

with the seven unit kernels T_u of ``oracle.greens``. The block table follows
from the basis components (x: 1 on x; 2D: xi_x on x, -xi_y on y; 3D: xi_x on
x, xi_y on y, -2 xi_z on z) and reproduces the zero pattern of Eq. 8:

            x        y        z        2D             3D
    x     G00       .        .        Sx             Sx
    y      .       G00       .       -Sy             Sy
    z      .        .       G00        .            -2Sz
    2D   -Sx       Sy        .       Qx+Qy          Qx-Qy
    3D   -Sx      -Sy      2Sz       Qx-Qy        Qx+Qy+4Qz

Eq. 9: each block product is a 3-D convolution over the grid; embedding the
Toeplitz kernel in a circulant of size P_i >= 2K_i - 1 (C[i] = T(i) for
0 <= i < K, C[P - i] = T(-i) for 1 <= i < K, zero elsewhere) turns it into a
cyclic convolution evaluated by FFTs:

    CC^beta = z^beta I^beta + j omega mu dx * IFFT{ sum_alpha Zhat^{beta alpha} * FFT{I^alpha} }.

The full operator (Eq. 7) is [Z, -A^T; A, 0] acting on [I; Phi].
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp

from . import greens, twofluid

# BLOCKS[beta][alpha] = 7-vector of coefficients on (G00, Sx, Sy, Sz, Qx, Qy, Qz)
BLOCKS = np.zeros((5, 5, 7))
_G, _SX, _SY, _SZ, _QX, _QY, _QZ = range(7)
BLOCKS[0, 0, _G] = BLOCKS[1, 1, _G] = BLOCKS[2, 2, _G] = 1.0
BLOCKS[0, 3, _SX] = 1.0
BLOCKS[0, 4, _SX] = 1.0
BLOCKS[1, 3, _SY] = -1.0
BLOCKS[1, 4, _SY] = 1.0
BLOCKS[2, 4, _SZ] = -2.0
BLOCKS[3, 0, _SX] = -1.0
BLOCKS[3, 1, _SY] = 1.0
BLOCKS[4, 0, _SX] = -1.0
BLOCKS[4, 1, _SY] = -1.0
BLOCKS[4, 2, _SZ] = 2.0
BLOCKS[3, 3, _QX] = BLOCKS[3, 3, _QY] = 1.0
BLOCKS[3, 4, _QX] = 1.0
BLOCKS[3, 4, _QY] = -1.0
BLOCKS[4, 3, _QX] = 1.0
BLOCKS[4, 3, _QY] = -1.0
BLOCKS[4, 4, _QX] = BLOCKS[4, 4, _QY] = 1.0
BLOCKS[4, 4, _QZ] = 4.0


def fft_size(K, smooth=(2, 3, 5, 7)):
    """Smallest P >= 2K - 1 with only the given prime factors, preferring 2K (Sec. II.A uses 2K)."""
    def ok(n):
        for p in smooth:
            while n % p == 0:
                n //= p
        return n == 1
    if ok(2 * K):
        return 2 * K
    n = 2 * K - 1
    while not ok(n):
        n += 1
    return n


def dense_Z(grid, Tsigned, omega, mu=twofluid.MU0):
    """Dense 5K x 5K Z (Eq. 8) from kernels at signed offsets (brute force, tiny grids)."""
    K = grid.K
    Kx, Ky, Kz = grid.Kx, grid.Ky, grid.Kz
    d = grid.pos[:, None, :] - grid.pos[None, :, :]              # obs - src
    T = Tsigned[:, d[..., 2] + Kz - 1, d[..., 1] + Ky - 1, d[..., 0] + Kx - 1]  # [7, K, K]
    Z = np.zeros((5 * K, 5 * K), complex)
    scale = 1j * omega * mu * grid.dx
    for b in range(5):
        for a in range(5):
            blk = np.tensordot(BLOCKS[b, a], T, axes=(0, 0))
            Z[b * K:(b + 1) * K, a * K:(a + 1) * K] = scale * blk
    zd = twofluid.zdiag(omega, grid.lam, grid.sigma0, grid.dx, mu)
    Z[np.arange(5 * K), np.arange(5 * K)] += zd.ravel()
    return Z


def dense_K(grid, Tsigned, omega, mu=twofluid.MU0):
    """Dense Eq. 7 operator [Z, -A^T; A, 0]."""
    Z = dense_Z(grid, Tsigned, omega, mu)
    A = grid.A.toarray()
    M = grid.M
    top = np.hstack([Z, -A.T])
    bot = np.hstack([A, np.zeros((M, M))])
    return np.vstack([top, bot])


def circulant(Tsigned, P):
    """Embed signed-offset kernels [7, 2Kz-1, 2Ky-1, 2Kx-1] in circulants [7, Pz, Py, Px]."""
    _, nz, ny, nx = Tsigned.shape
    Kz, Ky, Kx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
    Px, Py, Pz = P
    C = np.zeros((7, Pz, Py, Px))
    ix = np.concatenate([np.arange(Kx), Px - np.arange(1, Kx)])
    dxs = np.concatenate([np.arange(Kx), -np.arange(1, Kx)])
    iy = np.concatenate([np.arange(Ky), Py - np.arange(1, Ky)])
    dys = np.concatenate([np.arange(Ky), -np.arange(1, Ky)])
    iz = np.concatenate([np.arange(Kz), Pz - np.arange(1, Kz)])
    dzs = np.concatenate([np.arange(Kz), -np.arange(1, Kz)])
    C[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]] = \
        Tsigned[:, (dzs + Kz - 1)[:, None, None], (dys + Ky - 1)[None, :, None], (dxs + Kx - 1)[None, None, :]]
    return C


def spectra(Tsigned, P, workers=-1):
    """FFT of the 7 circulants -> complex [7, Pz, Py, Px] (the tensors Zhat of Eq. 9)."""
    return sfft.fftn(circulant(Tsigned, P), axes=(1, 2, 3), workers=workers)


def block_spectra(S7):
    """Zhat^{beta alpha} = sum_u BLOCKS[beta][alpha][u] * spectrum_u -> [5, 5, Pz, Py, Px]."""
    return np.tensordot(BLOCKS, S7, axes=(2, 0))


def apply_Z_fft(grid, S7, I, omega, P, mu=twofluid.MU0, workers=-1, Zh=None):
    """Z @ I via Eq. 9 (I: [5K] or [5, K] complex) -> [5, K].

    Zh: the block spectra block_spectra(S7), when the caller has formed them
    already (they depend on the kernels only); None forms them here."""
    K = grid.K
    I = np.asarray(I, complex).reshape(5, K)
    Px, Py, Pz = P
    grids = np.zeros((5, Pz, Py, Px), complex)
    x, y, z = grid.pos[:, 0], grid.pos[:, 1], grid.pos[:, 2]
    grids[:, z, y, x] = I
    Ihat = sfft.fftn(grids, axes=(1, 2, 3), workers=workers)
    if Zh is None:
        Zh = block_spectra(S7)
    Yhat = np.einsum("bapqr,apqr->bpqr", Zh, Ihat)
    Y = sfft.ifftn(Yhat, axes=(1, 2, 3), workers=workers)[:, z, y, x]
    zd = twofluid.zdiag(omega, grid.lam, grid.sigma0, grid.dx, mu)
    return zd * I + 1j * omega * mu * grid.dx * Y


def apply_K_fft(grid, S7, xvec, omega, P, mu=twofluid.MU0, workers=-1, Zh=None):
    """Eq. 7 operator on x = [I (5K); Phi (M)] using the FFT product for Z
    (Zh: optional pre-formed block spectra, as in apply_Z_fft)."""
    K, M = grid.K, grid.M
    xvec = np.asarray(xvec, complex)
    I = xvec[:5 * K]
    Phi = xvec[5 * K:]
    top = apply_Z_fft(grid, S7, I, omega, P, mu, workers, Zh).ravel() - grid.A.T @ Phi
    bot = grid.A @ I
    return np.concatenate([top, bot])


def direct_rows(grid, x, omega, vox_rows, node_rows, mu=twofluid.MU0):
    """Selected rows of the Eq. 7 product by direct summation (no FFT), for any x.

    vox_rows: voxel indices l (all five basis rows of each are returned,
    shape [5, len]); node_rows: node indices m (rows of A I). The sum runs
    only over the non-zero entries of x, so sparse inputs are cheap at any
    grid size."""
    K, M = grid.K, grid.M
    x = np.asarray(x, complex)
    I = x[:5 * K].reshape(5, K)
    Phi = x[5 * K:]
    supp = np.flatnonzero(np.any(I != 0, axis=0))
    vox_rows = np.asarray(vox_rows)
    d = grid.pos[vox_rows][:, None, :] - grid.pos[supp][None, :, :]          # obs - src
    T = greens.kernels_at_offsets(d.reshape(-1, 3)).reshape(7, vox_rows.size, supp.size)
    out = np.zeros((5, vox_rows.size), complex)
    scale = 1j * omega * mu * grid.dx
    for b in range(5):
        for a in range(5):
            coef = BLOCKS[b, a]
            if not coef.any():
                continue
            blk = np.tensordot(coef, T, axes=(0, 0))                      # [rows, supp]
            out[b] += scale * (blk @ I[a, supp])
    zd = twofluid.zdiag(omega, grid.lam[vox_rows], grid.sigma0[vox_rows], grid.dx, mu)
    out += zd * I[:, vox_rows]
    AT = grid.A.T.tocsr()
    for b in range(5):
        out[b] -= AT[b * K + vox_rows] @ Phi
    nodes = grid.A.tocsr()[np.asarray(node_rows)] @ x[:5 * K]
    return out, nodes


def direct_rows_table(grid, T, x, omega, vox_rows, node_rows, mu=twofluid.MU0):
    """Selected rows of the Eq. 7 product by direct summation over every voxel,
    with the unit kernels taken from a table instead of integrated per pair.

    T: the kernels at the non-negative offsets, [7, Kz, Ky, Kx]
    (greens.toeplitz_octant); a signed offset d reads T at |d|, negated for
    S_a when d_a < 0 (S_a is odd along a, every other kernel even). x: [N]
    or [nb, N]. Returns ([nb, 5, len(vox_rows)], [nb, len(node_rows)]) for a
    2-D x, else the shapes of direct_rows. The cost is O(rows * K), so dense
    inputs stay cheap at any grid size."""
    K = grid.K
    x = np.asarray(x, complex)
    one = x.ndim == 1
    X = np.atleast_2d(x)
    nb = X.shape[0]
    I = X[:, :5 * K].reshape(nb, 5, K)
    Phi = X[:, 5 * K:]
    vox_rows = np.asarray(vox_rows)
    out = np.zeros((nb, 5, vox_rows.size), complex)
    scale = 1j * omega * mu * grid.dx
    for i, l in enumerate(vox_rows):
        d = grid.pos[l][None, :] - grid.pos                        # obs - src, [K, 3]
        a = np.abs(d)
        Tl = T[:, a[:, 2], a[:, 1], a[:, 0]]                         # [7, K]
        for u, ax in ((1, 0), (2, 1), (3, 2)):                       # S_x, S_y, S_z
            Tl[u] = np.where(d[:, ax] < 0, -Tl[u], Tl[u])
        for b in range(5):
            for al in range(5):
                coef = BLOCKS[b, al]
                if coef.any():
                    out[:, b, i] += scale * (I[:, al, :] @ (coef @ Tl))
    zd = twofluid.zdiag(omega, grid.lam[vox_rows], grid.sigma0[vox_rows], grid.dx, mu)   # [5, rows]
    out += zd[None] * I[:, :, vox_rows]
    AT = grid.A.T.tocsr()
    for b in range(5):
        out[:, b, :] -= (AT[b * K + vox_rows] @ Phi.T).T
    nodes = (grid.A.tocsr()[np.asarray(node_rows)] @ X[:, :5 * K].T).T
    if one:
        return out[0], nodes[0]
    return out, nodes
