"""Port solves of Eq. 7: GMRES(50) with the Schur-complement preconditioner (oracle).

Excitation (Sec. II.A; the entries of V and Phi are deferred to VoxHenry, so
this is the reading used here): for port j the nodes of its plus terminal get
Phi = 1, every other terminal node (its minus terminal, the terminals of the
other ports, and gauge nodes of floating islands) gets Phi = 0. Those known
potentials leave the unknowns: with T the terminal nodes and F the free ones,

    [ Z   -A_F^T ] [ I   ]   [ A_T^T Phi_T ]
    [ A_F   0    ] [Phi_F] = [      0      ].

Port current: I_p = sum over the plus nodes of port p of (A I)_m, the net
outward flux there; Y[p, j] = I_p under excitation j; Z_port = Y^{-1};
L = Im(Z_port) / omega.

Preconditioner (Eq. 12-15): P = Q^{-1}, Q = [Y, -A_F^T; A_F, 0] with Y =
diag(|Z_kk|). Apply: e = d - A_F Y^{-1} c, b = S^{-1} e with S = A_F Y^{-1} A_F^T,
a = Y^{-1}(c + A_F^T b). The oracle solves S exactly (sparse LU); the paper uses
AGMG there, which only changes the iteration count.

Solver (Sec. III): GMRES restarted every 50 iterations until the relative
residual ||b - K x|| / ||b|| <= rre (1e-8); right preconditioning and x0 = 0
are this reading's choices.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import geometry, operator, twofluid


class PortSystem:
    def __init__(self, grid, S7, P, omega, mu=twofluid.MU0, workers=-1):
        self.g = grid
        self.S7 = S7
        self.P = P
        self.omega = omega
        self.mu = mu
        self.workers = workers
        K, M = grid.K, grid.M
        self.term = geometry.terminal_nodes(grid)
        self.free = np.flatnonzero(~self.term)
        self.AF = grid.A[self.free].tocsr()
        self.AT = grid.A[np.flatnonzero(self.term)].tocsr()
        self.tidx = np.flatnonzero(self.term)
        # Y = |diag Z| including the Green self terms
        T0 = S7.real.sum(axis=(1, 2, 3)) / np.prod(P)   # kernels at offset 0 (inverse FFT at 0)
        self.T0 = T0
        zd = twofluid.zdiag(omega, grid.lam, grid.sigma0, grid.dx, mu)
        self_g = np.array([
            operator.BLOCKS[b, b] @ T0 for b in range(5)])
        diag = zd + 1j * omega * mu * grid.dx * self_g[:, None]
        self.Ydiag = np.abs(diag).ravel()
        Yinv = sp.diags(1.0 / self.Ydiag)
        self.S = (self.AF @ Yinv @ self.AF.T).tocsc()
        self.S_lu = spla.splu(self.S)
        self.n = 5 * K + self.free.size

    def matvec(self, xr):
        K, M = self.g.K, self.g.M
        full = np.zeros(5 * K + M, complex)
        full[:5 * K] = xr[:5 * K]
        full[5 * K + self.free] = xr[5 * K:]
        y = operator.apply_K_fft(self.g, self.S7, full, self.omega, self.P, self.mu, self.workers)
        return np.concatenate([y[:5 * K], y[5 * K + self.free]])

    def precond(self, v):
        K = self.g.K
        c = v[:5 * K]
        d = v[5 * K:]
        yi = 1.0 / self.Ydiag
        e = d - self.AF @ (yi * c)
        b = self.S_lu.solve(e.real.copy()) + 1j * self.S_lu.solve(e.imag.copy())
        a = yi * (c + self.AF.T @ b)
        return np.concatenate([a, b])

    def rhs(self, j):
        phiT = np.zeros(self.tidx.size)
        plus = np.isin(self.tidx, self.g.port_plus[j])
        phiT[plus] = 1.0
        bI = self.AT.T @ phiT
        return np.concatenate([bI.astype(complex), np.zeros(self.free.size, complex)])

    def port_currents(self, xr):
        K = self.g.K
        AI = self.g.A @ xr[:5 * K]
        return np.array([AI[p].sum() for p in self.g.port_plus])


def gmres(matvec, precond, b, restart=50, rre=1e-8, maxiter=5000):
    """Right-preconditioned restarted GMRES (Arnoldi with modified Gram-Schmidt,
    Givens rotations), x0 = 0. Returns (x, iterations, true relative residual)."""
    n = b.size
    x = np.zeros(n, complex)
    nb = np.linalg.norm(b)
    if nb == 0:
        return x, 0, 0.0
    it = 0
    while it < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / nb <= rre:
            return x, it, beta / nb
        V = np.zeros((restart + 1, n), complex)
        Zs = np.zeros((restart, n), complex)
        H = np.zeros((restart + 1, restart), complex)
        cs = np.zeros(restart, complex)
        sn = np.zeros(restart, complex)
        g = np.zeros(restart + 1, complex)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            Zs[k] = precond(V[k])
            w = matvec(Zs[k])
            for i in range(k + 1):
                H[i, k] = np.vdot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + np.conj(cs[i]) * H[i + 1, k]
                H[i, k] = t
            a, bb = H[k, k], H[k + 1, k]
            cs[k], sn[k] = _givens(a, bb)
            H[k, k] = cs[k] * a + sn[k] * bb
            H[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) / nb <= rre or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + Zs[:k_used].T @ y
    r = b - matvec(x)
    return x, it, np.linalg.norm(r) / nb


def _givens(a, b):
    """Complex Givens pair (c, s) with [c s; -conj(s) conj(c)] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0 + 0j, 0.0 + 0j
    if a == 0:
        return 0.0 + 0j, np.conj(b) / abs(b)
    t = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c + 0j, s


def port_inductance(structure, S7=None, P=None, freq=None, rre=1e-8, restart=50,
                    Tsigned=None, workers=-1):
    """Solve every port of ``structure`` at ``freq`` -> dict(Y, Z, L, iters, resid, x)."""
    g = geometry.build_grid(structure)
    if P is None:
        P = (operator.fft_size(g.Kx), operator.fft_size(g.Ky), operator.fft_size(g.Kz))
    if S7 is None:
        from . import greens
        T = Tsigned if Tsigned is not None else greens.toeplitz_signed(g.Kx, g.Ky, g.Kz)
        S7 = operator.spectra(T, P, workers)
    f = structure.freqs[0] if freq is None else freq
    omega = 2 * np.pi * f
    ps = PortSystem(g, S7, P, omega, workers=workers)
    npt = len(g.port_plus)
    Y = np.zeros((npt, npt), complex)
    iters, res, xs = [], [], []
    for j in range(npt):
        b = ps.rhs(j)
        x, it, rr = gmres(ps.matvec, ps.precond, b, restart=restart, rre=rre)
        Y[:, j] = ps.port_currents(x)
        iters.append(it)
        res.append(rr)
        xs.append(x)
    Zp = np.linalg.inv(Y)
    return dict(Y=Y, Z=Zp, L=Zp.imag / omega, R=Zp.real, iters=iters, resid=res, x=xs,
                system=ps, grid=g, omega=omega)
