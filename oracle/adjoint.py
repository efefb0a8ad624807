"""Gradient of the port impedance / inductance with respect to per-voxel lambda and sigma0 (oracle).

With Kt x_j = b_j the masked system of each port and Y_pj = c_p^T x_j the port
currents, the identity Kt^T = D Kt D (D = diag(I, -I): negating the continuity
rows makes Eq. 7 complex-symmetric) and c_p = b_p (both are A_T^T 1 on port
p's plus nodes) make the adjoint solutions equal the forward ones. Only the
diagonal two-fluid term z^beta_k = c_k s_beta / dx depends on the materials, so

    dY_pq / d lambda_k = - sum_beta x_p^(k,beta) x_q^(k,beta) dz^beta_k / d lambda_k,
    dZ = -Z dY Z  =>  dZ_ij / d lambda_k = sum_beta dz^beta_k/d lambda_k w_i^(k,beta) w_j^(k,beta),

with w_i = sum_p Z_ip x_p (I parts only), and dL = Im(dZ) / omega. The same holds
for sigma0 with dc/d sigma0 = -1/sigma^2.
"""
from __future__ import annotations

import numpy as np

from . import solve, twofluid


def inductance_gradient(structure, i, j, freq=None, rre=1e-12, res=None):
    """(dL_ij/dlambda[K], dL_ij/dsigma0[K], solve result) at one frequency."""
    if res is None:
        res = solve.port_inductance(structure, freq=freq, rre=rre)
    g = res["grid"]
    om = res["omega"]
    Z = res["Z"]
    K = g.K
    X = np.array([x[:5 * K].reshape(5, K) for x in res["x"]])      # [ports, 5, K]
    wi = np.tensordot(Z[i, :], X, axes=(0, 0))
    wj = np.tensordot(Z[:, j], X, axes=(0, 0))
    sb = twofluid.S_BETA[:, None] / g.dx
    dc_dlam = twofluid.dc_dlambda(om, g.lam, g.sigma0)
    sig = twofluid.sigma(om, g.lam, g.sigma0)
    dc_dsig = -1.0 / (sig * sig)
    dZ_lam = (sb * dc_dlam[None, :] * wi * wj).sum(0)
    dZ_sig = (sb * dc_dsig[None, :] * wi * wj).sum(0)
    return dZ_lam.imag / om, dZ_sig.imag / om, res
