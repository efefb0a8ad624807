"""Pin of the oracle's adjoint inductance gradient: central finite differences
(relative step 1e-4) of full oracle solves, on a two-port structure."""
import numpy as np

import svh_synth as S
from oracle import adjoint as adj
from oracle import geometry as G
from oracle import solve as so


def _two_bars(lam):
    s = S.bar(10, 8, 3, 1, 8, 1, 2, 0, 1, lam=lam, sigma0=2e6)
    s2 = S.bar(10, 8, 3, 1, 8, 5, 6, 0, 1, lam=lam, sigma0=2e6)
    s.occ |= s2.occ
    s.lam += s2.lam
    s.sigma0 += s2.sigma0
    s.ports += s2.ports
    rng = np.random.default_rng(4)
    s.lam *= np.exp(rng.normal(0, 0.3, s.lam.shape))     # per-voxel lambda
    return s


def test_adjoint_gradient_matches_finite_differences():
    s = _two_bars(90e-9)
    f = 3e9
    gl, gs, res = adj.inductance_gradient(s, 0, 1, freq=f)
    g = res["grid"]
    vox = g.vox
    for k in [0, 5, 17, g.K - 1]:
        cell = np.unravel_index(vox[k], s.occ.shape)
        # sigma0 moves L ~1e-13 relative per 1e-4 step (the solve's noise floor): larger step there
        for name, arr, grad, rel, tol in (("lam", s.lam, gl, 1e-4, 1e-4), ("sigma0", s.sigma0, gs, 1e-2, 1e-3)):
            v0 = arr[cell]
            hstep = rel * v0
            arr[cell] = v0 + hstep
            Lp = so.port_inductance(s, freq=f, rre=1e-12)["L"][0, 1]
            arr[cell] = v0 - hstep
            Lm = so.port_inductance(s, freq=f, rre=1e-12)["L"][0, 1]
            arr[cell] = v0
            fd = (Lp - Lm) / (2 * hstep)
            assert abs(fd - grad[k]) <= tol * np.abs(grad).max(), (name, k, fd, grad[k])
    # a random direction over all voxels (directional derivative)
    rng = np.random.default_rng(9)
    d = rng.standard_normal(g.K)
    eps = 1e-4
    lam0 = s.lam.copy()
    flat = s.lam.reshape(-1)
    flat[vox] = lam0.reshape(-1)[vox] * (1 + eps * d)
    Lp = so.port_inductance(s, freq=f, rre=1e-12)["L"][0, 1]
    flat[vox] = lam0.reshape(-1)[vox] * (1 - eps * d)
    Lm = so.port_inductance(s, freq=f, rre=1e-12)["L"][0, 1]
    s.lam[...] = lam0
    fd = (Lp - Lm) / (2 * eps)
    an = np.sum(gl * lam0.reshape(-1)[vox] * d)
    assert abs(fd - an) <= 1e-5 * abs(an)
