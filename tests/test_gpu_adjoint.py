"""Adjoint gradient of a port inductance (row a11) on the GPU, through the C ABI
and through torch.autograd, against the oracle's adjoint gradient and central
finite differences (relative step 1e-4) of library solves."""
import numpy as np
import pytest

import svh_synth as S
from gpu_util import handle_for
from oracle import adjoint as adj

pytestmark = pytest.mark.gpu


def _two_bars():
    s = S.bar(10, 8, 3, 1, 8, 1, 2, 0, 1, lam=90e-9, sigma0=2e6)
    s2 = S.bar(10, 8, 3, 1, 8, 5, 6, 0, 1, lam=90e-9, sigma0=2e6)
    s.occ |= s2.occ
    s.lam += s2.lam
    s.sigma0 += s2.sigma0
    s.ports += s2.ports
    rng = np.random.default_rng(4)
    s.lam *= np.exp(rng.normal(0, 0.3, s.lam.shape))
    return s


OPTS = dict(rre=1e-12, inner_precision=1)


def test_gradient_matches_oracle_adjoint():
    s = _two_bars()
    f = 3e9
    gl_o, gs_o, ref = adj.inductance_gradient(s, 0, 1, freq=f)
    h = handle_for(s)
    res = h.solve([f], **OPTS)
    assert abs(res["L"][0, 0, 1] - ref["L"][0, 1]) <= 1e-8 * abs(ref["L"][0, 1])
    gl, gs = h.grad_inductance(0, 1)
    assert np.abs(gl - gl_o).max() <= 1e-6 * np.abs(gl_o).max()
    assert np.abs(gs - gs_o).max() <= 1e-6 * np.abs(gs_o).max()
    h.close()


def test_gradient_matches_library_finite_differences():
    s = _two_bars()
    f = 3e9
    h = handle_for(s)
    lam, sig = h.materials()
    h.solve([f], **OPTS)
    gl, _ = h.grad_inductance(1, 1)
    for k in (0, 7, 31, lam.size - 1):
        step = 1e-4 * lam[k]
        lp = lam.copy(); lp[k] += step
        lm = lam.copy(); lm[k] -= step
        h.set_materials(lp, sig)
        Lp = h.solve([f], **OPTS)["L"][0, 1, 1]
        h.set_materials(lm, sig)
        Lm = h.solve([f], **OPTS)["L"][0, 1, 1]
        fd = (Lp - Lm) / (2 * step)
        assert abs(fd - gl[k]) <= 1e-4 * np.abs(gl).max(), (k, fd, gl[k])
    h.close()


def test_torch_autograd_function():
    import torch

    from paper_2105_08627_gb300.autograd import port_inductance
    s = _two_bars()
    f = 3e9
    h = handle_for(s)
    lam0, sig0 = h.materials()
    lam = torch.tensor(lam0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sig0, dtype=torch.float64, requires_grad=True)
    L = port_inductance(lam, sig, h, f, 0, 1, **OPTS)
    L.backward()
    gl, gs = h.grad_inductance(0, 1)
    assert np.allclose(lam.grad.numpy(), gl, rtol=0, atol=1e-12 * np.abs(gl).max())
    # directional derivative through the Function
    rng = np.random.default_rng(2)
    d = torch.tensor(rng.standard_normal(lam0.size) * lam0 * 1e-4)
    with torch.no_grad():
        Lp = port_inductance(lam + d, sig, h, f, 0, 1, **OPTS)
        Lm = port_inductance(lam - d, sig, h, f, 0, 1, **OPTS)
    fd = (Lp - Lm).item() / 2
    an = float((lam.grad * d).sum())
    assert abs(fd - an) <= 1e-5 * abs(an)
    h.close()


@pytest.mark.slow
def test_two_meanders_128x128x16_gradient_spot_checks():
    """cfg 4 shape: dL12/dlambda by adjoint vs central differences on seeded voxels and directions."""
    s = S.pair_cfg4()
    f = 1e9
    h = handle_for(s)
    lam, sig = h.materials()
    opts = dict(rre=1e-11, inner_precision=1)
    h.solve([f], **opts)
    gl, _ = h.grad_inductance(0, 1)
    rng = np.random.default_rng(404)
    scale = np.abs(gl).max()
    top = np.argsort(-np.abs(gl))[:4]                     # voxels that matter most
    for k in list(top) + list(rng.choice(lam.size, 4, replace=False)):
        step = 1e-4 * lam[k]
        lp = lam.copy(); lp[k] += step
        lm = lam.copy(); lm[k] -= step
        h.set_materials(lp, sig)
        Lp = h.solve([f], **opts)["L"][0, 0, 1]
        h.set_materials(lm, sig)
        Lm = h.solve([f], **opts)["L"][0, 0, 1]
        assert abs((Lp - Lm) / (2 * step) - gl[k]) <= 1e-3 * scale
    for _ in range(2):
        d = rng.standard_normal(lam.size) * lam * 1e-4
        h.set_materials(lam + d, sig)
        Lp = h.solve([f], **opts)["L"][0, 0, 1]
        h.set_materials(lam - d, sig)
        Lm = h.solve([f], **opts)["L"][0, 0, 1]
        an = float(np.sum(gl * d))
        assert abs((Lp - Lm) / 2 - an) <= 1e-3 * abs(an)
    h.close()
