"""Pins for the oracle's unit Green's-function kernels (Eq. 19-21, App. B).

Each kernel value is checked against a route that shares no code with the
oracle's Duffy/Gauss-Legendre quadrature: the exact box-box integral of
1/|r - r'| (sixfold antiderivative), the unit-cube closed form, 1-D/2-D
integrals of box-box closed forms for the linear moments, far-field
multipole expansions, and parity.
"""
import numpy as np
import pytest

import closed_forms as cf
from oracle import greens as g


def test_cube_self_closed_form():
    # two independent closed forms of int int_{unit cube} 1/|r-r'| agree
    assert abs(cf.bar_self(1, 1, 1) - cf.CUBE_SELF) < 1e-13
    # Monte Carlo mean inverse distance (weak, independent of both)
    rng = np.random.default_rng(0)
    p, q = rng.random((2, 400000, 3))
    mc = np.mean(1.0 / np.linalg.norm(p - q, axis=1))
    assert abs(mc - cf.CUBE_SELF) < 0.01


def test_g00_self_term_matches_cube_closed_form():
    T = g.unit_kernels_at((0, 0, 0))
    assert abs(T[0] - cf.CUBE_SELF / (4 * np.pi)) < 1e-15


@pytest.mark.parametrize("d", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1),
                               (2, 0, 0), (2, 1, 0), (3, 2, 1), (0, 4, 2)])
def test_g00_matches_box_box_closed_form(d):
    T = g.unit_kernels_at(d)
    ref = cf.g00_closed(d, mpmode=max(map(abs, d)) > 2)   # float64 F cancels beyond |d| ~ 3
    assert abs(T[0] - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("d", [(11, 7, 3), (40, 3, 1), (65, 70, 20)])
def test_g00_far_closed_form_highprec(d):
    T = g.unit_kernels_at(d)
    ref = cf.g00_closed(d, mpmode=True)
    assert abs(T[0] - ref) <= 1e-11 * abs(ref)


@pytest.mark.parametrize("d", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (1, 1, 1), (2, 1, 0), (-1, 2, 1)])
def test_source_linear_kernels_match_closed_form_integral(d):
    T = g.unit_kernels_at(d)
    for a in range(3):
        ref = cf.s_closed(d, a)
        assert abs(T[1 + a] - ref) <= 1e-13 * T[0], (a, T[1 + a], ref)   # scale: the integrand's size


@pytest.mark.parametrize("d", [(0, 0, 0), (1, 0, 0), (0, 1, 1)])
def test_linear_linear_kernels_match_closed_form_integral(d):
    T = g.unit_kernels_at(d)
    for a in range(3):
        ref = cf.q_closed(d, a)
        assert abs(T[4 + a] - ref) <= 1e-11 * abs(ref), (a, T[4 + a], ref)


def _grad_G(d):
    """Derivatives of G = 1/(4 pi r) needed by the far-field expansions."""
    d = np.asarray(d, float)
    r = np.linalg.norm(d)
    G = 1 / (4 * np.pi * r)
    g1 = -d / (4 * np.pi * r ** 3)
    H = (3 * np.outer(d, d) / r ** 5 - np.eye(3) / r ** 3) / (4 * np.pi)
    g3 = np.zeros(3)   # d^3 G / d a^3
    for a in range(3):
        x = d[a]
        g3[a] = (-15 * x ** 3 / r ** 7 + 9 * x / r ** 5) / (4 * np.pi)
    return G, g1, H, g3


@pytest.mark.parametrize("d", [(30, 20, 10), (-25, 40, 7), (60, -5, 33)])
def test_far_field_expansions(d):
    # with m2(w0) = 1/6, m1(w1) = -1/12, m3(w1) = -1/30, m2(w2) = -1/72 and
    # harmonicity of G: G00 = G + O(r^-5), S_a = -G_a/12 + G_aaa/720 + O(r^-6),
    # Q_a = -G_aa/144 + O(r^-5)
    T = g.unit_kernels_at(d)
    G, g1, H, g3 = _grad_G(d)
    r = np.linalg.norm(d)
    assert abs(T[0] - G) <= 0.05 * G / r ** 4
    for a in range(3):
        s_ref = -g1[a] / 12 + g3[a] / 720
        assert abs(T[1 + a] - s_ref) <= 0.05 * G / r ** 5
        q_ref = -H[a, a] / 144
        assert abs(T[4 + a] - q_ref) <= 0.05 * G / r ** 4


def test_parity_of_directly_integrated_signed_offsets():
    Ts = g.toeplitz_signed(4, 5, 3)
    for k in range(7):
        ax_w = g.AXIS_WEIGHTS[k]
        for ax, arr_ax in ((0, 2), (1, 1), (2, 0)):
            flipped = np.flip(Ts[k], axis=arr_ax)
            sgn = -1.0 if ax_w[ax] == 1 else 1.0
            assert np.allclose(flipped, sgn * Ts[k], rtol=0, atol=1e-14 * np.abs(Ts[k]).max()), (k, ax)
    # octant + parity reproduces the direct signed integration
    To = g.toeplitz_octant(4, 5, 3)
    assert np.allclose(g.signed_from_octant(To), Ts, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d", [(2, 0, 0), (2, 2, 1), (3, 0, 0), (4, 1, 0), (5, 0, 0), (10, 3, 2), (11, 0, 0),
                               (40, 1, 0), (41, 0, 0), (200, 7, 3)])
def test_gauss_legendre_order_converged(d):
    a = g.unit_kernels_at(d)
    b = g.unit_kernels_at(d, n_gl=20)
    scale = np.abs(b[0])
    assert np.max(np.abs(a - b)) <= 1e-13 * scale


def test_duffy_order_converged():
    for d in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)]:
        a = g.unit_kernels_at(d)
        b = g.unit_kernels_at(d, n_duffy=28)
        assert np.max(np.abs(a - b)) <= 1e-16


def test_direct_six_dimensional_block_entries():
    """Blocks of Z from the basis definitions (Eq. 4-6 with Eq. 16-18 normalisation)
    by a direct 6-D Gauss-Legendre rule on two separated voxels, against the
    oracle's block table. Pins the table's signs, axes and transposes."""
    from oracle import operator as op
    n = 6
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * x
    w = 0.5 * w
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()

    def comps(beta, xi):   # basis component polynomials (unit-free, times dx^2)
        one = np.ones(len(xi))
        zero = np.zeros(len(xi))
        return {0: (one, zero, zero), 1: (zero, one, zero), 2: (zero, zero, one),
                3: (xi[:, 0], -xi[:, 1], zero), 4: (xi[:, 0], xi[:, 1], -2 * xi[:, 2])}[beta]

    for d in [(3, 1, 2), (-2, 3, 4)]:
        d = np.asarray(d, float)
        R = d[None, None, :] + X[:, None, :] - X[None, :, :]
        Gm = 1.0 / (4 * np.pi * np.linalg.norm(R, axis=-1))
        WW = W[:, None] * W[None, :]
        T = g.unit_kernels_at(d)
        for b in range(5):
            for a in range(5):
                pb = comps(b, X)
                pa = comps(a, X)
                val = sum(np.sum(WW * Gm * pb[i][:, None] * pa[i][None, :]) for i in range(3))
                ref = op.BLOCKS[b, a] @ T
                assert abs(val - ref) <= 1e-9 * abs(T[0]), (d, b, a, val, ref)
