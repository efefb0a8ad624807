"""Pins for the oracle's two-fluid terms, incidence, operator, Tucker-SVD and solver.

Every check compares the oracle with something other than itself: a second
formula, a closed form, brute force, a direct dense solve, or an invariant
that the paper's equations imply.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import closed_forms as cf
import svh_synth as S
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op
from oracle import solve as so
from oracle import tucker as tk
from oracle import twofluid as tf

MU = tf.MU0


# ---------------------------------------------------------------- two-fluid (Eq. 3, 22-23)
def test_two_fluid_identity():
    rng = np.random.default_rng(1)
    lam = rng.uniform(20e-9, 500e-9, 50)
    s0 = rng.uniform(0, 1e8, 50)
    om = 2 * np.pi * rng.uniform(1e6, 1e11, 50)
    c = tf.c_of(om, lam, s0)
    inv_sigma = 1.0 / tf.sigma(om, lam, s0)
    assert np.allclose(c, inv_sigma, rtol=1e-13, atol=0)


def test_two_fluid_limits():
    om = 2 * np.pi * 1e9
    lam = 90e-9
    # no normal channel: purely kinetic, 1/sigma = j omega mu lambda^2
    assert np.isclose(tf.c_of(om, lam, 0.0), 1j * om * MU * lam ** 2, rtol=1e-14)
    # lambda -> infinity: normal conductor 1/sigma0
    assert np.isclose(tf.c_of(om, 1e3, 1e7), 1e-7, rtol=1e-12)


def test_dc_dlambda_finite_difference():
    om, lam, s0 = 2 * np.pi * 3e9, 80e-9, 2e6
    h = lam * 1e-5
    fd = (tf.c_of(om, lam + h, s0) - tf.c_of(om, lam - h, s0)) / (2 * h)
    assert np.isclose(tf.dc_dlambda(om, lam, s0), fd, rtol=1e-8)


# ---------------------------------------------------------------- face nodes and A (Eq. 7)
def test_node_numbering_two_voxels():
    s = S.bar(2, 1, 1, 0, 1, 0, 0, 0, 0)
    g = G.build_grid(s)
    assert g.K == 2 and g.M == 11
    assert g.node.tolist() == [[0, 1, 2, 3, 4, 5], [1, 6, 7, 8, 9, 10]]
    assert g.port_minus[0].tolist() == [0] and g.port_plus[0].tolist() == [6]


@pytest.mark.parametrize("abc", [(1, 1, 1), (3, 2, 1), (4, 3, 2), (5, 1, 3)])
def test_node_count_of_a_box(abc):
    a, b, c = abc
    s = S.bar(a + 2, b + 2, c + 1, 1, a, 1, b, 0, c - 1)
    g = G.build_grid(s)
    assert g.M == (a + 1) * b * c + a * (b + 1) * c + a * b * (c + 1)
    assert g.A.nnz == 16 * g.K
    assert np.abs(np.asarray(g.A.sum(axis=0))).max() == 0.0     # divergence-free bases


def test_flux_table_from_surface_integrals():
    """Outward flux of each normalised basis through each face, by quadrature of f.n."""
    x, w = np.polynomial.legendre.leggauss(4)
    x = 0.5 * x
    w = 0.5 * w
    A, B = np.meshgrid(x, x, indexing="ij")
    W = (w[:, None] * w[None, :]).ravel()
    A, B = A.ravel(), B.ravel()

    def f(beta, xi):   # basis in local coordinates, times dx^2 (so a face has unit area)
        one = np.ones(len(xi))
        zero = np.zeros(len(xi))
        return np.stack({0: (one, zero, zero), 1: (zero, one, zero), 2: (zero, zero, one),
                         3: (xi[:, 0], -xi[:, 1], zero),
                         4: (xi[:, 0], xi[:, 1], -2 * xi[:, 2])}[beta], -1)

    for face in range(6):
        ax, side = face // 2, (1 if face % 2 else -1)
        xi = np.zeros((A.size, 3))
        others = [i for i in range(3) if i != ax]
        xi[:, ax] = 0.5 * side
        xi[:, others[0]] = A
        xi[:, others[1]] = B
        n = np.zeros(3)
        n[ax] = side
        for beta in range(5):
            flux = np.sum(W * (f(beta, xi) @ n))
            assert abs(flux - G.FLUX[beta, face]) < 1e-14, (beta, face)


def test_gauge_for_floating_island():
    s = S.bar(8, 6, 3, 0, 5, 0, 1, 0, 0)
    s.occ[2, 4:6, 0:4] = 1      # a separate island without terminals
    s.lam[2, 4:6, 0:4] = 90e-9
    s.sigma0[2, 4:6, 0:4] = 1e7
    g = G.build_grid(s)
    assert g.gauge.size == 1


# ---------------------------------------------------------------- operator (Eq. 7-9)
@pytest.fixture(scope="module")
def strip():
    s = S.strip_cfg1()
    g = G.build_grid(s)
    T = gr.toeplitz_signed(s.Kx, s.Ky, s.Kz)
    return s, g, T


def test_dense_equals_fft_various_padding(strip):
    s, g, T = strip
    om = 2 * np.pi * 1e9
    Kd = op.dense_K(g, T, om)
    x = S.random_complex(7, g.N)
    y = Kd @ x
    for P in [(32, 32, 8), (31, 31, 7), (35, 36, 9)]:
        S7 = op.spectra(T, P)
        y2 = op.apply_K_fft(g, S7, x, om, P)
        assert np.linalg.norm(y - y2) <= 1e-13 * np.linalg.norm(y)


def test_fft_equals_dense_on_random_blob():
    s = S.random_blob(11, 7, 5, 4, fill=0.6)
    g = G.build_grid(s)
    T = gr.toeplitz_signed(7, 5, 4)
    om = 2 * np.pi * 5e9
    P = (op.fft_size(7), op.fft_size(5), op.fft_size(4))
    x = S.random_complex(3, g.N)
    y = op.dense_K(g, T, om) @ x
    y2 = op.apply_K_fft(g, op.spectra(T, P), x, om, P)
    assert np.linalg.norm(y - y2) <= 1e-13 * np.linalg.norm(y)


def test_Z_symmetric_and_inductive_part_positive_definite(strip):
    s, g, T = strip
    om = 2 * np.pi * 1e9
    Z = op.dense_Z(g, T, om)
    assert np.abs(Z - Z.T).max() <= 1e-15 * np.abs(Z).max()
    zd = tf.zdiag(om, g.lam, g.sigma0, g.dx).ravel()
    Lm = (Z - np.diag(zd)) / (1j * om * MU * g.dx)
    assert np.abs(Lm.imag).max() < 1e-14 * np.abs(Lm).max()
    sla.cholesky(Lm.real)                                    # raises if not SPD
    assert np.linalg.eigvalsh(Lm.real).min() > 0


def test_zero_block_pattern_of_eq8(strip):
    s, g, T = strip
    Z = op.dense_Z(g, T, 2 * np.pi * 1e9)
    K = g.K
    zero = [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1), (2, 3), (3, 2)]
    for b in range(5):
        for a in range(5):
            blk = Z[b * K:(b + 1) * K, a * K:(a + 1) * K]
            if (b, a) in zero:
                assert np.abs(blk).max() == 0
            else:
                assert np.abs(blk).max() > 0


def test_self_term_eq16_scaling(strip):
    """Z^{xx}_kk = a/dx + j omega mu (b/dx + I1/dx^4) with I1 = dx^5 * (unit-cube integral)/4pi."""
    s, g, T = strip
    om = 2 * np.pi * 1e9
    Z = op.dense_Z(g, T, om)
    a, b = tf.ab(om, g.lam[0], g.sigma0[0])
    I1 = g.dx ** 5 * cf.CUBE_SELF / (4 * np.pi)
    ref = a / g.dx + 1j * om * MU * (b / g.dx + I1 / g.dx ** 4)
    assert np.isclose(Z[0, 0], ref, rtol=1e-13)


def test_bar_sum_rule_matches_exact_bar_integral():
    """sum over voxel pairs of G00 = (1/4pi) int int_bar 1/|r-r'| (exact, closed form)."""
    a, b, c = 6, 2, 3
    T = gr.toeplitz_signed(a, b, c)
    pos = np.stack(np.meshgrid(np.arange(a), np.arange(b), np.arange(c), indexing="ij"), -1).reshape(-1, 3)
    d = pos[:, None, :] - pos[None, :, :]
    tot = T[0][d[..., 2] + c - 1, d[..., 1] + b - 1, d[..., 0] + a - 1].sum()
    assert abs(tot - cf.bar_self(a, b, c) / (4 * np.pi)) <= 1e-12 * tot


def test_fft_size():
    assert op.fft_size(16) == 32 and op.fft_size(24) == 48
    assert op.fft_size(37) == 75        # 74 = 2 * 37 is not smooth
    for K in range(2, 200):
        P = op.fft_size(K)
        assert P >= 2 * K - 1


# ---------------------------------------------------------------- Tucker (Alg. 1, Eq. 10-11)
def test_mode_product_brute_force():
    rng = np.random.default_rng(0)
    Tn = rng.standard_normal((3, 4, 5))
    F = rng.standard_normal((6, 4))
    out = tk.mode_product(Tn, F, 1)
    ref = np.zeros((3, 6, 5))
    for i in range(3):
        for v in range(6):
            for k in range(5):
                ref[i, v, k] = sum(Tn[i, j, k] * F[v, j] for j in range(4))
    assert np.allclose(out, ref, atol=1e-14)
    U = tk.unfold(Tn, 2)
    assert U.shape == (5, 12) and U[3, 0] == Tn[0, 0, 3] and U[3, 5] == Tn[1, 1, 3]


def test_tucker_recovers_exact_low_rank():
    rng = np.random.default_rng(5)
    C = rng.standard_normal((2, 3, 4))
    Fs = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in ((20, 2), (17, 3), (9, 4))]
    O = tk.tucker_restore(C, Fs)
    C2, F2 = tk.tucker_svd(O, 1e-10)
    assert [f.shape[1] for f in F2] == [2, 3, 4]
    assert np.linalg.norm(tk.tucker_restore(C2, F2) - O) <= 1e-13 * np.linalg.norm(O)


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
def test_tucker_error_bound_on_kernel_spectrum(tol):
    T = gr.toeplitz_octant(24, 20, 6)
    Ts = gr.signed_from_octant(T)
    P = (48, 40, 12)
    spec = op.spectra(Ts, P)[0].real[:7, :21, :25]       # an octant of the G00 spectrum
    C, Fs = tk.tucker_svd(spec, tol)
    err = np.linalg.norm(tk.tucker_restore(C, Fs) - spec) / np.linalg.norm(spec)
    assert err <= tol
    assert C.size < spec.size


# ---------------------------------------------------------------- solver (Eq. 12-15, Sec. III)
def test_schur_preconditioner_inverts_Q(strip):
    s, g, T = strip
    P = (32, 32, 8)
    ps = so.PortSystem(g, op.spectra(T, P), P, 2 * np.pi * 1e9)
    v = S.random_complex(4, ps.n)
    # Q applied explicitly
    K = g.K
    a = ps.precond(v)
    Qa = np.concatenate([ps.Ydiag * a[:5 * K] - ps.AF.T @ a[5 * K:], ps.AF @ a[:5 * K]])
    assert np.linalg.norm(Qa - v) <= 1e-12 * np.linalg.norm(v)


def test_gmres_matches_dense_direct_solve(strip):
    s, g, T = strip
    res = so.port_inductance(s, Tsigned=T)
    ps = res["system"]
    om = res["omega"]
    Kd = op.dense_K(g, T, om)
    keep = np.concatenate([np.arange(5 * g.K), 5 * g.K + ps.free])
    Kr = Kd[np.ix_(keep, keep)]
    x = np.linalg.solve(Kr, ps.rhs(0))
    Ydir = ps.port_currents(x)[0]
    assert abs(res["Y"][0, 0] - Ydir) <= 1e-7 * abs(Ydir)
    assert res["resid"][0] <= 1e-8
    assert res["L"][0, 0] > 0 and res["R"][0, 0] >= 0


def test_dc_normal_bar_matches_exact_partial_inductance():
    """lambda -> inf, small omega mu sigma0 (w t): uniform current, L = mu dx bar/(4 pi b^2 c^2)."""
    a, b, c = 8, 3, 2
    s = S.bar(a + 2, b + 2, c + 2, 1, a, 1, b, 1, c, dx=0.1e-6, lam=1e3, sigma0=3e6, freqs=(1e9,))
    res = so.port_inductance(s, rre=1e-12)
    Lbar = MU * s.dx * cf.bar_self(a, b, c) / (4 * np.pi * b * b * c * c)
    assert abs(res["L"][0, 0] - Lbar) <= 2e-5 * Lbar
    assert np.isclose(res["R"][0, 0], a / (3e6 * b * c * s.dx), rtol=1e-5)


def test_kinetic_limit_and_lambda_trend():
    """sigma0 = 0: L -> mu lambda^2 l/(w t) + L_bar as lambda grows; L falls with lambda.

    (A section of 4 x 2 voxels: in a 2 x 2 section every column is a corner
    column and symmetry alone makes the current uniform.)"""
    a, b, c = 8, 4, 2
    dx = 0.1e-6
    Lbar = MU * dx * cf.bar_self(a, b, c) / (4 * np.pi * b * b * c * c)
    gaps, Ls = [], []
    for lam in (0.05e-6, 0.1e-6, 0.4e-6, 1.6e-6):
        s = S.bar(a + 2, b + 2, c + 2, 1, a, 1, b, 1, c, dx=dx, lam=lam, sigma0=0.0)
        res = so.port_inductance(s, rre=1e-12)
        L = res["L"][0, 0]
        Lk = MU * lam ** 2 * (a * dx) / (b * c * dx * dx)
        Ls.append(L)
        gaps.append(abs((L - Lk) - Lbar) / Lbar)
        assert abs(res["R"][0, 0]) <= 1e-9 * abs(res["Z"][0, 0])     # lossless
    assert all(np.diff(Ls) > 0)
    assert all(np.diff(gaps) < 0) and gaps[-1] < 1e-3


def test_two_port_admittance_symmetric():
    s = S.bar(10, 8, 3, 1, 8, 1, 2, 0, 1)
    s2 = S.bar(10, 8, 3, 1, 8, 5, 6, 0, 1)
    s.occ |= s2.occ
    s.lam += s2.lam
    s.sigma0 += s2.sigma0
    s.ports += s2.ports
    res = so.port_inductance(s, rre=1e-11)
    Y = res["Y"]
    assert abs(Y[0, 1] - Y[1, 0]) <= 1e-7 * abs(Y[0, 1])
    L = res["L"]
    assert L[0, 0] > 0 and L[1, 1] > 0 and 0 < L[0, 1] < np.sqrt(L[0, 0] * L[1, 1])


def test_direct_rows_equal_dense_product(strip):
    """The direct-summation rows used at full size agree with the dense product."""
    s, g, T = strip
    om = 2 * np.pi * 1e9
    rng = np.random.default_rng(12)
    x = np.zeros(g.N, complex)
    sup = rng.choice(g.K, 30, replace=False)
    for a in range(5):
        x[a * g.K + sup] = S.random_complex(a, 30)
    x[5 * g.K + rng.choice(g.M, 40, replace=False)] = S.random_complex(9, 40)
    y = op.dense_K(g, T, om) @ x
    rows = rng.choice(g.K, 25, replace=False)
    nodes = rng.choice(g.M, 25, replace=False)
    yv, yn = op.direct_rows(g, x, om, rows, nodes)
    for b in range(5):
        assert np.allclose(yv[b], y[b * g.K + rows], rtol=1e-12, atol=1e-12 * np.abs(y).max())
    assert np.allclose(yn, y[5 * g.K + nodes], rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_direct_rows_table_equals_dense_product():
    """The table-driven direct rows (kernels looked up at |d| with the parity of S_a) agree with
    the dense product, whose kernels are integrated at every signed offset, for a dense
    multi-item input on a ragged blob (odd kernels change sign across every axis)."""
    s = S.random_blob(31, 9, 7, 5, fill=0.6)
    g = G.build_grid(s)
    Ts = gr.toeplitz_signed(g.Kx, g.Ky, g.Kz)
    To = gr.toeplitz_octant(g.Kx, g.Ky, g.Kz)
    om = 2 * np.pi * 3e9
    x = S.random_complex(32, (3, g.N))
    Kd = op.dense_K(g, Ts, om)
    y = x @ Kd.T
    rng = np.random.default_rng(33)
    rows = rng.choice(g.K, 20, replace=False)
    nodes = rng.choice(g.M, 20, replace=False)
    yv, yn = op.direct_rows_table(g, To, x, om, rows, nodes)
    for b in range(3):
        scale = np.abs(y[b]).max()
        for be in range(5):
            assert np.allclose(yv[b, be], y[b, be * g.K + rows], rtol=0, atol=1e-12 * scale)
        assert np.allclose(yn[b], y[b, 5 * g.K + nodes], rtol=0, atol=1e-12 * scale)
    # a 1-D x gives the shapes of direct_rows, and both direct forms agree
    v1, n1 = op.direct_rows_table(g, To, x[1], om, rows[:5], nodes[:5])
    v2, n2 = op.direct_rows(g, x[1], om, rows[:5], nodes[:5])
    assert v1.shape == v2.shape == (5, 5) and np.allclose(v1, v2, rtol=0, atol=1e-12 * np.abs(v2).max())
    assert np.allclose(n1, n2, rtol=0, atol=1e-12 * np.abs(n2).max())


def test_toeplitz_octant_in_worker_processes_is_bit_identical():
    a = gr.toeplitz_octant(7, 5, 4)
    b = gr.toeplitz_octant(7, 5, 4, processes=2)
    assert np.array_equal(a, b)


def test_preformed_block_spectra_give_the_same_product(strip):
    s, g, T = strip
    P = (op.fft_size(g.Kx), op.fft_size(g.Ky), op.fft_size(g.Kz))
    S7 = op.spectra(T, P)
    x = S.random_complex(34, g.N)
    om = 2 * np.pi * 1e9
    a = op.apply_K_fft(g, S7, x, om, P)
    b = op.apply_K_fft(g, S7, x, om, P, Zh=op.block_spectra(S7))
    assert np.array_equal(a, b)
