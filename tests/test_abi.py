"""CPU tests of the C ABI library: it builds, loads, exports every declared
symbol, and its host-side logic (face nodes, circulant spectra, Tucker-SVD)
matches the oracle. No device call is made."""
import os
import re

import numpy as np
import pytest

import svh_synth as S
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op
from oracle import tucker as tk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def svh():
    from paper_2105_08627_gb300 import build, svh as mod
    build.build()
    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "svh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char)\s*\*?\s*(svh_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol(svh):
    L = svh.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(svh.SIGNATURES), set(names) ^ set(svh.SIGNATURES)


@pytest.mark.parametrize("seed,shape", [(1, (7, 6, 4)), (2, (9, 3, 5)), (3, (16, 16, 4))])
def test_face_nodes_match_oracle(svh, seed, shape):
    s = S.random_blob(seed, *shape, fill=0.55)
    node, M = svh.host_face_nodes(s.occ)
    g = G.build_grid(s)
    assert M == g.M
    assert np.array_equal(node, g.node)


@pytest.mark.parametrize("K,P", [((7, 6, 4), (14, 12, 8)), ((5, 4, 3), (9, 7, 5)), ((6, 5, 3), (15, 10, 6))])
def test_host_spectra_match_oracle_fft(svh, K, P):
    T = gr.toeplitz_octant(*K)
    Sl = svh.host_spectra(T, P)
    S7 = op.spectra(gr.signed_from_octant(T), P)
    Hx, Hy, Hz = P[0] // 2 + 1, P[1] // 2 + 1, P[2] // 2 + 1
    for k in range(7):
        a = S7[k][:Hz, :Hy, :Hx]
        ref = -a.imag if k in (1, 2, 3) else a.real
        assert np.abs(Sl[k] - ref).max() <= 1e-14 * np.abs(ref).max() + 1e-300
        # the other part vanishes: spectra are real (even kernels) or imaginary (S kernels)
        other = a.real if k in (1, 2, 3) else a.imag
        assert np.abs(other).max() <= 1e-14 * np.abs(ref).max()


def test_host_tucker_matches_oracle(svh):
    T = gr.toeplitz_octant(20, 18, 6)
    P = (40, 36, 12)
    spec = svh.host_spectra(T, P)
    for k in (0, 1, 4):
        O = spec[k]
        for tol in (1e-4, 1e-8):
            core, F = svh.host_tucker_svd(O, tol)
            rec = tk.tucker_restore(np.transpose(core, (2, 1, 0)), F)      # oracle restore, modes (x, y, z)
            err = np.linalg.norm(np.transpose(rec, (2, 1, 0)) - O) / np.linalg.norm(O)
            assert err <= tol
            Co, Fo = tk.tucker_svd(np.transpose(O, (2, 1, 0)), tol)
            # ranks agree with the oracle's SVD-based ones (the library's QR + one-sided Jacobi
            # keeps the singular values accurate to eps sigma_max, below the cut at tol 1e-8);
            # a tie at the threshold may move one vector
            assert all(abs(a - b) <= 1 for a, b in zip(core.shape[::-1], Co.shape))
            if tol >= 1e-6:
                assert core.shape[::-1] == Co.shape
            for f in F:
                assert np.allclose(f.T @ f, np.eye(f.shape[1]), atol=1e-10)


def test_toeplitz_store_crop_and_errors(svh, tmp_path):
    """Algorithm 2: the stored large-domain tensors, restored and cropped, give the
    small domain's tensors (T_u depends only on the offset) within the Tucker bound."""
    big = gr.toeplitz_octant(14, 12, 6)
    path = str(tmp_path / "unit.svhstore")
    tol = 1e-9
    svh.toeplitz_store_write(path, (14, 12, 6), tol, T=big)
    small = gr.toeplitz_octant(9, 7, 4)
    T, ranks = svh.toeplitz_store_read(path, (9, 7, 4))
    assert ranks.shape == (7, 3) and np.all(ranks >= 1) and np.all(ranks <= [14, 12, 6])
    for u in range(7):
        assert np.linalg.norm(T[u] - small[u]) <= tol * np.linalg.norm(big[u])
    Tfull, _ = svh.toeplitz_store_read(path, (14, 12, 6))
    for u in range(7):
        assert np.linalg.norm(Tfull[u] - big[u]) <= tol * np.linalg.norm(big[u])
    with pytest.raises(svh.SVHError):
        svh.toeplitz_store_read(path, (15, 12, 6))          # larger than the stored domain
    bad = tmp_path / "bad.svhstore"
    bad.write_bytes(b"not a store" * 8)
    with pytest.raises(svh.SVHError):
        svh.toeplitz_store_read(str(bad), (4, 4, 4))


# ---------------------------------------------------------------- failures made on the host
def test_null_handle_and_null_arrays_are_rejected(svh):
    """Every handle call checks its handle before touching a device; host utilities check their
    arrays (no GPU is needed for either)."""
    import ctypes as C
    L = svh.lib()
    null = svh._P()
    z = (C.c_double * 4)()
    opt = svh.svh_options()
    L.svh_default_options(C.byref(opt))
    assert L.svh_solve(null, z, 1, C.byref(opt), z, z, None) == svh.SVH_ERR_ARG
    assert L.svh_matvec(null, 1e9, 1, None, None, svh.SVH_FP32) == svh.SVH_ERR_ARG
    assert L.svh_matvec_noalloc(null, 1e9, 1, None, None, svh.SVH_FP32) == svh.SVH_ERR_ARG
    assert L.svh_grad_inductance(null, 0, 0, z, z) == svh.SVH_ERR_ARG
    assert L.svh_set_materials(null, z, z) == svh.SVH_ERR_ARG
    assert L.svh_get_solution(null, 0, z) == svh.SVH_ERR_ARG
    K = C.c_int64()
    assert L.svh_host_face_nodes(2, 2, 2, None, C.byref(K), C.byref(K), None) == svh.SVH_ERR_ARG
    assert L.svh_host_spectra(2, 2, 2, 4, 4, 4, None, z) == svh.SVH_ERR_ARG
    assert L.svh_host_spectra(2, 2, 2, 2, 4, 4, z, z) == svh.SVH_ERR_ARG        # P < 2K - 1
    d = (C.c_int32 * 3)()
    assert L.svh_host_tucker_svd(z, 2, 2, 1, -1.0, d, z, z, z, z) == svh.SVH_ERR_ARG
    assert L.svh_host_amg_solve(0, None, None, None, None, None, 1e-8, 10, None, None) == svh.SVH_ERR_ARG


def test_host_amg_stops_at_maxit_with_not_converged(svh):
    """A CG that runs out of iterations reports SVH_ERR_NOT_CONVERGED (the Schur solves of the
    preconditioner, Eq. 14)."""
    import scipy.sparse as sp
    n = 4000
    rng = np.random.default_rng(3)
    main = 2.0 + 1e-6 * rng.random(n)
    S_ = sp.diags([-np.ones(n - 1), main, -np.ones(n - 1)], [-1, 0, 1], format="csr")   # 1-D Laplacian
    b = rng.standard_normal(n)
    with pytest.raises(svh.SVHError) as e:
        svh.host_amg_solve(S_, b, tol=1e-14, maxit=1)
    assert e.value.code == svh.SVH_ERR_NOT_CONVERGED
    x, it, lv = svh.host_amg_solve(S_, b, tol=1e-8, maxit=500)
    assert np.linalg.norm(S_ @ x - b) <= 2e-8 * np.linalg.norm(b)
