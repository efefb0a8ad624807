"""GPU parity of the operator product (Eq. 7-9) against the CPU oracle, through the C ABI.

Tolerances: FP64 path 1e-11 relative (quadrature of two independent kernel
generators and FFT round-off); FP32 path 1e-5 relative in the 2-norm per
batch item (the bound stated for the mixed-precision matvec), and every
element within 2e-5 of the item's max-norm.
"""
import numpy as np
import pytest

import svh_synth as S
from gpu_util import handle_for, oracle_reference, rel_err
from oracle import greens as gr
from oracle import operator as op

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-11


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _check_fp32(y, yref):
    for b in range(yref.shape[0]):
        assert rel_err(y[b], yref[b]) <= FP32_TOL, (b, rel_err(y[b], yref[b]))
        assert np.abs(y[b] - yref[b]).max() <= 2 * FP32_TOL * np.abs(yref[b]).max()


def test_device_toeplitz_matches_oracle():
    for shape in [(16, 16, 4), (13, 9, 5), (41, 3, 2)]:
        s = S.random_blob(7, *shape, fill=0.3)
        h = handle_for(s)
        T = h.toeplitz()
        To = gr.toeplitz_octant(*shape)
        scale = np.abs(To[0])
        assert np.all(np.abs(T - To) <= 1e-12 * scale[None]), np.max(np.abs(T - To) / scale[None])
        h.close()


def test_grid_info_matches_oracle():
    s = S.strip_cfg1()
    h = handle_for(s)
    g, _, P, _ = oracle_reference(s)
    i = h.info()
    assert (i["K"], i["M"], i["N"]) == (g.K, g.M, g.N) == (128, 488, 1128)
    assert (i["Px"], i["Py"], i["Pz"]) == P
    assert np.array_equal(h.nodes(), g.node)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_strip_matvec_vs_dense_oracle(prec):
    torch = _torch()
    s = S.strip_cfg1()
    g, S7, P, T = oracle_reference(s)
    om = 2 * np.pi * 1e9
    Kd = op.dense_K(g, gr.signed_from_octant(T), om)
    nb = 3
    x = S.random_complex(11, (nb, g.N))
    yref = x @ Kd.T
    h = handle_for(s)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    y = h.matvec(om, torch.from_numpy(x).to(dt).cuda()).cpu().numpy().astype(np.complex128)
    if prec == "fp64":
        for b in range(nb):
            assert rel_err(y[b], yref[b]) <= FP64_TOL
    else:
        _check_fp32(y, yref)
    h.close()


@pytest.mark.parametrize("seed,shape,P", [
    (21, (13, 9, 5), None),          # ragged, P = 26, 18, 10
    (22, (37, 11, 3), (75, 21, 6)),  # 2*37, 2*11 not smooth: the oracle's P (generic kernels)
    (23, (24, 20, 6), (48, 40, 12)),
    (24, (10, 14, 7), (21, 27, 14)),  # odd FFT sizes 2K - 1 (radix 3 and 7)
    (25, (70, 33, 4), None),         # several x-lines per block, ragged y tiles
])
def test_random_blob_matvec_fp64_fp32(seed, shape, P):
    torch = _torch()
    s = S.random_blob(seed, *shape, fill=0.45)
    g, S7, Pr, T = oracle_reference(s, P)
    om = 2 * np.pi * 3e9
    nb = 2
    x = S.random_complex(seed, (nb, g.N))
    yref = np.stack([op.apply_K_fft(g, S7, x[b], om, Pr) for b in range(nb)])
    h = handle_for(s, toeplitz=T, P=P)
    y64 = h.matvec(om, torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(nb):
        assert rel_err(y64[b], yref[b]) <= FP64_TOL
    y32 = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    _check_fp32(y32, yref)
    h.close()


def test_empty_planes_and_rows():
    """Planes and rows without voxels are skipped; the product must not change."""
    torch = _torch()
    s = S.random_blob(31, 12, 10, 8, fill=0.5)
    s.occ[2:5] = 0
    s.occ[:, 3:6, :] = 0
    s.lam *= s.occ
    s.sigma0 *= s.occ
    g, S7, P, T = oracle_reference(s)
    om = 2 * np.pi * 1e9
    x = S.random_complex(3, (1, g.N))
    yref = op.apply_K_fft(g, S7, x[0], om, P)[None]
    h = handle_for(s, toeplitz=T)
    assert h.info()["n_active_planes"] == 5
    y = h.matvec(om, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_err(y[0], yref[0]) <= FP64_TOL
    h.close()


def test_matvec_host_equals_device():
    torch = _torch()
    s = S.random_blob(41, 9, 8, 3, fill=0.5)
    h = handle_for(s)
    N = h.info()["N"]
    x = S.random_complex(5, (2, N))
    for dt, npdt in ((torch.complex64, np.complex64), (torch.complex128, np.complex128)):
        yd = h.matvec(2e9, torch.from_numpy(x.astype(npdt)).cuda()).cpu().numpy()
        yh = h.matvec_host(2e9, x.astype(npdt))
        assert np.array_equal(yd, yh)
    h.close()


def test_argument_errors():
    torch = _torch()
    from paper_2105_08627_gb300 import svh
    h = svh.Handle(0)
    s = S.strip_cfg1()
    with pytest.raises(svh.SVHError) as e:
        h.setup_grid(s.Kx, s.Ky, s.Kz, -1.0, s.occ, s.lam, s.sigma0, s.ports)
    assert e.value.code == svh.SVH_ERR_ARG
    h.setup_structure(s)
    x = torch.zeros(h.info()["N"], dtype=torch.complex64, device="cuda")
    with pytest.raises(svh.SVHError) as e:
        h.matvec(1e9, x)
    assert e.value.code == svh.SVH_ERR_STATE
    h.generate_toeplitz()
    with pytest.raises(svh.SVHError) as e:
        h.matvec_ptr(-1.0, 1, x.data_ptr(), x.data_ptr(), svh.SVH_FP32)
    assert e.value.code == svh.SVH_ERR_ARG
    with pytest.raises(svh.SVHError) as e:      # x and y overlap
        h.matvec_ptr(1e9, 1, x.data_ptr(), x.data_ptr(), svh.SVH_FP32)
    assert e.value.code == svh.SVH_ERR_ARG
    bad = s.ports[0].plus.copy()
    bad[0] = 0                                   # voxel 0 of the grid is empty
    with pytest.raises(svh.SVHError):
        h.setup_grid(s.Kx, s.Ky, s.Kz, s.dx, s.occ, s.lam, s.sigma0, [(bad, s.ports[0].minus)])
    h.close()


def test_tucker_rebuild_matches_oracle_restore():
    """a1: the device restore (Eq. 10) of Tucker data made by the oracle's Algorithm 1."""
    torch = _torch()
    from oracle import tucker as tk
    from paper_2105_08627_gb300 import svh
    s = S.random_blob(51, 24, 20, 6, fill=0.4)
    h = handle_for(s)
    spec = h.spectra()
    for u in range(7):
        C, Fs = tk.tucker_svd(np.transpose(spec[u], (2, 1, 0)), 1e-9)
        h.load_tucker(u, np.transpose(C, (2, 1, 0)), Fs)
    h.rebuild_spectra()
    torch.cuda.synchronize()
    # compare the FP32 matvec using rebuilt spectra with the oracle restore
    g, S7, P, T = oracle_reference(s)
    om = 2 * np.pi * 1e9
    x = S.random_complex(8, (1, g.N))
    yref = op.apply_K_fft(g, S7, x[0], om, P)[None]
    y = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    _check_fp32(y, yref)
    # rebuild-every-matvec mode gives the same result, in every stream schedule
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    for sched in (0, 1, 2, 3):
        h.set_pass_variant(6, sched)
        y2 = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        assert np.array_equal(y, y2), sched
    # every z-pass variant, the direct one reading z-space kernels made from each restore
    counts = h.pass_variants()[0]
    assert counts[2] == 4
    for zv in range(counts[2]):
        h.set_pass_variant(2, zv)
        y3 = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        _check_fp32(y3, yref)
    h.close()


def test_direct_z_pass_with_empty_planes():
    """a4: the direct z pass (block-Toeplitz product over the active planes) when the active
    planes are not consecutive (z = 2 and 5 empty: offsets up to 7 between active planes),
    against the oracle, resident and after a Tucker restore."""
    torch = _torch()
    from paper_2105_08627_gb300 import svh
    s = S.random_blob(66, 40, 24, 8, fill=0.5)
    for z in (2, 5):
        s.occ[z] = 0
        s.lam[z] = 0
        s.sigma0[z] = 0
    g, S7, P, T = oracle_reference(s)
    om = 2 * np.pi * 1.5e9
    nb = 2
    x = S.random_complex(67, (nb, g.N))
    yref = np.stack([op.apply_K_fft(g, S7, x[b], om, P) for b in range(nb)])
    h = handle_for(s, toeplitz=T)
    assert h.info()["n_active_planes"] == 6
    counts = h.pass_variants()[0]
    assert counts[2] == 4
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    for zv in range(4):
        h.set_pass_variant(2, zv)
        _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)
    h.tucker_compress(1e-9)
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    h.set_pass_variant(2, 3)
    _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)
    assert h.device_status() == 0
    h.close()


@pytest.mark.parametrize("case", ["blob", "meander256"])
def test_tucker_restore_elementwise(case):
    """a1: the tensor-core restore (Eq. 10-11: modes 1 and 2 as tcgen05 GEMMs, mode 3 folded
    into the core at load) of every FP32 spectrum value, against the oracle's FP64 restore
    of the same Tucker data. The blob's octant (25 x 25 x 7) is one masked 128-row tile; the
    256x256x8 meander's (257 x 257 x 9) has two full row tiles and a Nyquist row done by the
    FP32 edge blocks; G00's low ranks end in a partial k slice."""
    torch = _torch()
    from oracle import tucker as tk
    s = S.random_blob(53, 24, 20, 6, fill=0.4) if case == "blob" else S.meander_cfg2()
    h = handle_for(s)
    ranks = h.tucker_compress(1e-8)
    h.rebuild_spectra()
    got = h.spectra32().astype(np.float64)
    for u in range(7):
        C, Fs = h.get_tucker(u)
        ref = np.transpose(tk.tucker_restore(np.transpose(C, (2, 1, 0)), Fs), (2, 1, 0))
        err = np.abs(got[u] - ref).max() / np.abs(ref).max()
        assert err <= 1e-5, (u, tuple(ranks[u]), err)
    assert h.device_status() == 0
    h.close()


def _restore(C, Fs):
    """S[z][y][x] from core[d3][d2][d1] and F1 [Hx][d1], F2 [Hy][d2], F3 [Hz][d3] (mode products)."""
    X = np.tensordot(C, Fs[0], axes=([2], [1]))          # [d3][d2][Hx]
    X = np.tensordot(X, Fs[1], axes=([1], [1]))          # [d3][Hx][Hy]
    X = np.tensordot(X, Fs[2], axes=([0], [1]))          # [Hx][Hy][Hz]
    return np.transpose(X, (2, 1, 0))


@pytest.mark.parametrize("case", ["blob", "meander256"])
def test_device_tucker_svd_matches_oracle(case):
    """f1: Algorithm 1 on the device (QR of each unfolding's transpose, SVD of the triangle,
    ranks from the residual row norms, projections) gives the oracle's ranks (SVD of the
    unfoldings, same truncation rule) and meets ||S - restore|| <= tol ||S|| for every
    kernel at tol 1e-4 and 1e-8, with orthonormal factors."""
    torch = _torch()
    from oracle import tucker as tk
    s = S.random_blob(54, 28, 22, 5, fill=0.4) if case == "blob" else S.meander_cfg2()
    h = handle_for(s)
    spec = h.spectra()
    for tol in (1e-4, 1e-8):
        rd = h.tucker_compress(tol, device=True)
        for u in range(7):
            C, Fs = h.get_tucker(u)
            assert tuple(rd[u]) == C.shape[::-1]
            Co, _ = tk.tucker_svd(np.transpose(spec[u], (2, 1, 0)), tol)
            assert np.abs(np.array(Co.shape) - rd[u]).max() <= 1, (tol, u, Co.shape, rd[u])   # threshold ties
            err = np.linalg.norm(_restore(C, Fs) - spec[u]) / np.linalg.norm(spec[u])
            assert err <= tol, (tol, u, err)
            for i in range(3):
                assert np.abs(Fs[i].T @ Fs[i] - np.eye(Fs[i].shape[1])).max() < 1e-10
    h.close()


def test_tucker_compress_error_bound():
    torch = _torch()
    from paper_2105_08627_gb300 import svh
    s = S.random_blob(52, 30, 26, 5, fill=0.4)
    h = handle_for(s)
    spec = h.spectra()
    ranks = h.tucker_compress(1e-6)
    for u in range(7):
        C, Fs = h.get_tucker(u)
        rec = np.einsum("cba,ia,jb,kc->kji", C, Fs[0], Fs[1], Fs[2])
        assert np.linalg.norm(rec - spec[u]) <= 1e-6 * np.linalg.norm(spec[u])
        assert tuple(ranks[u]) == C.shape[::-1]
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    g, S7, P, T = oracle_reference(s)
    x = S.random_complex(9, (1, g.N))
    yref = op.apply_K_fft(g, S7, x[0], 2e9, P)[None]
    y = h.matvec(2e9, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    _check_fp32(y, yref)
    h.close()


@pytest.mark.slow
def test_meander_256x256x8_full_size():
    """cfg 2 size (256x256x8, P = 512x512x16) in the bench's launch shape: FP32 and FP64 vs the oracle."""
    torch = _torch()
    s = S.meander_cfg2()
    g, S7, P, T = oracle_reference(s)
    om = 2 * np.pi * 1e9
    nb = 2
    x = S.random_complex(202, (nb, g.N))
    yref = np.stack([op.apply_K_fft(g, S7, x[b], om, P) for b in range(nb)])
    h = handle_for(s)           # device-generated kernels: fully independent of the oracle
    y64 = h.matvec(om, torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(nb):
        assert rel_err(y64[b], yref[b]) <= FP64_TOL
    y32 = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    _check_fp32(y32, yref)
    assert h.pass_variants()[0][5] == 2          # the fused y/z/y path applies
    h.set_pass_variant(5, 1)                     # fused y/z/y (the separate passes ran above)
    y32s = h.matvec(om, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    _check_fp32(y32s, yref)
    h.close()


@pytest.mark.slow
def test_esfq_512x512x24_sampled_rows():
    """cfg 5 size (512x512x24, P = 1024x1024x48) in one FP64 and one FP32 product of a
    sparse input (1500 voxels, 500 nodes); 60 voxel rows (all 5 bases) and 40 node
    rows are summed directly by the oracle (no FFT)."""
    torch = _torch()
    from oracle import geometry as G
    from oracle import operator as opo
    s = S.esfq_cfg5()
    g = G.build_grid(s)
    h = handle_for(s)
    rng = np.random.default_rng(505)
    x = np.zeros(g.N, complex)
    sup = rng.choice(g.K, 1500, replace=False)
    for a in range(5):
        x[a * g.K + sup] = S.random_complex(10 + a, 1500)
    x[5 * g.K + rng.choice(g.M, 500, replace=False)] = S.random_complex(20, 500)
    om = 2 * np.pi * 1e9
    rows = np.concatenate([rng.choice(sup, 30, replace=False), rng.choice(g.K, 30, replace=False)])
    nodes = rng.choice(g.M, 40, replace=False)
    yv, yn = opo.direct_rows(g, x, om, rows, nodes)
    ref = np.concatenate([yv.ravel(), yn])
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 2e-5)):
        y = h.matvec(om, torch.from_numpy(x).to(dt).cuda()).cpu().numpy().astype(np.complex128)
        got = np.concatenate([np.stack([y[b * g.K + rows] for b in range(5)]).ravel(), y[5 * g.K + nodes]])
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (dt, np.abs(got - ref).max() / np.abs(ref).max())
    h.close()


@pytest.mark.parametrize("seed,shape,fused", [
    (61, (64, 16, 8), False),     # P = 128, 32, 16: transposed-split variants on x and y
    (62, (48, 24, 12), False),    # P = 96, 48, 24: x inverse without a grouped kernel
    (63, (64, 64, 8), True),      # P = 128, 128, 16: the fused y/z/y path applies
    (64, (128, 128, 4), True),    # P = 256, 256, 8
    (65, (32, 16, 16), False),    # P = 64, 32, 32: the z pass with pencils split over two threads
    (66, (24, 16, 24), False),    # P = 48, 32, 48: the same at Pz = 48
])
def test_every_tile_variant_and_autotune(seed, shape, fused):
    """a12: each FFT tile variant and path the autotuner may pick gives the oracle's product."""
    torch = _torch()
    s = S.random_blob(seed, *shape, fill=0.5)
    g, S7, Pr, T = oracle_reference(s)
    om = 2 * np.pi * 2e9
    nb = 3
    x = S.random_complex(seed, (nb, g.N))
    yref = np.stack([op.apply_K_fft(g, S7, x[b], om, Pr) for b in range(nb)])
    h = handle_for(s, toeplitz=T)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    counts, chosen = h.pass_variants()
    assert np.all(counts[:5] >= 2) and np.all(chosen == 0)
    assert counts[5] == (2 if fused else 1)
    _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)   # default: separate passes
    if fused:
        h.set_pass_variant(5, 1)                                                # fused y/z/y
        _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)
        h.set_pass_variant(5, 0)
    for p in range(5):
        for v in range(counts[p]):
            h.set_pass_variant(p, v)
            y = h.matvec(om, xd).cpu().numpy().astype(np.complex128)
            _check_fp32(y, yref)
            assert h.device_status() == 0          # no bounded wait (TMA z pass) expired
        h.set_pass_variant(p, 0)
    h.set_pass_variant(5, 0)
    assert counts[6] == 4
    for v in (1, 2, 3, 0):                                                      # stream schedules
        h.set_pass_variant(6, v)
        _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)
    with pytest.raises(Exception):
        h.set_pass_variant(0, counts[0])
    with pytest.raises(Exception):
        h.set_pass_variant(5, counts[5])
    v, ms = h.autotune(nb)
    assert np.all((v >= 0) & (v < np.maximum(counts, 1))) and np.all(ms[:5] > 0) and ms[6] > 0
    assert np.array_equal(h.pass_variants()[1], v)
    _check_fp32(h.matvec(om, xd).cpu().numpy().astype(np.complex128), yref)
    # FP64 products ignore the FP32 tile choices and the fused path
    y64 = h.matvec(om, torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(nb):
        assert rel_err(y64[b], yref[b]) <= FP64_TOL
    h.close()


def test_toeplitz_store_from_device_quadrature(tmp_path):
    """Algorithm 2 end to end: store computed by the device quadrature for a larger
    domain, cropped to a structure's grid at set-up; the FP64 product matches the oracle's
    (own quadrature, exact crop) within the Tucker tolerance."""
    torch = _torch()
    from paper_2105_08627_gb300 import build, svh
    build.build()
    path = str(tmp_path / "unit.svhstore")
    svh.toeplitz_store_write(path, (40, 36, 10), 1e-11)
    s = S.random_blob(71, 24, 20, 6, fill=0.5)
    g, S7, P, T = oracle_reference(s)
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    h.setup_structure(s)
    h.load_toeplitz_store(path)
    om = 2 * np.pi * 1e9
    x = S.random_complex(71, (2, g.N))
    y = h.matvec(om, torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(2):
        assert rel_err(y[b], op.apply_K_fft(g, S7, x[b], om, P)) <= 1e-9
    Tst, _ = svh.toeplitz_store_read(path, (24, 20, 6))
    assert np.abs(Tst - T).max() <= 1e-9 * np.abs(T).max()
    h.close()
