"""svh_matvec_noalloc: the operator product for callers that cannot allocate
device memory at call time (for example a plug-in whose host application owns
the device-memory budget). It must give the same result as svh_matvec, call
after call, while working in the library's fixed device scratch array.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it; it also passes on its own in a
fresh process."""
import numpy as np
import pytest

import svh_synth as S

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5    # the matvec tolerance used by the other GPU tests
FP64_TOL = 1e-11


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_matvec_on_consecutive_calls(prec):
    import torch

    from paper_2105_08627_gb300 import build, svh
    build.build()
    s = S.random_blob(61, 20, 18, 6, fill=0.45)
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    h.setup_structure(s)
    h.generate_toeplitz()
    N = h.info()["N"]
    dt, code, tol = ((torch.complex64, svh.SVH_FP32, FP32_TOL) if prec == "fp32"
                     else (torch.complex128, svh.SVH_FP64, FP64_TOL))
    nb = 3
    for call in range(2):                      # two calls in a row share the scratch
        x = torch.from_numpy(S.random_complex(100 + call, (nb, N))).to(dt).cuda()
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        h.matvec_ptr(2 * np.pi * 1e9, nb, x.data_ptr(), y_ref.data_ptr(), code)
        h.matvec_noalloc_ptr(2 * np.pi * 1e9, nb, x.data_ptr(), y_new.data_ptr(), code)
        torch.cuda.synchronize()
        a = y_new.cpu().numpy().astype(np.complex128)
        b = y_ref.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(a))
        for i in range(nb):
            assert _rel(a[i], b[i]) <= tol, (call, i, _rel(a[i], b[i]))
    h.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch

    from paper_2105_08627_gb300 import build, svh
    build.build()
    s = S.random_blob(62, 128, 128, 8, fill=0.5)     # 5*8*256*(128+256)*8 B = 31 MB per right-hand side
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    h.setup_structure(s)
    h.generate_toeplitz()
    N = h.info()["N"]
    x = torch.zeros((4, N), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(svh.SVHError) as e:
        h.matvec_noalloc_ptr(1e9, 4, x.data_ptr(), y.data_ptr(), svh.SVH_FP32)
    assert e.value.code == svh.SVH_ERR_ARG and "64 MiB" in str(e.value)
    h.close()


def _noalloc_case(h, svh, torch, nb, seed):
    """One noalloc product on a handle that has never run svh_matvec: the free device memory must
    not change across the call, and the result must match svh_matvec (run after it)."""
    N = h.info()["N"]
    x = torch.from_numpy(S.random_complex(seed, (nb, N))).to(torch.complex64).cuda()
    y_new = torch.full_like(x, float("nan"))
    y_ref = torch.empty_like(x)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    h.matvec_noalloc_ptr(2 * np.pi * 1e9, nb, x.data_ptr(), y_new.data_ptr(), svh.SVH_FP32)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    h.matvec_ptr(2 * np.pi * 1e9, nb, x.data_ptr(), y_ref.data_ptr(), svh.SVH_FP32)
    torch.cuda.synchronize()
    a = y_new.cpu().numpy().astype(np.complex128)
    b = y_ref.cpu().numpy().astype(np.complex128)
    assert free0 == free1, (free0, free1)
    assert np.all(np.isfinite(a))
    for i in range(nb):
        assert _rel(a[i], b[i]) <= FP32_TOL, (i, _rel(a[i], b[i]))


def test_noalloc_allocates_nothing_with_tuned_or_forced_direct_z_pass():
    """A fresh handle whose tile choices come from the autotuner's cache, or whose z pass is set
    to the direct form, has no z-space kernel buffers yet: the call must still allocate nothing
    (it takes the FFT form of the z pass) and give svh_matvec's product."""
    import torch

    from paper_2105_08627_gb300 import build, svh
    build.build()
    s = S.random_blob(63, 20, 18, 6, fill=0.45)
    nb = 2
    stream = torch.cuda.current_stream().cuda_stream
    h0 = svh.Handle(0, stream)
    h0.setup_structure(s)
    h0.generate_toeplitz()
    N = h0.info()["N"]
    x0 = torch.zeros((nb, N), dtype=torch.complex64, device="cuda")
    y0 = torch.empty_like(x0)
    # load the kernels and the scratch symbol once (module loading may allocate), tune the grid
    h0.matvec_ptr(1e9, nb, x0.data_ptr(), y0.data_ptr(), svh.SVH_FP32)
    h0.matvec_noalloc_ptr(1e9, nb, x0.data_ptr(), y0.data_ptr(), svh.SVH_FP32)
    h0.set_pass_variant(2, 3)
    h0.matvec_ptr(1e9, nb, x0.data_ptr(), y0.data_ptr(), svh.SVH_FP32)
    h0.set_pass_variant(2, 0)
    h0.autotune(nb)
    torch.cuda.synchronize()
    for route in ("autotune-cache", "forced-direct"):
        h = svh.Handle(0, stream)
        h.setup_structure(s)
        h.generate_toeplitz()
        if route == "autotune-cache":
            h.autotune(nb, timings=False)       # cache hit: tile choices set, no buffers sized
        else:
            assert h.pass_variants()[0][2] >= 4
            h.set_pass_variant(2, 3)            # the direct z pass
        _noalloc_case(h, svh, torch, nb, 200 + len(route))
        h.close()
    h0.close()


def test_noalloc_in_tucker_restore_mode():
    """In Tucker-restore mode the call refuses until the restored spectra are on the device, then
    applies the same (restored) operator as svh_matvec."""
    import torch

    from paper_2105_08627_gb300 import build, svh
    build.build()
    s = S.random_blob(64, 20, 18, 6, fill=0.45)
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    h.setup_structure(s)
    h.generate_toeplitz()
    h.tucker_compress(1e-6)
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    N = h.info()["N"]
    x = torch.from_numpy(S.random_complex(301, (2, N))).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    with pytest.raises(svh.SVHError) as e:
        h.matvec_noalloc_ptr(2 * np.pi * 1e9, 2, x.data_ptr(), y.data_ptr(), svh.SVH_FP32)
    assert e.value.code == svh.SVH_ERR_STATE
    h.rebuild_spectra()
    for call in range(2):
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        h.matvec_ptr(2 * np.pi * 1e9, 2, x.data_ptr(), y_ref.data_ptr(), svh.SVH_FP32)
        h.matvec_noalloc_ptr(2 * np.pi * 1e9, 2, x.data_ptr(), y_new.data_ptr(), svh.SVH_FP32)
        torch.cuda.synchronize()
        a = y_new.cpu().numpy().astype(np.complex128)
        b = y_ref.cpu().numpy().astype(np.complex128)
        for i in range(2):
            assert _rel(a[i], b[i]) <= FP32_TOL, (call, i, _rel(a[i], b[i]))
    h.close()
