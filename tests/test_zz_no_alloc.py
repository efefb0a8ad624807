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
