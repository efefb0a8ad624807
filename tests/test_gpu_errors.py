"""Failure paths of the C ABI on the GPU, all made on the host (SURVEY-planned error tests):
invalid materials, a solve that runs out of iterations, a device AMG that runs out of
iterations. None of them faults or stalls the device; each call returns its status code and
the handle stays usable afterwards."""
import numpy as np
import pytest

import svh_synth as S
from gpu_util import handle_for, oracle_reference

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bad", ["nan_lambda", "neg_lambda", "zero_lambda", "inf_lambda", "nan_sigma",
                                 "neg_sigma"])
def test_invalid_materials_are_rejected(bad):
    import torch
    from paper_2105_08627_gb300 import build, svh
    build.build()
    s = S.strip_cfg1()
    lam, sig = s.lam.copy(), s.sigma0.copy()
    occ = s.occ.astype(bool)
    first = np.flatnonzero(occ.ravel())[3]
    field, val = {"nan_lambda": ("lam", np.nan), "neg_lambda": ("lam", -90e-9), "zero_lambda": ("lam", 0.0),
                  "inf_lambda": ("lam", np.inf), "nan_sigma": ("sig", np.nan), "neg_sigma": ("sig", -1.0)}[bad]
    (lam if field == "lam" else sig).ravel()[first] = val
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(svh.SVHError) as e:
        h.setup_grid(s.Kx, s.Ky, s.Kz, s.dx, s.occ, lam, sig, s.ports)
    assert e.value.code == svh.SVH_ERR_ARG
    # the handle stays usable; svh_set_materials checks the same values per voxel
    h.setup_structure(s)
    K = h.info()["K"]
    lv, sv = np.full(K, 90e-9), np.full(K, 1e7)
    (lv if field == "lam" else sv)[5] = val
    with pytest.raises(svh.SVHError) as e:
        h.set_materials(lv, sv)
    assert e.value.code == svh.SVH_ERR_ARG
    got_l, got_s = h.materials()
    assert np.all(got_l > 0) and np.all(np.isfinite(got_l)) and np.all(got_s >= 0)
    h.close()


def test_solve_out_of_iterations_reports_not_converged_with_outputs_filled():
    from paper_2105_08627_gb300 import svh
    s = S.strip_cfg1()
    h = handle_for(s)
    res = h.solve([1e9], max_iterations=2, max_refinements=1, restart=2, allow_unconverged=True)
    st = res["stats"]
    assert st["status"] == svh.SVH_ERR_NOT_CONVERGED
    assert st["final_rre"] > 1e-8
    assert np.all(np.isfinite(res["Z"])) and np.all(np.isfinite(res["L"]))
    assert np.all(res["L"] == res["Z"].imag / (2 * np.pi * 1e9))
    with pytest.raises(svh.SVHError) as e:       # without allow_unconverged the binding raises
        h.solve([1e9], max_iterations=2, max_refinements=1, restart=2)
    assert e.value.code == svh.SVH_ERR_NOT_CONVERGED
    # the same handle then converges to the oracle's inductance
    from oracle import solve as so
    ref = so.port_inductance(s, freq=1e9, rre=1e-10)
    ok = h.solve([1e9])
    assert ok["stats"]["status"] == svh.SVH_OK
    assert abs(ok["L"][0, 0, 0] - ref["L"][0, 0]) <= 1e-6 * abs(ref["L"][0, 0])
    h.close()


def test_device_amg_stops_at_maxit_with_not_converged():
    import scipy.sparse as sp
    from paper_2105_08627_gb300 import build, svh
    build.build()
    n = 6000
    rng = np.random.default_rng(4)
    S_ = sp.diags([-np.ones(n - 1), 2.0 + 1e-6 * rng.random(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    b = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    with pytest.raises(svh.SVHError) as e:
        svh.device_amg_solve(S_, b, tol=1e-14, maxit=1)
    assert e.value.code == svh.SVH_ERR_NOT_CONVERGED
    x, it, lv = svh.device_amg_solve(S_, b, tol=1e-8, maxit=500)
    for r in range(2):
        for part in (np.real, np.imag):
            assert np.linalg.norm(S_ @ part(x[r]) - part(b[r])) <= 2e-8 * np.linalg.norm(part(b[r]))
