"""Batching (row a12): per-item frequencies in one product, all (port, frequency)
pairs in one solve, and batches of unevenly sized structures (graph-captured
products, concurrent solves), each against the unbatched library calls and the
oracle."""
import numpy as np
import pytest

import svh_synth as S
from gpu_util import handle_for, oracle_reference, rel_err
from oracle import operator as op
from oracle import solve as so

pytestmark = pytest.mark.gpu


def test_per_item_frequencies_equal_separate_products():
    import torch
    s = S.random_blob(71, 20, 14, 5, fill=0.5)
    h = handle_for(s)
    N = h.info()["N"]
    oms = 2 * np.pi * np.array([1e9, 10e9, 50e9])
    x = S.random_complex(5, (3, N))
    g, S7, P, T = oracle_reference(s)
    for dt, tol in ((torch.complex128, 1e-13), (torch.complex64, 1e-6)):
        xd = torch.from_numpy(x).to(dt).cuda()
        y = h.matvec_omegas(oms, xd).cpu().numpy().astype(np.complex128)
        for b in range(3):
            yb = h.matvec(oms[b], xd[b].contiguous()).cpu().numpy().astype(np.complex128)
            assert rel_err(y[b], yb) <= tol
            yref = op.apply_K_fft(g, S7, x[b], oms[b], P)
            assert rel_err(y[b], yref) <= (1e-11 if dt == torch.complex128 else 1e-5)
    h.close()


def test_multi_frequency_solve_equals_single_frequency_solves():
    s = S.bar(12, 9, 3, 1, 10, 1, 2, 0, 1)
    s2 = S.bar(12, 9, 3, 1, 10, 5, 7, 0, 1)
    s.occ |= s2.occ
    s.lam += s2.lam
    s.sigma0 += s2.sigma0
    s.ports += s2.ports
    freqs = [1e9, 10e9, 50e9]
    h = handle_for(s)
    res = h.solve(freqs)
    for fi, f in enumerate(freqs):
        one = h.solve([f])
        assert np.abs(res["Z"][fi] - one["Z"][0]).max() <= 1e-7 * np.abs(one["Z"][0]).max()
        ref = so.port_inductance(s, freq=f, rre=1e-10)
        assert np.abs(res["Z"][fi] - ref["Z"]).max() <= 1e-6 * np.abs(ref["Z"]).max()
    h.close()


def _items():
    return S.batch_cfg3(seed=303, n_items=6)[:3]


def test_batch_matvec_graph_equals_individual_products():
    import torch

    from paper_2105_08627_gb300 import svh
    items = _items()
    hs = [handle_for(s) for s in items]
    b = svh.Batch(0)
    for h in hs:
        b.add(h)
    oms = [2 * np.pi * 1e9, 2 * np.pi * 10e9, 2 * np.pi * 50e9]
    xs, ys = [], []
    for i, h in enumerate(hs):
        N = h.info()["N"]
        xs.append(torch.from_numpy(S.random_complex(i, (2, N)).astype(np.complex64)).cuda())
        ys.append(torch.zeros((2, N), dtype=torch.complex64, device="cuda"))
    for rep in range(2):                  # capture, then replay
        for y in ys:
            y.zero_()
        torch.cuda.synchronize()
        b.matvec(oms, xs, ys, svh.SVH_FP32, nb=2)
        b.sync()
        for i, h in enumerate(hs):
            ref = h.matvec(oms[i], xs[i]).cpu().numpy()
            assert np.array_equal(ys[i].cpu().numpy(), ref), (rep, i)
    b.close()
    for h in hs:
        h.close()


def test_batch_solve_equals_individual_solves():
    from paper_2105_08627_gb300 import svh
    items = _items()
    hs = [handle_for(s) for s in items]
    b = svh.Batch(0)
    for h in hs:
        b.add(h)
    freqs = [1e9, 10e9]
    res = b.solve(freqs, n_workers=3)
    assert res["stats"]["final_rre"] <= 1e-8
    for i, h in enumerate(hs):
        one = h.solve(freqs)
        assert np.abs(res["Z"][i] - one["Z"]).max() <= 1e-7 * np.abs(one["Z"]).max()
        assert np.all(np.diagonal(res["L"][i], axis1=1, axis2=2) > 0)
    b.close()
    for h in hs:
        h.close()
