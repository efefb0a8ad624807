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
    items = S.batch_cfg3(seed=303, n_items=8)
    return [items[3], items[5], items[0]]        # 33x65x14, 56x35x10, 71x52x15: uneven grids


def test_batch_matvec_persistent_launch_vs_oracle():
    """One persistent launch applies three unevenly sized structures, each with its own number of
    right-hand sides and per-right-hand-side frequencies; every item equals the oracle's FFT
    product (FP32 1e-5, FP64 1e-11), on the capturing call and on a graph replay."""
    import torch

    from paper_2105_08627_gb300 import svh
    items = _items()
    nbs = [2, 3, 1]
    refs, xs = [], []
    hs = [handle_for(s) for s in items]
    for i, (s, nb) in enumerate(zip(items, nbs)):
        g, S7, P, T = oracle_reference(s, processes=4)
        oms = 2 * np.pi * np.array(s.freqs)[np.arange(nb) % 3]
        x = S.random_complex(900 + i, (nb, g.N))
        refs.append((oms, np.stack([op.apply_K_fft(g, S7, x[r], oms[r], P) for r in range(nb)])))
        xs.append(x)
    b = svh.Batch(0)
    for h in hs:
        b.add(h)
    for mode, dt, tol in ((0, torch.complex64, 1e-5), (0, torch.complex128, 1e-11),
                          (1, torch.complex64, 1e-5), (1, torch.complex128, 1e-11)):
        b.set_mode(mode)                           # 0: persistent queue, 1: per-structure chains
        xd = [torch.from_numpy(x).to(dt).cuda() for x in xs]
        yd = [torch.full_like(x, float("nan")) for x in xd]
        prec = svh.SVH_FP32 if dt == torch.complex64 else svh.SVH_FP64
        for rep in range(2):                       # capture, then replay
            for y in yd:
                y.fill_(float("nan"))
            torch.cuda.synchronize()
            b.matvec([r[0] for r in refs], xd, yd, prec)
            b.sync()
            for i, (oms, yref) in enumerate(refs):
                y = yd[i].cpu().numpy().astype(np.complex128)
                for r in range(nbs[i]):
                    assert rel_err(y[r], yref[r]) <= tol, (mode, dt, rep, i, r, rel_err(y[r], yref[r]))
                    if dt == torch.complex64:
                        assert np.abs(y[r] - yref[r]).max() <= 2 * tol * np.abs(yref[r]).max()
    ms = b.autotune([r[0] for r in refs], xd, yd, svh.SVH_FP64)
    assert np.all(ms > 0) and b.mode == (1 if ms[1] < ms[0] else 0)
    b.close()
    for h in hs:
        h.close()


def test_batch_queue_wait_runs_out_with_timeout_status():
    """A wait of the batch queue on a pass whose completion nothing counts ends after its bound
    with SVH_ERR_TIMEOUT (no fault, no hang); the batch then runs correctly again."""
    import time

    import torch

    from paper_2105_08627_gb300 import svh
    items = _items()[:2]
    hs = [handle_for(s) for s in items]
    b = svh.Batch(0)
    for h in hs:
        b.add(h)
    xs = [torch.from_numpy(S.random_complex(950 + i, (2, h.info()["N"])).astype(np.complex64)).cuda()
          for i, h in enumerate(hs)]
    ys = [torch.empty_like(x) for x in xs]
    oms = [2 * np.pi * 1e9] * 2
    b.set_wait(50.0, hold_item=1, hold_phase=2)     # y-forward of item 1 never counts as done
    t0 = time.perf_counter()
    b.matvec(oms, xs, ys)
    with pytest.raises(svh.SVHError) as e:
        b.sync()
    assert e.value.code == svh.SVH_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    b.set_wait(1000.0)
    b.matvec(oms, xs, ys)
    b.sync()
    for i, h in enumerate(hs):
        ref = h.matvec(oms[i], xs[i]).cpu().numpy()
        got = ys[i].cpu().numpy()
        for r in range(2):
            assert rel_err(got[r], ref[r]) <= 1e-6
    b.close()
    for h in hs:
        h.close()


def test_batch_solve_vs_oracle():
    """Port inductances of every structure of a batch solve against the oracle's solves
    (L within 1e-6), at two frequencies."""
    from paper_2105_08627_gb300 import svh
    items = _items()[:2]
    hs = [handle_for(s) for s in items]
    b = svh.Batch(0)
    for h in hs:
        b.add(h)
    freqs = [1e9, 10e9]
    res = b.solve(freqs, n_workers=2)
    assert res["stats"]["final_rre"] <= 1e-8
    for i, s in enumerate(items):
        for fi, f in enumerate(freqs):
            ref = so.port_inductance(s, freq=f, rre=1e-10)
            L = res["L"][i][fi]
            assert np.abs(L - ref["L"]).max() <= 1e-6 * np.abs(np.diag(ref["L"])).max(), (i, f)
            assert np.allclose(L, res["Z"][i][fi].imag / (2 * np.pi * f), rtol=1e-14, atol=0)
    b.close()
    for h in hs:
        h.close()
