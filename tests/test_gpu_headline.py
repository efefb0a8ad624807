"""Parity of the exact path the benchmark times, at the benchmark's sizes, against the oracle.

The benchmark's step is one FP32 product of nb right-hand sides with the kernel spectra
Tucker-compressed on the device at tol 1e-8 (Algorithm 1) and restored by the tensor-core
GEMMs in every product (Eq. 10-11, SVH_KERNELS_TUCKER_REBUILD), on the FFT tiles that the
autotuner picks. These tests run that path (and every z-pass form the autotuner may pick at
that size) on dense random inputs, distinct per right-hand side, and compare element by element
with the oracle: on the 512 x 512 x 24 eSFQ-like block (P = 1024 x 1024 x 48, nb = 16) through
the oracle's direct row sums with its own quadrature table, and on the 256 x 256 x 8 meander
(nb = 4) through its full FFT product. Bound: every compared value within 2e-5 of the
largest compared value of its right-hand side (the FP32 tolerance of the other tests), plus
the 1e-5 relative 2-norm bound where the whole vector is compared.
"""
import os

import numpy as np
import pytest

import svh_synth as S
from gpu_util import handle_for, oracle_reference, rel_err
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP32_TOL = 1e-5


def _bench_handle(s, nb):
    from paper_2105_08627_gb300 import svh
    h = handle_for(s)                               # device quadrature: independent of the oracle
    h.tucker_compress(1e-8)                         # Algorithm 1 on the device
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    tiles, _ = h.autotune(nb)
    return h, tiles


def test_esfq512_bench_path_dense_input():
    import torch
    from paper_2105_08627_gb300 import svh
    s = S.esfq_cfg5()
    g = G.build_grid(s)
    T = gr.toeplitz_octant(g.Kx, g.Ky, g.Kz, processes=os.cpu_count() or 1)
    nb = 16
    h, tiles = _bench_handle(s, nb)
    info = h.info()
    assert (info["Px"], info["Py"], info["Pz"]) == (1024, 1024, 48)
    om = 2 * np.pi * s.freqs[0]
    x = S.random_complex(5050, (nb, g.N))
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    rng = np.random.default_rng(5051)
    rows = np.concatenate([[0, g.K - 1], rng.choice(g.K, 30, replace=False)])
    nodes = np.concatenate([[0, g.M - 1], rng.choice(g.M, 30, replace=False)])
    yv, yn = op.direct_rows_table(g, T, x, om, rows, nodes)
    K = g.K

    def check(y, what):
        y = y.cpu().numpy().astype(np.complex128)
        for b in range(nb):
            got = np.concatenate([y[b, :5 * K].reshape(5, K)[:, rows].ravel(), y[b, 5 * K + nodes]])
            ref = np.concatenate([yv[b].ravel(), yn[b]])
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= 2 * FP32_TOL, (what, b, err)

    check(h.matvec(om, xd), f"autotuned tiles {tiles.tolist()}")
    assert h.device_status() == 0
    counts, chosen = h.pass_variants()
    for sched in range(counts[6]):                   # stream schedules
        h.set_pass_variant(6, sched)
        check(h.matvec(om, xd), f"schedule {sched}")
    h.set_pass_variant(6, int(chosen[6]))
    for p in (2, 1, 3, 0, 4):                        # every tile variant of every pass at this size
        for v in range(counts[p]):
            h.set_pass_variant(p, v)
            check(h.matvec(om, xd), f"pass {p} variant {v}")
            assert h.device_status() == 0
        h.set_pass_variant(p, int(chosen[p]))
    h.close()


def test_meander256_bench_path_dense_input():
    import torch
    from paper_2105_08627_gb300 import svh
    s = S.meander_cfg2()
    g, S7, P, T = oracle_reference(s, processes=os.cpu_count() or 1)
    nb = 4
    h, tiles = _bench_handle(s, nb)
    om = 2 * np.pi * s.freqs[0]
    x = S.random_complex(2020, (nb, g.N))
    Zh = op.block_spectra(S7)
    yref = np.stack([op.apply_K_fft(g, S7, x[b], om, P, Zh=Zh) for b in range(nb)])
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()

    def check(what):
        y = h.matvec(om, xd).cpu().numpy().astype(np.complex128)
        for b in range(nb):
            assert rel_err(y[b], yref[b]) <= FP32_TOL, (what, b, rel_err(y[b], yref[b]))
            assert np.abs(y[b] - yref[b]).max() <= 2 * FP32_TOL * np.abs(yref[b]).max(), (what, b)
        assert h.device_status() == 0

    check(f"autotuned tiles {tiles.tolist()}")
    counts, chosen = h.pass_variants()
    for p in (2, 1, 3, 0, 4):                        # every tile variant (z: FFT forms and the direct pass)
        for v in range(counts[p]):
            h.set_pass_variant(p, v)
            check(f"pass {p} variant {v}")
        h.set_pass_variant(p, int(chosen[p]))
    for sched in range(counts[6]):                   # stream schedules with the restore
        h.set_pass_variant(6, sched)
        check(f"schedule {sched}")
    h.close()
