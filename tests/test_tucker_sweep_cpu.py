"""Row f4 (Sec. III.B, Figs. 2-3): the compression ratio the benchmark's sweep reports is the
count of octant-spectrum values over the count of values the Tucker data holds. Checked on a
plate's spectra against the oracle's own Tucker-SVD (Algorithm 1): its ranks give the library's
host Tucker-SVD ranks (to a tie at the threshold), and the arrays it returns hold exactly the
values the ratio's denominator counts. CR rises as the tolerance loosens."""
import os
import sys

import numpy as np
import pytest

import svh_synth as S
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op
from oracle import tucker as tk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _octant_spectra(Kx, Ky, Kz):
    T = gr.toeplitz_octant(Kx, Ky, Kz)
    P = (op.fft_size(Kx), op.fft_size(Ky), op.fft_size(Kz))
    S7 = op.spectra(gr.signed_from_octant(T), P)
    H = (P[0] // 2 + 1, P[1] // 2 + 1, P[2] // 2 + 1)
    octs = []
    for u in range(7):
        a = S7[u][:H[2], :H[1], :H[0]]
        octs.append(-a.imag if u in (1, 2, 3) else a.real)      # S kernels are imaginary
    return H, octs


def test_compression_ratio_counts_the_tucker_values():
    bench = _bench()
    H, octs = _octant_spectra(20, 20, 4)
    prev = None
    for tol in (1e-8, 1e-6, 1e-4):
        ranks, stored = [], 0
        for O in octs:
            C, Fs = tk.tucker_svd(O.transpose(2, 1, 0), tol)    # oracle modes (x, y, z)
            ranks.append(tuple(int(v) for v in C.shape))
            stored += C.size + sum(F.size for F in Fs)
        cr = bench.tucker_compression_ratio(H, ranks)
        assert cr == pytest.approx(7 * H[0] * H[1] * H[2] / stored, rel=1e-15)
        if prev is not None:
            assert cr >= prev                                     # looser tolerance, fewer values
        prev = cr


def test_library_host_tucker_ranks_match_the_oracle():
    from paper_2105_08627_gb300 import build, svh
    build.build()
    H, octs = _octant_spectra(20, 20, 4)
    for tol in (1e-8, 1e-4):
        for O in octs:
            C, Fs = tk.tucker_svd(O.transpose(2, 1, 0), tol)
            core, F = svh.host_tucker_svd(np.ascontiguousarray(O), tol)    # O[z, y, x]: mode 1 = x
            d = (core.shape[2], core.shape[1], core.shape[0])
            assert np.all(np.abs(np.asarray(d) - np.asarray(C.shape)) <= 1), (tol, d, C.shape)
