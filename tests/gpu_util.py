"""Helpers shared by the GPU tests (library handles and oracle references)."""
import numpy as np

import svh_synth as S
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op


def handle_for(structure, toeplitz=None, P=None):
    import torch

    from paper_2105_08627_gb300 import build, svh
    build.build()
    h = svh.Handle(0, torch.cuda.current_stream().cuda_stream)
    h.setup_structure(structure)
    if P is not None:
        h.set_fft_sizes(*P)
    if toeplitz is None:
        h.generate_toeplitz()
    else:
        h.load_toeplitz(toeplitz)
    return h


def oracle_reference(structure, P=None, processes=1):
    """(grid, S7, P, T) of the oracle for a structure, with its own kernels (their z planes
    integrated in `processes` spawned worker processes)."""
    g = G.build_grid(structure)
    if P is None:
        P = (op.fft_size(g.Kx), op.fft_size(g.Ky), op.fft_size(g.Kz))
    T = gr.toeplitz_octant(g.Kx, g.Ky, g.Kz, processes=processes)
    S7 = op.spectra(gr.signed_from_octant(T), P)
    return g, S7, P, T


def rel_err(y, yref):
    return np.linalg.norm(y - yref) / np.linalg.norm(yref)
