"""The oracle against values the paper prints (fixtures in tests/golden/, each citing its equation).

- Eq. 8: which of the 25 blocks of Z are zero.
- Eq. 16-18: the resistive self-term factors a/dx, a/(6 dx), a/(2 dx) of the diagonal blocks.
The oracle builds Z from the basis definitions and the Green's function integrals, so both are
independent checks of its basis normalisation and block assembly.
"""
import os

import numpy as np
import pytest

import svh_synth as S
from oracle import geometry as G
from oracle import greens as gr
from oracle import operator as op
from oracle import twofluid as tf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=1)


@pytest.fixture(scope="module")
def strip_Z():
    s = S.strip_cfg1()
    g = G.build_grid(s)
    T = gr.toeplitz_signed(s.Kx, s.Ky, s.Kz)
    om = 2 * np.pi * 1e9
    return g, op.dense_Z(g, T, om), om


def test_eq8_block_pattern(strip_Z):
    g, Z, _ = strip_Z
    pattern = _load("eq8_block_pattern.txt").reshape(5, 5)
    K = g.K
    for b in range(5):
        for a in range(5):
            blk = np.abs(Z[b * K:(b + 1) * K, a * K:(a + 1) * K]).max()
            assert (blk > 0) == bool(pattern[b, a]), (b, a, blk)


def test_eq16_18_resistive_self_terms(strip_Z):
    g, Z, om = strip_Z
    s_beta = _load("eq16_18_self_term_scale.txt")
    assert s_beta.shape == (5,)
    K = g.K
    for k in (0, K // 2, K - 1):
        a, _ = tf.ab(om, g.lam[k], g.sigma0[k])
        for beta in range(5):
            # the Green and kinetic parts are j omega mu (...), so the real part is the resistive term
            re = Z[beta * K + k, beta * K + k].real
            assert np.isclose(re, a * s_beta[beta] / g.dx, rtol=1e-12), (k, beta, re)
