"""Tucker-SVD (Algorithm 1) and Tucker restore (Eq. 10-11), oracle.

Algorithm 1 unfolds the ORIGINAL tensor O along each mode i, takes its SVD,
keeps d_i left singular vectors as the factor F^i and projects the core onto
them in turn (C = C x_i F^i*). Reading of the truncation rule (the printed
"index of maximum normalized value smaller than tol/sqrt(3)" is ambiguous):
d_i is the smallest rank whose discarded singular values satisfy

    || sigma_{> d_i} ||_2 <= (tol / sqrt(3)) * || O ||_F,

which makes the three truncations together give ||O - O~||_F <= tol ||O||_F
(HOSVD error bound: the squared errors of the modes add up).
"""
from __future__ import annotations

import numpy as np


def unfold(O, mode):
    """Mode-i unfolding: rows indexed by axis ``mode``, columns by the others."""
    return np.moveaxis(O, mode, 0).reshape(O.shape[mode], -1)


def mode_product(T, F, mode):
    """(T x_mode F)[.., v, ..] = sum_i T[.., i, ..] F[v, i]   (Eq. 11)."""
    Tm = np.moveaxis(T, mode, 0)
    out = np.tensordot(F, Tm, axes=(1, 0))
    return np.moveaxis(out, 0, mode)


def tucker_svd(O, tol):
    """Algorithm 1 -> (core, [F1, F2, F3]) for a real or complex 3-D array."""
    O = np.asarray(O)
    normO = np.linalg.norm(O)
    thr = tol / np.sqrt(3.0) * normO
    C = O
    Fs = []
    for i in range(3):
        U, s, _ = np.linalg.svd(unfold(O, i), full_matrices=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]   # tail[r] = ||s[r:]||
        d = s.size
        for r in range(1, s.size + 1):
            rest = tail[r] if r < s.size else 0.0
            if rest <= thr:
                d = r
                break
        F = U[:, :d]
        Fs.append(F)
        C = mode_product(C, F.conj().T, i)
    return C, Fs


def tucker_restore(C, Fs):
    """Eq. 10: O = C x1 F1 x2 F2 x3 F3."""
    O = C
    for i, F in enumerate(Fs):
        O = mode_product(O, F, i)
    return O
