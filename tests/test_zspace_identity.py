"""The direct z pass's reading of Eq. 9 (CPU, numpy only): along z, the circulant
product over the active planes equals a plain block-Toeplitz product with z-space
kernels. With the transforms' conventions (forward e^-, inverse e^+ unnormalised), the
z-even octant spectra give r(dz) = sum_az c_az S(az) cos(2 pi az dz / Pz) and the odd
S_z spectrum (carrying -i sign(kz)) gives i rho(dz), rho(dz) = sum_az c_az S(az)
sin(2 pi az dz / Pz), c_az = 2 inside the octant and 1 at az = 0 and Pz / 2. The +-i
factors of the S_z terms then cancel. Checked against the frequency-domain 5 x 5 block
product (the block structure of Eq. 7: G00 on the diagonal, S_a coupling the
divergence bases, Q on the 2-D/3-D bases), for consecutive and gapped active planes."""
import numpy as np
import pytest


def _mi(v):
    return -1j * v


def _pi(v):
    return 1j * v


def _block_freq(I, g, sx, sy, sz, qx, qy, qz):
    Ix, Iy, Iz, I2, I3 = I
    qs, qd = qx + qy, qx - qy
    return np.array([
        g * Ix + sx * _mi(I2 + I3),
        g * Iy + sy * _mi(I3 - I2),
        g * Iz + 2 * sz * _pi(I3),
        sx * _pi(Ix) - sy * _pi(Iy) + qs * I2 + qd * I3,
        sx * _pi(Ix) + sy * _pi(Iy) - 2 * sz * _pi(Iz) + qd * I2 + (qs + 4 * qz) * I3,
    ])


@pytest.mark.parametrize("Pz,zl", [(16, [0, 1, 2, 3, 4, 5]), (16, [0, 1, 3, 4, 6, 7]), (12, [1, 2, 3]),
                                   (8, [0, 1, 2, 3]), (48, [2, 5, 9, 17, 20, 23])])
def test_direct_z_product_equals_fft_form(Pz, zl):
    rng = np.random.default_rng(Pz + len(zl))
    Hz = Pz // 2 + 1
    S = rng.standard_normal((7, Hz))
    S[3, 0] = S[3, Pz // 2] = 0.0                    # the odd S_z spectrum vanishes there
    sgx, sgy = -1.0, 1.0                             # x/y signs of the odd S_x, S_y at this (kx, ky)
    kz = np.arange(Pz)
    az = np.minimum(kz, Pz - kz)
    sgn = np.where(2 * kz <= Pz, 1.0, -1.0)
    s = np.array([S[u, az] for u in range(7)])
    s[1] *= sgx
    s[2] *= sgy
    s[3] *= sgn
    nza = len(zl)
    X = rng.standard_normal((5, nza)) + 1j * rng.standard_normal((5, nza))
    xf = np.zeros((5, Pz), complex)
    xf[:, zl] = X
    Yfft = (np.fft.ifft(_block_freq(np.fft.fft(xf, axis=1), *s), axis=1) * Pz)[:, zl]
    D = zl[-1] - zl[0] + 1
    c = np.array([1.0 if (a == 0 or 2 * a == Pz) else 2.0 for a in range(Hz)])
    th = 2 * np.pi * np.outer(np.arange(D), np.arange(Hz)) / Pz
    wc, ws = c * np.cos(th), np.where(c == 2.0, 2.0, 0.0) * np.sin(th)
    R = np.array([(ws if u == 3 else wc) @ S[u] for u in range(7)])
    Yd = np.zeros((5, nza), complex)
    for i in range(nza):
        for j in range(nza):
            dz = zl[i] - zl[j]
            g, sx, sy, rho = R[0, abs(dz)], sgx * R[1, abs(dz)], sgy * R[2, abs(dz)], np.sign(dz) * R[3, abs(dz)]
            qx, qy, qz = R[4, abs(dz)], R[5, abs(dz)], R[6, abs(dz)]
            Ix, Iy, Iz, I2, I3 = X[:, j]
            Yd[:, i] += [g * Ix + sx * _mi(I2 + I3), g * Iy + sy * _mi(I3 - I2), g * Iz - 2 * rho * I3,
                         sx * _pi(Ix) - sy * _pi(Iy) + (qx + qy) * I2 + (qx - qy) * I3,
                         sx * _pi(Ix) + sy * _pi(Iy) + 2 * rho * Iz + (qx - qy) * I2 + (qx + qy + 4 * qz) * I3]
    assert np.abs(Yd - Yfft).max() <= 1e-13 * np.abs(Yfft).max()
