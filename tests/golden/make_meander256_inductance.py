"""Writes meander256_inductance.txt: the port inductance of the 256 x 256 x 8 thin-film meander
(seed 202, 1 GHz) from the CPU oracle alone (its own kernel quadrature, FFT products and
right-preconditioned GMRES(50) with the exact Schur-complement preconditioner, RRE 1e-10).

Run from the repository root:  python tests/golden/make_meander256_inductance.py
The GPU test test_gpu_solve.py::test_meander256_inductance_vs_stored_oracle compares the
library's solve with the stored value at 1e-6 (the inductance bound of the mixed-precision solve).
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def main():
    import numpy as np

    import svh_synth as S
    from oracle import geometry as G
    from oracle import greens as gr
    from oracle import operator as op
    from oracle import solve as so

    s = S.meander_cfg2()
    g = G.build_grid(s)
    P = (op.fft_size(g.Kx), op.fft_size(g.Ky), op.fft_size(g.Kz))
    t0 = time.time()
    T = gr.toeplitz_octant(g.Kx, g.Ky, g.Kz, processes=os.cpu_count() or 1)
    S7 = op.spectra(gr.signed_from_octant(T), P)
    res = so.port_inductance(s, S7=S7, P=P, freq=s.freqs[0], rre=1e-10)
    L = np.asarray(res["L"])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "meander256_inductance.txt")
    with open(out, "w") as f:
        f.write("# Port inductance (H) of the 256x256x8 meander (svh_synth.meander_cfg2, seed 202) at 1 GHz,\n")
        f.write("# CPU oracle: own kernel quadrature, FFT products (Eq. 9), GMRES(50) to RRE 1e-10 with the\n")
        f.write("# exact Schur-complement preconditioner (Eq. 12-15); written by make_meander256_inductance.py\n")
        f.write(f"# oracle GMRES iterations: {res['iters']}, wall {time.time() - t0:.0f} s\n")
        for row in np.atleast_2d(L):
            f.write(" ".join(f"{v:.15e}" for v in row) + "\n")
    print(out, L)


if __name__ == "__main__":
    main()
