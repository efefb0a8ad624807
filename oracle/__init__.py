"""CPU FP64 oracle for the SuperVoxHenry operator (arXiv 2105.08627).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package. The CUDA
library never calls it, and it never calls the CUDA library. The two share no
code; only the seeded input generators in ``svh_synth`` feed both.

Everything here is plain, slow and in float64 / complex128:

* ``twofluid``  -- two-fluid conductivity (Eq. 3) and the diagonal terms (Eq. 9, 16-18, 22-23)
* ``greens``    -- unit Green's-function Toeplitz kernels over voxel pairs (Eq. 19-21, App. B)
* ``geometry``  -- voxel list, face-node numbering, incidence matrix A (Eq. 7), ports
* ``operator``  -- dense Z (Eq. 8), circulant embedding + FFT matvec (Eq. 9), full Eq. 7 operator,
                   selected rows of the product by direct summation
* ``tucker``    -- Tucker-SVD (Algorithm 1) and the restore by mode products (Eq. 10-11)
* ``solve``     -- right-preconditioned GMRES(50) (Sec. III), the Schur-complement
                   preconditioner (Eq. 12-15, exact sparse solve), port admittance -> inductance

Pins: every function is checked in ``tests/`` against something other than
itself (closed forms, far-field expansions, brute force, invariants). Parity
is unpinned only where stated in the docstring of the function concerned.
"""
