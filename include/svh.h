/*
 * svh.h -- C ABI of the GB300 library for the FFT-accelerated voxel VIE
 * operator of SuperVoxHenry (arXiv 2105.08627).
 *
 * The library applies the operator of Eq. 7,
 *
 *     [ Z   -A^T ] [ I   ]
 *     [ A    0   ] [ Phi ],
 *
 * where Z (Eq. 8) is the two-fluid diagonal (Eq. 3, 9, 16-18, 22-23) plus
 * j*omega*mu*dx times Green's-function convolutions over the voxel grid,
 * evaluated as in Eq. 9 by zero-padded 3-D FFTs whose kernel spectra are
 * rebuilt from a Tucker representation (Eq. 10-11), and A is the face-node
 * incidence matrix of current continuity (Eq. 7, Eq. 2).
 *
 * Conventions (all calls):
 *  - Every call returns SVH_OK (0) or one of the SVH_ERR_* codes below; on
 *    error svh_last_error() gives a message owned by the handle (valid until
 *    the next call on that handle).
 *  - Complex numbers are interleaved (re, im) pairs of float (SVH_FP32) or
 *    double (SVH_FP64).
 *  - Grid arrays are row-major with x fastest: index x + Kx*(y + Ky*z).
 *  - Voxels (the K non-empty cells) are numbered in that raster order. Face
 *    nodes are numbered by scanning voxels in order and, per voxel, its faces
 *    in the order -x,+x,-y,+y,-z,+z: a face takes the next id the first time
 *    it is met (a face shared by two voxels is one node).
 *  - A vector of the operator has N = 5K + M entries laid out as
 *    [I^x (K), I^y (K), I^z (K), I^2D (K), I^3D (K), Phi (M)].
 *  - Pointer arguments ending in _dev are device pointers on the handle's
 *    device, used in stream order on the handle's stream; all other pointers
 *    are host memory, read or written before the call returns. The caller
 *    keeps ownership of every array it passes; the library owns all of its
 *    internal buffers and frees them in svh_destroy().
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 *  - The seven unit kernels are indexed 0..6 = G00, Sx, Sy, Sz, Qx, Qy, Qz:
 *    G00 couples constant moments, S_a a constant observer moment with the
 *    source moment xi_a, Q_a the moments xi_a and xi'_a (App. A, Eq. 19-21).
 *    They are dx-free (unit voxel, App. B): the library multiplies the
 *    convolution by j*omega*mu*dx, which together with the basis
 *    normalisation of Eq. 16-18 realises the dx^5 scale of App. B.
 */
#ifndef SVH_H
#define SVH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svh_handle svh_handle;

#define SVH_OK                 0
#define SVH_ERR_ARG            1  /* invalid argument or size mismatch */
#define SVH_ERR_CUDA           2  /* a CUDA runtime call failed */
#define SVH_ERR_OOM            3  /* device or host allocation failed */
#define SVH_ERR_NOT_CONVERGED  4  /* iterative solve stopped above its tolerance */
#define SVH_ERR_TIMEOUT        5  /* a bounded device wait ran out */
#define SVH_ERR_SINGULAR       6  /* singular port matrix or preconditioner */
#define SVH_ERR_STATE          7  /* call made before a prerequisite call */

#define SVH_FP32 0
#define SVH_FP64 1

/* Kernel-spectrum modes for svh_set_kernel_mode(). */
#define SVH_KERNELS_RESIDENT        0 /* octant spectra stay in HBM (default) */
#define SVH_KERNELS_TUCKER_REBUILD  1 /* every FP32 matvec first rebuilds the spectra from
                                         their Tucker cores and factors (Sec. II.B.2) */

/* One port: a unit voltage source between the faces of its plus terminal and
 * the faces of its minus terminal (Sec. II.A). Each face is encoded as
 * voxel_linear_index*6 + face, face order -x,+x,-y,+y,-z,+z. */
typedef struct {
    int32_t n_plus;
    const int32_t* plus;
    int32_t n_minus;
    const int32_t* minus;
} svh_port;

typedef struct {
    int32_t Kx, Ky, Kz;        /* voxel grid */
    int32_t Px, Py, Pz;        /* FFT sizes, each >= 2K_i - 1 (2K_i when smooth) */
    int32_t Hx, Hy, Hz;        /* octant sizes P_i/2 + 1 of the stored spectra */
    int64_t K, M, N;           /* non-empty voxels, face nodes, unknowns 5K+M */
    int32_t nports;
    int32_t n_fixed_nodes;     /* terminal nodes plus one gauge node per floating island */
    int32_t n_active_planes;   /* z planes holding at least one voxel */
    int32_t n_active_rows;     /* (z, y) rows holding at least one voxel */
    double dx;                 /* voxel edge (m) */
} svh_grid_info;

/* Create a handle bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL means the legacy default stream). */
int svh_create(svh_handle** h, int device, void* stream);
int svh_destroy(svh_handle* h);
const char* svh_last_error(const svh_handle* h);
int svh_set_stream(svh_handle* h, void* stream);

/* Voxel grid, materials and ports (Sec. II.A; Eq. 3 materials).
 *  occ[Kz*Ky*Kx]   : 1 for a non-empty voxel, 0 otherwise;
 *  lambda, sigma0  : London depth (m) and normal conductivity (S/m) per grid
 *                    cell (read only at non-empty cells; lambda > 0 there);
 *  ports[nports]   : terminal face lists (may be NULL when nports == 0).
 * Builds the voxel list, face nodes, the implicit incidence A, the port
 * terminals and gauge nodes, and picks FFT sizes: per axis the smallest
 * P >= 2K - 1 with size-specialised kernels (x, y: 16, 32, 48, 64, 96, 128,
 * 192, 256, 384, 512, 768, 1024; z: 8, 12, 16, 24, 32, 48), else the
 * smallest 2,3,5,7-smooth P >= 2K - 1 (2K first). Errors: SVH_ERR_ARG for
 * non-positive sizes or dx, an empty grid, lambda <= 0 on a voxel, or a port
 * face on an empty voxel. Invalidates previously loaded kernels. */
int svh_setup_grid(svh_handle* h, int Kx, int Ky, int Kz, double dx,
                   const uint8_t* occ, const double* lambda, const double* sigma0,
                   const svh_port* ports, int nports);
/* Override the FFT sizes chosen by svh_setup_grid (each P_i >= 2K_i - 1 with
 * prime factors 2, 3, 5, 7 only). Must precede the kernel calls below. */
int svh_set_fft_sizes(svh_handle* h, int Px, int Py, int Pz);
int svh_get_grid_info(const svh_handle* h, svh_grid_info* info);
/* Face-node ids of every voxel, node[K*6] (for tests and post-processing). */
int svh_get_nodes(const svh_handle* h, int32_t* node);

/* Unit Toeplitz kernels (App. B, Eq. 19-21 and the off-diagonal blocks of
 * Eq. 8) at the non-negative lattice offsets 0 <= d < K, T[7][Kz][Ky][Kx]
 * (double). svh_generate_toeplitz computes them on the device by quadrature
 * (Duffy transform at the singular offsets, Gauss-Legendre elsewhere);
 * svh_load_toeplitz takes them from the caller. Either call also embeds them
 * in the 2K circulant and transforms it (Eq. 9), storing the octant spectra
 * described at svh_get_spectra. Requires svh_setup_grid. */
int svh_generate_toeplitz(svh_handle* h);
int svh_load_toeplitz(svh_handle* h, const double* T);
int svh_get_toeplitz(const svh_handle* h, double* T);

/* Octant spectra S[7][Hz][Hy][Hx] (double): the FFT of kernel u's circulant
 * at frequency k is S_u(|k|) for the even kernels G00, Qx, Qy, Qz and
 * -j*sign_a(k)*S_u(|k|) for S_a, with |k|_i = min(k_i, P_i - k_i) and
 * sign_a(k) = +1 for k_a <= P_a/2, -1 otherwise. */
int svh_get_spectra(const svh_handle* h, double* S);
/* The FP32 copy of the octant spectra on the device, which the FFT forms of
 * the FP32 z pass read (same layout, float S[7][Hz][Hy][Hx]; S host memory,
 * 7 Hz Hy Hx floats, owned by the caller). After svh_rebuild_spectra, or a
 * product in SVH_KERNELS_TUCKER_REBUILD mode with an FFT z pass, it holds the
 * Tucker restore (a rebuild-mode product with the direct z pass restores its
 * z-space kernels instead and leaves these as they were). Synchronises the
 * handle's stream. SVH_ERR_ARG for a null S, SVH_ERR_STATE without kernels. */
int svh_get_spectra32(svh_handle* h, float* S);

/* Tucker representation (Eq. 10) of kernel `kernel_id`'s octant spectrum:
 * S = core x1 F1 x2 F2 x3 F3 with core[d3][d2][d1] (d1 index fastest),
 * F1[Hx][d1], F2[Hy][d2], F3[Hz][d3] row-major (double). Loading switches
 * that kernel to Tucker storage; svh_rebuild_spectra (or every FP32 matvec
 * in SVH_KERNELS_TUCKER_REBUILD mode) restores it on the device (Eq. 11). */
int svh_load_tucker(svh_handle* h, int kernel_id, int d1, int d2, int d3,
                    const double* core, const double* F1, const double* F2, const double* F3);
/* Algorithm 1 (Tucker-SVD) applied to the current FP64 octant spectra with
 * truncation ||sigma_discarded|| <= tol/sqrt(3) * ||S||_F per mode; installs
 * the result as by svh_load_tucker. ranks[7*3] (may be NULL) receives d1,d2,d3.
 * Per mode the left singular vectors of the unfolding come from a Householder
 * QR of its transpose and an SVD of the triangle (accurate to eps sigma_max,
 * so the ranks are those of an SVD of the unfolding also at tol 1e-8), the
 * rank from the residual rows u_r^T S_(i). svh_tucker_compress runs on the
 * device (cuSOLVER QR and SVD, cuBLAS GEMMs, the library's row-norm kernels, on
 * the handle's stream; synchronises it); svh_tucker_compress_on(..., 0) runs
 * the same steps on the host cores (one-sided Jacobi for the SVD). Errors:
 * SVH_ERR_STATE without kernels, SVH_ERR_ARG unless 0 < tol < 1. */
int svh_tucker_compress(svh_handle* h, double tol, int32_t* ranks);
int svh_tucker_compress_on(svh_handle* h, double tol, int32_t* ranks, int on_device);
/* Copy out the Tucker data of one kernel; pass NULL arrays to query d1,d2,d3. */
int svh_get_tucker(const svh_handle* h, int kernel_id, int32_t* d, double* core,
                   double* F1, double* F2, double* F3);
int svh_set_kernel_mode(svh_handle* h, int mode);
/* Restore the FP32 octant spectra of all Tucker-stored kernels now (Eq. 10). */
int svh_rebuild_spectra(svh_handle* h);

/* y = Kop x for nb vectors (Eq. 7 with Z applied by Eq. 9):
 *   rows of I:   y^beta = z^beta I^beta + j omega mu dx * (conv)^beta - (A^T Phi)^beta
 *   rows of Phi: y = A I.
 * x_dev, y_dev: nb*N complex values (interleaved) of the chosen precision,
 * item b at offset b*N; x_dev and y_dev must not overlap. omega > 0 (rad/s).
 * precision: SVH_FP32 (FFT and multiply in float, spectra in float) or
 * SVH_FP64. Asynchronous on the handle's stream. Requires kernels. */
int svh_matvec(svh_handle* h, double omega, int nb, const void* x_dev, void* y_dev,
               int precision);
/* Same product with a different angular frequency per batch item
 * (omegas[nb], host memory): many ports and frequencies of one structure in
 * one launch sequence. The kernel spectra do not depend on omega (the Green
 * function is static, Sec. II.A); only the j omega mu dx scale and the
 * two-fluid diagonal change per item. */
int svh_matvec_omegas(svh_handle* h, const double* omegas, int nb, const void* x_dev, void* y_dev,
                      int precision);
/* Same product from and to host memory: copies x to the device, applies the
 * operator and copies y back before returning (synchronous). */
int svh_matvec_host(svh_handle* h, double omega, int nb, const void* x, void* y,
                    int precision);

/* ---- Port solves (Sec. II.C and Sec. III).
 * For each angular frequency and each port j, solves Eq. 7 with a unit
 * potential on port j's plus-terminal nodes and zero on every other fixed
 * node (all ports' terminals and one gauge node per floating island); fixed
 * nodes leave the unknowns. The solver is right-preconditioned flexible
 * GMRES(restart) with FP64 Arnoldi on the device; the preconditioner is the
 * sparse P = Q^{-1}, Q = [Y, -A^T; A, 0], Y = diag(|Z_kk|) (Eq. 12), applied
 * through the Schur complement S = A Y^{-1} A^T (Eq. 13-15) whose solves run
 * by AMG-preconditioned CG to amg_tol: the aggregation hierarchy is built on
 * the host once per frequency and the CG with its K-cycle runs on the device
 * (amg_on_device = 1) or on the host cores (0). With inner_precision =
 * SVH_FP32 the Krylov products use the FP32 operator and an FP64 refinement
 * loop restores the FP64 residual. The iteration stops when every port's
 * relative residual ||b - K x|| / ||b||, measured with the FP64 operator, is
 * <= rre. Port currents I_p = sum of (A I) over port p's plus-terminal nodes
 * give the admittance Y[p][j]; Zport = Y^{-1} (the inductance is Im(Z)/omega). */
typedef struct {
    int32_t restart;           /* GMRES restart length (default 50, Sec. III) */
    int32_t max_iterations;    /* inner iterations per refinement step (default 2000) */
    int32_t max_refinements;   /* FP64 refinement steps (default 8) */
    int32_t inner_precision;   /* SVH_FP32 (default) or SVH_FP64 */
    double rre;                /* relative residual target (default 1e-8, Sec. III) */
    double amg_tol;            /* relative tolerance of each Schur solve (default 1e-8, Sec. II.C) */
    int32_t amg_on_device;     /* 1 (default): Schur solves by AMG-CG on the device; 0: on the host cores */
} svh_options;

typedef struct {
    int32_t iterations;        /* inner GMRES iterations, all frequencies */
    int32_t refinements;       /* refinement steps, all frequencies */
    int32_t amg_levels;        /* levels of the last AMG hierarchy */
    double amg_avg_iterations; /* CG iterations per Schur solve, last frequency */
    double final_rre;          /* largest final relative residual over ports and frequencies */
    double setup_seconds;      /* preconditioner set-up time */
    double solve_seconds;      /* everything else */
} svh_stats;

void svh_default_options(svh_options* opt);
/* omegas[nfreq] (rad/s, > 0); Zport receives nfreq * nports * nports complex
 * values (interleaved), Zport[f][p][q]; Lport (may be NULL) receives the port
 * inductances nfreq * nports * nports doubles, Lport[f][p][q] =
 * Im(Zport[f][p][q]) / omegas[f] (H; the quantity whose error Sec. III
 * reports). opt may be NULL (defaults), st may be NULL. Returns
 * SVH_ERR_NOT_CONVERGED (with Zport and Lport filled) if some residual stays
 * above rre. Requires kernels and at least one port. */
int svh_solve(svh_handle* h, const double* omegas, int nfreq, const svh_options* opt, double* Zport,
              double* Lport, svh_stats* st);
/* Solution vector x[N] (complex interleaved double) of port `port` at the
 * last frequency of the last svh_solve (fixed-node potentials are 0). */
int svh_get_solution(const svh_handle* h, int port, double* x);
/* Per-voxel materials (voxel order, length K): London depth (m, > 0) and
 * normal conductivity (S/m, >= 0). Replaces those given to svh_setup_grid
 * (kernels and FFT sizes are unaffected; the next svh_solve uses them). */
int svh_set_materials(svh_handle* h, const double* lambda_vox, const double* sigma0_vox);
int svh_get_materials(const svh_handle* h, double* lambda_vox, double* sigma0_vox);
/* Adjoint gradient of L_ij = Im(Zport_ij)/omega at the last frequency of the
 * last svh_solve with respect to each voxel's lambda (dL_dlambda[K], H/m) and
 * sigma0 (dL_dsigma0[K], may be NULL). Uses the stored forward solutions as
 * the adjoint ones (negating the continuity rows makes Eq. 7 complex
 * symmetric): dZ_ij/dp_k = sum_beta dz^beta_k/dp_k w_i w_j, w_i = sum_p
 * Z_ip I_p, with z^beta the two-fluid diagonal (Eq. 3, 9, 22-23). */
int svh_grad_inductance(svh_handle* h, int i, int j, double* dL_dlambda, double* dL_dsigma0);
/* Host reference of the preconditioner apply out = P in (Eq. 13-15) at
 * omega for nb vectors of length N (complex interleaved double), with the
 * Schur solves run to 1e-12 (for tests). */
int svh_precond_apply(svh_handle* h, double omega, int nb, const double* in, double* out);

/* ---- Batches of independent structures (unevenly sized grids; Sec. III's
 * many ports and frequencies of many structures at once).
 * A batch borrows handles (each set up with its grid, ports and kernels) and
 * must be destroyed before them. svh_batch_matvec applies structure i's
 * operator (Eq. 7 with Z by Eq. 9, as svh_matvec_omegas) to its own nbs[i]
 * right-hand sides x_dev[i] -> y_dev[i] (device pointers, nbs[i] * N_i complex
 * values of the precision, item r at offset r * N_i) at the angular
 * frequencies omegas[i][0 .. nbs[i]) (host arrays, > 0). All products of the
 * batch run in ONE persistent launch: a device work queue holds the tiles of
 * every pass of every structure (x-forward, node rows, y-forward, z pass,
 * y-inverse, x-inverse with the epilogue), phase by phase; each CTA takes the
 * next tile, waits (bounded in time) until the pass that tile reads is
 * complete for its structure, runs it and counts it done. The first call with
 * a given argument set builds the queue (growing each handle's intermediate
 * grids) and captures the launch in a CUDA graph on the batch stream; that
 * call and later calls with the same arguments launch the graph
 * (asynchronous). The spectra are each handle's resident ones (the batch
 * runs no Tucker restore). svh_batch_sync waits for the batch stream and
 * returns SVH_ERR_TIMEOUT (the products of that launch are incomplete, the
 * device stays usable) when a wait of the queue ran out.
 * svh_batch_set_wait sets the bound of each wait (limit_ms, default 1000)
 * and, for diagnostics, a (hold_item, hold_phase) pair whose completion count
 * is never reached (-1, -1: none; phases numbered 0 x-forward, 1 node rows,
 * 2 y-forward, 3 z pass, 4 y-inverse, 5 x-inverse), so that the waits on it
 * run out and the launch ends with SVH_ERR_TIMEOUT.
 * svh_batch_set_mode selects how svh_batch_matvec runs: 0 (default) the one
 * persistent launch above; 1 every structure's own launch sequence (the
 * size-specialised, tile-tuned kernels of svh_matvec_omegas) on up to 16
 * streams forked from and joined to the batch stream, captured as one CUDA
 * graph. svh_batch_autotune times both modes on the given arguments (three
 * graph launches each after a warm-up; ms[2], may be NULL, receives the
 * milliseconds per launch) and keeps the faster; svh_batch_get_mode reports
 * the current mode.
 * svh_batch_solve runs svh_solve for every structure at the same
 * frequencies with n_workers host threads (<= 0: 4), each on its own stream,
 * so one structure's host preconditioner work overlaps the others' device
 * work; Zports[i] receives structure i's nfreq*np_i*np_i complex values and
 * Lports[i] (Lports may be NULL) its inductances as in svh_solve; the
 * stats are summed (final_rre: the largest). */
#define SVH_STATUS_QUEUE_TIMEOUT 4
typedef struct svh_batch svh_batch;
int svh_batch_create(svh_batch** b, int device);
int svh_batch_destroy(svh_batch* b);
const char* svh_batch_last_error(const svh_batch* b);
int svh_batch_add(svh_batch* b, svh_handle* h);
int svh_batch_size(const svh_batch* b);
int svh_batch_matvec(svh_batch* b, const int32_t* nbs, const double* const* omegas, const void* const* x_dev,
                     void* const* y_dev, int precision);
int svh_batch_sync(svh_batch* b);
int svh_batch_set_wait(svh_batch* b, double limit_ms, int hold_item, int hold_phase);
int svh_batch_set_mode(svh_batch* b, int mode);
int svh_batch_get_mode(const svh_batch* b);
int svh_batch_autotune(svh_batch* b, const int32_t* nbs, const double* const* omegas, const void* const* x_dev,
                       void* const* y_dev, int precision, double* ms);
void* svh_batch_stream(svh_batch* b);
int svh_batch_solve(svh_batch* b, const double* omegas, int nfreq, const svh_options* opt, double* const* Zports,
                    double* const* Lports, int n_workers, svh_stats* st);

/* ---- Product for callers that cannot allocate device memory at call time.
 * (An interface of this library; the paper has no counterpart.)
 * svh_matvec allocates its intermediate FFT grids with cudaMalloc the first
 * time it sees a larger batch. A caller that may not allocate then -- a
 * plug-in inside a host application that owns the device-memory budget, or
 * a latency-critical loop that must not enter the allocator, which can
 * synchronise the device -- can call svh_matvec_noalloc instead: the same
 * product as svh_matvec with the same arguments, computed on a fixed scratch
 * array of SVH_NOALLOC_SCRATCH_BYTES (64 MiB) compiled into the library's
 * device code. Every GPU that loads the library holds that array until the
 * process exits. The call makes no cudaMalloc/cudaFree and no allocating
 * library call; the handle's second stream and events it uses are created
 * by svh_setup_grid. Its first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture. The scratch needs 5 * nza * Px * (Ky + Py) complex values per
 * right-hand side (nza = planes holding voxels); larger requests return
 * SVH_ERR_ARG. All calls share the one array: calls that may run
 * concurrently on the GPU (different streams or handles) race and must be
 * serialised by the caller. Nothing in the array needs clearing between
 * calls: every value a call reads it has written itself. It applies the
 * FP32 spectra on the device as they are and never runs the per-product
 * Tucker restore: in SVH_KERNELS_TUCKER_REBUILD mode (FP32, Tucker data
 * loaded) it returns SVH_ERR_STATE until svh_rebuild_spectra has restored
 * them, and then applies the restored operator, as svh_matvec does. When
 * the direct z pass is chosen but its z-space kernels have no buffers yet
 * (svh_matvec has not run it on this handle), the call takes the FFT form
 * of the z pass, which gives the same product. */
#define SVH_NOALLOC_SCRATCH_BYTES (64u << 20)
int svh_matvec_noalloc(svh_handle* h, double omega, int nb, const void* x_dev, void* y_dev, int precision);

/* ---- FFT tile autotuning (batching of Sec. II.B.1 products on this GPU).
 * The five FFT passes (0 x-forward with gather, 1 y-forward, 2 z pass,
 * 3 y-inverse, 4 x-inverse with epilogue) have size-specialised FP32 kernels
 * in several tile variants (radix split N1 x N2, threads per block, pruned
 * or full z pencils). Choice 5 is the path: 0 runs the passes separately,
 * 1 fuses passes 1-3 into one kernel per (kx, item) that keeps the column's
 * (basis, plane, y) slab in shared memory (offered when it fits and the
 * active planes are contiguous). Choice 6 is the stream schedule of a
 * product: 0 runs the Tucker restore and the node rows on the handle's second
 * stream, overlapping passes 1-2; 1 overlaps only the node rows; 2 uses one
 * stream; 3 overlaps the node rows with pass 1 only (joined before pass 2, so
 * that a persistent y pass starts on every SM). svh_autotune times every variant of every pass on this handle's
 * grid for nb right-hand sides (zero data, 5 launches each, CUDA events on
 * the handle's stream), then the fused path against the separate passes,
 * then the four schedules on whole products, and keeps the fastest for
 * later FP32 products; results are cached per process for equal grids and
 * nb. variants[7] and ms[7] (may be NULL) receive the choices and their
 * milliseconds per launch. svh_set_pass_variant forces one (SVH_ERR_ARG if
 * the pass has no such variant at this size); svh_get_pass_variants reports
 * the number of variants per pass (0: generic kernel) and the current choice.
 * FP64 products always use variant 0. */
#define SVH_NFFTPASS 7
/* Device status word of the handle: bit 0 (SVH_STATUS_TMA_TIMEOUT) is set
 * when a kernel's bounded wait for a TMA copy expired, bit 1
 * (SVH_STATUS_MMA_TIMEOUT) when the Tucker restore's bounded wait for its
 * tensor-core MMAs expired (results are then invalid). clear != 0 resets it. */
#define SVH_STATUS_TMA_TIMEOUT 1
#define SVH_STATUS_MMA_TIMEOUT 2
int svh_get_device_status(svh_handle* h, int32_t* status, int clear);
int svh_autotune(svh_handle* h, int nb, int32_t* variants, double* ms);
int svh_set_pass_variant(svh_handle* h, int pass, int variant);
int svh_get_pass_variants(const svh_handle* h, int32_t* counts, int32_t* chosen);

/* ---- Per-pass timing of svh_matvec with CUDA events (begin and end of each
 * pass on the stream it runs on).
 * Passes: 0 Tucker rebuild (Eq. 10), 1 x-forward with gather, 2 y-forward,
 * 3 z-FFT + block multiply + inverse z-FFT, 4 y-inverse, 5 x-inverse with
 * the diagonal and A^T epilogue, 6 node rows (A I). Passes 0 and 6 run on
 * the handle's second stream, overlapping passes 1-2 (the sum of the pass
 * times can exceed the call's duration). svh_profile_begin
 * starts recording for up to max_calls matvec calls (events are recorded
 * without synchronising); svh_profile_end waits for them and returns the
 * summed milliseconds per pass in ms[SVH_NPASS] and the calls recorded. */
#define SVH_NPASS 7
int svh_profile_begin(svh_handle* h, int max_calls);
int svh_profile_end(svh_handle* h, double* ms, int* ncalls);

/* ---- Host utilities (no device needed; safe to call on a machine without a GPU) */

/* Voxel count and face-node numbering of an occupancy grid, with the
 * conventions above. Call with node == NULL to learn K and M, then again with
 * node[K*6]. */
int svh_host_face_nodes(int Kx, int Ky, int Kz, const uint8_t* occ, int64_t* K_out, int64_t* M_out,
                        int32_t* node);
/* Octant spectra S[7][Pz/2+1][Py/2+1][Px/2+1] of the circulant embeddings of
 * unit kernels T[7][Kz][Ky][Kx] (same definition as svh_get_spectra). */
int svh_host_spectra(int Kx, int Ky, int Kz, int Px, int Py, int Pz, const double* T, double* S);
/* S x = b for a real symmetric positive definite CSR matrix (rowptr[n+1],
 * colidx, vals) by conjugate gradients preconditioned with the library's
 * aggregation AMG K-cycle (the inner solver of the Schur complement, Eq. 14),
 * x0 = 0, to ||b - S x|| <= tol ||b||. iters, levels (may be NULL) receive the
 * CG iterations and the number of AMG levels. SVH_ERR_NOT_CONVERGED after
 * maxit iterations; SVH_ERR_SINGULAR if the coarsest level is not SPD. */
int svh_host_amg_solve(int n, const int32_t* rowptr, const int32_t* colidx, const double* vals, const double* b,
                       double* x, double tol, int maxit, int32_t* iters, int32_t* levels);
/* The same solver with the CG and its K-cycle on the current CUDA device (the
 * hierarchy is built on the host): nrhs complex right-hand sides b[nrhs][n]
 * (host, interleaved re, im), whose real and imaginary parts are separate real
 * systems, each solved to ||b - S x|| <= tol ||b||; x[nrhs][n] (host) receives
 * the solutions. iters receives the mean CG iterations per real system.
 * Errors as svh_host_amg_solve, plus SVH_ERR_CUDA. */
int svh_device_amg_solve(int n, const int32_t* rowptr, const int32_t* colidx, const double* vals, const double* b,
                         double* x, int nrhs, double tol, int maxit, int32_t* iters, int32_t* levels);
/* ---- Algorithm 2: install-time store of the unit Toeplitz tensors.
 * svh_toeplitz_store_write compresses the 7 unit Toeplitz tensors of a
 * Kx x Ky x Kz domain, T[7][Kz][Ky][Kx] (the layout of svh_load_toeplitz),
 * with Algorithm 1 at tol and writes their Tucker cores and factors to path;
 * T = NULL computes them on the current CUDA device first (the quadrature of
 * svh_generate_toeplitz). svh_toeplitz_store_read restores (Eq. 10) the
 * leading Kx x Ky x Kz block of each tensor into T (host, 7*Kx*Ky*Kz
 * doubles); ranks[21] (may be NULL) receives the stored ranks. The unit
 * kernels are dimensionless (the voxel size enters the product as
 * j omega mu dx), so a store serves every voxel size and the crop needs no
 * scaling. svh_load_toeplitz_store reads the handle's grid size from a store
 * and installs the result as svh_load_toeplitz does. All return SVH_ERR_ARG
 * for an unreadable or foreign file or a grid larger than the stored one.
 * The file is in host byte order. */
int svh_toeplitz_store_write(const char* path, int Kx, int Ky, int Kz, const double* T, double tol);
int svh_toeplitz_store_read(const char* path, int Kx, int Ky, int Kz, double* T, int32_t* ranks);
int svh_load_toeplitz_store(svh_handle* h, const char* path);

/* Algorithm 1 (Tucker-SVD) of a real D1 x D2 x D3 array O stored with the
 * mode-1 index fastest, O[(i3*D2 + i2)*D1 + i1]. The rank of mode i is the
 * smallest d_i whose discarded singular values have 2-norm <= tol/sqrt(3) *
 * ||O||_F, so ||O - restore||_F <= tol ||O||_F. Outputs (caller-allocated,
 * worst-case sizes): d[3]; core[d3][d2][d1] (<= D1*D2*D3); F1[D1][d1] (<= D1*D1),
 * F2[D2][d2], F3[D3][d3]. The singular vectors of each unfolding come from a
 * Householder QR of its transpose and a one-sided Jacobi SVD of the triangle
 * (host cores, OpenMP); SVH_ERR_ARG for null arrays, non-positive sizes or
 * tol <= 0. */
int svh_host_tucker_svd(const double* O, int D1, int D2, int D3, double tol, int32_t* d, double* core,
                        double* F1, double* F2, double* F3);

#ifdef __cplusplus
}
#endif

#endif /* SVH_H */
