// svh_internal.h -- handle state and helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/svh.h"

namespace svh {

struct FftPlanHost {
    int N = 0;
    std::vector<int> R;
};

// Device arrays owned by a handle (freed in svh_destroy).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Tucker {
    int d[3] = {0, 0, 0};
    std::vector<double> core, F[3];
};

struct Handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // ---- grid (svh_setup_grid)
    bool have_grid = false;
    int Kx = 0, Ky = 0, Kz = 0, Px = 0, Py = 0, Pz = 0, Hx = 0, Hy = 0, Hz = 0;
    double dx = 0;
    int64_t K = 0, M = 0;
    std::vector<int32_t> vox;         // grid linear index of each voxel
    std::vector<int32_t> node;        // [K*6]
    std::vector<double> lam, sig0;    // [K]
    std::vector<int32_t> zlist;       // active planes (z values)
    std::vector<int32_t> rows;        // active rows, zi*Ky + y
    std::vector<uint8_t> fixed;       // [M] 1 for terminal/gauge nodes
    std::vector<std::vector<int32_t>> port_plus, port_minus;   // node ids
    std::vector<int32_t> gauge;

    // device copies
    DevBuf d_vidx;      // int32 [nza][Ky][Kx]  voxel index or -1
    DevBuf d_rows;      // int32 [nrows]
    DevBuf d_rinfo;     // int2 [nrows]: first voxel index and voxel count of each active row
    DevBuf d_vx;        // int32 [K]: x of each voxel (a row's voxels are consecutive, ordered by x)
    DevBuf d_rowmask;   // uint8 [nza][Ky] 1 for rows holding voxels
    DevBuf d_zlist;     // int32 [nza]
    DevBuf d_node;      // int32 [K*6]
    DevBuf d_ninc;      // int32 [M*2]  voxel*6+face touching each node, or -1
    DevBuf d_free;      // uint8 [M] 1 for free nodes
    DevBuf d_lam, d_sig0;   // double [K]

    // ---- kernels
    bool have_kernels = false;
    std::vector<double> toep;          // [7][Kz][Ky][Kx]
    std::vector<double> spec;          // [7][Hz][Hy][Hx]
    DevBuf d_spec32, d_spec64;         // float / double [7][Hz][Hy][Hx]
    int spec_version = 0;              // bumped whenever d_spec32 is rewritten
    int spec32_tk_version = -1;        // tk_version whose Tucker restore d_spec32 holds (-1: exact spectra)
    // z-space kernels of the direct z pass: float [7][zk_D][Hy][Hx], made from d_spec32
    // with the weights d_zkw [2][zk_D][Hz] (cosines, sines); current when zk_version == spec_version
    DevBuf d_zk32, d_zkw;
    int zk_D = 0, zk_version = -1;
    DevBuf d_tw32[3], d_tw64[3];       // twiddles per axis
    FftPlanHost plan[3];
    bool tucker_on[7] = {false, false, false, false, false, false, false};
    Tucker tk[7];
    // device form of the Tucker data (float, rows padded to 8): core x_3 F3 as
    // [Hz][d2p][d1p], F1 as [Hx][d1p], F2 as [Hy][d2p] (d_tk_F[u][2] unused)
    DevBuf d_tk_core[7], d_tk_F[7][3];
    // core x_3 (W_u F3) for a restore straight to the z-space kernels of the direct z pass
    // (W_u the [zk_D][Hz] weights of zk_weights), planes [2][zk_D d2p][d1p]; built for tk_zk_D planes
    DevBuf d_tk_core_zk[7];
    int tk_zk_D = 0;
    int tk_probs_target = -1;            // 0: the descriptors write the spectra, 1: the z-space kernels
    DevBuf d_tk_w1;                      // restore intermediate [Hx][Hz][d2p] per kernel (float)
    DevBuf d_tk_probs;                   // GEMM descriptors of the restore
    std::vector<char> tk_probs;          // host copy of the descriptors
    int tk_probs_split[3] = {0, 0, 0};
    int tk_version = 0, tk_probs_version = -1;
    int kernel_mode = SVH_KERNELS_RESIDENT;

    // ---- per-pass profiling (svh_profile_begin/end)
    bool prof_on = false;
    int prof_max = 0, prof_calls = 0;
    std::vector<cudaEvent_t> prof_ev;   // [prof_max][SVH_NPASS][begin, end]
    // second stream of the product: the Tucker restore and the node rows run on it,
    // overlapping the x and y passes (joined by events before the z pass and at the end)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_spec = nullptr, ev_done = nullptr, ev_x = nullptr;
    // set by the host-buffer entry point: the second stream was forked before the input
    // copy (the restore overlaps it) and ev_x marks the input on the device
    bool preforked = false;
    // copy streams of the host-buffer entry point: the items go in up to kHostChunks chunks,
    // each copied in on cpy_in (ev_in), multiplied on the handle's stream (ev_out) and copied out
    // on cpy_out while the next chunk is multiplied
    cudaStream_t cpy_in = nullptr, cpy_out = nullptr;
    cudaEvent_t ev_in[4] = {nullptr, nullptr, nullptr, nullptr}, ev_out[4] = {nullptr, nullptr, nullptr, nullptr};

    // ---- sparse preconditioner (amg.cpp), built per frequency by the solver
    void* precond = nullptr;
    // ---- cuBLAS / cuSOLVER handles of the device Tucker-SVD (tucker_svd_dev.cu)
    void* tsvd = nullptr;

    // ---- last solve (svh_get_solution)
    std::vector<double> last_x;   // [nb][N] complex interleaved
    std::vector<double> last_Z;   // [nb][nb] complex interleaved, at last_omega
    double last_omega = 0;
    int last_nb = 0;

    // ---- scratch for the matvec
    DevBuf d_B1, d_B2;
    DevBuf d_xin, d_yout;              // staging for svh_matvec_host
    DevBuf d_omegas;                   // per-item frequencies for svh_matvec_omegas
    DevBuf d_status;                   // int32 status word set by kernels (bounded waits that expired)
    // FP32 tile variant per FFT pass; [5]: 0 separate passes, 1 fused y/z/y; [6] stream
    // schedule: 0 restore + node rows on the second stream, 1 node rows only, 2 one stream,
    // 3 node rows beside pass 1 only
    int tune32[7] = {0, 0, 0, 0, 0, 0, 0};
    size_t smem_optin = 0;                // opt-in shared memory per block of the device
};

int set_err(Handle* h, int code, const std::string& msg);
// record the begin (end = 0) or end (end = 1) event of pass p on stream s when profiling
void prof_at(Handle* h, int p, int end, cudaStream_t s);
int cuda_err(Handle* h, cudaError_t e, const char* what);
int dev_alloc(Handle* h, DevBuf& b, size_t bytes);
void dev_free(DevBuf& b);
int dev_upload(Handle* h, DevBuf& b, const void* src, size_t bytes);

// launchers (matvec.cu)
// d_omegas (device, nb entries): per-item angular frequency; nullptr -> omega for all items
int launch_matvec32(Handle* h, double omega, int nb, const void* x, void* y, int masked,
                    const double* d_omegas = nullptr);
int launch_matvec64(Handle* h, double omega, int nb, const void* x, void* y, int masked,
                    const double* d_omegas = nullptr);
// same product on caller-provided intermediate grids (no allocation, no Tucker restore)
int launch_matvec_on(Handle* h, double omega, int nb, const void* x, void* y, int precision, void* B1, void* B2);
void matvec_scratch_bytes(const Handle* h, int nb, int precision, size_t* b1, size_t* b2);
// fork the product's second stream now (before an input copy the caller enqueues next);
// mark_input_ready records, after that copy, the event the node rows wait for
int matvec_prefork(Handle* h);
// the product's second stream and its events, and the device's shared-memory limit (made once
// per handle at grid set-up, so that no product call creates them)
int matvec_streams(Handle* h);
int matvec_mark_input_ready(Handle* h);
constexpr int kHostChunks = 4;
// the product with the kernels that an earlier product of the same call prepared (no restore)
int launch_matvec_reuse(Handle* h, double omega, int nb, const void* x, void* y, int precision);
// FFT tile variants (matvec.cu)
int autotune(Handle* h, int nb, int32_t* variants, double* ms);
int set_pass_variant(Handle* h, int pass, int variant);
void get_pass_variants(const Handle* h, int32_t* counts, int32_t* chosen);
#define SVH_NTUNE 7
// quadrature of the unit kernels (kernels_gen.cu): fills T[7][Kz][Ky][Kx] (host)
int generate_toeplitz_device(Handle* h, std::vector<double>& T);
// sparse preconditioner (amg.cpp)
void precond_free(Handle* h);
int precond_setup(Handle* h, const double* omegas, int nfreq, double tol);
int precond_schur_solve(Handle* h, int nb, int per_freq, const double* e, double* b);
const double* precond_Y(Handle* h, int freq_index);
const int* precond_free_nodes(Handle* h, int* nf);
int precond_levels(Handle* h);
double precond_avg_iters(Handle* h);
int precond_apply_host(Handle* h, int nb, const double* in, double* out);
// read-only view of frequency fi's AMG hierarchy (amg.cpp) for the device solver
struct AmgLevelView {
    int n = 0, nc = 0;
    const int *rp = nullptr, *ci = nullptr;
    const double *v = nullptr, *l1 = nullptr;
    const int *agg = nullptr, *crp = nullptr, *cidx = nullptr;
};
struct AmgView {
    std::vector<AmgLevelView> lv;
    const double* chol = nullptr;   // coarsest Cholesky factor, row-major lower, nco x nco
    int nco = 0;
    double tol = 1e-8;
    int maxit = 500;
};
int precond_nfreq(Handle* h);
int precond_view(Handle* h, int fi, AmgView& out);
// device copy of frequency fi's hierarchy, owned by the preconditioner (amg_dev.cu)
void*& precond_dev(Handle* h, int fi);
void precond_count(Handle* h, int fi, long long calls, long long iters);
void amg_dev_destroy(void* d);
// b = S^{-1} e on the device; e, b: double2 [nb][nf] device arrays
int precond_schur_solve_dev(Handle* h, int nb, int per_freq, const void* e_dev, void* b_dev);
// Tucker rebuild (tucker.cu)
// restore the FP32 spectra from Tucker data (Eq. 10) into d_spec32
// restore of the kernels with Tucker data on `s`: into the FP32 octant spectra (to_zk false,
// bumps spec_version) or straight into the z-space kernels d_zk32 (to_zk true; needs zk_D set)
int launch_tucker_rebuild(Handle* h, cudaStream_t s, bool to_zk = false);
// plane span of the active planes (the z offsets the direct z pass needs: 0 .. span - 1)
inline int zk_planes(const Handle* h) {
    return h->zlist.empty() ? 0 : h->zlist.back() - h->zlist.front() + 1;
}
// weights of the z-space kernels r_u(dz) = sum_az w[dz][az] S_u(az), dz < D, az < Hz, for the
// z-even kernels (w[0 .. D Hz)) and for S_z (w[D Hz .. 2 D Hz)): c_az cos(2 pi az dz / Pz) and
// c_az sin(2 pi az dz / Pz), c_az = 2 inside the octant, 1 at az = 0 and az = Pz / 2 (where the
// odd S_z spectrum vanishes, so its weight is 0)
inline void zk_weights(int Pz, int Hz, int D, std::vector<double>& w) {
    w.assign((size_t)2 * D * Hz, 0.0);
    const double pi = 3.14159265358979323846;
    for (int d = 0; d < D; ++d)
        for (int az = 0; az < Hz; ++az) {
            const bool edge = az == 0 || 2 * az == Pz;
            const double th = 2.0 * pi * az * d / Pz;
            w[(size_t)d * Hz + az] = (edge ? 1.0 : 2.0) * std::cos(th);
            w[(size_t)(D + d) * Hz + az] = edge ? 0.0 : 2.0 * std::sin(th);
        }
}
// uploads the device form of h->tk[u] (tucker.cu)
int upload_tucker_device(Handle* h, int u);
// Algorithm 1 on kernel u's FP64 octant spectra on the device (tucker_svd_dev.cu)
int tucker_svd_device(Handle* h, int u, double tol, Tucker& out);
void tsvd_free(void* p);

}  // namespace svh

#define SVH_CUDA_TRY(h, call)                                   \
    do {                                                        \
        cudaError_t e__ = (call);                               \
        if (e__ != cudaSuccess) return svh::cuda_err((h), e__, #call); \
    } while (0)
