// adjoint.cu -- gradient of a port inductance with respect to per-voxel lambda and sigma0.
//
// Negating the continuity rows makes Eq. 7 complex-symmetric (Kt^T = D Kt D,
// D = diag(I, -I)) and a port's right-hand side equals its current
// functional, so the adjoint solutions are the forward ones of the last
// svh_solve. Only the two-fluid diagonal z^beta_k = c_k s_beta / dx (Eq. 9,
// 22-23, c = 1/sigma, sigma = sigma0 - j/(omega mu lambda^2), Eq. 3) depends on
// the materials, so with w_i = sum_p Z_ip I_p:
//   dZ_ij / d lambda_k = sum_beta (s_beta/dx) dc_k/d lambda_k w_i^(k,beta) w_j^(k,beta),
//   dc/d lambda = -(1/sigma^2) * 2j/(omega mu lambda^3),  dc/d sigma0 = -1/sigma^2,
//   dL_ij = Im(dZ_ij) / omega.
// One thread per voxel, FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "svh_internal.h"

namespace svh {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    double2 c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    double2 c; c.x = (a.x * b.x + a.y * b.y) / d; c.y = (a.y * b.x - a.x * b.y) / d; return c;
}

__global__ void k_grad_inductance(const double2* __restrict__ XI, int64_t K, int np, const double2* __restrict__ zi,
                                  const double2* __restrict__ zj, const double* __restrict__ lam,
                                  const double* __restrict__ sig0, double omega, double mu, double dx,
                                  double* __restrict__ dl, double* __restrict__ ds) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double l = lam[k];
    const double wm = omega * mu;
    double2 sig; sig.x = sig0[k]; sig.y = -1.0 / (wm * l * l);
    const double2 s2 = zmul(sig, sig);
    double2 dsig; dsig.x = 0; dsig.y = 2.0 / (wm * l * l * l);
    double2 one; one.x = 1; one.y = 0;
    double2 dcl = zdiv(dsig, s2); dcl.x = -dcl.x; dcl.y = -dcl.y;     // -(dsigma/dlambda)/sigma^2
    double2 dcs = zdiv(one, s2); dcs.x = -dcs.x; dcs.y = -dcs.y;     // -1/sigma^2
    const double sb[5] = {1.0, 1.0, 1.0, 1.0 / 6.0, 0.5};
    double2 accl; accl.x = 0; accl.y = 0;
    double2 accs = accl;
    for (int b = 0; b < 5; ++b) {
        double2 a; a.x = 0; a.y = 0;
        double2 c = a;
        for (int p = 0; p < np; ++p) {
            const double2 x = XI[((int64_t)p * 5 + b) * K + k];
            const double2 u = zmul(zi[p], x), v = zmul(zj[p], x);
            a.x += u.x; a.y += u.y;
            c.x += v.x; c.y += v.y;
        }
        const double2 ab = zmul(a, c);
        const double f = sb[b] / dx;
        const double2 tl = zmul(dcl, ab), ts = zmul(dcs, ab);
        accl.x += f * tl.x; accl.y += f * tl.y;
        accs.x += f * ts.x; accs.y += f * ts.y;
    }
    dl[k] = accl.y / omega;
    if (ds) ds[k] = accs.y / omega;
}

int grad_inductance(Handle* h, int i, int j, double* dl_host, double* ds_host) {
    const int np = h->last_nb;
    const int64_t K = h->K, N = 5 * K + h->M;
    // I parts of the stored solutions
    std::vector<double> XI((size_t)np * 5 * K * 2);
    for (int p = 0; p < np; ++p)
        std::memcpy(XI.data() + (size_t)p * 5 * K * 2, h->last_x.data() + (size_t)p * N * 2, (size_t)5 * K * 16);
    std::vector<double> zi(2 * np), zj(2 * np);
    for (int p = 0; p < np; ++p) {
        zi[2 * p] = h->last_Z[((size_t)i * np + p) * 2];
        zi[2 * p + 1] = h->last_Z[((size_t)i * np + p) * 2 + 1];
        zj[2 * p] = h->last_Z[((size_t)p * np + j) * 2];
        zj[2 * p + 1] = h->last_Z[((size_t)p * np + j) * 2 + 1];
    }
    DevBuf dX, dzi, dzj, ddl, dds;
    auto cleanup = [&]() { dev_free(dX); dev_free(dzi); dev_free(dzj); dev_free(ddl); dev_free(dds); };
    int rc;
    if ((rc = dev_upload(h, dX, XI.data(), XI.size() * 8)) || (rc = dev_upload(h, dzi, zi.data(), zi.size() * 8)) ||
        (rc = dev_upload(h, dzj, zj.data(), zj.size() * 8)) || (rc = dev_alloc(h, ddl, (size_t)K * 8)) ||
        (rc = dev_alloc(h, dds, (size_t)K * 8))) {
        cleanup();
        return rc;
    }
    const double mu = 4e-7 * 3.14159265358979323846;
    k_grad_inductance<<<(unsigned)((K + 255) / 256), 256, 0, h->stream>>>(
        static_cast<double2*>(dX.p), K, np, static_cast<double2*>(dzi.p), static_cast<double2*>(dzj.p),
        static_cast<double*>(h->d_lam.p), static_cast<double*>(h->d_sig0.p), h->last_omega, mu, h->dx,
        static_cast<double*>(ddl.p), static_cast<double*>(dds.p));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl_host, ddl.p, (size_t)K * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && ds_host) e = cudaMemcpyAsync(ds_host, dds.p, (size_t)K * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cleanup();
    if (e != cudaSuccess) return cuda_err(h, e, "svh_grad_inductance");
    return SVH_OK;
}

}  // namespace svh

using namespace svh;

extern "C" int svh_grad_inductance(svh_handle* hh, int i, int j, double* dL_dlambda, double* dL_dsigma0) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !dL_dlambda) return SVH_ERR_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaSetDevice");
    if (h->last_nb == 0 || h->last_Z.empty()) return set_err(h, SVH_ERR_STATE, "svh_grad_inductance: run svh_solve first");
    if (i < 0 || j < 0 || i >= h->last_nb || j >= h->last_nb) return set_err(h, SVH_ERR_ARG, "svh_grad_inductance: bad port");
    return grad_inductance(h, i, j, dL_dlambda, dL_dsigma0);
}

extern "C" int svh_set_materials(svh_handle* hh, const double* lambda_vox, const double* sigma0_vox) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !lambda_vox || !sigma0_vox) return SVH_ERR_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaSetDevice");
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_set_materials: no grid");
    for (int64_t v = 0; v < h->K; ++v)
        if (!(lambda_vox[v] > 0) || !(sigma0_vox[v] >= 0) || !std::isfinite(lambda_vox[v]) || !std::isfinite(sigma0_vox[v]))
            return set_err(h, SVH_ERR_ARG, "svh_set_materials: lambda must be > 0 and sigma0 >= 0");
    h->lam.assign(lambda_vox, lambda_vox + h->K);
    h->sig0.assign(sigma0_vox, sigma0_vox + h->K);
    SVH_CUDA_TRY(h, cudaMemcpyAsync(h->d_lam.p, lambda_vox, (size_t)h->K * 8, cudaMemcpyHostToDevice, h->stream));
    SVH_CUDA_TRY(h, cudaMemcpyAsync(h->d_sig0.p, sigma0_vox, (size_t)h->K * 8, cudaMemcpyHostToDevice, h->stream));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->last_nb = 0;
    h->last_Z.clear();
    return SVH_OK;
}

extern "C" int svh_get_materials(const svh_handle* hh, double* lambda_vox, double* sigma0_vox) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !lambda_vox || !sigma0_vox) return SVH_ERR_ARG;
    if (!h->have_grid) return SVH_ERR_STATE;
    std::memcpy(lambda_vox, h->lam.data(), (size_t)h->K * 8);
    std::memcpy(sigma0_vox, h->sig0.data(), (size_t)h->K * 8);
    return SVH_OK;
}
