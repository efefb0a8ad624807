// kernels_gen.cu -- device quadrature of the seven unit Green's-function kernels.
//
// Each kernel is a 6-D integral over two unit voxels of polynomial moments
// times G = 1/(4 pi |r - r'|) (App. A Eq. 19-21, App. B Eq. 24-27 with dx = 1),
// folded to 3-D over u = xi - xi' in [-1,1]^3 with the 1-D overlap weights
//   w0(t) = 1 - |t|,  w1(t) = -t(1 - |t|)/2,  w2(t) = 1/12 - |t|/4 + |t|^3/6
// (G00 = w0 w0 w0; S_a = w1 on axis a; Q_a = w2 on axis a). On each of the 8
// octant boxes of [-1,1]^3 the weight is a polynomial. The singular point
// u = -d is either a box vertex (|d|_inf <= 1: Duffy map into three pyramids
// removes the 1/r singularity) or at sup-distance >= 1 (tensor Gauss-Legendre,
// order falling with distance). One thread integrates one far offset; one
// block integrates one near offset.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "svh_internal.h"

namespace svh {

// Gauss-Legendre rule on [0, 1]: roots of P_n by Newton's method from the
// Chebyshev-like guess cos(pi (i + 3/4) / (n + 1/2)), weights 2/((1-x^2) P_n'(x)^2).
static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // P_n(z) = p1, P_{n-1}(z) = p0
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // = 0.5 * 2 / ((1 - z^2) P_n'^2)
    }
}

__host__ __device__ inline double wt0(double t) { return 1.0 - fabs(t); }
__host__ __device__ inline double wt1(double t) { return -t * (1.0 - fabs(t)) * 0.5; }
__host__ __device__ inline double wt2(double t) {
    double a = fabs(t);
    return 1.0 / 12.0 - a * 0.25 + a * a * a / 6.0;
}

// weights of the 7 kernels at u
__host__ __device__ inline void kernel_weights(const double u[3], double W[7]) {
    double a0[3], a1[3], a2[3];
    for (int k = 0; k < 3; ++k) { a0[k] = wt0(u[k]); a1[k] = wt1(u[k]); a2[k] = wt2(u[k]); }
    W[0] = a0[0] * a0[1] * a0[2];
    W[1] = a1[0] * a0[1] * a0[2];
    W[2] = a0[0] * a1[1] * a0[2];
    W[3] = a0[0] * a0[1] * a1[2];
    W[4] = a2[0] * a0[1] * a0[2];
    W[5] = a0[0] * a2[1] * a0[2];
    W[6] = a0[0] * a0[1] * a2[2];
}

// far offsets: tables of (u, 7 weights) per Gauss-Legendre order
struct FarTables {
    const double* tab;   // [sum nq][10]
    int off[5];          // row offset of each table
    int nq[5];           // nodes per table
};

__device__ __forceinline__ int far_table(int rinf) {
    if (rinf <= 2) return 0;   // 12 points per axis
    if (rinf <= 4) return 1;   // 8
    if (rinf <= 10) return 2;  // 6
    if (rinf <= 40) return 3;  // 5
    return 4;                  // 4
}

__global__ void k_far(FarTables ft, int Kx, int Ky, int Kz, double* __restrict__ T) {
    const int64_t Kt = (int64_t)Kx * Ky * Kz;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kt) return;
    int dx = (int)(i % Kx), dy = (int)((i / Kx) % Ky), dz = (int)(i / ((int64_t)Kx * Ky));
    int rinf = max(dx, max(dy, dz));
    if (rinf <= 1) return;
    int t = far_table(rinf);
    const double* tab = ft.tab + (int64_t)ft.off[t] * 10;
    const int nq = ft.nq[t];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const double fx = dx, fy = dy, fz = dz;
    for (int q = 0; q < nq; ++q) {
        const double* e = tab + q * 10;
        double rx = fx + e[0], ry = fy + e[1], rz = fz + e[2];
        double inv = rsqrt(rx * rx + ry * ry + rz * rz);
#pragma unroll
        for (int k = 0; k < 7; ++k) acc[k] += e[3 + k] * inv;
    }
    const double s = 0.07957747154594766788;   // 1 / (4 pi)
#pragma unroll
    for (int k = 0; k < 7; ++k) T[k * Kt + i] = acc[k] * s;
}

// near offsets d in {0,1}^3: Duffy on boxes with the singular vertex, Gauss-Legendre elsewhere
__global__ void k_near(const double* __restrict__ gx, const double* __restrict__ gw, int nd,
                       const double* __restrict__ hx, const double* __restrict__ hw, int ng,
                       int Kx, int Ky, int Kz, double* __restrict__ T) {
    const int o = blockIdx.x;
    const int d[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    if (d[0] >= Kx || d[1] >= Ky || d[2] >= Kz) return;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int box = 0; box < 8; ++box) {
        const double sg[3] = {(box & 1) ? 1.0 : -1.0, (box & 2) ? 1.0 : -1.0, (box & 4) ? 1.0 : -1.0};
        double vloc[3];
        bool vertex = true;
        for (int k = 0; k < 3; ++k) {
            vloc[k] = -sg[k] * d[k];
            if (!(vloc[k] == 0.0 || vloc[k] == 1.0)) vertex = false;
        }
        if (vertex) {
            double dirs[3];
            for (int k = 0; k < 3; ++k) dirs[k] = sg[k] * (vloc[k] == 1.0 ? -1.0 : 1.0);
            const int nq = nd * nd * nd;
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3, c = (a + 2) % 3;
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    int i0 = q / (nd * nd), i1 = (q / nd) % nd, i2 = q % nd;
                    double S = gx[i0], T1 = gx[i1], T2 = gx[i2];
                    double v[3];
                    v[a] = S; v[b] = S * T1; v[c] = S * T2;
                    double u[3];
                    for (int k = 0; k < 3; ++k) u[k] = -d[k] + v[k] * dirs[k];
                    double wq = gw[i0] * gw[i1] * gw[i2] * S / sqrt(1.0 + T1 * T1 + T2 * T2);
                    double W[7];
                    kernel_weights(u, W);
                    for (int k = 0; k < 7; ++k) acc[k] += W[k] * wq;
                }
            }
        } else {
            const int nq = ng * ng * ng;
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                int i0 = q / (ng * ng), i1 = (q / ng) % ng, i2 = q % ng;
                double u[3] = {sg[0] * hx[i0], sg[1] * hx[i1], sg[2] * hx[i2]};
                double rx = d[0] + u[0], ry = d[1] + u[1], rz = d[2] + u[2];
                double wq = hw[i0] * hw[i1] * hw[i2] / sqrt(rx * rx + ry * ry + rz * rz);
                double W[7];
                kernel_weights(u, W);
                for (int k = 0; k < 7; ++k) acc[k] += W[k] * wq;
            }
        }
    }
    __shared__ double red[7][256];
    for (int k = 0; k < 7; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t Kt = (int64_t)Kx * Ky * Kz;
        const int64_t idx = ((int64_t)d[2] * Ky + d[1]) * Kx + d[0];
        for (int k = 0; k < 7; ++k) T[k * Kt + idx] = red[k][0] * 0.07957747154594766788;
    }
}

int generate_toeplitz_device(Handle* h, std::vector<double>& Tout) {
    const int orders[5] = {12, 8, 6, 5, 4};
    std::vector<double> tab;
    FarTables ft{};
    int rows = 0;
    for (int t = 0; t < 5; ++t) {
        std::vector<double> x, w;
        gauss_legendre01(orders[t], x, w);
        const int n = orders[t];
        ft.off[t] = rows;
        ft.nq[t] = 8 * n * n * n;
        for (int box = 0; box < 8; ++box) {
            const double sg[3] = {(box & 1) ? 1.0 : -1.0, (box & 2) ? 1.0 : -1.0, (box & 4) ? 1.0 : -1.0};
            for (int i0 = 0; i0 < n; ++i0)
                for (int i1 = 0; i1 < n; ++i1)
                    for (int i2 = 0; i2 < n; ++i2) {
                        double u[3] = {sg[0] * x[i0], sg[1] * x[i1], sg[2] * x[i2]};
                        double W[7];
                        kernel_weights(u, W);
                        double wq = w[i0] * w[i1] * w[i2];
                        tab.push_back(u[0]);
                        tab.push_back(u[1]);
                        tab.push_back(u[2]);
                        for (int k = 0; k < 7; ++k) tab.push_back(W[k] * wq);
                    }
        }
        rows += ft.nq[t];
    }
    std::vector<double> gx, gw, hx, hw;
    gauss_legendre01(16, gx, gw);
    gauss_legendre01(12, hx, hw);
    DevBuf d_tab, d_gx, d_gw, d_hx, d_hw, d_T;
    const int64_t Kt = (int64_t)h->Kx * h->Ky * h->Kz;
    int rc = 0;
    auto cleanup = [&]() {
        dev_free(d_tab); dev_free(d_gx); dev_free(d_gw); dev_free(d_hx); dev_free(d_hw); dev_free(d_T);
    };
    if ((rc = dev_upload(h, d_tab, tab.data(), tab.size() * 8)) || (rc = dev_upload(h, d_gx, gx.data(), gx.size() * 8)) ||
        (rc = dev_upload(h, d_gw, gw.data(), gw.size() * 8)) || (rc = dev_upload(h, d_hx, hx.data(), hx.size() * 8)) ||
        (rc = dev_upload(h, d_hw, hw.data(), hw.size() * 8)) || (rc = dev_alloc(h, d_T, (size_t)7 * Kt * 8))) {
        cleanup();
        return rc;
    }
    ft.tab = static_cast<const double*>(d_tab.p);
    double* T = static_cast<double*>(d_T.p);
    k_far<<<(unsigned)((Kt + 127) / 128), 128, 0, h->stream>>>(ft, h->Kx, h->Ky, h->Kz, T);
    k_near<<<8, 256, 0, h->stream>>>(static_cast<const double*>(d_gx.p), static_cast<const double*>(d_gw.p), 16,
                                     static_cast<const double*>(d_hx.p), static_cast<const double*>(d_hw.p), 12,
                                     h->Kx, h->Ky, h->Kz, T);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        Tout.resize((size_t)7 * Kt);
        e = cudaMemcpyAsync(Tout.data(), T, Tout.size() * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    cleanup();
    if (e != cudaSuccess) return cuda_err(h, e, "generate_toeplitz_device");
    return SVH_OK;
}

}  // namespace svh
