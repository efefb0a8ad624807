// tucker_svd_dev.cu -- Algorithm 1 (Tucker-SVD) of the FP64 octant spectra on the device.
//
// For each mode i of S (x, y, z): the left singular vectors of the mode-i
// unfolding S_(i) of the original tensor, the rank d_i as the smallest d whose
// discarded part ||(I - U_d U_d^T) S_(i)||_F^2 = sum_{r >= d} ||u_r^T S_(i)||^2
// stays within tol^2 / 3 ||S||_F^2 (the rows u_r^T S_(i) formed from S
// itself), and the projection of the core onto the d_i leading vectors
// (Eq. 10; modes taken in order x, y, z on the shrinking core). The singular
// vectors come from a Householder QR of S_(i)^T = Q R (tall: D_i columns) and
// the SVD of the small triangle R = U_R Sigma V_R^T, since S_(i) = V_R Sigma
// (Q U_R)^T: both steps are backward stable, so the singular values carry an
// absolute error ~ eps sigma_max, far below the threshold (~ 6e-9 ||S|| at
// tol 1e-8). The Gram matrix S_(i) S_(i)^T would not do: its round-off,
// eps ||S||^2, exceeds tol^2 / 3 ||S||^2, and the trailing eigenvectors it
// yields mix with the leading ones. QR, SVD and GEMMs are library calls
// (cuSOLVER, cuBLAS); the copies and row norms are kernels of this file.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "svh_internal.h"

namespace svh {

struct TsvdHandles {
    cublasHandle_t bl = nullptr;
    cusolverDnHandle_t so = nullptr;
    ~TsvdHandles() {
        if (bl) cublasDestroy(bl);
        if (so) cusolverDnDestroy(so);
    }
};

void tsvd_free(void* p) { delete static_cast<TsvdHandles*>(p); }

constexpr int RS_BLOCKS = 64, RS_THREADS = 128;

// partial[b][i] = sum over the columns j = b, b + RS_BLOCKS, ... of T[i + j ld]^2 (column-major
// T, m rows); one block per column residue, the rows spread over the threads (coalesced)
__global__ void k_row_sumsq_partial(const double* __restrict__ T, int m, int64_t n, int64_t ld,
                                    double* __restrict__ partial) {
    for (int i = threadIdx.x; i < m; i += RS_THREADS) {
        double s = 0;
        for (int64_t j = blockIdx.x; j < n; j += RS_BLOCKS) {
            const double v = T[i + j * ld];
            s = fma(v, v, s);
        }
        partial[(int64_t)blockIdx.x * m + i] = s;
    }
}
// out[i] (+)= sum_b partial[b][i], in a fixed order
__global__ void k_row_sumsq_final(const double* __restrict__ partial, int m, double* __restrict__ out, int add) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0;
    for (int b = 0; b < RS_BLOCKS; ++b) s += partial[(int64_t)b * m + i];
    out[i] = add ? out[i] + s : s;
}

// R (n x n, column-major, zero below the diagonal) from the upper triangle of a QR-factored
// column-major m x n matrix A (ld m)
__global__ void k_upper(const double* __restrict__ A, int64_t lda, double* __restrict__ R, int n) {
    const int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || j >= n) return;
    R[(int64_t)j * n + i] = i <= j ? A[(int64_t)j * lda + i] : 0.0;
}

namespace {

struct Buf {
    double* p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    bool alloc(size_t n) { return cudaMalloc(&p, n * sizeof(double)) == cudaSuccess; }
};

}  // namespace

#define TSVD_BL(call) do { if ((call) != CUBLAS_STATUS_SUCCESS) return set_err(h, SVH_ERR_CUDA, "device Tucker-SVD: cuBLAS call failed"); } while (0)
#define TSVD_SO(call) do { if ((call) != CUSOLVER_STATUS_SUCCESS) return set_err(h, SVH_ERR_CUDA, "device Tucker-SVD: cuSOLVER call failed"); } while (0)

// Algorithm 1 on kernel u's FP64 octant spectrum (d_spec64, [Hz][Hy][Hx], x fastest):
// dims (D1, D2, D3) = (Hx, Hy, Hz); the result in the host Tucker layout
// (core [d3][d2][d1], F_i [D_i][d_i] row-major)
int tucker_svd_device(Handle* h, int u, double tol, Tucker& out) {
    if (!h->d_spec64.p) return set_err(h, SVH_ERR_STATE, "device Tucker-SVD: no FP64 spectra on the device");
    if (!h->tsvd) h->tsvd = new TsvdHandles();
    TsvdHandles* H = static_cast<TsvdHandles*>(h->tsvd);
    if (!H->bl) TSVD_BL(cublasCreate(&H->bl));
    if (!H->so) TSVD_SO(cusolverDnCreate(&H->so));
    cudaStream_t s = h->stream;
    TSVD_BL(cublasSetStream(H->bl, s));
    TSVD_SO(cusolverDnSetStream(H->so, s));
    const int D[3] = {h->Hx, h->Hy, h->Hz};
    const int64_t Ht = (int64_t)D[0] * D[1] * D[2];
    const double* O = static_cast<const double*>(h->d_spec64.p) + u * Ht;
    double norm = 0;
    TSVD_BL(cublasDnrm2(H->bl, (int)Ht, O, 1, &norm));
    const double thr2 = tol * tol / 3.0 * norm * norm;
    const int Dmax = std::max(D[0], std::max(D[1], D[2]));
    Buf M, Rm, Sg, VT, T, rown, part, F, C0, C1, C2, tau;
    int* info = nullptr;
    if (!M.alloc(Ht) || !Rm.alloc((size_t)Dmax * Dmax) || !Sg.alloc(Dmax) || !VT.alloc((size_t)Dmax * Dmax) ||
        !T.alloc(Ht) || !rown.alloc(Dmax) || !part.alloc((size_t)RS_BLOCKS * Dmax) || !F.alloc((size_t)Dmax * Dmax) ||
        !C0.alloc(Ht) || !C1.alloc(Ht) || !C2.alloc(Ht) || !tau.alloc(Dmax) ||
        cudaMalloc(&info, sizeof(int)) != cudaSuccess) {
        if (info) cudaFree(info);
        return set_err(h, SVH_ERR_OOM, "device Tucker-SVD: out of device memory");
    }
    struct InfoFree { int* p; ~InfoFree() { cudaFree(p); } } info_guard{info};
    const double one = 1.0, zero = 0.0;
    const int D1 = D[0], D2 = D[1], D3 = D[2];
    auto row_norms = [&](const double* Tm, int m, int64_t n, int64_t ld, int add) {
        k_row_sumsq_partial<<<RS_BLOCKS, RS_THREADS, 0, s>>>(Tm, m, n, ld, part.p);
        k_row_sumsq_final<<<(m + 127) / 128, 128, 0, s>>>(part.p, m, rown.p, add);
    };
    int d[3] = {0, 0, 0};
    std::vector<double> V, w, rn;
    for (int mode = 0; mode < 3; ++mode) {
        const int Dm = D[mode];
        const int Rr = (int)(Ht / Dm);   // columns of the unfolding
        // M = S_(mode)^T, column-major Rr x Dm
        if (mode == 0) {          // S as column-major D1 x (D2 D3), transposed
            TSVD_BL(cublasDgeam(H->bl, CUBLAS_OP_T, CUBLAS_OP_N, Rr, D1, &one, O, D1, &zero, M.p, Rr, M.p, Rr));
        } else if (mode == 1) {   // rows (c, a), column y: slab c (D1 x D2, ld D1) to rows c D1 .. of each column
            for (int c = 0; c < D3; ++c)
                SVH_CUDA_TRY(h, cudaMemcpy2DAsync(M.p + (int64_t)c * D1, (size_t)Rr * 8, O + (int64_t)c * D1 * D2,
                                                  (size_t)D1 * 8, (size_t)D1 * 8, D2, cudaMemcpyDeviceToDevice, s));
        } else {                  // S as column-major (D1 D2) x D3
            SVH_CUDA_TRY(h, cudaMemcpyAsync(M.p, O, (size_t)Ht * 8, cudaMemcpyDeviceToDevice, s));
        }
        // M = Q R, then R = U_R Sigma V_R^T: the rows of V_R^T are the left singular vectors of S_(mode)
        int lw_qr = 0, lw_svd = 0;
        TSVD_SO(cusolverDnDgeqrf_bufferSize(H->so, Rr, Dm, M.p, Rr, &lw_qr));
        TSVD_SO(cusolverDnDgesvd_bufferSize(H->so, Dm, Dm, &lw_svd));
        Buf work, rwork;
        if (!work.alloc((size_t)std::max(std::max(lw_qr, lw_svd), 1)) || !rwork.alloc((size_t)Dm))
            return set_err(h, SVH_ERR_OOM, "device Tucker-SVD: workspace");
        TSVD_SO(cusolverDnDgeqrf(H->so, Rr, Dm, M.p, Rr, tau.p, work.p, lw_qr, info));
        k_upper<<<dim3((Dm + 31) / 32, (Dm + 7) / 8), dim3(32, 8), 0, s>>>(M.p, Rr, Rm.p, Dm);
        signed char jn = 'N', ja = 'A';
        TSVD_SO(cusolverDnDgesvd(H->so, jn, ja, Dm, Dm, Rm.p, Dm, Sg.p, nullptr, Dm, VT.p, Dm, work.p, lw_svd,
                                 rwork.p, info));
        // rows u_r^T S_(mode) = (V_R^T S_(mode))_r and their squared norms
        if (mode == 0) {
            TSVD_BL(cublasDgemm(H->bl, CUBLAS_OP_N, CUBLAS_OP_N, D1, D2 * D3, D1, &one, VT.p, D1, O, D1, &zero, T.p, D1));
            row_norms(T.p, D1, (int64_t)D2 * D3, D1, 0);
        } else if (mode == 1) {   // per slab: V_R^T S_c^T (D2 x D1)
            for (int c = 0; c < D3; ++c) {
                TSVD_BL(cublasDgemm(H->bl, CUBLAS_OP_N, CUBLAS_OP_T, D2, D1, D2, &one, VT.p, D2,
                                    O + (int64_t)c * D1 * D2, D1, &zero, T.p, D2));
                row_norms(T.p, D2, D1, D2, c > 0);
            }
        } else {
            TSVD_BL(cublasDgemm(H->bl, CUBLAS_OP_N, CUBLAS_OP_T, D3, D1 * D2, D3, &one, VT.p, D3, O, D1 * D2, &zero,
                                T.p, D3));
            row_norms(T.p, D3, (int64_t)D1 * D2, D3, 0);
        }
        V.resize((size_t)Dm * Dm);
        w.resize(Dm);
        rn.resize(Dm);
        int inf = 0;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(V.data(), VT.p, V.size() * 8, cudaMemcpyDeviceToHost, s));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(w.data(), Sg.p, w.size() * 8, cudaMemcpyDeviceToHost, s));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(rn.data(), rown.p, rn.size() * 8, cudaMemcpyDeviceToHost, s));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(&inf, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        SVH_CUDA_TRY(h, cudaStreamSynchronize(s));
        if (inf != 0) return set_err(h, SVH_ERR_CUDA, "device Tucker-SVD: SVD did not converge");
        // vectors by decreasing singular value; rank from the tail of the row norms
        std::vector<int> idx(Dm);
        for (int k = 0; k < Dm; ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
        int dm = Dm;
        double tail = 0;
        for (int r = Dm - 1; r >= 1; --r) {
            tail += rn[idx[r]];
            if (tail <= thr2) dm = r;
            else break;
        }
        d[mode] = dm;
        // factor F [Dm][dm] (row-major, the host layout) and its column-major copy for the projection
        std::vector<double> Fr((size_t)Dm * dm), Fc((size_t)Dm * dm);
        for (int i = 0; i < Dm; ++i)
            for (int k = 0; k < dm; ++k) {
                const double v = V[(size_t)i * Dm + idx[k]];   // component i of vector idx[k]: V_R^T (k, i)
                Fr[(size_t)i * dm + k] = v;
                Fc[(size_t)k * Dm + i] = v;
            }
        out.F[mode] = Fr;
        out.d[mode] = dm;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(F.p, Fc.data(), Fc.size() * 8, cudaMemcpyHostToDevice, s));
        // projection of the core (x, then y, then z)
        if (mode == 0) {          // C0 [D3][D2][d1] = F1^T applied along x
            TSVD_BL(cublasDgemm(H->bl, CUBLAS_OP_T, CUBLAS_OP_N, dm, D2 * D3, D1, &one, F.p, D1, O, D1, &zero, C0.p, dm));
        } else if (mode == 1) {   // C1 [D3][d2][d1]: per slab C0_c (d1 x D2) F2
            TSVD_BL(cublasDgemmStridedBatched(H->bl, CUBLAS_OP_N, CUBLAS_OP_N, d[0], dm, D2, &one, C0.p, d[0],
                                              (long long)d[0] * D2, F.p, D2, 0, &zero, C1.p, d[0],
                                              (long long)d[0] * dm, D3));
        } else {                  // core [d3][d2][d1] = C1 ((d1 d2) x D3) F3
            TSVD_BL(cublasDgemm(H->bl, CUBLAS_OP_N, CUBLAS_OP_N, d[0] * d[1], dm, D3, &one, C1.p, d[0] * d[1], F.p, D3,
                                &zero, C2.p, d[0] * d[1]));
        }
        SVH_CUDA_TRY(h, cudaStreamSynchronize(s));   // F is rewritten by the next mode
    }
    out.core.resize((size_t)d[0] * d[1] * d[2]);
    SVH_CUDA_TRY(h, cudaMemcpyAsync(out.core.data(), C2.p, out.core.size() * 8, cudaMemcpyDeviceToHost, s));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(s));
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

}  // namespace svh
