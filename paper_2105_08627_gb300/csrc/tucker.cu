// tucker.cu -- device restore of the kernel spectra from their Tucker form (Eq. 10-11).
//
// S[kz][ky][kx] = sum_{a,b,c} core[c][b][a] F1[kx][a] F2[ky][b] F3[kz][c] is
// evaluated as three successive mode products (Eq. 11), each a small batched
// contraction out[o][i][n] = sum_j F[i][j] in[o][j][n]:
//   W1[c][b][kx]  = sum_a core[c][b][a] F1[kx][a]
//   W2[c][ky][kx] = sum_b W1[c][b][kx] F2[ky][b]
//   S[kz][ky][kx] = sum_c W2[c][ky][kx] F3[kz][c]
// Each stage is a batch of FP32 GEMMs (one launch per stage for all kernels).
// The S and Q spectra keep ranks of 100-250 per mode at tol = 1e-8 (only G00
// compresses to ~20), so the restore is a real dense contraction of about
// 2.5 GFLOP at 512 x 512 x 16. FP32 keeps the rebuilt spectra within ~1e-7
// of the FP64 ones, which the 1e-5 product bound needs; single-pass TF32 or
// BF16 tensor-core products (10 or 7 mantissa bits) would not.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "svh_internal.h"

namespace svh {

// ---------------------------------------------------------------- batched FP32 GEMM
// C[m][n] = sum_k A[m][k] B(k, n) for a list of independent problems; A is
// row-major (lda), B(k, n) = B[k*bsk + n*bsn], C row-major (ldc). Tiles of
// 64 x 64 outputs per block, 16-deep k steps staged in shared memory, 4 x 4
// outputs per thread. blockIdx.z selects the problem; blocks past a
// problem's tile count return at once.
struct GemmProb {
    const float* A;
    const float* B;
    float* C;
    int M, N, K, lda, bsk, bsn, ldc;
};

constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

__global__ void __launch_bounds__(256) k_gemm_batched(const GemmProb* __restrict__ probs) {
    const GemmProb p = probs[blockIdx.z];
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    if (m0 >= p.M || n0 >= p.N) return;
    __shared__ float As[GB_K][GB_M + 4];
    __shared__ float Bs[GB_K][GB_N + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < p.K; k0 += GB_K) {
        for (int i = threadIdx.x; i < GB_M * GB_K; i += 256) {
            const int mm = i / GB_K, kk = i % GB_K;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < p.M && k < p.K) ? __ldg(p.A + (int64_t)m * p.lda + k) : 0.f;
        }
        for (int i = threadIdx.x; i < GB_N * GB_K; i += 256) {
            int nn, kk;
            if (p.bsn == 1) { kk = i / GB_N; nn = i % GB_N; }   // n contiguous: coalesce over n
            else { nn = i / GB_K; kk = i % GB_K; }              // k contiguous: coalesce over k
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < p.N && k < p.K) ? __ldg(p.B + (int64_t)k * p.bsk + (int64_t)n * p.bsn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= p.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < p.N) p.C[(int64_t)m * p.ldc + n] = acc[i][j];
        }
    }
}

int launch_tucker_rebuild(Handle* h) {
    const int Hx = h->Hx, Hy = h->Hy, Hz = h->Hz;
    const int64_t Ht = (int64_t)Hx * Hy * Hz;
    size_t n1 = 0, n2 = 0;
    for (int u = 0; u < 7; ++u)
        if (h->tucker_on[u]) {
            n1 += (size_t)h->tk[u].d[2] * h->tk[u].d[1] * Hx;
            n2 += (size_t)h->tk[u].d[2] * Hy * Hx;
        }
    if (n1 == 0) return SVH_OK;
    bool fresh = false;
    if (h->d_tk_w1.bytes < n1 * 4) { int rc = dev_alloc(h, h->d_tk_w1, n1 * 4); if (rc) return rc; fresh = true; }
    if (h->d_tk_w2.bytes < n2 * 4) { int rc = dev_alloc(h, h->d_tk_w2, n2 * 4); if (rc) return rc; fresh = true; }
    if (fresh || h->tk_probs_version != h->tk_version) {
        float* w1 = static_cast<float*>(h->d_tk_w1.p);
        float* w2 = static_cast<float*>(h->d_tk_w2.p);
        float* spec = static_cast<float*>(h->d_spec32.p);
        std::vector<GemmProb> px, py, pz;
        size_t o1 = 0, o2 = 0;
        for (int u = 0; u < 7; ++u) {
            if (!h->tucker_on[u]) continue;
            const int d1 = h->tk[u].d[0], d2 = h->tk[u].d[1], d3 = h->tk[u].d[2];
            const float* core = static_cast<const float*>(h->d_tk_core[u].p);
            const float* F1 = static_cast<const float*>(h->d_tk_F[u][0].p);
            const float* F2 = static_cast<const float*>(h->d_tk_F[u][1].p);
            const float* F3 = static_cast<const float*>(h->d_tk_F[u][2].p);
            float* W1 = w1 + o1;
            float* W2 = w2 + o2;
            o1 += (size_t)d3 * d2 * Hx;
            o2 += (size_t)d3 * Hy * Hx;
            // mode 1: W1[(c,b)][kx] = sum_a core[(c,b)][a] F1[kx][a]
            px.push_back(GemmProb{core, F1, W1, d3 * d2, Hx, d1, d1, 1, d1, Hx});
            // mode 2: W2[c][ky][kx] = sum_b F2[ky][b] W1[(c,b)][kx]
            for (int c = 0; c < d3; ++c)
                py.push_back(GemmProb{F2, W1 + (size_t)c * d2 * Hx, W2 + (size_t)c * Hy * Hx, Hy, Hx, d2, d2, Hx, 1, Hx});
            // mode 3: S[kz][(ky,kx)] = sum_c F3[kz][c] W2[c][(ky,kx)]
            pz.push_back(GemmProb{F3, W2, spec + u * Ht, Hz, Hy * Hx, d3, d3, Hy * Hx, 1, Hy * Hx});
        }
        h->tk_probs.clear();
        h->tk_probs_split[0] = (int)px.size();
        h->tk_probs_split[1] = (int)py.size();
        h->tk_probs_split[2] = (int)pz.size();
        for (auto* v : {&px, &py, &pz}) {
            const char* b = reinterpret_cast<const char*>(v->data());
            h->tk_probs.insert(h->tk_probs.end(), b, b + v->size() * sizeof(GemmProb));
        }
        const size_t bytes = h->tk_probs.size();
        if (h->d_tk_probs.bytes < bytes) { int rc = dev_alloc(h, h->d_tk_probs, bytes); if (rc) return rc; }
        SVH_CUDA_TRY(h, cudaMemcpyAsync(h->d_tk_probs.p, h->tk_probs.data(), bytes, cudaMemcpyHostToDevice, h->stream));
        SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->tk_probs_version = h->tk_version;
    }
    const GemmProb* all = reinterpret_cast<const GemmProb*>(h->tk_probs.data());
    const GemmProb* dev = static_cast<const GemmProb*>(h->d_tk_probs.p);
    int off = 0;
    for (int st = 0; st < 3; ++st) {
        const int n = h->tk_probs_split[st];
        int mt = 0, nt = 0;
        for (int i = 0; i < n; ++i) {
            mt = std::max(mt, (all[off + i].M + GB_M - 1) / GB_M);
            nt = std::max(nt, (all[off + i].N + GB_N - 1) / GB_N);
        }
        if (n) k_gemm_batched<<<dim3(nt, mt, n), 256, 0, h->stream>>>(dev + off);
        off += n;
    }
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

}  // namespace svh
