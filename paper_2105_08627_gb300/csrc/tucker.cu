// tucker.cu -- device restore of the kernel spectra from their Tucker form (Eq. 10-11).
//
// S[kz][ky][kx] = sum_{a,b,c} core[c][b][a] F1[kx][a] F2[ky][b] F3[kz][c] is
// evaluated as three successive mode products (Eq. 11), each a small batched
// contraction out[o][i][n] = sum_j F[i][j] in[o][j][n]:
//   W1[c][b][kx]  = sum_a core[c][b][a] F1[kx][a]
//   W2[c][ky][kx] = sum_b W1[c][b][kx] F2[ky][b]
//   S[kz][ky][kx] = sum_c W2[c][ky][kx] F3[kz][c]
// One launch per stage covers all Tucker-stored kernels (blockIdx.y). The
// work is < 1 % of a matvec's and FP32 keeps the rebuilt spectra within
// ~1e-7 of the FP64 ones, which the 1e-5 matvec bound needs; TF32 or BF16
// tensor-core products (10 or 7 mantissa bits) would not.
#include <cuda_runtime.h>

#include "svh_internal.h"

namespace svh {

struct ModeProd {
    const float* in[7];
    float* out[7];
    const float* F[7];
    int outer[7], J[7], I[7], inner[7];
    int nk;
    int map[7];   // kernel slot -> kernel id
};

__global__ void k_modeprod(ModeProd a) {
    const int s = blockIdx.y;
    const int64_t inner = a.inner[s], I = a.I[s], J = a.J[s];
    const int64_t n_out = (int64_t)a.outer[s] * I * inner;
    const float* __restrict__ in = a.in[s];
    const float* __restrict__ F = a.F[s];
    float* __restrict__ out = a.out[s];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_out; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = e % inner;
        int64_t t = e / inner;
        int64_t i = t % I, o = t / I;
        const float* src = in + o * J * inner + n;
        const float* f = F + i * J;
        float acc = 0.f;
        for (int j = 0; j < J; ++j) acc = fmaf(__ldg(f + j), __ldg(src + (int64_t)j * inner), acc);
        out[e] = acc;
    }
}

int launch_tucker_rebuild(Handle* h) {
    const int Hx = h->Hx, Hy = h->Hy, Hz = h->Hz;
    const int64_t Ht = (int64_t)Hx * Hy * Hz;
    size_t n1 = 0, n2 = 0;
    int nk = 0;
    for (int u = 0; u < 7; ++u)
        if (h->tucker_on[u]) {
            n1 += (size_t)h->tk[u].d[2] * h->tk[u].d[1] * Hx;
            n2 += (size_t)h->tk[u].d[2] * Hy * Hx;
            ++nk;
        }
    if (nk == 0) return SVH_OK;
    if (h->d_tk_w1.bytes < n1 * 4) { int rc = dev_alloc(h, h->d_tk_w1, n1 * 4); if (rc) return rc; }
    if (h->d_tk_w2.bytes < n2 * 4) { int rc = dev_alloc(h, h->d_tk_w2, n2 * 4); if (rc) return rc; }
    float* w1 = static_cast<float*>(h->d_tk_w1.p);
    float* w2 = static_cast<float*>(h->d_tk_w2.p);
    float* spec = static_cast<float*>(h->d_spec32.p);
    ModeProd s1{}, s2{}, s3{};
    size_t o1 = 0, o2 = 0;
    int k = 0;
    int64_t max_out = 0;
    for (int u = 0; u < 7; ++u) {
        if (!h->tucker_on[u]) continue;
        const int d1 = h->tk[u].d[0], d2 = h->tk[u].d[1], d3 = h->tk[u].d[2];
        float* W1 = w1 + o1;
        float* W2 = w2 + o2;
        o1 += (size_t)d3 * d2 * Hx;
        o2 += (size_t)d3 * Hy * Hx;
        s1.in[k] = static_cast<const float*>(h->d_tk_core[u].p); s1.out[k] = W1;
        s1.F[k] = static_cast<const float*>(h->d_tk_F[u][0].p);
        s1.outer[k] = d3 * d2; s1.J[k] = d1; s1.I[k] = Hx; s1.inner[k] = 1;
        s2.in[k] = W1; s2.out[k] = W2; s2.F[k] = static_cast<const float*>(h->d_tk_F[u][1].p);
        s2.outer[k] = d3; s2.J[k] = d2; s2.I[k] = Hy; s2.inner[k] = Hx;
        s3.in[k] = W2; s3.out[k] = spec + u * Ht; s3.F[k] = static_cast<const float*>(h->d_tk_F[u][2].p);
        s3.outer[k] = 1; s3.J[k] = d3; s3.I[k] = Hz; s3.inner[k] = Hy * Hx;
        max_out = std::max<int64_t>(max_out, std::max<int64_t>((int64_t)d3 * d2 * Hx, std::max<int64_t>((int64_t)d3 * Hy * Hx, Ht)));
        ++k;
    }
    s1.nk = s2.nk = s3.nk = nk;
    auto blocks = [](int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); };
    k_modeprod<<<dim3(blocks((int64_t)max_out), nk), 256, 0, h->stream>>>(s1);
    k_modeprod<<<dim3(blocks((int64_t)max_out), nk), 256, 0, h->stream>>>(s2);
    k_modeprod<<<dim3(blocks(Ht), nk), 256, 0, h->stream>>>(s3);
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

}  // namespace svh
