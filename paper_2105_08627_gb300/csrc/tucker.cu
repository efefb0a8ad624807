// tucker.cu -- device restore of the kernel spectra from their Tucker form (Eq. 10-11).
//
// S[kz][ky][kx] = sum_{a,b,c} core[c][b][a] F1[kx][a] F2[ky][b] F3[kz][c] is
// evaluated as three successive mode products (Eq. 11), each a small batched
// contraction out[o][i][n] = sum_j F[i][j] in[o][j][n]:
//   W1[c][b][kx]  = sum_a core[c][b][a] F1[kx][a]
//   W2[c][ky][kx] = sum_b W1[c][b][kx] F2[ky][b]
//   S[kz][ky][kx] = sum_c W2[c][ky][kx] F3[kz][c]
// Modes 1 and 2 are batches of GEMMs on the tensor cores (3xTF32, one launch
// per stage for all kernels); mode 3 (d3, Hz ~ Pz/2) is a streaming kernel
// (k_mode3_h, its plane count a compile-time constant).
// The S and Q spectra keep ranks of 100-250 per mode at tol = 1e-8 (only G00
// compresses to ~20), so the restore is a real dense contraction of about
// 2.5 GFLOP at 512 x 512 x 16. The three-way TF32 split keeps the rebuilt
// spectra within ~1e-7 of the FP64 ones, which the 1e-5 product bound needs;
// single-pass TF32 or BF16 products (10 or 7 mantissa bits) would not.
#include <cuda_runtime.h>

#include <stdint.h>

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

// Tensor-core tiles: mma.sync m16n8k8 with TF32 operands, split three ways
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi); D += lo*hi' + hi*lo' + hi*hi')
// so the products keep close to FP32 accuracy, which the 1e-5 bound on the
// operator product needs (a single TF32 pass keeps only 10 mantissa bits).
// 8 warps per 64 x 64 tile, warp w owns rows (w % 4)*16..+15 and columns
// (w / 4)*32..+31 (four n8 fragments); k tiles of 16 are staged in shared
// memory, the next one fetched into registers during the current MMAs.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_gemm_batched(const GemmProb* __restrict__ probs) {
    const GemmProb p = probs[blockIdx.z];
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    if (m0 >= p.M || n0 >= p.N) return;
    // As[k][m], Bs[k][n]; a row stride of 72 words puts the 32 fragment reads
    // (k8 + t, g) of a warp on 32 distinct banks
    __shared__ __align__(16) float As[2][GB_K][GB_M + 8];
    __shared__ __align__(16) float Bs[2][GB_K][GB_N + 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 32;
    float acc[4][4] = {};
    float ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = threadIdx.x + q * 256;
            const int mm = i / GB_K, kk = i % GB_K;
            const int m = m0 + mm, k = k0 + kk;
            ra[q] = (m < p.M && k < p.K) ? __ldg(p.A + (int64_t)m * p.lda + k) : 0.f;
            int nn, kb;
            if (p.bsn == 1) { kb = i / GB_N; nn = i % GB_N; }
            else { nn = i / GB_K; kb = i % GB_K; }
            const int n = n0 + nn, kq = k0 + kb;
            rb[q] = (n < p.N && kq < p.K) ? __ldg(p.B + (int64_t)kq * p.bsk + (int64_t)n * p.bsn) : 0.f;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = threadIdx.x + q * 256;
            As[buf][i % GB_K][i / GB_K] = ra[q];
            if (p.bsn == 1) Bs[buf][i / GB_N][i % GB_N] = rb[q];
            else Bs[buf][i % GB_K][i / GB_K] = rb[q];
        }
    };
    fetch(0);
    stash(0);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < p.K; k0 += GB_K) {
        const bool more = k0 + GB_K < p.K;
        if (more) fetch(k0 + GB_K);
#pragma unroll
        for (int k8 = 0; k8 < GB_K; k8 += 8) {
            const float af[4] = {As[cur][k8 + t][wm + g], As[cur][k8 + t][wm + g + 8], As[cur][k8 + t + 4][wm + g],
                                 As[cur][k8 + t + 4][wm + g + 8]};
            uint32_t ah[4], al[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ah[q] = to_tf32(af[q]);
                al[q] = to_tf32(af[q] - __uint_as_float(ah[q]));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float bf[2] = {Bs[cur][k8 + t][wn + j * 8 + g], Bs[cur][k8 + t + 4][wn + j * 8 + g]};
                uint32_t bh[2], bl[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    bh[q] = to_tf32(bf[q]);
                    bl[q] = to_tf32(bf[q] - __uint_as_float(bh[q]));
                }
                mma_tf32(acc[j], al, bh);
                mma_tf32(acc[j], ah, bl);
                mma_tf32(acc[j], ah, bh);
            }
        }
        if (more) {
            stash(cur ^ 1);
            __syncthreads();
            cur ^= 1;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int n = n0 + wn + j * 8 + 2 * t;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int m = m0 + wm + g + 8 * h2;
            if (m >= p.M) continue;
            if (n < p.N) p.C[(int64_t)m * p.ldc + n] = acc[j][2 * h2];
            if (n + 1 < p.N) p.C[(int64_t)m * p.ldc + n + 1] = acc[j][2 * h2 + 1];
        }
    }
}

// Mode-3 product S[kz][n] = sum_c F3[kz][c] W2[c][n] (d3 and Hz small): a
// streaming kernel, one output column n per thread, F3 in shared memory.
struct Mode3 {
    const float* W2[7];
    const float* F3[7];
    float* out[7];
    int d3[7];
    int64_t n;     // Hy * Hx
    int Hz;
};

__global__ void __launch_bounds__(256) k_mode3(const __grid_constant__ Mode3 a) {
    const int s = blockIdx.y;
    __shared__ float f3[64 * 64];
    const int d3 = a.d3[s];
    for (int i = threadIdx.x; i < a.Hz * d3; i += 256) f3[i] = a.F3[s][i];
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (n >= a.n) return;
    float w[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) w[c] = c < d3 ? __ldg(a.W2[s] + (int64_t)c * a.n + n) : 0.f;
    for (int kz = 0; kz < a.Hz; ++kz) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 64; ++c)
            if (c < d3) acc = fmaf(f3[kz * d3 + c], w[c], acc);
        a.out[s][(int64_t)kz * a.n + n] = acc;
    }
}

// k_mode3 with the plane count a compile-time constant (Hz = Pz / 2 + 1 of
// the specialised z sizes): d3 <= Hz values per point in registers, no
// shared memory, the same fmaf order as k_mode3.
template <int NH>
__global__ void __launch_bounds__(256) k_mode3_h(const __grid_constant__ Mode3 a) {
    const int s = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (n >= a.n) return;
    const int d3 = a.d3[s];
    const float* F3 = a.F3[s];
    float w[NH];
#pragma unroll
    for (int c = 0; c < NH; ++c) w[c] = c < d3 ? __ldg(a.W2[s] + (int64_t)c * a.n + n) : 0.f;
#pragma unroll
    for (int kz = 0; kz < NH; ++kz) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < NH; ++c)
            if (c < d3) acc = fmaf(__ldg(F3 + kz * d3 + c), w[c], acc);
        a.out[s][(int64_t)kz * a.n + n] = acc;
    }
}

static bool launch_mode3_h(const Mode3& m3, int nz, cudaStream_t st) {
    const dim3 grid((unsigned)((m3.n + 255) / 256), nz);
    switch (m3.Hz) {
        case 5: k_mode3_h<5><<<grid, 256, 0, st>>>(m3); return true;
        case 7: k_mode3_h<7><<<grid, 256, 0, st>>>(m3); return true;
        case 9: k_mode3_h<9><<<grid, 256, 0, st>>>(m3); return true;
        case 13: k_mode3_h<13><<<grid, 256, 0, st>>>(m3); return true;
        case 17: k_mode3_h<17><<<grid, 256, 0, st>>>(m3); return true;
        case 25: k_mode3_h<25><<<grid, 256, 0, st>>>(m3); return true;
        default: return false;
    }
}

int launch_tucker_rebuild(Handle* h, cudaStream_t strm) {
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
            // mode 3: S[kz][(ky,kx)] = sum_c F3[kz][c] W2[c][(ky,kx)] (k_mode3 when small)
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
        SVH_CUDA_TRY(h, cudaMemcpyAsync(h->d_tk_probs.p, h->tk_probs.data(), bytes, cudaMemcpyHostToDevice, strm));
        SVH_CUDA_TRY(h, cudaStreamSynchronize(strm));
        h->tk_probs_version = h->tk_version;
    }
    const GemmProb* all = reinterpret_cast<const GemmProb*>(h->tk_probs.data());
    const GemmProb* dev = static_cast<const GemmProb*>(h->d_tk_probs.p);
    int off = 0;
    for (int st = 0; st < 2; ++st) {
        const int n = h->tk_probs_split[st];
        int mt = 0, nt = 0;
        for (int i = 0; i < n; ++i) {
            mt = std::max(mt, (all[off + i].M + GB_M - 1) / GB_M);
            nt = std::max(nt, (all[off + i].N + GB_N - 1) / GB_N);
        }
        if (n) k_gemm_batched<<<dim3(nt, mt, n), 256, 0, strm>>>(dev + off);
        off += n;
    }
    // mode 3
    const int nz = h->tk_probs_split[2];
    bool small = Hz <= 64;
    for (int i = 0; i < nz; ++i) small = small && all[off + i].K <= 64;
    if (small && nz) {
        Mode3 m3{};
        for (int i = 0; i < nz; ++i) {
            m3.W2[i] = all[off + i].B;
            m3.F3[i] = all[off + i].A;
            m3.out[i] = all[off + i].C;
            m3.d3[i] = all[off + i].K;
        }
        m3.n = (int64_t)Hy * Hx;
        m3.Hz = Hz;
        if (!launch_mode3_h(m3, nz, strm))
            k_mode3<<<dim3((unsigned)((m3.n + 255) / 256), nz), 256, 0, strm>>>(m3);
    } else if (nz) {
        int mt = 0, nt = 0;
        for (int i = 0; i < nz; ++i) {
            mt = std::max(mt, (all[off + i].M + GB_M - 1) / GB_M);
            nt = std::max(nt, (all[off + i].N + GB_N - 1) / GB_N);
        }
        k_gemm_batched<<<dim3(nt, mt, nz), 256, 0, strm>>>(dev + off);
    }
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

}  // namespace svh
