// tucker.cu -- device restore of the kernel spectra from their Tucker form (Eq. 10-11).
//
// S[kz][ky][kx] = sum_{a,b,c} core[c][b][a] F1[kx][a] F2[ky][b] F3[kz][c]
// is a chain of mode products (Eq. 11), which commute. The z extent of the
// octant is small (Hz = Pz/2 + 1 <= 25 planes), so the mode-3 product is
// applied once when the Tucker data is loaded, in FP64 on the host:
//   core'[kz][b][a] = sum_c F3[kz][c] core[c][b][a]      (Hz x d2 x d1 values)
// and every restore is two GEMM stages on the tensor cores, one GEMM per kernel:
//   stage 1: W1[kz][kx][b] = sum_a F1[kx][a] core'[(kz, b)][a]        (M = Hx, N = Hz d2)
//   stage 2: S[kz][ky][kx] = sum_b F2[ky][b] W1[(kz, kx)][b]          (M = Hy, N = Hz Hx)
// Both are D = A B^T with A and B K-major (rows of contiguous k), the form
// tcgen05.mma reads from shared memory; the epilogue scatters column n of D
// to (n / g) s1 + (n % g) s2, which lays W1 out as stage 2's B operand and S
// as the octant spectra.
//
// The S and Q spectra keep ranks of 100-250 per mode at tol = 1e-8 (only G00
// compresses to ~20), so the restore is a dense contraction. The products use
// TF32 operands split two ways (x = hi + lo, hi = tf32(x), lo = tf32(x - hi);
// D += lo hi' + hi lo' + hi hi', FP32 accumulation in tensor memory), which
// keeps the restored spectra within ~1e-7 of the FP64 ones; a single TF32 or
// BF16 pass (10 or 7 mantissa bits) would break the 1e-5 product bound. The
// operands are stored split, as two planes [hi; lo]: the constant factors and
// core' when the Tucker data is loaded, W1 by stage 1's epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "svh_internal.h"
#include "tc_async.cuh"

namespace svh {

constexpr int TC_BM = 128;       // rows of a tile = MMA M = TMEM lanes
constexpr int TC_BK = 32;        // k per pipeline stage: one 128-byte swizzled row of FP32
#ifndef SVH_TC_MAXN
#define SVH_TC_MAXN 160
#endif
constexpr int TC_MAXN = SVH_TC_MAXN;   // widest tile: 160 leaves room for three pipeline stages, 256 for two
constexpr int TC_TMEM_COLS = 256;
constexpr int TC_EDGE = 8;       // up to this many rows past the last full tile: FP32 rows
constexpr int TC_THREADS = 192;  // warps 0-3 epilogue (+ edge rows), 4 TMA producer, 5 MMA issuer + TMEM
constexpr int TC_NPROB = 7;
constexpr int TC_MAX_STAGES = 4;
constexpr int TC_A_TILE = TC_BM * TC_BK * 4;   // 16 KB per plane
constexpr int TC_SMEM = 226 * 1024;            // dynamic shared memory per block
constexpr int TC_SPIN_LIMIT = 1 << 20;

static inline int pad8(int x) { return (x + 7) & ~7; }
constexpr int TC_E_TILE = TC_EDGE * TC_BK * 4;   // 1 KB per plane: the rows past the last full tile
// a stage: A hi, A lo (128 rows), B hi, B lo (ntw rows), E hi, E lo (TC_EDGE rows), all 1024-byte aligned
__host__ __device__ inline int tc_stage_bytes(int ntw) { return 2 * TC_A_TILE + 2 * ntw * TC_BK * 4 + 2 * TC_E_TILE; }
__host__ __device__ inline int tc_stages(int ntw) {
    const int n = (TC_SMEM - 1024 - ntw * 8) / tc_stage_bytes(ntw);
    return n < TC_MAX_STAGES ? n : TC_MAX_STAGES;
}

// One launch: one GEMM per kernel. A, B: planes [2][rows][K] (hi, lo), row
// stride K (a multiple of 8); mapA / mapB: their 3-D TMA views {K, rows, 2},
// boxes {32, 128, 1} and {32, ntw, 1}, 128-byte swizzle; mapE: A's view with
// box {32, TC_EDGE, 1} for the rows past the last full tile. Output (m, n) goes to
// C[m ldc + (n / g) s1 + (n % g) s2], and its lo part to c_lo further when
// c_lo != 0 (a split output).
struct TcStage {
    CUtensorMap mapA[TC_NPROB];
    CUtensorMap mapB[TC_NPROB];
    CUtensorMap mapE[TC_NPROB];
    const float* A[TC_NPROB];
    const float* B[TC_NPROB];
    float* C[TC_NPROB];
    int64_t a_plane[TC_NPROB], b_plane[TC_NPROB], ldc[TC_NPROB], s1[TC_NPROB], s2[TC_NPROB], c_lo[TC_NPROB];
    int M[TC_NPROB], N[TC_NPROB], K[TC_NPROB], ntw[TC_NPROB], g[TC_NPROB];
    int* status;
};

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void store_out(float* p, int64_t c_lo, float v) {
    if (c_lo) {
        const float h = tf32_round(v);
        p[0] = h;
        p[c_lo] = tf32_round(v - h);
    } else {
        p[0] = v;
    }
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int spins = 0; !mbar_try_wait(bar, parity);)
        if (++spins > TC_SPIN_LIMIT) return false;
    return true;
}

// FP32 rows [mr0, mr0 + nr) x columns [n0, n0 + nw) of D (nr <= TC_EDGE) from the
// hi + lo planes in global memory: one warp per column, the lanes split k and
// add up with shuffles (only used when M <= TC_EDGE, i.e. no tensor-core tile)
__device__ void tc_edge_rows_global(const TcStage& P, int u, int nr, int n0, int nw, const int64_t* col_off) {
    const int K = P.K[u], lane = threadIdx.x & 31;
    const int64_t ap = P.a_plane[u], bp = P.b_plane[u];
    for (int c = threadIdx.x >> 5; c < nw; c += TC_THREADS / 32) {
        const float* b = P.B[u] + (int64_t)(n0 + c) * K;
        float acc[TC_EDGE];
#pragma unroll
        for (int r = 0; r < TC_EDGE; ++r) acc[r] = 0.f;
        for (int k = 4 * lane; k < K; k += 128) {
            const float4 bh = __ldg(reinterpret_cast<const float4*>(b + k));
            const float4 bl = __ldg(reinterpret_cast<const float4*>(b + bp + k));
#pragma unroll
            for (int r = 0; r < TC_EDGE; ++r)
                if (r < nr) {
                    const float* a = P.A[u] + (int64_t)r * K + k;
                    const float4 ah = __ldg(reinterpret_cast<const float4*>(a));
                    const float4 al = __ldg(reinterpret_cast<const float4*>(a + ap));
                    acc[r] = fmaf(ah.x + al.x, bh.x + bl.x, acc[r]);
                    acc[r] = fmaf(ah.y + al.y, bh.y + bl.y, acc[r]);
                    acc[r] = fmaf(ah.z + al.z, bh.z + bl.z, acc[r]);
                    acc[r] = fmaf(ah.w + al.w, bh.w + bl.w, acc[r]);
                }
        }
#pragma unroll
        for (int r = 0; r < TC_EDGE; ++r) {
            float v = acc[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && r < nr) store_out(P.C[u] + (int64_t)r * P.ldc[u] + col_off[c], P.c_lo[u], v);
        }
    }
}

// One 128 x ntw tile of one kernel's GEMM per block (blockIdx.x: column tile,
// y: row tile, z: kernel). Warp 4 streams k-slices of the four operand planes
// (A hi, A lo, B hi, B lo) by TMA into a ring of shared-memory stages; warp 5
// issues the three tcgen05 MMAs per k-step of 8 as each stage lands and
// commits them to the stage's "empty" barrier, which lets the producer refill
// it; warps 0-3 compute the few rows past the last full tile (if any) in FP32
// meanwhile, then read the accumulator (TMEM lanes 32 w .. +31, w = warp),
// stage it in shared memory and write coalesced rows. Every wait is bounded:
// on expiry the block sets SVH_STATUS_MMA_TIMEOUT, skips its output, drains its
// copies (bounded), frees its TMEM and returns.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_restore(const __grid_constant__ TcStage P) {
    const int u = blockIdx.z;
    const int M = P.M[u], N = P.N[u], K = P.K[u], ntw = P.ntw[u];
    const int n0 = blockIdx.x * ntw;
    if (n0 >= N) return;
    const int nw = min(ntw, N - n0);
    const int mfull = M / TC_BM, mrem = M % TC_BM;
    const int mma_mt = mrem > TC_EDGE ? mfull + 1 : mfull;
    const int edge_rows = (mrem > 0 && mrem <= TC_EDGE) ? mrem : 0;
    if ((int)blockIdx.y >= max(mma_mt, 1)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* sm = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    const int sb = tc_stage_bytes(ntw), nst = tc_stages(ntw);
    int64_t* col_off = reinterpret_cast<int64_t*>(sm + nst * sb);
    const int g = P.g[u];
    for (int c = tid; c < nw; c += TC_THREADS) {
        const int n = n0 + c;
        col_off[c] = (int64_t)(n / g) * P.s1[u] + (int64_t)(n % g) * P.s2[u];
    }
    if (mma_mt == 0) {   // M <= TC_EDGE: FP32 rows only
        __syncthreads();
        tc_edge_rows_global(P, u, edge_rows, n0, nw, col_off);
        return;
    }
    // the block of the last full row tile also computes the rows past it, from the B
    // slices in shared memory; its stages are then released by two arrivals
    const bool do_edge = edge_rows > 0 && (int)blockIdx.y == mma_mt - 1;

    __shared__ uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag, n_issued, n_consumed;
    if (warp == 5) {
        tmem_alloc(&tmem_slot, TC_TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < nst; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], do_edge ? 2 : 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        n_issued = n_consumed = 0;
        fence_mbar_init();
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;
    const int m0 = blockIdx.y * TC_BM, mw = min(TC_BM, M - m0);
    const int nmma = (nw + 15) & ~15;
    const int nchunk = (K + TC_BK - 1) / TC_BK;
    const int bplane = ntw * TC_BK * 4;

    if (warp == 4) {
        if (lane == 0) {   // TMA producer
            const uint32_t bytes = (uint32_t)(sb - (do_edge ? 0 : 2 * TC_E_TILE));
            for (int s = 0; s < nchunk; ++s) {
                const int st = s % nst, it = s / nst;
                if (s >= nst && !wait_bounded(&empty[st], (uint32_t)(it - 1) & 1u)) {
                    atomicOr(P.status, SVH_STATUS_MMA_TIMEOUT);
                    *abort_v = 1;
                }
                if (*abort_v) break;
                uint8_t* base = sm + st * sb;
                mbar_expect_tx(&full[st], bytes);
                tma_load_3d(base, &P.mapA[u], &full[st], s * TC_BK, m0, 0);
                tma_load_3d(base + TC_A_TILE, &P.mapA[u], &full[st], s * TC_BK, m0, 1);
                tma_load_3d(base + 2 * TC_A_TILE, &P.mapB[u], &full[st], s * TC_BK, n0, 0);
                tma_load_3d(base + 2 * TC_A_TILE + bplane, &P.mapB[u], &full[st], s * TC_BK, n0, 1);
                if (do_edge) {
                    tma_load_3d(base + 2 * TC_A_TILE + 2 * bplane, &P.mapE[u], &full[st], s * TC_BK, mfull * TC_BM, 0);
                    tma_load_3d(base + 2 * TC_A_TILE + 2 * bplane + TC_E_TILE, &P.mapE[u], &full[st], s * TC_BK,
                                mfull * TC_BM, 1);
                }
                n_issued = s + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = idesc_tf32(TC_BM, nmma);
            for (int s = 0; s < nchunk; ++s) {
                const int st = s % nst, it = s / nst;
                if (!wait_bounded(&full[st], (uint32_t)it & 1u)) {
                    atomicOr(P.status, SVH_STATUS_MMA_TIMEOUT);
                    *abort_v = 1;
                }
                if (*abort_v) break;
                tc_fence_after();
                const uint32_t a_hi = smem_u32(sm + st * sb), a_lo = a_hi + TC_A_TILE;
                const uint32_t b_hi = a_hi + 2 * TC_A_TILE, b_lo = b_hi + bplane;
                const int ksteps = min(TC_BK / 8, (K - s * TC_BK) / 8);
                for (int j = 0; j < ksteps; ++j) {
                    const uint32_t o = 32u * j;   // 8 FP32 along the 128-byte row
                    tc_mma_tf32(tmem, smem_desc_sw128(a_lo + o), smem_desc_sw128(b_hi + o), idesc,
                                (s > 0 || j > 0) ? 1u : 0u);
                    tc_mma_tf32(tmem, smem_desc_sw128(a_hi + o), smem_desc_sw128(b_lo + o), idesc, 1u);
                    tc_mma_tf32(tmem, smem_desc_sw128(a_hi + o), smem_desc_sw128(b_hi + o), idesc, 1u);
                }
                tc_commit(&empty[st]);
                n_consumed = s + 1;
            }
            tc_commit(&done);   // arrives once every MMA issued above has completed
        }
    } else {
        // warps 0-3: the rows past the last full tile (FP32, while the MMAs run), then the epilogue
        float eacc[2][TC_EDGE];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < TC_EDGE; ++r) eacc[q][r] = 0.f;
        if (do_edge) {
            for (int s = 0; s < nchunk; ++s) {
                const int st = s % nst, it = s / nst;
                bool bad = !wait_bounded(&full[st], (uint32_t)it & 1u);
                if (bad) {
                    atomicOr(P.status, SVH_STATUS_MMA_TIMEOUT);
                    *abort_v = 1;
                }
                if (named_bar_or(2, 128, bad || *abort_v != 0)) break;
                const uint8_t* bhi = sm + st * sb + 2 * TC_A_TILE;
                const uint8_t* blo = bhi + bplane;
                const uint8_t* ehi = bhi + 2 * bplane;
                const uint8_t* elo = ehi + TC_E_TILE;
                const int nq = min(TC_BK, K - s * TC_BK) / 4;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = tid + 128 * q;
                    if (c >= nw) continue;
                    for (int j = 0; j < nq; ++j) {
                        // 16-byte chunk j of row c sits at chunk j ^ (c % 8) (128-byte swizzle)
                        const int off = c * 128 + ((j ^ (c & 7)) << 4);
                        const float4 h = *reinterpret_cast<const float4*>(bhi + off);
                        const float4 l = *reinterpret_cast<const float4*>(blo + off);
#pragma unroll
                        for (int r = 0; r < TC_EDGE; ++r)
                            if (r < edge_rows) {
                                const int eo = r * 128 + ((j ^ r) << 4);
                                const float4 ah = *reinterpret_cast<const float4*>(ehi + eo);
                                const float4 al = *reinterpret_cast<const float4*>(elo + eo);
                                eacc[q][r] = fmaf(ah.x + al.x, h.x + l.x, eacc[q][r]);
                                eacc[q][r] = fmaf(ah.y + al.y, h.y + l.y, eacc[q][r]);
                                eacc[q][r] = fmaf(ah.z + al.z, h.z + l.z, eacc[q][r]);
                                eacc[q][r] = fmaf(ah.w + al.w, h.w + l.w, eacc[q][r]);
                            }
                    }
                }
                named_bar(2, 128);   // all four warps are done with this stage
                if (tid == 0) mbar_arrive(&empty[st]);
            }
        }
        if (!wait_bounded(&done, 0u)) {
            atomicOr(P.status, SVH_STATUS_MMA_TIMEOUT);
            *abort_v = 1;
        }
        const bool ab = __any_sync(0xffffffffu, *abort_v != 0);
        const int srow = ntw + 1;   // odd row stride: the column writes below hit distinct banks
        float* stile = reinterpret_cast<float*>(sm);   // the ring is idle once every MMA has completed
        if (!ab) {
            tc_fence_after();
            const int row = 32 * warp + lane;
            for (int jc = 0; jc < nmma / 16; ++jc) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * jc), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) stile[row * srow + 16 * jc + i] = v[i];
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
        if (!*abort_v) {
            const int64_t ldc = P.ldc[u], c_lo = P.c_lo[u];
            float* C = P.C[u];
            for (int r = warp; r < mw; r += 4) {
                float* crow = C + (int64_t)(m0 + r) * ldc;
                for (int c = lane; c < nw; c += 32) store_out(crow + col_off[c], c_lo, stile[r * srow + c]);
            }
            if (do_edge)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = tid + 128 * q;
                    if (c >= nw) continue;
#pragma unroll
                    for (int r = 0; r < TC_EDGE; ++r)
                        if (r < edge_rows)
                            store_out(C + (int64_t)(mfull * TC_BM + r) * ldc + col_off[c], c_lo, eacc[q][r]);
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_v && tid == 128) {   // drain the loads still in flight (bounded)
        for (int s = n_consumed; s < n_issued; ++s) wait_bounded(&full[s % nst], (uint32_t)(s / nst) & 1u);
    }
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host side
static inline float tf32_rna_host(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}

// planes [2][rows][Kp] (hi, lo) of an FP64 matrix [rows][K], zero-padded to Kp
static std::vector<float> split_planes(const double* X, int rows, int K, int Kp) {
    std::vector<float> out((size_t)2 * rows * Kp, 0.f);
    const size_t plane = (size_t)rows * Kp;
    for (int i = 0; i < rows; ++i)
        for (int k = 0; k < K; ++k) {
            const float x = (float)X[(size_t)i * K + k];
            const float h = tf32_rna_host(x);
            out[(size_t)i * Kp + k] = h;
            out[plane + (size_t)i * Kp + k] = tf32_rna_host(x - h);
        }
    return out;
}

// core x_3 G (Eq. 11, mode 3, FP64) for a [P][d3] matrix G, rows (p, b) padded to d2p
static std::vector<double> fold_mode3(const Tucker& t, const double* G, int P, int d2p) {
    const int d1 = t.d[0], d2 = t.d[1], d3 = t.d[2];
    std::vector<double> cp((size_t)P * d2p * d1, 0.0);
    for (int p = 0; p < P; ++p)
        for (int c = 0; c < d3; ++c) {
            const double w = G[(size_t)p * d3 + c];
            for (int b = 0; b < d2; ++b) {
                const double* src = t.core.data() + ((size_t)c * d2 + b) * d1;
                double* dst = cp.data() + ((size_t)p * d2p + b) * d1;
                for (int a = 0; a < d1; ++a) dst[a] += w * src[a];
            }
        }
    return cp;
}

int upload_tucker_device(Handle* h, int u) {
    const Tucker& t = h->tk[u];
    const int d1 = t.d[0], d2 = t.d[1], d3 = t.d[2];
    const int d1p = pad8(d1), d2p = pad8(d2);
    const int Hx = h->Hx, Hy = h->Hy, Hz = h->Hz;
    // core' = core x_3 F3: the restore of the octant spectra
    const std::vector<double> cp = fold_mode3(t, t.F[2].data(), Hz, d2p);
    const std::vector<float> core_s = split_planes(cp.data(), Hz * d2p, d1, d1p);
    const std::vector<float> f1_s = split_planes(t.F[0].data(), Hx, d1, d1p);
    const std::vector<float> f2_s = split_planes(t.F[1].data(), Hy, d2, d2p);
    int rc = dev_upload(h, h->d_tk_core[u], core_s.data(), core_s.size() * sizeof(float));
    if (!rc) rc = dev_upload(h, h->d_tk_F[u][0], f1_s.data(), f1_s.size() * sizeof(float));
    if (!rc) rc = dev_upload(h, h->d_tk_F[u][1], f2_s.data(), f2_s.size() * sizeof(float));
    // core x_3 (W_u F3): the restore straight to the z-space kernels r_u(dz), dz < D (the
    // cosine weights for the z-even kernels, the sine weights for S_z)
    const int D = zk_planes(h);
    if (!rc && D >= 1 && D <= Hz) {
        std::vector<double> w;
        zk_weights(h->Pz, Hz, D, w);
        const double* Wu = w.data() + (u == 3 ? (size_t)D * Hz : 0);
        std::vector<double> G((size_t)D * d3, 0.0);
        for (int d = 0; d < D; ++d)
            for (int c = 0; c < d3; ++c) {
                double acc = 0;
                for (int az = 0; az < Hz; ++az) acc += Wu[(size_t)d * Hz + az] * t.F[2][(size_t)az * d3 + c];
                G[(size_t)d * d3 + c] = acc;
            }
        const std::vector<double> cz = fold_mode3(t, G.data(), D, d2p);
        const std::vector<float> cz_s = split_planes(cz.data(), D * d2p, d1, d1p);
        rc = dev_upload(h, h->d_tk_core_zk[u], cz_s.data(), cz_s.size() * sizeof(float));
        h->tk_zk_D = D;
    }
    return rc;
}

// tile width: columns split evenly into ceil(N / TC_MAXN) tiles, rounded up to 16
static int tile_width(int N) {
    const int nt = (N + TC_MAXN - 1) / TC_MAXN;
    return std::min(TC_MAXN, ((N + nt - 1) / nt + 15) & ~15);
}

// TMA view {K, rows, 2} of split planes, box {32, box_rows, 1}, 128-byte swizzle
static bool plane_map(CUtensorMap* m, const float* base, int K, int rows, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, 2};
    const cuuint64_t strides[2] = {(cuuint64_t)K * sizeof(float), (cuuint64_t)K * rows * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static void add_problem(TcStage& S, int i, const float* A, int rowsA, const float* B, int rowsB, int K, float* C,
                        int64_t ldc, int g, int64_t s1, int64_t s2, int64_t c_lo, bool& ok) {
    const int ntw = tile_width(rowsB);
    ok = ok && plane_map(&S.mapA[i], A, K, rowsA, TC_BM) && plane_map(&S.mapB[i], B, K, rowsB, ntw) &&
         plane_map(&S.mapE[i], A, K, rowsA, TC_EDGE);
    S.A[i] = A;
    S.B[i] = B;
    S.C[i] = C;
    S.a_plane[i] = (int64_t)rowsA * K;
    S.b_plane[i] = (int64_t)rowsB * K;
    S.ldc[i] = ldc;
    S.s1[i] = s1;
    S.s2[i] = s2;
    S.c_lo[i] = c_lo;
    S.M[i] = rowsA;
    S.N[i] = rowsB;
    S.K[i] = K;
    S.ntw[i] = ntw;
    S.g[i] = g;
}

static void launch_stage(const TcStage& S, int n, cudaStream_t strm) {
    if (n == 0) return;
    int nt = 0, mt = 0;
    for (int i = 0; i < n; ++i) {
        nt = std::max(nt, (S.N[i] + S.ntw[i] - 1) / S.ntw[i]);
        const int mrem = S.M[i] % TC_BM;
        mt = std::max(mt, std::max(1, S.M[i] / TC_BM + (mrem > TC_EDGE ? 1 : 0)));
    }
    k_tc_restore<<<dim3(nt, mt, n), TC_THREADS, TC_SMEM, strm>>>(S);
}

// the two launch descriptors, kept in the handle's host buffer at a 64-byte boundary
static TcStage* stages_of(Handle* h) {
    const uintptr_t p = reinterpret_cast<uintptr_t>(h->tk_probs.data());
    return reinterpret_cast<TcStage*>((p + 63) & ~uintptr_t(63));
}

int launch_tucker_rebuild(Handle* h, cudaStream_t strm, bool to_zk) {
    const int Hx = h->Hx, Hy = h->Hy, Hz = h->Hz;
    // planes of the restored octant: Hz spectra planes, or D z-offsets of the z-space kernels
    const int NP = to_zk ? h->zk_D : Hz;
    if (to_zk && (NP < 1 || NP > Hz || h->tk_zk_D != NP || !h->d_zk32.p))
        return set_err(h, SVH_ERR_STATE, "Tucker restore: no z-space form of the Tucker data for these planes");
    float* out = static_cast<float*>(to_zk ? h->d_zk32.p : h->d_spec32.p);
    const int64_t Ht = (int64_t)Hx * Hy * NP;
    size_t n1 = 0;
    for (int u = 0; u < 7; ++u)
        if (h->tucker_on[u]) n1 += (size_t)2 * Hz * Hx * pad8(h->tk[u].d[1]);
    if (n1 == 0) return SVH_OK;
    bool fresh = false;
    if (h->d_tk_w1.bytes < n1 * 4) {
        int rc = dev_alloc(h, h->d_tk_w1, n1 * 4);
        if (rc) return rc;
        fresh = true;
    }
    if (fresh || h->tk_probs_version != h->tk_version || h->tk_probs_target != (int)to_zk) {
        float* w1 = static_cast<float*>(h->d_tk_w1.p);
        h->tk_probs.assign(2 * sizeof(TcStage) + 64, 0);   // tensor maps want 64-byte alignment
        TcStage* st = stages_of(h);
        bool ok = true;
        int n = 0;
        size_t o1 = 0;
        for (int u = 0; u < 7; ++u) {
            if (!h->tucker_on[u]) continue;
            const int d1p = pad8(h->tk[u].d[0]), d2p = pad8(h->tk[u].d[1]);
            const float* core = static_cast<const float*>((to_zk ? h->d_tk_core_zk[u] : h->d_tk_core[u]).p);
            const float* F1 = static_cast<const float*>(h->d_tk_F[u][0].p);
            const float* F2 = static_cast<const float*>(h->d_tk_F[u][1].p);
            float* W1 = w1 + o1;
            const int64_t w1_plane = (int64_t)NP * Hx * d2p;
            o1 += (size_t)2 * Hz * Hx * d2p;
            // stage 1: D[kx][(kz, b)] -> W1[kz][kx][b] (split: stage 2 reads it as TF32 planes)
            add_problem(st[0], n, F1, Hx, core, NP * d2p, d1p, W1, d2p, d2p, (int64_t)Hx * d2p, 1, w1_plane, ok);
            // stage 2: D[ky][(kz, kx)] -> out[kz][ky][kx]
            add_problem(st[1], n, F2, Hy, W1, NP * Hx, d2p, out + u * Ht, Hx, Hx, (int64_t)Hy * Hx, 1, 0, ok);
            ++n;
        }
        if (!ok) return set_err(h, SVH_ERR_CUDA, "Tucker restore: TMA descriptor encoding failed");
        st[0].status = st[1].status = static_cast<int*>(h->d_status.p);
        h->tk_probs_split[0] = h->tk_probs_split[1] = n;
        h->tk_probs_split[2] = 0;
        SVH_CUDA_TRY(h, cudaFuncSetAttribute(k_tc_restore, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        h->tk_probs_version = h->tk_version;
        h->tk_probs_target = (int)to_zk;
    }
    const TcStage* st = stages_of(h);
    launch_stage(st[0], h->tk_probs_split[0], strm);
    launch_stage(st[1], h->tk_probs_split[1], strm);
    SVH_CUDA_TRY(h, cudaGetLastError());
    if (to_zk) {
        h->zk_version = -2;   // the z-space kernels now come from the Tucker data, not the spectra
    } else {
        ++h->spec_version;
        h->spec32_tk_version = h->tk_version;
    }
    return SVH_OK;
}

}  // namespace svh
