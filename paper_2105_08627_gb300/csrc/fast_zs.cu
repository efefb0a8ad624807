// fast_zs.cu -- the FFT z pass with each pencil split over two threads
// (FP32; a tile variant of pass 3 for the long z sizes, Pz = 32 and 48).
//
// Same arithmetic as k_zpass_half (z-FFT, 5 x 5 block product, inverse
// z-FFT on shifted pencils whose inputs and kept outputs lie in the lower
// half), with each length-Pz transform split in two by decimation in time:
// with H = Pz / 2 and W = exp(-2 pi i / Pz),
//   X[k] = E[k] + W^k O[k],  X[k + H] = E[k] - W^k O[k]     (k < H)
// where E, O are the length-H DFTs of the even and odd samples, and for the
// inverse, split by output parity,
//   x[2m] = IDFT_H(Y[k] + Y[k + H])[m],  x[2m + 1] = IDFT_H((Y[k] - Y[k + H]) W^-k)[m].
// Thread (basis, parity, column) transforms its half (pruned: the inputs and
// the kept outputs are the first half of each length-H line); the block
// product task for (k, column) combines E and W^k O of all 5 bases into the
// pair X[k], X[k + H], multiplies both and writes back the sum and the
// twiddled difference. Half the registers of the one-thread form at Pz = 48,
// so twice the warps fit an SM.
#include <cuda_runtime.h>

#include "fastpass.cuh"

namespace svh {

bool z_split_ok(int Pz, int nza, int zcontig) { return (Pz == 32 || Pz == 48) && zcontig && 2 * nza <= Pz; }

template <int PZ>
__global__ void __launch_bounds__(320, 2) k_zpass_split(const __grid_constant__ PassArgs a) {
    using C = float2;
    constexpr int H = PZ / 2, Q = H / 2, TS = 96 / PZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C(*buf)[2][H][32] = reinterpret_cast<C(*)[2][H][32]>(smem_raw);   // [5][parity][k][column]
    float(*sp)[PZ][32] = reinterpret_cast<float(*)[PZ][32]>(smem_raw + sizeof(C) * 5 * 2 * H * 32);
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int al = wp >> 1, par = wp & 1;
    const int kx0 = blockIdx.x * 32, ky = blockIdx.y, kx = kx0 + lane;
    const bool ok = kx < a.Px;
    load_tile_spectra<float, PZ>(a, sp, kx0, ky);
    C* B2 = static_cast<C*>(a.B2);
    const int64_t plane = (int64_t)a.Py * a.Px;
    const int nza = a.nza;
    C pre[Q];
    auto fetch = [&](int b) {
        const int64_t base = ((int64_t)(b * 5 + al) * nza * a.Py + ky) * a.Px + kx;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const int zi = 2 * m + par;
            C z;
            z.x = 0;
            z.y = 0;
            if (ok && zi < nza) z = B2[base + zi * plane];
            pre[m] = z;
        }
    };
    fetch(0);
    for (int b = 0; b < a.nb; ++b) {
        {
            C v[H];
            reg_fft_lowin<H, false>(pre, v);
            if (b + 1 < a.nb) fetch(b + 1);
#pragma unroll
            for (int k = 0; k < H; ++k) buf[al][par][k][lane] = (par && k) ? cmul(v[k], w96<C>(k * TS)) : v[k];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < H * 32; task += 320) {
            const int k = task >> 5, ln = task & 31;
            C lo[5], hi[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const C e = buf[q][0][k][ln], o = buf[q][1][k][ln];
                lo[q] = cadd(e, o);
                hi[q] = csub(e, o);
            }
            block_multiply5<float>(lo, sp[0][k][ln], sp[1][k][ln], sp[2][k][ln], sp[3][k][ln], sp[4][k][ln],
                                   sp[5][k][ln], sp[6][k][ln]);
            block_multiply5<float>(hi, sp[0][k + H][ln], sp[1][k + H][ln], sp[2][k + H][ln], sp[3][k + H][ln],
                                   sp[4][k + H][ln], sp[5][k + H][ln], sp[6][k + H][ln]);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                buf[q][0][k][ln] = cadd(lo[q], hi[q]);
                const C d = csub(lo[q], hi[q]);
                buf[q][1][k][ln] = k ? cmulc(d, w96<C>(k * TS)) : d;
            }
        }
        __syncthreads();
        // each thread reads back only its own (basis, parity, column) line, which it alone writes
        // in the next item's forward step: no further barrier is needed
        C v[H], w[Q];
#pragma unroll
        for (int k = 0; k < H; ++k) v[k] = buf[al][par][k][lane];
        reg_fft_lowout<H, true>(v, w);
        if (ok) {
            const int64_t base = ((int64_t)(b * 5 + al) * nza * a.Py + ky) * a.Px + kx;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const int zi = 2 * m + par;
                if (zi < nza) B2[base + zi * plane] = w[m];
            }
        }
    }
}

// Variants 5 and 6: the same split-pencil transform on tiles of TC kx columns (TC = 16: blocks
// of 160 threads, 44 KB of shared memory), with the tile's octant spectra packed per frequency
// point as two float4 (G00, Sx, Sy, Sz | Qx, Qy, Qz, 0): two 16-byte shared loads per point
// instead of seven.
// PREF: the next item's inputs are loaded into registers while the current item is transformed
// (4 blocks per SM); without it the loads come right before each item's transform and the
// register budget allows 5 blocks per SM (variant 6), whose other warps cover the latency.
template <int PZ, int TC, bool PREF>
__global__ void __launch_bounds__(10 * TC, PREF ? 4 : 5) k_zpass_split4(const __grid_constant__ PassArgs a) {
    using C = float2;
    constexpr int NT = 10 * TC, H = PZ / 2, Q = H / 2, TS = 96 / PZ, NH = PZ / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C(*buf)[2][H][TC] = reinterpret_cast<C(*)[2][H][TC]>(smem_raw);   // [5][parity][k][column]
    // octant spectra of the tile, az = 0 .. PZ / 2: frequency kz reads az = min(kz, PZ - kz), with
    // S_z negated for kz > PZ / 2 (at kz = PZ / 2 itself the odd S_z spectrum vanishes)
    float4(*sp)[NH][TC] = reinterpret_cast<float4(*)[NH][TC]>(smem_raw + sizeof(C) * 5 * 2 * H * TC);  // [2][az][col]
    const int q = threadIdx.x / TC, lane = threadIdx.x % TC;
    const int al = q >> 1, par = q & 1;
    const int kx0 = blockIdx.x * TC, ky = blockIdx.y, kx = kx0 + lane;
    const bool ok = kx < a.Px;
    {
        // spectra of the tile with the odd-kernel signs folded in (Sx by column, Sy by row, Sz by
        // the upper half of kz); each octant value is loaded once
        const float* spec = static_cast<const float*>(a.spec);
        const int64_t plane = (int64_t)a.Hx * a.Hy, Sk = plane * a.Hz;
        const int ay = min(ky, a.Py - ky);
        const float sgy = (2 * ky <= a.Py) ? 1.f : -1.f;
        float* spf = reinterpret_cast<float*>(sp);
        for (int task = threadIdx.x; task < 7 * TC; task += NT) {
            const int u = task / TC, ln = task % TC;
            const int kxx = min(kx0 + ln, a.Px - 1);
            const int ax = min(kxx, a.Px - kxx);
            const float sgx = (2 * kxx <= a.Px) ? 1.f : -1.f;
            const float sg = u == 1 ? sgx : (u == 2 ? sgy : 1.f);
            const int64_t off = (int64_t)ay * a.Hx + ax;
            const int half = u / 4, comp = u % 4;
            float val[NH];
#pragma unroll
            for (int az = 0; az < NH; ++az) val[az] = __ldg(spec + u * Sk + az * plane + off);
#pragma unroll
            for (int az = 0; az < NH; ++az) spf[((half * NH + az) * TC + ln) * 4 + comp] = sg * val[az];
        }
        for (int i = threadIdx.x; i < NH * TC; i += NT) spf[((NH + i / TC) * TC + i % TC) * 4 + 3] = 0.f;
    }
    C* B2 = static_cast<C*>(a.B2);
    const int64_t plane = (int64_t)a.Py * a.Px;
    const int nza = a.nza;
    C pre[Q];
    auto fetch = [&](int b) {
        const int64_t base = ((int64_t)(b * 5 + al) * nza * a.Py + ky) * a.Px + kx;
#pragma unroll
        for (int m = 0; m < Q; ++m) {
            const int zi = 2 * m + par;
            C z;
            z.x = 0;
            z.y = 0;
            if (ok && zi < nza) z = B2[base + zi * plane];
            pre[m] = z;
        }
    };
    if (PREF) fetch(0);
    for (int b = 0; b < a.nb; ++b) {
        {
            C v[H];
            if (!PREF) fetch(b);
            reg_fft_lowin<H, false>(pre, v);
            if (PREF && b + 1 < a.nb) fetch(b + 1);
            // a thread writes only its own (basis, parity, column) line here, which after the
            // previous item's second barrier only it reads: no barrier is needed before this (the
            // odd line's twiddles W^k are applied by the block-product tasks)
#pragma unroll
            for (int k = 0; k < H; ++k) buf[al][par][k][lane] = v[k];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < H * TC; task += NT) {
            const int k = task / TC, ln = task % TC;
            const C w = w96<C>(k * TS);   // W^k of the odd-sample half (1 at k = 0)
            C lo[5], hi[5];
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                const C e = buf[p][0][k][ln], o = cmul(buf[p][1][k][ln], w);
                lo[p] = cadd(e, o);
                hi[p] = csub(e, o);
            }
            // k reads az = k; k + H (> PZ / 2 for k > 0) reads az = H - k with S_z negated
            const float4 l0 = sp[0][k][ln], l1 = sp[1][k][ln], h0 = sp[0][H - k][ln], h1 = sp[1][H - k][ln];
            block_multiply5_fma(lo, l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z);
            block_multiply5_fma(hi, h0.x, h0.y, h0.z, -h0.w, h1.x, h1.y, h1.z);
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                buf[p][0][k][ln] = cadd(lo[p], hi[p]);
                const C d = csub(lo[p], hi[p]);
                buf[p][1][k][ln] = k ? cmulc(d, w96<C>(k * TS)) : d;
            }
        }
        __syncthreads();
        C v[H], w[Q];
#pragma unroll
        for (int k = 0; k < H; ++k) v[k] = buf[al][par][k][lane];
        reg_fft_lowout<H, true>(v, w);
        if (ok) {
            const int64_t base = ((int64_t)(b * 5 + al) * nza * a.Py + ky) * a.Px + kx;
#pragma unroll
            for (int m = 0; m < Q; ++m) {
                const int zi = 2 * m + par;
                if (zi < nza) B2[base + zi * plane] = w[m];
            }
        }
    }
}

template <int PZ, int TC, bool PREF>
static void run_zsplit4(const PassArgs& a, cudaStream_t s) {
    const size_t sm = (size_t)5 * PZ * TC * sizeof(float2) + (size_t)2 * (PZ / 2 + 1) * TC * sizeof(float4);
    cudaFuncSetAttribute(k_zpass_split4<PZ, TC, PREF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_zpass_split4<PZ, TC, PREF><<<dim3((unsigned)((a.Px + TC - 1) / TC), (unsigned)a.Py), 10 * TC, sm, s>>>(a);
}

bool launch_z_split16(const PassArgs& a, cudaStream_t s, bool prefetch) {
    if (!z_split_ok(a.Pz, a.nza, a.zcontig)) return false;
    if (a.Pz == 32) prefetch ? run_zsplit4<32, 16, true>(a, s) : run_zsplit4<32, 16, false>(a, s);
    else prefetch ? run_zsplit4<48, 16, true>(a, s) : run_zsplit4<48, 16, false>(a, s);
    return true;
}

template <int PZ>
static void run_zsplit(const PassArgs& a, cudaStream_t s) {
    const size_t sm = (size_t)5 * PZ * 32 * sizeof(float2) + (size_t)7 * PZ * 32 * sizeof(float);
    cudaFuncSetAttribute(k_zpass_split<PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_zpass_split<PZ><<<dim3((unsigned)((a.Px + 31) / 32), (unsigned)a.Py), 320, sm, s>>>(a);
}

bool launch_z_split(const PassArgs& a, cudaStream_t s) {
    if (!z_split_ok(a.Pz, a.nza, a.zcontig)) return false;
    if (a.Pz == 32) run_zsplit<32>(a, s);
    else run_zsplit<48>(a, s);
    return true;
}

}  // namespace svh
