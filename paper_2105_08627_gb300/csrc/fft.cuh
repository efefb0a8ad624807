// fft.cuh -- batched mixed-radix FFTs in shared memory (device side).
//
// The 3-D transforms of Eq. 9 are split into 1-D passes; each pass stages a
// tile of lines in shared memory and runs a Stockham auto-sort FFT over it.
// Stage s with radix R (Ns = product of the earlier radices) reads, for each
// butterfly j in [0, N/R), the R inputs data[j + r N/R], multiplies them by
// w^(r m) with m = (j mod Ns) * N/(Ns R), takes a length-R DFT and writes
// the results to data[(j div Ns) Ns R + (j mod Ns) + r Ns]. A stage holds its
// inputs in registers between a read phase and a write phase separated by a
// barrier, so one shared buffer serves in place.
//
// Two line layouts: ROWS (element n of line l at buf[l*ld + n]) for lines that
// are contiguous in HBM, COLS (buf[n*ld + l]) for lines strided in HBM whose
// batch index is contiguous. Tasks are mapped so that a warp touches
// consecutive shared-memory words in both layouts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_plan.h"

namespace svh {

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmk(double x, double y) { C c; c.x = x; c.y = y; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { C c; c.x = a.x * s; c.y = a.y * s; return c; }
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
    C c;
    if (INV) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
    return c;
}

// FP32 complex add, subtract and real scale as packed two-lane FP32 instructions
// (add/sub/mul.rn.f32x2, sm_100 and later): one instruction per complex operation instead of
// two, with the same round-to-nearest result in each lane. SVH_F32X2=0 keeps the scalar forms.
#ifndef SVH_F32X2
#define SVH_F32X2 1
#endif
#if SVH_F32X2
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(d);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(d);
}
template <> __device__ __forceinline__ float2 cscale<float2, float>(float2 a, float s) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(make_float2(s, s))));
    return f2_unpack(d);
}
#endif

// ---------------------------------------------------------------- small DFTs
// Forward: V[k] = sum_r v[r] exp(-2 pi i r k / R); inverse uses +i.
template <typename C, bool INV> __device__ __forceinline__ void dft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
    C t3 = mul_mi<C, INV>(csub(v1, v3));
    v0 = cadd(t0, t2); v2 = csub(t0, t2); v1 = cadd(t1, t3); v3 = csub(t1, t3);
}

template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
    using T = decltype(v[0].x);
    const T h = (T)0.70710678118654752440;
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    // twiddles w8^k, k = 0..3, with w8 = exp(-+ i pi/4)
    C t1, t2, t3;
    if (!INV) {
        t1.x = h * (o1.x + o1.y); t1.y = h * (o1.y - o1.x);     // (1 - i)/sqrt2
        t2.x = o2.y; t2.y = -o2.x;                              // -i
        t3.x = h * (o3.y - o3.x); t3.y = -h * (o3.x + o3.y);    // (-1 - i)/sqrt2
    } else {
        t1.x = h * (o1.x - o1.y); t1.y = h * (o1.y + o1.x);     // (1 + i)/sqrt2
        t2.x = -o2.y; t2.y = o2.x;                              // +i
        t3.x = -h * (o3.x + o3.y); t3.y = h * (o3.x - o3.y);    // (-1 + i)/sqrt2
    }
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

template <typename C, bool INV> __device__ __forceinline__ void dft3(C* v) {
    using T = decltype(v[0].x);
    const T s3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
    C s = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m; m.x = v[0].x - (T)0.5 * s.x; m.y = v[0].y - (T)0.5 * s.y;
    C r = mul_mi<C, INV>(cscale(d, s3));     // -+ i sin(2pi/3) (v1 - v2)
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

// generic odd radix (5, 7) by pairing conjugate-symmetric terms
template <typename C, bool INV, int R> __device__ __forceinline__ void dft_odd(C* v) {
    using T = decltype(v[0].x);
    constexpr int H = (R - 1) / 2;
    // cos/sin(2 pi k / R), k = 1..H
    T cs[H], sn[H];
    if (R == 5) {
        cs[0] = (T)0.30901699437494742410; sn[0] = (T)0.95105651629515357212;
        cs[1] = (T)-0.80901699437494742410; sn[1] = (T)0.58778525229247312917;
    } else {  // R == 7
        cs[0] = (T)0.62348980185873353053; sn[0] = (T)0.78183148246802980871;
        cs[1] = (T)-0.22252093395631440429; sn[1] = (T)0.97492791218182360702;
        cs[2] = (T)-0.90096886790241912624; sn[2] = (T)0.43388373911755812048;
    }
    C a[H], b[H];
#pragma unroll
    for (int k = 1; k <= H; ++k) { a[k - 1] = cadd(v[k], v[R - k]); b[k - 1] = csub(v[k], v[R - k]); }
    C out[R];
    C s0 = v[0];
#pragma unroll
    for (int k = 0; k < H; ++k) s0 = cadd(s0, a[k]);
    out[0] = s0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        C re = v[0];
        C im; im.x = 0; im.y = 0;
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            int idx = (r * k) % R;          // angle index of w^(r k)
            T c, s;
            if (idx <= H) { c = cs[idx - 1]; s = sn[idx - 1]; }
            else { c = cs[R - idx - 1]; s = -sn[R - idx - 1]; }
            re.x += c * a[r - 1].x; re.y += c * a[r - 1].y;
            im.x += s * b[r - 1].x; im.y += s * b[r - 1].y;
        }
        // forward: V[k] = re - i*im, V[R-k] = re + i*im (inverse: signs swap)
        C t = mul_mi<C, INV>(im);
        out[k] = cadd(re, t);
        out[R - k] = csub(re, t);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename C, bool INV, int R> __device__ __forceinline__ void dft(C* v) {
    if constexpr (R == 2) dft2<C, INV>(v);
    else if constexpr (R == 3) dft3<C, INV>(v);
    else if constexpr (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<C, INV>(v);
    else dft_odd<C, INV, R>(v);
}

// ---------------------------------------------------------------- one Stockham stage
enum { ROWS = 0, COLS = 1 };

template <typename C, int R, bool INV, int MAXB, int LAYOUT>
__device__ __forceinline__ void fft_stage(C* buf, int N, int Ns, int nlines, int ld,
                                          const C* tw, int tid, int nthr) {
    const int NR = N / R;
    const int ntask = nlines * NR;
    const int tstride = N / (Ns * R);
    C v[MAXB][R];
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        int task = tid + i * nthr;
        if (task < ntask) {
            int l, j;
            if (LAYOUT == ROWS) { l = task / NR; j = task - l * NR; }
            else { j = task / nlines; l = task - j * nlines; }
            int m = (j % Ns) * tstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int n = j + r * NR;
                C x = (LAYOUT == ROWS) ? buf[l * ld + n] : buf[n * ld + l];
                if (r > 0) {
                    C w = tw[m * r];
                    x = INV ? cmulc(x, w) : cmul(x, w);
                }
                v[i][r] = x;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        int task = tid + i * nthr;
        if (task < ntask) {
            int l, j;
            if (LAYOUT == ROWS) { l = task / NR; j = task - l * NR; }
            else { j = task / nlines; l = task - j * nlines; }
            dft<C, INV, R>(v[i]);
            int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int n = base + r * Ns;
                if (LAYOUT == ROWS) buf[l * ld + n] = v[i][r];
                else buf[n * ld + l] = v[i][r];
            }
        }
    }
    __syncthreads();
}

// Full transform of nlines lines of length p.N held in `buf`; `tw` holds
// exp(-2 pi i m / N), m = 0..N-1 (the inverse uses its conjugate).
// Requires nlines * N <= MAXPTS * nthr. Ends with a barrier.
template <typename C, bool INV, int MAXPTS, int LAYOUT>
__device__ __forceinline__ void fft_run(C* buf, const FftPlan& p, int nlines, int ld, const C* tw, int tid, int nthr) {
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.R[s];
        switch (R) {
            case 8: fft_stage<C, 8, INV, (MAXPTS + 7) / 8, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            case 4: fft_stage<C, 4, INV, (MAXPTS + 3) / 4, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            case 2: fft_stage<C, 2, INV, (MAXPTS + 1) / 2, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            case 3: fft_stage<C, 3, INV, (MAXPTS + 2) / 3, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            case 5: fft_stage<C, 5, INV, (MAXPTS + 4) / 5, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            case 7: fft_stage<C, 7, INV, (MAXPTS + 6) / 7, LAYOUT>(buf, p.N, Ns, nlines, ld, tw, tid, nthr); break;
            default: break;
        }
        Ns *= R;
    }
}

}  // namespace svh
