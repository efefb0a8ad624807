// batch_persist.cu -- one persistent launch for the operator products (Eq. 7, 9) of a whole
// batch of independent, unevenly sized structures, each with its own right-hand sides
// (ports x frequencies).
//
// The work of every structure i is cut into tiles of six phases:
//   0 x-forward (gather from the voxel list, FFT along x)     -> B1_i
//   1 node rows y_m = (A I)_m                                   (no dependency)
//   2 y-forward (FFT along y)                          B1_i    -> B2_i   after phase 0 of i
//   3 z pass (z-FFT, 5 x 5 block product, inverse)     B2_i in place     after phase 2 of i
//   4 y-inverse, keep y < Ky                           B2_i    -> B1_i   after phase 3 of i
//   5 x-inverse, keep x < Kx, diagonal and A^T epilogue B1_i   -> y_i    after phase 4 of i
// A device queue lists the tiles phase by phase (all phase-0 tiles of all structures, then
// all phase-1 tiles, ...; within a phase the largest structures first). Every CTA of the
// persistent grid takes the next tile index from an atomic counter, waits until the phase its
// tile depends on is complete for that structure (a per-structure, per-phase completion count),
// runs the tile and adds one to its own count. A dependency always lies earlier in the queue,
// so it was taken by a CTA that is running or has finished, whatever the grid size: the queue
// cannot deadlock. Every wait is bounded in time (globaltimer); on expiry the CTA sets bit
// SVH_STATUS_QUEUE_TIMEOUT of the batch's status word and leaves the queue, so the launch
// always ends and the host reports SVH_ERR_TIMEOUT.
//
// The tile bodies are the generic mixed-radix passes (runtime FFT plans, one shared-memory
// budget for every size), so one kernel serves every grid of the batch. Intermediate grids
// written by other CTAs during the launch are read with ld.global.cg (L2, never a stale L1 line).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "batch_persist.h"
#include "fft.cuh"

namespace svh {

namespace {

constexpr int QT = 256;   // threads per CTA of the persistent kernel

template <typename T> struct QCfg;
// points per thread of one tile (8 FP32 / 4 FP64 complex): the shared FFT code then fits
// 128 registers, two CTAs per SM
template <> struct QCfg<float> { static constexpr int MAXPTS = 8; };
template <> struct QCfg<double> { static constexpr int MAXPTS = 4; };

__constant__ float c_qflux[5][6] = {
    {-1.f, 1.f, 0.f, 0.f, 0.f, 0.f},
    {0.f, 0.f, -1.f, 1.f, 0.f, 0.f},
    {0.f, 0.f, 0.f, 0.f, -1.f, 1.f},
    {0.5f, 0.5f, -0.5f, -0.5f, 0.f, 0.f},
    {0.5f, 0.5f, 0.5f, 0.5f, -1.f, -1.f},
};

template <typename C> __device__ __forceinline__ C ldcg(const C* p);
template <> __device__ __forceinline__ float2 ldcg<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg<double2>(const double2* p) { return __ldcg(p); }

template <typename C> __device__ __forceinline__ C qzero() { C c; c.x = 0; c.y = 0; return c; }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename C>
__device__ __forceinline__ void load_tw(C* s, const void* g, int N) {
    const C* t = static_cast<const C*>(g);
    for (int i = threadIdx.x; i < N; i += QT) s[i] = t[i];
}

// ------------------------------------------------------------------ one FFT for every tile
// Forward transforms of `nlines` lines of length p->N held in shared memory, element n of
// line l at buf[l * sl + n * sn] (runtime strides: rows and columns alike), by the Stockham
// stages of fft.cuh. An inverse transform is taken as conj(FFT(conj(x))) by its caller, so
// that the kernel holds a single copy of the FFT code (one register allocation for all
// tiles). lfast: consecutive threads take consecutive lines (column layouts).
template <typename C, int R, int MAXB>
__device__ __forceinline__ void stage_rt(C* buf, int N, int Ns, int nlines, int sl, int sn, bool lfast,
                                         const C* tw) {
    const int NR = N / R;
    const int ntask = nlines * NR;
    const int tstride = N / (Ns * R);
    C v[MAXB][R];
    int lv[MAXB], jv[MAXB];
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int task = threadIdx.x + i * QT;
        lv[i] = 0;
        jv[i] = -1;
        if (task < ntask) {
            const int l = lfast ? task % nlines : task / NR;
            const int j = lfast ? task / nlines : task - l * NR;
            lv[i] = l;
            jv[i] = j;
            const int m = (j % Ns) * tstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = buf[l * sl + (j + r * NR) * sn];
                if (r > 0) x = cmul(x, tw[m * r]);
                v[i][r] = x;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        if (jv[i] >= 0) {
            const int j = jv[i];
            dft<C, false, R>(v[i]);
            const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[lv[i] * sl + (base + r * Ns) * sn] = v[i][r];
        }
    }
    __syncthreads();
}

template <typename C, int MAXPTS>
__device__ __noinline__ void fft_lines(C* buf, const FftPlan* p, int nlines, int sl, int sn, bool lfast,
                                       const C* tw) {
    const int N = p->N, nst = p->nst;
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = p->R[s];
        switch (R) {
            case 8: stage_rt<C, 8, (MAXPTS + 7) / 8>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
            case 4: stage_rt<C, 4, (MAXPTS + 3) / 4>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
            case 2: stage_rt<C, 2, (MAXPTS + 1) / 2>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
            case 3: stage_rt<C, 3, (MAXPTS + 2) / 3>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
            case 5: stage_rt<C, 5, (MAXPTS + 4) / 5>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
            default: stage_rt<C, 7, (MAXPTS + 6) / 7>(buf, N, Ns, nlines, sl, sn, lfast, tw); break;
        }
        Ns *= R;
    }
}

template <typename C> __device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }

// ------------------------------------------------------------------ tiles
// phase 0: lpb x-lines of Px: gather the voxels of active row `rows[ri]`, forward FFT
template <typename T>
__device__ __forceinline__ void tile_xfwd(const BItem& it, int tile, unsigned char* smem) {
    using C = typename CT<T>::type;
    const int N = it.px.N, ld = N + 1;
    C* tw = reinterpret_cast<C*>(smem);
    C* buf = tw + N;
    const int64_t nlines = (int64_t)it.nb * 5 * it.nrows;
    const int64_t line0 = (int64_t)tile * it.lpb;
    const int nl = (int)min((int64_t)it.lpb, nlines - line0);
    const C* x = static_cast<const C*>(it.x);
    load_tw<C>(tw, it.tw[0], N);
    for (int i = threadIdx.x; i < nl * N; i += QT) {
        const int l = i / N, n = i - l * N;
        const int64_t line = line0 + l;
        const int64_t ba = line / it.nrows;
        const int ri = (int)(line - ba * it.nrows);
        C v = qzero<C>();
        if (n < it.Kx) {
            const int vi = __ldg(it.vidx + (int64_t)__ldg(it.rows + ri) * it.Kx + n);
            if (vi >= 0) {
                const int64_t b = ba / 5, a = ba - 5 * b;
                v = x[b * it.Nvec + a * it.K + vi];
            }
        }
        buf[l * ld + n] = v;
    }
    __syncthreads();
    fft_lines<C, QCfg<T>::MAXPTS>(buf, &it.px, nl, ld, 1, false, tw);
    C* B1 = static_cast<C*>(it.B1);
    for (int i = threadIdx.x; i < nl * N; i += QT) {
        const int l = i / N, n = i - l * N;
        const int64_t line = line0 + l;
        const int64_t ba = line / it.nrows;
        const int ri = (int)(line - ba * it.nrows);
        B1[(ba * it.nza * it.Ky + __ldg(it.rows + ri)) * (int64_t)N + n] = buf[l * ld + n];
    }
}

// phase 1: QT (node, item) pairs of the continuity rows (A I)_m
template <typename T>
__device__ __forceinline__ void tile_nodes(const BItem& it, int tile) {
    using C = typename CT<T>::type;
    const int64_t i = (int64_t)tile * QT + threadIdx.x;
    if (i >= it.M * it.nb) return;
    const int64_t b = i / it.M, m = i - b * it.M;
    const C* xb = static_cast<const C*>(it.x) + b * it.Nvec;
    C acc = qzero<C>();
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int code = __ldg(it.ninc + m * 2 + e);
        if (code < 0) continue;
        const int v = code / 6, f = code - 6 * v;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            const float fl = c_qflux[a][f];
            if (fl != 0.f) {
                const C I = xb[a * it.K + v];
                acc.x += (T)fl * I.x;
                acc.y += (T)fl * I.y;
            }
        }
    }
    static_cast<C*>(it.y)[b * it.Nvec + 5 * it.K + m] = acc;
}

// phases 2 / 4: tby kx columns of one (item, basis, plane): FFT along y
template <typename T, bool INV>
__device__ __forceinline__ void tile_y(const BItem& it, int tile, unsigned char* smem) {
    using C = typename CT<T>::type;
    const int Py = it.py.N, Px = it.Px, Ky = it.Ky, tb = it.tby;
    C* tw = reinterpret_cast<C*>(smem);
    C* buf = tw + Py;
    const int nkx = (Px + tb - 1) / tb;
    const int kxt = tile % nkx;
    const int r = tile / nkx;
    const int zi = r % it.nza;
    const int64_t ba = r / it.nza;
    const int kx0 = kxt * tb;
    const int nt = min(tb, Px - kx0);
    const C* in = static_cast<const C*>(INV ? it.B2 : it.B1);
    C* out = static_cast<C*>(INV ? it.B1 : it.B2);
    const int64_t plane_in = (ba * it.nza + zi) * (int64_t)(INV ? Py : Ky);
    const int64_t plane_out = (ba * it.nza + zi) * (int64_t)(INV ? Ky : Py);
    const uint8_t* rm = it.rowmask + (int64_t)zi * Ky;
    load_tw<C>(tw, it.tw[1], Py);
    for (int i = threadIdx.x; i < Py * tb; i += QT) {
        const int n = i / tb, t = i - n * tb;
        C v = qzero<C>();
        if (t < nt) {
            if (INV) v = conjc(ldcg(in + (plane_in + n) * Px + kx0 + t));
            else if (n < Ky && __ldg(rm + n)) v = ldcg(in + (plane_in + n) * Px + kx0 + t);
        }
        buf[i] = v;
    }
    __syncthreads();
    fft_lines<C, QCfg<T>::MAXPTS>(buf, &it.py, tb, 1, tb, true, tw);
    const int nout = INV ? Ky : Py;
    for (int i = threadIdx.x; i < nout * tb; i += QT) {
        const int n = i / tb, t = i - n * tb;
        if (t < nt && (!INV || __ldg(rm + n)))
            out[(plane_out + n) * Px + kx0 + t] = INV ? conjc(buf[n * tb + t]) : buf[n * tb + t];
    }
}

// the 5 x 5 block product of Eq. 9 at one frequency point (spectra of S_a are -i sign R)
template <typename T>
__device__ __forceinline__ void qblock5(typename CT<T>::type* io, T g, T sx, T sy, T sz, T qx, T qy, T qz) {
    using C = typename CT<T>::type;
    auto mi = [](C a) { C c; c.x = a.y; c.y = -a.x; return c; };
    auto pi = [](C a) { C c; c.x = -a.y; c.y = a.x; return c; };
    const C Ix = io[0], Iy = io[1], Iz = io[2], I2 = io[3], I3 = io[4];
    const C Yx = cadd(cscale(Ix, g), cscale(mi(cadd(I2, I3)), sx));
    const C Yy = cadd(cscale(Iy, g), cscale(mi(csub(I3, I2)), sy));
    const C Yz = cadd(cscale(Iz, g), cscale(pi(I3), (T)2 * sz));
    const C pX = pi(Ix), pY = pi(Iy), pZ = pi(Iz);
    const T qs = qx + qy, qd = qx - qy;
    const C Y2 = cadd(cadd(cscale(pX, sx), cscale(pY, -sy)), cadd(cscale(I2, qs), cscale(I3, qd)));
    const C Y3 = cadd(cadd(cscale(pX, sx), cscale(pY, sy)),
                      cadd(cscale(pZ, (T)-2 * sz), cadd(cscale(I2, qd), cscale(I3, qs + (T)4 * qz))));
    io[0] = Yx; io[1] = Yy; io[2] = Yz; io[3] = Y2; io[4] = Y3;
}

// phase 3: tbz kx columns of one (item, ky): the 5 basis pencils along z
template <typename T>
__device__ __forceinline__ void tile_z(const BItem& it, int tile, unsigned char* smem) {
    using C = typename CT<T>::type;
    const int Pz = it.pz.N, Px = it.Px, Py = it.Py, tb = it.tbz, nza = it.nza;
    C* tw = reinterpret_cast<C*>(smem);
    C* buf = tw + Pz;
    const int nkx = (Px + tb - 1) / tb;
    const int kxt = tile % nkx;
    const int r = tile / nkx;
    const int ky = r % Py;
    const int64_t b = r / Py;
    const int kx0 = kxt * tb;
    const int nt = min(tb, Px - kx0);
    const int ld = 5 * tb;
    C* B2 = static_cast<C*>(it.B2);
    load_tw<C>(tw, it.tw[2], Pz);
    for (int i = threadIdx.x; i < Pz * ld; i += QT) buf[i] = qzero<C>();
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * nza * tb; i += QT) {
        const int t = i % tb, q = i / tb;
        const int zi = q % nza, a = q / nza;
        if (t < nt)
            buf[__ldg(it.zlist + zi) * ld + a * tb + t] =
                ldcg(B2 + (((b * 5 + a) * nza + zi) * (int64_t)Py + ky) * Px + kx0 + t);
    }
    __syncthreads();
    fft_lines<C, QCfg<T>::MAXPTS>(buf, &it.pz, ld, 1, ld, true, tw);
    const T* spec = static_cast<const T*>(it.spec);
    const int64_t Sk = (int64_t)it.Hx * it.Hy * it.Hz;
    const int ay = min(ky, Py - ky);
    const T sgy = (2 * ky <= Py) ? (T)1 : (T)-1;
    for (int i = threadIdx.x; i < Pz * tb; i += QT) {
        const int kz = i / tb, t = i - kz * tb;
        if (t >= nt) continue;
        const int kx = kx0 + t;
        const int ax = min(kx, Px - kx), az = min(kz, Pz - kz);
        const T sgx = (2 * kx <= Px) ? (T)1 : (T)-1;
        const T sgz = (2 * kz <= Pz) ? (T)1 : (T)-1;
        const int64_t off = ((int64_t)az * it.Hy + ay) * it.Hx + ax;
        C io[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) io[a] = buf[kz * ld + a * tb + t];
        qblock5<T>(io, __ldg(spec + off), sgx * __ldg(spec + Sk + off), sgy * __ldg(spec + 2 * Sk + off),
                   sgz * __ldg(spec + 3 * Sk + off), __ldg(spec + 4 * Sk + off), __ldg(spec + 5 * Sk + off),
                   __ldg(spec + 6 * Sk + off));
#pragma unroll
        for (int a = 0; a < 5; ++a) buf[kz * ld + a * tb + t] = conjc(io[a]);   // inverse by conjugation
    }
    __syncthreads();
    fft_lines<C, QCfg<T>::MAXPTS>(buf, &it.pz, ld, 1, ld, true, tw);
    for (int i = threadIdx.x; i < 5 * nza * tb; i += QT) {
        const int t = i % tb, q = i / tb;
        const int zi = q % nza, a = q / nza;
        if (t < nt)
            B2[(((b * 5 + a) * nza + zi) * (int64_t)Py + ky) * Px + kx0 + t] =
                conjc(buf[__ldg(it.zlist + zi) * ld + a * tb + t]);
    }
}

// phase 5: lpb x-lines: inverse FFT, keep x < Kx, then per voxel
// y^beta = j omega mu dx / P conv + z^beta I^beta - (A^T Phi)^beta (Eq. 7, 9, 16-18, 22-23)
template <typename T>
__device__ __forceinline__ void tile_xinv(const BItem& it, int tile, unsigned char* smem) {
    using C = typename CT<T>::type;
    const int N = it.px.N, ld = N + 1, Kx = it.Kx;
    C* tw = reinterpret_cast<C*>(smem);
    C* buf = tw + N;
    const int64_t nlines = (int64_t)it.nb * 5 * it.nrows;
    const int64_t line0 = (int64_t)tile * it.lpb;
    const int nl = (int)min((int64_t)it.lpb, nlines - line0);
    const C* B1 = static_cast<const C*>(it.B1);
    load_tw<C>(tw, it.tw[0], N);
    for (int i = threadIdx.x; i < nl * N; i += QT) {
        const int l = i / N, n = i - l * N;
        const int64_t line = line0 + l;
        const int64_t ba = line / it.nrows;
        const int ri = (int)(line - ba * it.nrows);
        buf[l * ld + n] = conjc(ldcg(B1 + (ba * it.nza * it.Ky + __ldg(it.rows + ri)) * (int64_t)N + n));
    }
    __syncthreads();
    fft_lines<C, QCfg<T>::MAXPTS>(buf, &it.px, nl, ld, 1, false, tw);
    const C* x = static_cast<const C*>(it.x);
    C* y = static_cast<C*>(it.y);
    for (int i = threadIdx.x; i < nl * Kx; i += QT) {
        const int l = i / Kx, n = i - l * Kx;
        const int64_t line = line0 + l;
        const int64_t ba = line / it.nrows;
        const int ri = (int)(line - ba * it.nrows);
        const int vi = __ldg(it.vidx + (int64_t)__ldg(it.rows + ri) * Kx + n);
        if (vi < 0) continue;
        const int64_t b = ba / 5;
        const int be = (int)(ba - 5 * b);
        const C* xb = x + b * it.Nvec;
        const C cv = conjc(buf[l * ld + n]);
        const double omega = it.omegas[b];
        const T cs = (T)(omega * it.mu * it.dx * it.inv_P);
        C val;
        val.x = -cs * cv.y;
        val.y = cs * cv.x;
        // two-fluid diagonal: c = a + j omega mu b (Eq. 22-23), z^beta = c s_beta / dx
        const double lm = it.lam[vi], s0 = it.sig0[vi];
        const double wml2 = omega * it.mu * lm * lm;
        const double tt = s0 * wml2;
        const double den = 1.0 + tt * tt;
        const double sb = be < 3 ? 1.0 : (be == 3 ? 1.0 / 6.0 : 0.5);
        const double sc = sb / it.dx;
        const T zr = (T)(s0 * wml2 * wml2 / den * sc), zi_ = (T)(omega * it.mu * (lm * lm / den) * sc);
        const C I = xb[be * it.K + vi];
        val.x += zr * I.x - zi_ * I.y;
        val.y += zr * I.y + zi_ * I.x;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const float fl = c_qflux[be][f];
            if (fl != 0.f) {
                const C ph = xb[5 * it.K + __ldg(it.node + (int64_t)vi * 6 + f)];
                val.x -= (T)fl * ph.x;
                val.y -= (T)fl * ph.y;
            }
        }
        y[b * it.Nvec + be * it.K + vi] = val;
    }
}

// ------------------------------------------------------------------ the queue
// waits (thread 0, bounded in time) until *cnt >= need; false on expiry (status bit set)
__device__ __forceinline__ bool wait_count(const int* cnt, int need, const BQueue& q) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (*(volatile const int*)cnt < need) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned ns = 64;
            while (*(volatile const int*)cnt < need) {
                if (globaltimer_ns() - t0 > q.wait_ns) {
                    atomicOr(q.status, SVH_STATUS_QUEUE_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 2048) ns *= 2;
            }
        }
        __threadfence();   // the dependency's writes are visible before this CTA reads them
        s_ok = ok;
    }
    __syncthreads();
    const int ok = s_ok;
    __syncthreads();
    return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(QT, 2) k_batch_queue(const __grid_constant__ BQueue q) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx;
    const int64_t total = q.seg_start[q.nseg];
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(q.counter, 1);
        __syncthreads();
        const int64_t g = s_idx;
        __syncthreads();
        if (g >= total) break;
        // segment of g (segments are (phase, item) in queue order): binary search
        int lo = 0, hi = q.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (q.seg_start[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int phase = q.seg_phase[lo];
        const int item = q.seg_item[lo];
        const int tile = (int)(g - q.seg_start[lo]);
        const BItem& it = q.items[item];
        // dependency: the previous phase of the same structure (phases 0 and 1 have none)
        const int dep = phase >= 2 ? (phase == 2 ? 0 : phase - 1) : -1;
        if (dep >= 0) {
            int need = it.ntile[dep];
            if (item == q.hold_item && dep == q.hold_phase) ++need;   // diagnostic: a count nothing reaches
            if (!wait_count(q.done + item * kBatchPhases + dep, need, q)) return;
        }
        switch (phase) {
            case 0: tile_xfwd<T>(it, tile, smem); break;
            case 1: tile_nodes<T>(it, tile); break;
            case 2: tile_y<T, false>(it, tile, smem); break;
            case 3: tile_z<T>(it, tile, smem); break;
            case 4: tile_y<T, true>(it, tile, smem); break;
            default: tile_xinv<T>(it, tile, smem); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();   // this tile's writes are visible before its completion is counted
            atomicAdd(q.done + item * kBatchPhases + phase, 1);
        }
    }
}

}  // namespace

// Tile shapes and shared memory of one structure (the same limits as the generic passes).
void batch_item_shape(BItem& it, int precision) {
    const int maxpts = (precision == SVH_FP32 ? QCfg<float>::MAXPTS : QCfg<double>::MAXPTS) * QT;
    const size_t csz = precision == SVH_FP32 ? 8 : 16;
    it.lpb = std::max(1, maxpts / it.px.N);
    it.tby = std::max(1, std::min(32, maxpts / it.py.N));
    it.tbz = std::max(1, std::min(64, maxpts / (5 * it.pz.N)));
    const int64_t nlines = (int64_t)it.nb * 5 * it.nrows;
    it.ntile[0] = (int)((nlines + it.lpb - 1) / it.lpb);
    it.ntile[1] = (int)((it.M * it.nb + QT - 1) / QT);
    it.ntile[2] = ((it.Px + it.tby - 1) / it.tby) * it.nza * it.nb * 5;
    it.ntile[3] = ((it.Px + it.tbz - 1) / it.tbz) * it.Py * it.nb;
    it.ntile[4] = it.ntile[2];
    it.ntile[5] = it.ntile[0];
    const size_t sx = (size_t)(it.px.N + it.lpb * (it.px.N + 1)) * csz;
    const size_t sy = (size_t)(it.py.N + it.py.N * it.tby) * csz;
    const size_t sz = (size_t)(it.pz.N + it.pz.N * 5 * it.tbz) * csz;
    it.smem = std::max(sx, std::max(sy, sz));
}

bool batch_fits(const BItem& it, int precision) {
    const int maxpts = (precision == SVH_FP32 ? QCfg<float>::MAXPTS : QCfg<double>::MAXPTS) * QT;
    return it.px.N <= maxpts && it.py.N <= maxpts && 5 * it.pz.N <= maxpts && it.px.nst <= MAX_STAGES;
}

int batch_queue_grid(int precision, size_t smem, int device, int* grid) {
    const void* fn = precision == SVH_FP32 ? reinterpret_cast<const void*>(&k_batch_queue<float>)
                                           : reinterpret_cast<const void*>(&k_batch_queue<double>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SVH_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, QT, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return SVH_ERR_CUDA;
    *grid = std::max(1, per_sm) * sms;
    return SVH_OK;
}

int batch_queue_launch(const BQueue& q, int precision, size_t smem, int grid, cudaStream_t s) {
    if (cudaMemsetAsync(q.counter, 0, sizeof(int) * (1 + (size_t)q.nitems * kBatchPhases), s) != cudaSuccess)
        return SVH_ERR_CUDA;
    if (precision == SVH_FP32) k_batch_queue<float><<<grid, QT, smem, s>>>(q);
    else k_batch_queue<double><<<grid, QT, smem, s>>>(q);
    return cudaGetLastError() == cudaSuccess ? SVH_OK : SVH_ERR_CUDA;
}

}  // namespace svh
