// fastpass.cuh -- size-specialised FFT passes of the operator product (Eq. 9).
//
// x and y passes use the four-step split N = N1 * N2 (N1 >= N2, both <= 32):
//   step 1: each thread loads the N1 points n1*N2 + n2 (n2 fixed) straight
//           from HBM, takes a register DFT of length N1, multiplies by
//           w_N^(n2 k1) and parks the result in shared memory;
//   step 3: each thread gathers the N2 points (n2, k1) of one k1, takes a
//           register DFT of length N2 and writes X[k1 + N1 k2] straight to HBM.
// Lines contiguous in HBM (x) map n2 / k1 to consecutive threads; strided
// lines (y) map the contiguous kx column index to consecutive threads. So
// every HBM access is a coalesced row segment and each point crosses shared
// memory once. The z pass keeps one whole Pz-point line per thread.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fft_reg.cuh"
#include "svh.h"
#include "tc_async.cuh"

namespace svh {

// Everything a pass kernel reads, passed by value.
struct PassArgs {
    const void* x;           // input vectors, nb * Nvec complex
    void* y;                 // output vectors
    void* B1;                // [nb*5][nza][Ky][Px]
    void* B2;                // [nb*5][nza][Py][Px]
    const void* spec;        // octant spectra [7][Hz][Hy][Hx] (float or double)
    const void* twx;         // exp(-2 pi i m / Px), m < Px
    const void* twy;
    const void* twz;
    const int32_t* vidx;     // [nza][Ky][Kx] voxel index or -1
    const int32_t* rows;     // active rows zi*Ky + y
    const int2* rinfo;       // per active row: first voxel index, voxel count
    const int32_t* vx;       // per voxel: x
    const uint8_t* rowmask;  // [nza][Ky]
    const int32_t* zlist;    // active planes
    const int32_t* node;     // [K][6]
    const uint8_t* freem;    // [M]
    const double* lam;
    const double* sig0;
    int64_t K, M, Nvec;
    int64_t nlines;          // nb * 5 * nrows
    int nb, nza, nrows, Kx, Ky, Kz, Px, Py, Pz, Hx, Hy, Hz;
    double omega, mu, dx, conv_scale;
    const double* omegas;    // per-item angular frequency (device, nb entries) or nullptr
    double inv_P;            // 1 / (Px Py Pz)
    int masked;
    int zcontig;             // 1 when the active planes are consecutive
    int var;                 // tile variant of the pass being launched (0: default)
    int* status;             // device status word: kernels set bits on a bounded wait that timed out
    const float* zk;         // z-space kernels [7][zkD][Hy][Hx] of the direct z pass (FP32) or nullptr
    int zkD;                 // their plane offsets 0 .. zkD - 1
};

// direct z pass (fast_zd.cu): up to ZD_MAX_NZA active planes spanning at most ZK_MAX_D
// planes, octants of at most ZK_MAX_HZ z planes
constexpr int ZD_MAX_NZA = 8, ZK_MAX_D = 16, ZK_MAX_HZ = 25;


// outward flux of basis alpha through face f (-x,+x,-y,+y,-z,+z)
__device__ __forceinline__ float face_flux(int a, int f) {
    // x: -1,+1 on x faces; y: on y faces; z: on z faces; 2D: +1/2 on x, -1/2 on y;
    // 3D: +1/2 on x and y faces, -1 on z faces
    const int ax = f >> 1;
    const float sgn = (f & 1) ? 1.f : -1.f;
    switch (a) {
        case 0: return ax == 0 ? sgn : 0.f;
        case 1: return ax == 1 ? sgn : 0.f;
        case 2: return ax == 2 ? sgn : 0.f;
        case 3: return ax == 0 ? 0.5f : (ax == 1 ? -0.5f : 0.f);
        default: return ax == 2 ? -1.f : 0.5f;
    }
}

// y^beta = j conv_scale conv + z^beta I^beta - (A^T Phi)^beta for voxel vi, item b (Eq. 7, 9, 16-18, 22-23)
template <typename T>
__device__ __forceinline__ typename CT<T>::type epilogue(const PassArgs& a, int64_t b, int be, int vi,
                                                         typename CT<T>::type cv) {
    using C = typename CT<T>::type;
    const C* xb = static_cast<const C*>(a.x) + b * a.Nvec;
    const double om = a.omegas ? a.omegas[b] : a.omega;
    const T cs = a.omegas ? (T)(om * a.mu * a.dx * a.inv_P) : (T)a.conv_scale;
    C val;
    val.x = -cs * cv.y;
    val.y = cs * cv.x;
    // two-fluid c = a + j omega mu b (Eq. 22-23), z^beta = c s_beta / dx
    const T lm = (T)a.lam[vi], s0 = (T)a.sig0[vi];
    const T wml2 = (T)(om * a.mu) * lm * lm;
    const T tt = s0 * wml2;
    const T den = (T)1 + tt * tt;
    const T sb = be < 3 ? (T)1 : (be == 3 ? (T)(1.0 / 6.0) : (T)0.5);
    const T sc = sb / (T)a.dx;
    const T zr = s0 * wml2 * wml2 / den * sc;
    const T zi = (T)(om * a.mu) * (lm * lm / den) * sc;
    const C I = xb[be * a.K + vi];
    val.x += zr * I.x - zi * I.y;
    val.y += zr * I.y + zi * I.x;
    const int32_t* nd = a.node + (int64_t)vi * 6;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const float fl = face_flux(be, f);
        if (fl != 0.f) {
            const int m = nd[f];
            if (!a.masked || a.freem[m]) {
                const C ph = xb[5 * a.K + m];
                val.x -= (T)fl * ph.x;
                val.y -= (T)fl * ph.y;
            }
        }
    }
    return val;
}

// ---------------------------------------------------------------- x passes (contiguous lines)
// INV = false: gather I^alpha from the voxel list, forward FFT, write B1 rows.
// INV = true : read B1 rows, inverse FFT, keep x < Kx, epilogue to y.
template <typename T, int N1, int N2, bool INV, int NT>
__global__ void __launch_bounds__(NT) k_xrow(const __grid_constant__ PassArgs a) {
    using C = typename CT<T>::type;
    constexpr int N = N1 * N2;
    constexpr int L = NT / N2;            // lines per block
    constexpr int LDS = N1 + 1;           // padded stride of n2 rows in shared memory
    constexpr int TPT = (L * N1 + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const C* twg = static_cast<const C*>(a.twx);
    // twiddles of the N1 x N2 step in [k1][n2] order: tw[k1 N2 + n2] = W^(n2 k1) (n2 k1 < N), so a
    // thread's N1 factors sit at constant offsets and a warp's lanes read consecutive entries
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[(i / N2) * (i % N2)];
    const int64_t line0 = (int64_t)blockIdx.x * L;
    {
        const int l = threadIdx.x / N2, n2 = threadIdx.x % N2;
        const int64_t line = line0 + l;
        C v[N1];
        if constexpr (!INV) {
            // x < Kx <= N / 2: inputs n1 >= N1 / 2 are zero (input-pruned first stage). The row's
            // voxels are one index range in x order: they are read contiguously (with their x)
            // into the line's row in shared memory, then taken in the transform's order
            C* lrow = buf + l * (N / 2);
#pragma unroll
            for (int n1 = 0; n1 < N1 / 2; ++n1) {
                lrow[n1 * N2 + n2].x = 0;
                lrow[n1 * N2 + n2].y = 0;
            }
            __syncthreads();
            if (line < a.nlines) {
                const int64_t ba = line / a.nrows;
                const int2 ri = a.rinfo[line - ba * a.nrows];
                const int64_t b = ba / 5;
                const int al = (int)(ba - 5 * b);
                const C* xb = static_cast<const C*>(a.x) + b * a.Nvec + al * a.K + ri.x;
                const int32_t* xr = a.vx + ri.x;
                for (int j = n2; j < ri.y; j += N2) lrow[__ldg(xr + j)] = xb[j];
            }
            __syncthreads();
            C hv[N1 / 2];
#pragma unroll
            for (int n1 = 0; n1 < N1 / 2; ++n1) hv[n1] = lrow[n1 * N2 + n2];
            reg_fft_lowin<N1, false>(hv, v);
        } else {
            if (line < a.nlines) {
                const int64_t ba = line / a.nrows;
                const int row = a.rows[line - ba * a.nrows];
                const C* src = static_cast<const C*>(a.B1) + (ba * a.nza * a.Ky + row) * (int64_t)N;
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[n1 * N2 + n2];
            } else {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) { v[n1].x = 0; v[n1].y = 0; }
            }
            reg_fft<N1, true>(v);
        }
        __syncthreads();   // twiddle table ready
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            const C w = tw[k1 * N2 + n2];   // 1 for n2 = 0
            v[k1] = INV ? cmulc(v[k1], w) : cmul(v[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[(l * N2 + n2) * LDS + k1] = v[k1];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NT;
        if (task >= L * N1) break;
        const int l = task / N1, k1 = task % N1;
        const int64_t line = line0 + l;
        if (line >= a.nlines) continue;
        C u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = buf[(l * N2 + n2) * LDS + k1];
        const int64_t ba = line / a.nrows;
        const int row = a.rows[line - ba * a.nrows];
        if constexpr (!INV) {
            reg_fft<N2, false>(u);
            C* dst = static_cast<C*>(a.B1) + (ba * a.nza * a.Ky + row) * (int64_t)N;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) dst[k1 + N1 * k2] = u[k2];
        } else {
            // only x = k1 + N1 k2 < Kx <= N / 2 is kept: k2 < N2 / 2 (output-pruned)
            C w[N2 / 2];
            reg_fft_lowout<N2, true>(u, w);
            const int64_t b = ba / 5;
            const int be = (int)(ba - 5 * b);
            const int32_t* vr = a.vidx + (int64_t)row * a.Kx;
            C* yb = static_cast<C*>(a.y) + b * a.Nvec + be * a.K;
#pragma unroll
            for (int k2 = 0; k2 < N2 / 2; ++k2) {
                const int k = k1 + N1 * k2;
                if (k < a.Kx) {
                    const int vi = __ldg(vr + k);
                    if (vi >= 0) yb[vi] = epilogue<T>(a, b, be, vi, w[k2]);
                }
            }
        }
    }
}

// x inverse + epilogue, grouped: a block takes G (item, row) groups and the 5
// basis lines of each, runs the inverse x FFT of all 5G lines, parks the kept
// x < Kx values in shared memory and then finishes every voxel of its rows in
// one thread for all five bases (voxel index, face nodes, lambda, sigma0 and
// the two-fluid c are loaded or computed once per voxel, not once per basis).
template <typename T, int N1, int N2, int NT>
__global__ void __launch_bounds__(NT) k_xinv_grouped(const __grid_constant__ PassArgs a) {
    using C = typename CT<T>::type;
    constexpr int N = N1 * N2;
    constexpr int L = NT / N2;              // lines per block (a multiple of 5)
    constexpr int G = L / 5;                // (item, row) groups per block
    constexpr int LDS = N1 + 1;
    constexpr int TPT = (L * N1 + NT - 1) / NT;
    static_assert(L % 5 == 0, "lines per block must hold whole groups of 5 bases");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const C* twg = static_cast<const C*>(a.twx);
    // twiddles of the N1 x N2 step in [k1][n2] order: tw[k1 N2 + n2] = W^(n2 k1) (n2 k1 < N), so a
    // thread's N1 factors sit at constant offsets and a warp's lanes read consecutive entries
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[(i / N2) * (i % N2)];
    const int64_t ngroups = (int64_t)a.nb * a.nrows;
    const int64_t g0 = (int64_t)blockIdx.x * G;
    const int Kx = a.Kx;
    // the first epilogue task's per-voxel data (x, lambda, sigma0, face nodes) of group 0, loaded
    // now so that the loads overlap the transforms
    // (FP32 also its input values and face-node potentials: the FP64 form has no registers to spare)
    constexpr bool PFV = std::is_same<T, float>::value;
    int pf_vi = -1, pf_x = 0, pf_nd[6];
    T pf_lm = 0, pf_s0 = 0;
    C pf_I[5], pf_ph[6];
    if (g0 < ngroups) {
        const int64_t b = g0 / a.nrows;
        const int2 ri = a.rinfo[g0 - b * a.nrows];
        if ((int)threadIdx.x < ri.y) {
            pf_vi = ri.x + (int)threadIdx.x;
            pf_x = __ldg(a.vx + pf_vi);
            pf_lm = (T)a.lam[pf_vi];
            pf_s0 = (T)a.sig0[pf_vi];
            if constexpr (PFV) {
                const C* xb = static_cast<const C*>(a.x) + b * a.Nvec;
#pragma unroll
                for (int be = 0; be < 5; ++be) pf_I[be] = xb[be * a.K + pf_vi];
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) pf_nd[f] = __ldg(a.node + (int64_t)pf_vi * 6 + f);
        }
    }
    {
        const int l = threadIdx.x / N2, n2 = threadIdx.x % N2;
        const int64_t g = g0 + l / 5;
        const int be = l % 5;
        C v[N1];
        if (g < ngroups) {
            const int64_t b = g / a.nrows;
            const int row = a.rows[g - b * a.nrows];
            const C* src = static_cast<const C*>(a.B1) + ((b * 5 + be) * a.nza * a.Ky + row) * (int64_t)N;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[n1 * N2 + n2];
        } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) { v[n1].x = 0; v[n1].y = 0; }
        }
        if (PFV && pf_vi >= 0) {   // the prefetched voxel's face-node potentials (need its node indices)
            const C* xb = static_cast<const C*>(a.x) + (g0 / a.nrows) * a.Nvec;
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const int m = pf_nd[f];
                if (!a.masked || a.freem[m]) pf_ph[f] = xb[5 * a.K + m];
                else { pf_ph[f].x = 0; pf_ph[f].y = 0; }
            }
        }
        reg_fft<N1, true>(v);
        __syncthreads();
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            v[k1] = cmulc(v[k1], tw[k1 * N2 + n2]);   // 1 for n2 = 0
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[(l * N2 + n2) * LDS + k1] = v[k1];
    }
    __syncthreads();
    // only x = k1 + N1 k2 < Kx <= N / 2 is kept: k2 < N2 / 2 (output-pruned)
    C u[TPT][N2 / 2];
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NT;
        if (task < L * N1) {
            const int l = task / N1, k1 = task % N1;
            C t[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) t[n2] = buf[(l * N2 + n2) * LDS + k1];
            reg_fft_lowout<N2, true>(t, u[it]);
        }
    }
    __syncthreads();   // every step-3 read of buf is done; reuse it for the kept x < Kx values
    const int LDX = Kx + 1;
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NT;
        if (task < L * N1) {
            const int l = task / N1, k1 = task % N1;
#pragma unroll
            for (int k2 = 0; k2 < N2 / 2; ++k2) {
                const int k = k1 + N1 * k2;
                if (k < Kx) buf[l * LDX + k] = u[it][k2];
            }
        }
    }
    __syncthreads();
    const T inv_dx = (T)(1.0 / a.dx);
    // one task per voxel of the block's rows (each row's voxels are one index range, in x order)
    for (int gl = 0; gl < G; ++gl) {
        const int64_t g = g0 + gl;
        if (g >= ngroups) break;
        const int64_t b = g / a.nrows;
        const int2 ri = a.rinfo[g - b * a.nrows];
        for (int j = threadIdx.x; j < ri.y; j += NT) {
            const bool pf = gl == 0 && j == (int)threadIdx.x;   // data loaded at the start
            const int vi = ri.x + j;
            const int x = pf ? pf_x : __ldg(a.vx + vi);
            const double om = a.omegas ? a.omegas[b] : a.omega;
            const T cs = a.omegas ? (T)(om * a.mu * a.dx * a.inv_P) : (T)a.conv_scale;
            // two-fluid c = a + j omega mu b (Eq. 22-23), once per voxel
            const T lm = pf ? pf_lm : (T)a.lam[vi], s0 = pf ? pf_s0 : (T)a.sig0[vi];
            const T wm = (T)(om * a.mu);
            const T wml2 = wm * lm * lm;
            const T tt = s0 * wml2;
            const T den = (T)1 + tt * tt;
            const T cre = s0 * wml2 * wml2 / den * inv_dx, cim = wm * (lm * lm / den) * inv_dx;
            const C* xb = static_cast<const C*>(a.x) + b * a.Nvec;
            C* yb = static_cast<C*>(a.y) + b * a.Nvec;
            C ph[6];
            const int32_t* nd = a.node + (int64_t)vi * 6;
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (PFV && pf) {
                    ph[f] = pf_ph[f];
                } else {
                    const int m = nd[f];
                    if (!a.masked || a.freem[m]) ph[f] = xb[5 * a.K + m];
                    else { ph[f].x = 0; ph[f].y = 0; }
                }
            }
#pragma unroll
            for (int be = 0; be < 5; ++be) {
                const C cv = buf[(gl * 5 + be) * LDX + x];
                C val;
                val.x = -cs * cv.y;
                val.y = cs * cv.x;
                const T sb = be < 3 ? (T)1 : (be == 3 ? (T)(1.0 / 6.0) : (T)0.5);
                const C I = (PFV && pf) ? pf_I[be] : xb[be * a.K + vi];
                val.x += sb * (cre * I.x - cim * I.y);
                val.y += sb * (cre * I.y + cim * I.x);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const float fl = face_flux(be, f);
                    if (fl != 0.f) {
                        val.x -= (T)fl * ph[f].x;
                        val.y -= (T)fl * ph[f].y;
                    }
                }
                yb[be * a.K + vi] = val;
            }
        }
    }
}

// ---------------------------------------------------------------- y passes (strided lines, kx tiles)
// INV = false: B1 rows y < Ky (active) -> forward FFT -> B2 rows ky < Py.
// INV = true : B2 -> inverse FFT -> B1 active rows y < Ky.
// (256-thread blocks of lines up to 32 x 32 points: registers capped so that three blocks share
// an SM and one block's loads overlap another's transforms)
template <typename T, int N1, int N2, bool INV, int NT>
__global__ void __launch_bounds__(NT, (NT == 256 && N1 <= 32) ? 3 : 0)
    k_ycol_fast(const __grid_constant__ PassArgs a) {
    using C = typename CT<T>::type;
    constexpr int N = N1 * N2;
    constexpr int TB = NT / N2;           // kx columns per block
    constexpr int TPT = (TB * N1 + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;                      // [n2][k1][TB]
    const C* twg = static_cast<const C*>(a.twy);
    // twiddles of the N1 x N2 step in natural order, read at m = n2 k1 (with 512-thread blocks the
    // [k1][n2] order of the other passes measured slower here)
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
    const int kx0 = blockIdx.x * TB;
    const int zi = blockIdx.y;
    const int64_t ba = blockIdx.z;
    const int Px = a.Px;
    // the plane's row mask (rows y < Ky <= N / 2 holding voxels), staged once so that the
    // predicated loads and stores below do not wait on a global byte load each
    __shared__ uint8_t rm[N / 2];
    {
        const uint8_t* rmg = a.rowmask + (int64_t)zi * a.Ky;
        for (int i = threadIdx.x; i < N / 2; i += NT) rm[i] = i < a.Ky ? rmg[i] : 0;
    }
    __syncthreads();
    {
        const int c = threadIdx.x % TB, n2 = threadIdx.x / TB;
        const bool colok = kx0 + c < Px;
        C v[N1];
        if constexpr (!INV) {
            // y < Ky <= N / 2: inputs n1 >= N1 / 2 are zero (input-pruned first stage)
            const C* src = static_cast<const C*>(a.B1) + ((ba * a.nza + zi) * (int64_t)a.Ky) * Px + kx0 + c;
            C hv[N1 / 2];
#pragma unroll
            for (int n1 = 0; n1 < N1 / 2; ++n1) {
                const int n = n1 * N2 + n2;
                C z; z.x = 0; z.y = 0;
                if (colok && n < a.Ky && rm[n]) z = src[(int64_t)n * Px];
                hv[n1] = z;
            }
            reg_fft_lowin<N1, false>(hv, v);
        } else {
            const C* src = static_cast<const C*>(a.B2) + ((ba * a.nza + zi) * (int64_t)N) * Px + kx0 + c;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                C z; z.x = 0; z.y = 0;
                if (colok) z = src[(int64_t)(n1 * N2 + n2) * Px];
                v[n1] = z;
            }
            reg_fft<N1, true>(v);
        }
        __syncthreads();
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            const int m = (n2 * k1) % N;
            if (m) v[k1] = INV ? cmulc(v[k1], tw[m]) : cmul(v[k1], tw[m]);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[(n2 * N1 + k1) * TB + c] = v[k1];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NT;
        if (task >= TB * N1) break;
        const int c = task % TB, k1 = task / TB;
        if (kx0 + c >= Px) continue;
        C u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = buf[(n2 * N1 + k1) * TB + c];
        if constexpr (!INV) {
            reg_fft<N2, false>(u);
            C* dst = static_cast<C*>(a.B2) + ((ba * a.nza + zi) * (int64_t)N) * Px + kx0 + c;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) dst[(int64_t)(k1 + N1 * k2) * Px] = u[k2];
        } else {
            // only y = k1 + N1 k2 < Ky <= N / 2 is kept: k2 < N2 / 2 (output-pruned)
            C w[N2 / 2];
            reg_fft_lowout<N2, true>(u, w);
            C* dst = static_cast<C*>(a.B1) + ((ba * a.nza + zi) * (int64_t)a.Ky) * Px + kx0 + c;
#pragma unroll
            for (int k2 = 0; k2 < N2 / 2; ++k2) {
                const int k = k1 + N1 * k2;
                if (k < a.Ky && rm[k]) dst[(int64_t)k * Px] = w[k2];
            }
        }
    }
}

// ---------------------------------------------------------------- y passes, staged by cp.async
// The same four-step transform as k_ycol_fast (FP32), run by a persistent grid whose blocks walk
// the (item*basis, plane, kx tile) tiles with a stride of the grid size (kx tile fastest, so the
// grid sweeps one plane together). A tile's input rows travel by cp.async (16 bytes = two
// columns per copy, zero-filled for rows without voxels) into a shared buffer; as soon as the
// first stage has read the current tile from it, the copies of the block's NEXT tile are issued,
// so they land while this tile is twiddled, exchanged, transformed and stored.
template <int N1, int N2, bool INV, int NT>
__global__ void __launch_bounds__(NT, 2) k_ycol_async(const __grid_constant__ PassArgs a, int ntiles, int rbw_arg) {
    using C = float2;
    constexpr int N = N1 * N2;
    constexpr int TB = NT / N2;                 // kx columns per tile (even)
    constexpr int NROW = INV ? N : N / 2;        // input rows of a tile (forward: y < Ky <= N / 2)
    constexpr int SEG = TB / 2;                  // 16-byte segments per row
    constexpr int CPT = (NROW * SEG + NT - 1) / NT;
    constexpr int TPT = (TB * N1 + NT - 1) / NT;
    static_assert(TB % 2 == 0, "two columns per 16-byte copy");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* in = tw + N;                              // [NROW][TB]
    C* buf = in + NROW * TB;                     // [n2][k1][TB]
    // forward: the active-row masks of every plane as bits ([plane][Ky / 32] words), when the
    // launcher gave them room (rbw > 0), so that a copy's row test is a shared-memory read
    uint32_t* rbits = reinterpret_cast<uint32_t*>(buf + N * TB);
    const int rbw = INV ? 0 : rbw_arg;
    const C* twg = static_cast<const C*>(a.twy);
    // twiddles of the N1 x N2 step in [k1][n2] order: tw[k1 N2 + n2] = W^(n2 k1) (n2 k1 < N), so a
    // thread's N1 factors sit at constant offsets and a warp's lanes read consecutive entries
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[(i / N2) * (i % N2)];
    const int Px = a.Px, Ky = a.Ky, nza = a.nza;
    const int nkx = (Px + TB - 1) / TB;
    // the launcher takes this kernel only when Px is a multiple of TB: a tile's columns are all in range
    auto issue = [&](int t) {
        const int kxt = t % nkx, r = t / nkx;
        const int zi = r % nza;
        const int64_t ba = r / nza;
        const C* src = static_cast<const C*>(INV ? a.B2 : a.B1) +
                       ((ba * nza + zi) * (int64_t)(INV ? N : Ky)) * Px + (int64_t)kxt * TB;
        const uint8_t* rm = a.rowmask + (int64_t)zi * Ky;
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int e = threadIdx.x + i * NT;
            if (e < NROW * SEG) {
                const int row = e / SEG, sg = e % SEG;
                const bool valid =
                    INV || (row < Ky && (rbw ? (rbits[zi * rbw + (row >> 5)] >> (row & 31)) & 1u : __ldg(rm + row)));
                cp_async16_zfill(in + row * TB + 2 * sg, src + (int64_t)(valid ? row : 0) * Px + 2 * sg, valid);
            }
        }
        cp_async_commit();
    };
    const int c = threadIdx.x % TB, n2 = threadIdx.x / TB;
    for (int w = threadIdx.x; w < nza * rbw; w += NT) {
        const int zi = w / rbw, y0 = (w % rbw) * 32;
        const uint8_t* rm = a.rowmask + (int64_t)zi * Ky;
        uint32_t bits = 0;
        for (int b = 0; b < 32 && y0 + b < Ky; ++b) bits |= (uint32_t)(__ldg(rm + y0 + b) != 0) << b;
        rbits[w] = bits;
    }
    __syncthreads();
    int t = blockIdx.x;
    if (t < ntiles) issue(t);
    cp_async_wait<0>();
    __syncthreads();
    for (; t < ntiles; t += gridDim.x) {
        C v[N1];
        if constexpr (!INV) {
            C hv[N1 / 2];
#pragma unroll
            for (int n1 = 0; n1 < N1 / 2; ++n1) hv[n1] = in[(n1 * N2 + n2) * TB + c];
            reg_fft_lowin<N1, false>(hv, v);
        } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = in[(n1 * N2 + n2) * TB + c];
            reg_fft<N1, true>(v);
        }
        const int kxt = t % nkx, r = t / nkx;
        const int zi = r % nza;
        const int64_t ba = r / nza;
        const int kx0 = kxt * TB;
        __syncthreads();                                 // every read of `in` is done
        if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x);   // the next tile's rows, in flight
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            const C w = tw[k1 * N2 + n2];   // 1 for n2 = 0
            v[k1] = INV ? cmulc(v[k1], w) : cmul(v[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[(n2 * N1 + k1) * TB + c] = v[k1];
        __syncthreads();
#pragma unroll
        for (int it = 0; it < TPT; ++it) {
            const int task = threadIdx.x + it * NT;
            if (task >= TB * N1) break;
            const int cc = task % TB, k1 = task / TB;
            C u[N2];
#pragma unroll
            for (int q = 0; q < N2; ++q) u[q] = buf[(q * N1 + k1) * TB + cc];
            if constexpr (!INV) {
                reg_fft<N2, false>(u);
                C* dst = static_cast<C*>(a.B2) + ((ba * nza + zi) * (int64_t)N) * Px + kx0 + cc;
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) dst[(int64_t)(k1 + N1 * k2) * Px] = u[k2];
            } else {
                // only y = k1 + N1 k2 < Ky <= N / 2 is kept: k2 < N2 / 2 (output-pruned)
                C w[N2 / 2];
                reg_fft_lowout<N2, true>(u, w);
                C* dst = static_cast<C*>(a.B1) + ((ba * nza + zi) * (int64_t)Ky) * Px + kx0 + cc;
                const uint8_t* rm = a.rowmask + (int64_t)zi * Ky;
#pragma unroll
                for (int k2 = 0; k2 < N2 / 2; ++k2) {
                    const int k = k1 + N1 * k2;
                    if (k < Ky && __ldg(rm + k)) dst[(int64_t)k * Px] = w[k2];
                }
            }
        }
        cp_async_wait<0>();                              // the next tile's rows have landed
        __syncthreads();                                 // and every read of buf is done
    }
}

// ---------------------------------------------------------------- z pass (whole pencils per thread)
// Block: 5 warps (warp = basis alpha), lane = kx offset in a 32-wide tile, one ky.
template <typename T>
__device__ __forceinline__ void block_multiply5(typename CT<T>::type* io, T g, T sx, T sy, T sz, T qx, T qy, T qz) {
    using C = typename CT<T>::type;
    // the S-kernel spectra are -i*sign*R: mi(a) = -i a, pi(a) = +i a
    auto mi = [](C v) { C c; c.x = v.y; c.y = -v.x; return c; };
    auto pi = [](C v) { C c; c.x = -v.y; c.y = v.x; return c; };
    C Ix = io[0], Iy = io[1], Iz = io[2], I2 = io[3], I3 = io[4];
    C Yx = cadd(cscale(Ix, g), cscale(mi(cadd(I2, I3)), sx));
    C Yy = cadd(cscale(Iy, g), cscale(mi(csub(I3, I2)), sy));
    C Yz = cadd(cscale(Iz, g), cscale(pi(I3), (T)2 * sz));
    C pX = pi(Ix), pY = pi(Iy), pZ = pi(Iz);
    T qs = qx + qy, qd = qx - qy;
    C Y2 = cadd(cadd(cscale(pX, sx), cscale(pY, -sy)), cadd(cscale(I2, qs), cscale(I3, qd)));
    C Y3 = cadd(cadd(cscale(pX, sx), cscale(pY, sy)),
                cadd(cscale(pZ, (T)-2 * sz), cadd(cscale(I2, qd), cscale(I3, qs + (T)4 * qz))));
    io[0] = Yx; io[1] = Yy; io[2] = Yz; io[3] = Y2; io[4] = Y3;
}

// The same block product in scalar FP32 fused multiply-adds: the +-i factors become operand
// swaps and signs, so each complex-by-real term is two FMAs and no moves
__device__ __forceinline__ void block_multiply5_fma(float2* io, float g, float sx, float sy, float sz, float qx,
                                                    float qy, float qz) {
    const float2 Ix = io[0], Iy = io[1], Iz = io[2], I2 = io[3], I3 = io[4];
    const float px = I2.x + I3.x, py = I2.y + I3.y;   // I2 + I3
    const float mx = I3.x - I2.x, my = I3.y - I2.y;   // I3 - I2
    const float s2 = 2.f * sz, qs = qx + qy, qd = qx - qy, q3 = qs + 4.f * qz;
    float2 Y;
    // Yx = g Ix - i sx (I2 + I3)
    Y.x = fmaf(g, Ix.x, sx * py);
    Y.y = fmaf(g, Ix.y, -sx * px);
    io[0] = Y;
    // Yy = g Iy - i sy (I3 - I2)
    Y.x = fmaf(g, Iy.x, sy * my);
    Y.y = fmaf(g, Iy.y, -sy * mx);
    io[1] = Y;
    // Yz = g Iz + i 2 sz I3
    Y.x = fmaf(g, Iz.x, -s2 * I3.y);
    Y.y = fmaf(g, Iz.y, s2 * I3.x);
    io[2] = Y;
    // Y2 = i sx Ix - i sy Iy + qs I2 + qd I3
    Y.x = fmaf(qd, I3.x, fmaf(qs, I2.x, fmaf(sy, Iy.y, -sx * Ix.y)));
    Y.y = fmaf(qd, I3.y, fmaf(qs, I2.y, fmaf(-sy, Iy.x, sx * Ix.x)));
    io[3] = Y;
    // Y3 = i sx Ix + i sy Iy - i 2 sz Iz + qd I2 + q3 I3
    Y.x = fmaf(q3, I3.x, fmaf(qd, I2.x, fmaf(s2, Iz.y, fmaf(-sy, Iy.y, -sx * Ix.y))));
    Y.y = fmaf(q3, I3.y, fmaf(qd, I2.y, fmaf(-s2, Iz.x, fmaf(sy, Iy.x, sx * Ix.x))));
    io[4] = Y;
}

// Spectra of one z-pass tile (32 kx columns at one ky, all PZ planes) into
// shared memory sp[u][kz][lane], with the odd S-kernel signs folded in: only
// the octant |k| <= P/2 is stored, so kz and PZ - kz share the value at
// az = min(kz, PZ - kz) (Sz flips sign in the upper half, Sx/Sy by column/row).
// One task per (kernel, column), each octant value loaded once.
template <typename T, int PZ>
__device__ __forceinline__ void load_tile_spectra(const PassArgs& a, T (*sp)[PZ][32], int kx0, int ky) {
    constexpr int NH = PZ / 2 + 1;
    const T* spec = static_cast<const T*>(a.spec);
    const int Px = a.Px, Py = a.Py;
    const int64_t plane = (int64_t)a.Hx * a.Hy, Sk = plane * a.Hz;
    const int ay = min(ky, Py - ky);
    const T sgy = (2 * ky <= Py) ? (T)1 : (T)-1;
    for (int task = threadIdx.x; task < 7 * 32; task += blockDim.x) {
        const int u = task >> 5, ln = task & 31;
        const int kxx = min(kx0 + ln, Px - 1);
        const int ax = min(kxx, Px - kxx);
        const T sgx = (2 * kxx <= Px) ? (T)1 : (T)-1;
        const T sg = u == 1 ? sgx : (u == 2 ? sgy : (T)1);
        const int64_t off = (int64_t)ay * a.Hx + ax;
        T val[NH];
#pragma unroll
        for (int az = 0; az < NH; ++az) val[az] = __ldg(spec + u * Sk + az * plane + off);
#pragma unroll
        for (int az = 0; az < NH; ++az) {
            sp[u][az][ln] = sg * val[az];
            if (az > 0 && PZ - az != az) sp[u][PZ - az][ln] = (u == 3 ? -sg : sg) * val[az];
        }
    }
}

// The block's spectra (7 values at each of its PZ x 32 points) are loaded once
// into shared memory and reused for every batch item the block loops over.
template <typename T, int PZ>
__global__ void __launch_bounds__(160) k_zpass_fast(const __grid_constant__ PassArgs a) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C(*buf)[PZ][32] = reinterpret_cast<C(*)[PZ][32]>(smem_raw);            // [5][PZ][32]
    T(*sp)[PZ][32] = reinterpret_cast<T(*)[PZ][32]>(smem_raw + sizeof(C) * 5 * PZ * 32);  // [7][PZ][32]
    const int al = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kx0 = blockIdx.x * 32;
    const int ky = blockIdx.y;
    const int kx = kx0 + lane;
    const bool ok = kx < a.Px;
    const int Px = a.Px, Py = a.Py;
    // spectra of the tile, with the odd-kernel signs folded in
    load_tile_spectra<T, PZ>(a, sp, kx0, ky);
    C* B2 = static_cast<C*>(a.B2);
    const int64_t plane = (int64_t)Py * Px;
    // planes holding voxels: at most (Pz + 1) / 2 of them (Pz >= 2 Kz - 1)
    constexpr int NZ = PZ / 2 + 1;
    const int nza = a.nza;
    int zl[NZ];
#pragma unroll
    for (int zi = 0; zi < NZ; ++zi) zl[zi] = zi < nza ? a.zlist[zi] : 0;
    // the next item's active planes are fetched into registers while the
    // current item is transformed, so their latency overlaps the FFTs
    C pre[NZ];
    auto fetch = [&](int b) {
        const int64_t base = ((int64_t)(b * 5 + al) * nza * Py + ky) * Px + kx;
#pragma unroll
        for (int zi = 0; zi < NZ; ++zi)
            if (ok && zi < nza) pre[zi] = B2[base + zi * plane];
    };
    fetch(0);
    C v[PZ];
    for (int b = 0; b < a.nb; ++b) {
        // own column only until the first barrier: the previous item's
        // cross-column multiply finished before its second barrier
#pragma unroll
        for (int z = 0; z < PZ; ++z) { buf[al][z][lane].x = 0; buf[al][z][lane].y = 0; }
#pragma unroll
        for (int zi = 0; zi < NZ; ++zi)
            if (zi < nza && ok) buf[al][zl[zi]][lane] = pre[zi];
        if (b + 1 < a.nb) fetch(b + 1);
#pragma unroll
        for (int z = 0; z < PZ; ++z) v[z] = buf[al][z][lane];
        reg_fft<PZ, false>(v);
#pragma unroll
        for (int z = 0; z < PZ; ++z) buf[al][z][lane] = v[z];
        __syncthreads();
        for (int task = threadIdx.x; task < PZ * 32; task += 160) {
            const int kz = task >> 5, ln = task & 31;
            C io[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) io[q] = buf[q][kz][ln];
            block_multiply5<T>(io, sp[0][kz][ln], sp[1][kz][ln], sp[2][kz][ln], sp[3][kz][ln], sp[4][kz][ln],
                               sp[5][kz][ln], sp[6][kz][ln]);
#pragma unroll
            for (int q = 0; q < 5; ++q) buf[q][kz][ln] = io[q];
        }
        __syncthreads();
#pragma unroll
        for (int z = 0; z < PZ; ++z) v[z] = buf[al][z][lane];
        reg_fft<PZ, true>(v);
        if (ok) {
#pragma unroll
            for (int z = 0; z < PZ; ++z) buf[al][z][lane] = v[z];   // own column only
            const int64_t base = ((int64_t)(b * 5 + al) * nza * Py + ky) * Px + kx;
#pragma unroll
            for (int zi = 0; zi < NZ; ++zi)
                if (zi < nza) B2[base + zi * plane] = buf[al][zl[zi]][lane];
        }
    }
}

// Contiguous active planes z0 .. z0 + nza - 1 (the usual case: layers and the
// vias between them). A cyclic convolution commutes with shifts, so each
// pencil is shifted by -z0: its inputs then sit at [0, nza), inside the lower
// half of the PZ points (nza <= Kz <= PZ / 2), and only outputs [0, nza) are
// kept. The forward transform is then input-pruned and the inverse
// output-pruned (reg_fft_lowin / reg_fft_lowout), the pencil never passes
// through shared memory except for the cross-basis multiply, and the spectra
// indices kz are unchanged (a shift only multiplies each spectrum by a phase
// that the inverse removes).
template <typename T, int PZ>
__global__ void __launch_bounds__(160) k_zpass_half(const __grid_constant__ PassArgs a) {
    using C = typename CT<T>::type;
    constexpr int H = PZ / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C(*buf)[PZ][32] = reinterpret_cast<C(*)[PZ][32]>(smem_raw);            // [5][PZ][32]
    T(*sp)[PZ][32] = reinterpret_cast<T(*)[PZ][32]>(smem_raw + sizeof(C) * 5 * PZ * 32);  // [7][PZ][32]
    const int al = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kx0 = blockIdx.x * 32;
    const int ky = blockIdx.y;
    const int kx = kx0 + lane;
    const bool ok = kx < a.Px;
    const int Px = a.Px, Py = a.Py;
    load_tile_spectra<T, PZ>(a, sp, kx0, ky);
    C* B2 = static_cast<C*>(a.B2);
    const int64_t plane = (int64_t)Py * Px;
    const int nza = a.nza;
    C pre[H];
    auto fetch = [&](int b) {
        const int64_t base = ((int64_t)(b * 5 + al) * nza * Py + ky) * Px + kx;
#pragma unroll
        for (int zi = 0; zi < H; ++zi) {
            C z; z.x = 0; z.y = 0;
            if (ok && zi < nza) z = B2[base + zi * plane];
            pre[zi] = z;
        }
    };
    fetch(0);
    for (int b = 0; b < a.nb; ++b) {
        {
            C v[PZ];
            reg_fft_lowin<PZ, false>(pre, v);
            if (b + 1 < a.nb) fetch(b + 1);
#pragma unroll
            for (int z = 0; z < PZ; ++z) buf[al][z][lane] = v[z];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < PZ * 32; task += 160) {
            const int kz = task >> 5, ln = task & 31;
            C io[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) io[q] = buf[q][kz][ln];
            block_multiply5<T>(io, sp[0][kz][ln], sp[1][kz][ln], sp[2][kz][ln], sp[3][kz][ln], sp[4][kz][ln],
                               sp[5][kz][ln], sp[6][kz][ln]);
#pragma unroll
            for (int q = 0; q < 5; ++q) buf[q][kz][ln] = io[q];
        }
        __syncthreads();
        C v[PZ], w[H];
#pragma unroll
        for (int z = 0; z < PZ; ++z) v[z] = buf[al][z][lane];
        reg_fft_lowout<PZ, true>(v, w);
        if (ok) {
            const int64_t base = ((int64_t)(b * 5 + al) * nza * Py + ky) * Px + kx;
#pragma unroll
            for (int zi = 0; zi < H; ++zi)
                if (zi < nza) B2[base + zi * plane] = w[zi];
        }
    }
}

// ---------------------------------------------------------------- TMA-staged z pass
// Same arithmetic as k_zpass_half; the 5 nza active planes of a (32-kx, ky)
// tile of one item travel as one TMA box (cp.async.bulk.tensor, 3-D view of
// B2 as [planes][Py][2 Px] floats) into shared memory, double-buffered so the
// next item's box arrives while this one is transformed, and the results go
// back by a TMA store from the same buffer. One thread issues the copies;
// every wait is bounded (SVH_STATUS_TMA_TIMEOUT in a.status on expiry).
__device__ __forceinline__ void tma_store_3d(const void* tmap, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tmap),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// tmap: 3-D float view of B2, dims {2 Px, Py, nb 5 nza}, box {64, 1, 5 nza}
template <int PZ>
__global__ void __launch_bounds__(160) k_zpass_tma(const __grid_constant__ PassArgs a, const __grid_constant__ CUtensorMap tmap) {
    using C = float2;
    constexpr int NH = PZ / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // TMA boxes start on a 128-byte boundary (the launch adds 128 bytes of slack)
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int nza = a.nza, nq = 5 * nza;
    C* tile = reinterpret_cast<C*>(base);                                      // [2][nq][32]
    C(*buf)[PZ][32] = reinterpret_cast<C(*)[PZ][32]>(tile + 2 * nq * 32);      // [5][PZ][32]
    float(*sp)[PZ][32] = reinterpret_cast<float(*)[PZ][32]>(buf + 5);          // [7][PZ][32]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sp + 7);                       // [2]
    const int al = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kx0 = blockIdx.x * 32;
    const int ky = blockIdx.y;
    const uint32_t box_bytes = (uint32_t)nq * 32 * sizeof(C);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar[0], box_bytes);
        tma_load_3d(tile, &tmap, &bar[0], 2 * kx0, ky, 0);
    }
    load_tile_spectra<float, PZ>(a, sp, kx0, ky);
    bool failed = false;
    for (int b = 0; b < a.nb; ++b) {
        const int cur = b & 1;
        C* tb = tile + cur * nq * 32;
        if (threadIdx.x == 0 && b + 1 < a.nb) {
            bulk_wait_read0();   // item b - 1's store has read the other buffer
            mbar_expect_tx(&bar[cur ^ 1], box_bytes);
            tma_load_3d(tile + (cur ^ 1) * nq * 32, &tmap, &bar[cur ^ 1], 2 * kx0, ky, (b + 1) * nq);
        }
        // bounded wait for this item's box
        {
            const uint32_t parity = (uint32_t)(b >> 1) & 1u;
            int spins = 0;
            while (!mbar_try_wait(&bar[cur], parity)) {
                if (++spins > (1 << 20)) { failed = true; break; }
            }
        }
        if (__syncthreads_or(failed)) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, SVH_STATUS_TMA_TIMEOUT);
                // drain (bounded) the load issued for the next item before the CTA exits
                if (b + 1 < a.nb) {
                    int spins = 0;
                    while (!mbar_try_wait(&bar[cur ^ 1], (uint32_t)((b + 1) >> 1) & 1u) && ++spins < (1 << 20)) {
                    }
                }
            }
            break;
        }
        C pre[NH];
#pragma unroll
        for (int zi = 0; zi < NH; ++zi) pre[zi] = zi < nza ? tb[(al * nza + zi) * 32 + lane] : make_float2(0.f, 0.f);
        {
            C v[PZ];
            reg_fft_lowin<PZ, false>(pre, v);
#pragma unroll
            for (int z = 0; z < PZ; ++z) buf[al][z][lane] = v[z];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < PZ * 32; task += 160) {
            const int kz = task >> 5, ln = task & 31;
            C io[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) io[q] = buf[q][kz][ln];
            block_multiply5<float>(io, sp[0][kz][ln], sp[1][kz][ln], sp[2][kz][ln], sp[3][kz][ln], sp[4][kz][ln],
                                   sp[5][kz][ln], sp[6][kz][ln]);
#pragma unroll
            for (int q = 0; q < 5; ++q) buf[q][kz][ln] = io[q];
        }
        __syncthreads();
        {
            C v[PZ], w[NH];
#pragma unroll
            for (int z = 0; z < PZ; ++z) v[z] = buf[al][z][lane];
            reg_fft_lowout<PZ, true>(v, w);
#pragma unroll
            for (int zi = 0; zi < NH; ++zi)
                if (zi < nza) tb[(al * nza + zi) * 32 + lane] = w[zi];
        }
        fence_async_smem();   // this thread's writes to the box, visible to the TMA store
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_3d(&tmap, tb, 2 * kx0, ky, b * nq);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait0();   // the stores have finished before shared memory is released
}

// launchers (return false when the size has no specialised kernel)
template <typename T> bool launch_x_fast(const PassArgs& a, bool inv, cudaStream_t s);
template <typename T> bool launch_y_fast(const PassArgs& a, bool inv, cudaStream_t s);
template <typename T> bool launch_z_fast(const PassArgs& a, cudaStream_t s);
bool launch_z_direct(const PassArgs& a, cudaStream_t s);
// z pass with each pencil split over two threads (fast_zs.cu), FP32, Pz = 32 or 48 with the active
// planes consecutive and in the lower half
bool z_split_ok(int Pz, int nza, int zcontig);
bool launch_z_split(const PassArgs& a, cudaStream_t s);
bool launch_z_split16(const PassArgs& a, cudaStream_t s, bool prefetch);
void launch_spec_to_zk(const float* S, float* R, const float* W, int Hx, int Hy, int Hz, int D, cudaStream_t s);
bool z_fast_size(int Pz);
// number of tile variants of a pass at this size (0: no specialised kernel)
int x_fast_variants(int Px, bool inv, bool fp32);
int y_fast_variants(int Py, bool fp32);
int z_fast_variants(int Pz, bool fp32);

}  // namespace svh
