// fused.cuh -- the y forward, z and y inverse passes fused into one kernel.
//
// After the x pass the product needs, for every kx, the y-FFT of each
// (basis, plane) line, the z-FFT / 5 x 5 multiply / inverse z-FFT of each
// (kx, ky) pencil (Eq. 9) and the inverse y-FFT back to the voxel rows. For
// one kx these touch only that column's slab: 5 bases x nza planes x Py
// points (123 KB in FP32 at Py = 512, nza = 6), which fits one CTA's shared
// memory on GB300. So one CTA per (kx, item) loads the slab's active rows,
// runs all three passes in shared memory and writes the rows back: the
// padded y/z grids never reach HBM, which removes the 4 Q bytes per item the
// separate y, z, y passes move (Q = 5 nza Py Px 8 B).
//
// Layouts. B1T [nb][5][Px][nrows]: the x pass output transposed so a CTA's
// slab rows are contiguous (k_xfwd_t / k_xinv_t below). In shared memory a
// line of Py = NY1 x NY2 points is stored as an NY1 x (NY2 + 1) array (one
// pad column against bank conflicts); the forward transform leaves ky =
// k1 + NY1 k2 at (k1, k2) and the inverse takes that order back to natural.
// The z pencils use the shifted, pruned transforms of k_zpass_half (active
// planes contiguous), CH pencils at a time through a [5][PZ][CH] scratch.
#pragma once
#include "fastpass.cuh"

namespace svh {

template <int NY1, int NY2, int PZ, int NT>
struct YZCfg {
    static constexpr int NY = NY1 * NY2;
    static constexpr int LS = NY2 + 1;            // padded row of a line
    static constexpr int LINE = NY1 * LS;         // padded line
    static constexpr int CH = NT / 5;             // z pencils per chunk
    static_assert(NT % 5 == 0, "5 bases per pencil");
    static_assert(NY % CH == 0, "pencil chunks must tile the line");
};

// shared memory bytes of k_yz_fused for nza active planes
template <int NY1, int NY2, int PZ, int NT>
size_t yz_smem_bytes(int nza) {
    using Cf = YZCfg<NY1, NY2, PZ, NT>;
    return ((size_t)5 * nza * Cf::LINE + (size_t)5 * PZ * Cf::CH + Cf::NY) * sizeof(float2);
}

template <int NY1, int NY2, int PZ, int NT>
__global__ void __launch_bounds__(NT, 1) k_yz_fused(const __grid_constant__ PassArgs a) {
    using C = float2;
    using Cf = YZCfg<NY1, NY2, PZ, NT>;
    constexpr int NY = Cf::NY, LS = Cf::LS, LINE = Cf::LINE, CH = Cf::CH;
    constexpr int NH = PZ / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nza = a.nza, nlines = 5 * nza;
    C* buf = reinterpret_cast<C*>(smem_raw);               // [5 nza][LINE]
    C* zs = buf + (size_t)nlines * LINE;                   // [5][PZ][CH]
    C* tw = zs + 5 * PZ * CH;                              // [NY]
    const int kx = blockIdx.x;
    const int b = blockIdx.y;
    const int Px = a.Px, Ky = a.Ky, nrows = a.nrows;
    const C* twg = static_cast<const C*>(a.twy);
    for (int i = threadIdx.x; i < NY; i += NT) tw[i] = twg[i];
    // zero the lower half (n < NY / 2) of every line: rows without voxels and Ky <= y < NY / 2
    for (int i = threadIdx.x; i < nlines * (NY1 / 2) * NY2; i += NT) {
        const int line = i / ((NY1 / 2) * NY2), rem = i - line * ((NY1 / 2) * NY2);
        const int n1 = rem / NY2, n2 = rem - n1 * NY2;
        buf[(size_t)line * LINE + n1 * LS + n2] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    // load the slab's active rows: B1T[b][al][kx][r] -> line (al, zi), natural index y
    {
        const C* src = static_cast<const C*>(a.B1) + ((int64_t)b * 5 * Px + kx) * nrows;
        for (int i = threadIdx.x; i < 5 * nrows; i += NT) {
            const int al = i / nrows, r = i - al * nrows;
            const int row = __ldg(a.rows + r);
            const int zi = row / Ky, y = row - zi * Ky;
            buf[(size_t)(al * nza + zi) * LINE + (y / NY2) * LS + (y % NY2)] = src[(int64_t)al * Px * nrows + r];
        }
    }
    __syncthreads();
    // y forward, stage 1: per (line, n2), input-pruned NY1-point DFT over n1, twiddle W^(n2 k1)
    for (int t = threadIdx.x; t < nlines * NY2; t += NT) {
        const int line = t / NY2, n2 = t - line * NY2;
        C* L = buf + (size_t)line * LINE;
        C hv[NY1 / 2], v[NY1];
#pragma unroll
        for (int n1 = 0; n1 < NY1 / 2; ++n1) hv[n1] = L[n1 * LS + n2];
        reg_fft_lowin<NY1, false>(hv, v);
#pragma unroll
        for (int k1 = 0; k1 < NY1; ++k1) {
            const int m = (n2 * k1) % NY;
            L[k1 * LS + n2] = m ? cmul(v[k1], tw[m]) : v[k1];
        }
    }
    __syncthreads();
    // y forward, stage 2: per (line, k1), NY2-point DFT over n2 -> ky = k1 + NY1 k2 at (k1, k2)
    for (int t = threadIdx.x; t < nlines * NY1; t += NT) {
        const int line = t / NY1, k1 = t - line * NY1;
        C* R = buf + (size_t)line * LINE + k1 * LS;
        C u[NY2];
#pragma unroll
        for (int n2 = 0; n2 < NY2; ++n2) u[n2] = R[n2];
        reg_fft<NY2, false>(u);
#pragma unroll
        for (int k2 = 0; k2 < NY2; ++k2) R[k2] = u[k2];
    }
    __syncthreads();
    // z: CH pencils at a time; thread (al, j) transforms basis al of pencil p0 + j
    {
        const float* spec = static_cast<const float*>(a.spec);
        const int64_t plane = (int64_t)a.Hx * a.Hy, Sk = plane * a.Hz;
        const int ax = min(kx, Px - kx);
        const float sgx = (2 * kx <= Px) ? 1.f : -1.f;
        const int al = threadIdx.x / CH, j = threadIdx.x - al * CH;
        for (int p0 = 0; p0 < NY; p0 += CH) {
            {
                const int p = p0 + j, k1 = p / NY2, k2 = p - k1 * NY2;
                const C* col = buf + (size_t)(al * nza) * LINE + k1 * LS + k2;
                C hv[NH], v[PZ];
#pragma unroll
                for (int zi = 0; zi < NH; ++zi) hv[zi] = zi < nza ? col[(size_t)zi * LINE] : make_float2(0.f, 0.f);
                reg_fft_lowin<PZ, false>(hv, v);
#pragma unroll
                for (int kz = 0; kz < PZ; ++kz) zs[(al * PZ + kz) * CH + j] = v[kz];
            }
            __syncthreads();
            for (int t = threadIdx.x; t < PZ * CH; t += NT) {
                const int kz = t / CH, jj = t - kz * CH;
                const int p = p0 + jj, k1 = p / NY2, k2 = p - k1 * NY2;
                const int ky = k1 + NY1 * k2;
                const int ay = min(ky, NY - ky), az = min(kz, PZ - kz);
                const float sgy = (2 * ky <= NY) ? 1.f : -1.f;
                const float sgz = (2 * kz <= PZ) ? 1.f : -1.f;
                const int64_t off = (int64_t)az * plane + (int64_t)ay * a.Hx + ax;
                C io[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) io[q] = zs[(q * PZ + kz) * CH + jj];
                block_multiply5<float>(io, __ldg(spec + off), sgx * __ldg(spec + Sk + off),
                                       sgy * __ldg(spec + 2 * Sk + off), sgz * __ldg(spec + 3 * Sk + off),
                                       __ldg(spec + 4 * Sk + off), __ldg(spec + 5 * Sk + off),
                                       __ldg(spec + 6 * Sk + off));
#pragma unroll
                for (int q = 0; q < 5; ++q) zs[(q * PZ + kz) * CH + jj] = io[q];
            }
            __syncthreads();
            {
                const int p = p0 + j, k1 = p / NY2, k2 = p - k1 * NY2;
                C* col = buf + (size_t)(al * nza) * LINE + k1 * LS + k2;
                C v[PZ], w[NH];
#pragma unroll
                for (int kz = 0; kz < PZ; ++kz) v[kz] = zs[(al * PZ + kz) * CH + j];
                reg_fft_lowout<PZ, true>(v, w);
#pragma unroll
                for (int zi = 0; zi < NH; ++zi)
                    if (zi < nza) col[(size_t)zi * LINE] = w[zi];
            }
            // the next chunk's forward writes only this thread's own zs column
        }
    }
    __syncthreads();
    // y inverse, stage 1: per (line, k1), inverse NY2-point DFT over k2, twiddle W^-(n2 k1)
    for (int t = threadIdx.x; t < nlines * NY1; t += NT) {
        const int line = t / NY1, k1 = t - line * NY1;
        C* R = buf + (size_t)line * LINE + k1 * LS;
        C u[NY2];
#pragma unroll
        for (int k2 = 0; k2 < NY2; ++k2) u[k2] = R[k2];
        reg_fft<NY2, true>(u);
#pragma unroll
        for (int n2 = 0; n2 < NY2; ++n2) {
            const int m = (n2 * k1) % NY;
            R[n2] = m ? cmulc(u[n2], tw[m]) : u[n2];
        }
    }
    __syncthreads();
    // y inverse, stage 2: per (line, n2), output-pruned inverse NY1-point DFT -> y = NY2 n1 + n2 < NY / 2
    for (int t = threadIdx.x; t < nlines * NY2; t += NT) {
        const int line = t / NY2, n2 = t - line * NY2;
        C* L = buf + (size_t)line * LINE;
        C v[NY1], w[NY1 / 2];
#pragma unroll
        for (int k1 = 0; k1 < NY1; ++k1) v[k1] = L[k1 * LS + n2];
        reg_fft_lowout<NY1, true>(v, w);
#pragma unroll
        for (int n1 = 0; n1 < NY1 / 2; ++n1) L[n1 * LS + n2] = w[n1];
    }
    __syncthreads();
    // store the active rows back
    {
        C* dst = static_cast<C*>(a.B1) + ((int64_t)b * 5 * Px + kx) * nrows;
        for (int i = threadIdx.x; i < 5 * nrows; i += NT) {
            const int al = i / nrows, r = i - al * nrows;
            const int row = __ldg(a.rows + r);
            const int zi = row / Ky, y = row - zi * Ky;
            dst[(int64_t)al * Px * nrows + r] = buf[(size_t)(al * nza + zi) * LINE + (y / NY2) * LS + (y % NY2)];
        }
    }
}

// ---------------------------------------------------------------- x passes on the transposed layout
// Forward: gather I^alpha of NTX / N2 consecutive active rows, x-FFT, write
// B1T[ba][k][r] so that for every k the block's rows form one contiguous run.
template <int N1, int N2, int NTX>
__global__ void __launch_bounds__(NTX) k_xfwd_t(const __grid_constant__ PassArgs a) {
    using C = float2;
    constexpr int N = N1 * N2;
    constexpr int L = NTX / N2;            // lines per block
    constexpr int LDS = N1 + 1;
    constexpr int LST = N2 * LDS + 1;      // padded line stride (consecutive lines on different banks)
    constexpr int TPT = (L * N1 + NTX - 1) / NTX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const C* twg = static_cast<const C*>(a.twx);
    for (int i = threadIdx.x; i < N; i += NTX) tw[i] = twg[i];
    const int64_t line0 = (int64_t)blockIdx.x * L;
    {
        const int l = threadIdx.x / N2, n2 = threadIdx.x % N2;
        const int64_t line = line0 + l;
        C hv[N1 / 2], v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1 / 2; ++n1) hv[n1] = make_float2(0.f, 0.f);
        if (line < a.nlines) {
            const int64_t ba = line / a.nrows;
            const int row = a.rows[line - ba * a.nrows];
            const int64_t b = ba / 5;
            const int al = (int)(ba - 5 * b);
            const C* xb = static_cast<const C*>(a.x) + b * a.Nvec + al * a.K;
            const int32_t* vr = a.vidx + (int64_t)row * a.Kx;
#pragma unroll
            for (int n1 = 0; n1 < N1 / 2; ++n1) {
                const int n = n1 * N2 + n2;
                if (n < a.Kx) {
                    const int vi = __ldg(vr + n);
                    if (vi >= 0) hv[n1] = xb[vi];
                }
            }
        }
        reg_fft_lowin<N1, false>(hv, v);
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const int m = (n2 * k1) % N;
            buf[l * LST + n2 * LDS + k1] = m ? cmul(v[k1], tw[m]) : v[k1];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NTX;
        if (task >= L * N1) break;
        const int l = task % L, k1 = task / L;    // consecutive threads: consecutive rows
        const int64_t line = line0 + l;
        if (line >= a.nlines) continue;
        C u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = buf[l * LST + n2 * LDS + k1];
        reg_fft<N2, false>(u);
        const int64_t ba = line / a.nrows, r = line - ba * a.nrows;
        C* dst = static_cast<C*>(a.B1) + ba * (int64_t)a.Px * a.nrows + r;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) dst[(int64_t)(k1 + N1 * k2) * a.nrows] = u[k2];
    }
}

// Inverse x-FFT + epilogue from B1T: G (item, row) groups x 5 bases per block
// as k_xinv_grouped, with the row index fastest across threads when reading.
template <int N1, int N2, int NTX>
__global__ void __launch_bounds__(NTX) k_xinv_t(const __grid_constant__ PassArgs a) {
    using C = float2;
    using T = float;
    constexpr int N = N1 * N2;
    constexpr int L = NTX / N2;
    constexpr int G = L / 5;
    constexpr int LDS = N1 + 1;
    constexpr int LST = N2 * LDS + 1;
    constexpr int TPT = (L * N1 + NTX - 1) / NTX;
    static_assert(L % 5 == 0, "lines per block must hold whole groups of 5 bases");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const C* twg = static_cast<const C*>(a.twx);
    for (int i = threadIdx.x; i < N; i += NTX) tw[i] = twg[i];
    const int64_t ngroups = (int64_t)a.nb * a.nrows;
    const int64_t g0 = (int64_t)blockIdx.x * G;
    const int Kx = a.Kx;
    {
        const int gl = threadIdx.x % G, be = (threadIdx.x / G) % 5, n2 = threadIdx.x / L;
        const int l = gl * 5 + be;
        const int64_t g = g0 + gl;
        C v[N1];
        if (g < ngroups) {
            const int64_t b = g / a.nrows, r = g - b * a.nrows;
            const C* src = static_cast<const C*>(a.B1) + (b * 5 + be) * (int64_t)a.Px * a.nrows + r;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[(int64_t)(n1 * N2 + n2) * a.nrows];
        } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = make_float2(0.f, 0.f);
        }
        reg_fft<N1, true>(v);
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            const int m = (n2 * k1) % N;
            buf[l * LST + n2 * LDS + k1] = m ? cmulc(v[k1], tw[m]) : v[k1];
        }
    }
    __syncthreads();
    // only x = k1 + N1 k2 < Kx <= N / 2 is kept: k2 < N2 / 2 (output-pruned)
    C u[TPT][N2 / 2];
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NTX;
        if (task < L * N1) {
            const int l = task / N1, k1 = task % N1;
            C t[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) t[n2] = buf[l * LST + n2 * LDS + k1];
            reg_fft_lowout<N2, true>(t, u[it]);
        }
    }
    __syncthreads();
    const int LDX = Kx + 1;
#pragma unroll
    for (int it = 0; it < TPT; ++it) {
        const int task = threadIdx.x + it * NTX;
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
    for (int task = threadIdx.x; task < G * Kx; task += NTX) {
        const int gl = task / Kx, x = task % Kx;
        const int64_t g = g0 + gl;
        if (g >= ngroups) continue;
        const int64_t b = g / a.nrows;
        const int row = a.rows[g - b * a.nrows];
        const int vi = __ldg(a.vidx + (int64_t)row * Kx + x);
        if (vi < 0) continue;
        const double om = a.omegas ? a.omegas[b] : a.omega;
        const T cs = a.omegas ? (T)(om * a.mu * a.dx * a.inv_P) : (T)a.conv_scale;
        const T lm = (T)a.lam[vi], s0 = (T)a.sig0[vi];
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
            const int m = nd[f];
            if (!a.masked || a.freem[m]) ph[f] = xb[5 * a.K + m];
            else ph[f] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int be = 0; be < 5; ++be) {
            const C cv = buf[(gl * 5 + be) * LDX + x];
            C val;
            val.x = -cs * cv.y;
            val.y = cs * cv.x;
            const T sb = be < 3 ? (T)1 : (be == 3 ? (T)(1.0 / 6.0) : (T)0.5);
            const C I = xb[be * a.K + vi];
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

bool fused_path_ok(const PassArgs& a, size_t smem_limit);
void launch_x_t(const PassArgs& a, bool inv, cudaStream_t s);
void launch_yz(const PassArgs& a, size_t smem_limit, cudaStream_t s);

}  // namespace svh
