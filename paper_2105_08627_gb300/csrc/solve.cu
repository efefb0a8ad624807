// solve.cu -- port solves of Eq. 7: flexible GMRES(restart) with FP64 Arnoldi on the
// device, the Schur-complement preconditioner of Eq. 12-15, FP32 inner products
// with FP64 iterative refinement, and the port admittance -> impedance reduction.
//
// Excitation: for port j the plus-terminal nodes get Phi = 1 and every other
// fixed node (terminals of all ports, gauge nodes of floating islands) Phi = 0.
// Fixed nodes leave the unknowns; the library keeps the vector length N and
// solves the masked operator Kt = D K D + (I - D) (D zeroes fixed-node
// potentials and continuity rows) with right-hand side [A_T^T Phi_T; 0], so
// fixed-node entries of the solution are 0. Port current I_p = sum over the
// plus nodes of port p of (A I)_m; Y[p][j] = I_p under excitation j;
// Z_port = Y^{-1}.
//
// Right preconditioning with P applied exactly as Eq. 13-15, S^{-1} by the
// host AMG; because the AMG inner solve stops at a tolerance, the outer method
// is flexible GMRES (the preconditioned vectors Z_k are kept). Arnoldi uses
// classical Gram-Schmidt applied twice (CGS2) in FP64: each pass is one
// batched dot-product kernel over the basis and one linear-combination kernel.
// Givens rotations and the small least-squares solves run on the device (one thread per
// right-hand side); the host reads only the count of unconverged right-hand sides per step.
// Batching: every (frequency, port) pair is an item; one FGMRES runs all items
// in lock-step with batched operator products (per-item omega: the spectra do
// not depend on it), batched Arnoldi kernels and one AMG hierarchy per frequency.
// Refinement: r = b - Kt x in FP64, inner FGMRES on Kt (FP32 products) to a
// relative reduction of 1e-5 (or to the target), x += correction, until
// ||r|| / ||b|| <= rre measured with the FP64 product (Sec. III: RRE 1e-8).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "svh_internal.h"

namespace svh {

using cdbl = std::complex<double>;

static const double kFluxH[5][6] = {
    {-1, 1, 0, 0, 0, 0}, {0, 0, -1, 1, 0, 0}, {0, 0, 0, 0, -1, 1}, {0.5, 0.5, -0.5, -0.5, 0, 0}, {0.5, 0.5, 0.5, 0.5, -1, -1}};
__constant__ double c_fluxd[5][6] = {
    {-1, 1, 0, 0, 0, 0}, {0, 0, -1, 1, 0, 0}, {0, 0, 0, 0, -1, 1}, {0.5, 0.5, -0.5, -0.5, 0, 0}, {0.5, 0.5, 0.5, 0.5, -1, -1}};

constexpr int DOT_THREADS = 256;
constexpr int DOT_PER_THREAD = 8;

// partial[r][blk][i] = sum over the block's slice of conj(V[r][i][n]) * w[r][n], i < nv
__global__ void __launch_bounds__(DOT_THREADS) k_dots(const double2* __restrict__ V, int64_t ldv, int64_t rstride_v,
                                                      const double2* __restrict__ w, int64_t rstride_w, int nv,
                                                      int64_t n, double2* __restrict__ partial, int nblk) {
    const int r = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * DOT_THREADS * DOT_PER_THREAD;
    double2 wv[DOT_PER_THREAD];
    const double2* wr = w + r * rstride_w;
#pragma unroll
    for (int q = 0; q < DOT_PER_THREAD; ++q) {
        const int64_t idx = n0 + threadIdx.x + (int64_t)q * DOT_THREADS;
        if (idx < n) wv[q] = wr[idx];
        else { wv[q].x = 0; wv[q].y = 0; }
    }
    __shared__ double2 red[DOT_THREADS / 32];
    const double2* Vr = V + r * rstride_v;
    for (int i = 0; i < nv; ++i) {
        const double2* vi = Vr + (int64_t)i * ldv;
        double sr = 0, si = 0;
#pragma unroll
        for (int q = 0; q < DOT_PER_THREAD; ++q) {
            const int64_t idx = n0 + threadIdx.x + (int64_t)q * DOT_THREADS;
            if (idx < n) {
                const double2 a = vi[idx];
                sr += a.x * wv[q].x + a.y * wv[q].y;   // conj(a) * w
                si += a.x * wv[q].y - a.y * wv[q].x;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            si += __shfl_down_sync(0xffffffffu, si, o);
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5].x = sr; red[threadIdx.x >> 5].y = si; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 t; t.x = 0; t.y = 0;
            for (int q = 0; q < DOT_THREADS / 32; ++q) { t.x += red[q].x; t.y += red[q].y; }
            partial[((int64_t)r * nblk + blockIdx.x) * nv + i] = t;
        }
        __syncthreads();
    }
}

// out[r][i] = sum over blocks of partial[r][blk][i]
__global__ void k_dots_reduce(const double2* __restrict__ partial, int nblk, int nv, double2* __restrict__ out) {
    const int r = blockIdx.y, i = blockIdx.x;
    double sr = 0, si = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double2 p = partial[((int64_t)r * nblk + b) * nv + i];
        sr += p.x;
        si += p.y;
    }
    __shared__ double s1[256], s2[256];
    s1[threadIdx.x] = sr;
    s2[threadIdx.x] = si;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { s1[threadIdx.x] += s1[threadIdx.x + s]; s2[threadIdx.x] += s2[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[(int64_t)r * nv + i].x = s1[0]; out[(int64_t)r * nv + i].y = s2[0]; }
}

// out[r][n] = beta * out[r][n] + sum_i coef[r][i] * V[r][i][n]
__global__ void k_lincomb(double2* __restrict__ out, int64_t rstride_o, const double2* __restrict__ V, int64_t ldv,
                          int64_t rstride_v, const double2* __restrict__ coef, int ldc, int nv, double beta, int64_t n,
                          double csign = 1.0) {
    const int r = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double2* Vr = V + r * rstride_v;
    const double2* c = coef + (int64_t)r * ldc;
    double2 acc = out[r * rstride_o + idx];
    acc.x *= beta;
    acc.y *= beta;
    for (int i = 0; i < nv; ++i) {
        const double2 a = Vr[(int64_t)i * ldv + idx];
        double2 k = c[i];
        k.x *= csign;
        k.y *= csign;
        acc.x += k.x * a.x - k.y * a.y;
        acc.y += k.x * a.y + k.y * a.x;
    }
    out[r * rstride_o + idx] = acc;
}

// y[r][n] = x[r][n] * s[r] (real scale)
__global__ void k_scale(double2* __restrict__ y, int64_t rs_y, const double2* __restrict__ x, int64_t rs_x,
                        const double* __restrict__ s, int64_t n) {
    const int r = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = x[r * rs_x + i];
    v.x *= s[r];
    v.y *= s[r];
    y[r * rs_y + i] = v;
}

__global__ void k_to32(const double2* __restrict__ x, float2* __restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { y[i].x = (float)x[i].x; y[i].y = (float)x[i].y; }
}
__global__ void k_to64(const float2* __restrict__ x, double2* __restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { y[i].x = x[i].x; y[i].y = x[i].y; }
}

// a + b (elementwise) into a
__global__ void k_add(double2* __restrict__ a, const double2* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i].x += b[i].x; a[i].y += b[i].y; }
}

// a - b (elementwise) into a
__global__ void k_sub(double2* __restrict__ a, const double2* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i].x -= b[i].x; a[i].y -= b[i].y; }
}

// Preconditioner, first half (Eq. 14 right-hand side): e_m = d_m - sum over the
// voxel faces at free node m of flux * c / Y, for every free node (compact).
__global__ void k_prec_pre(const double2* __restrict__ v, int64_t Nvec, int64_t K, const double* __restrict__ Yall,
                           int per_freq, const int32_t* __restrict__ free_nodes, int nf,
                           const int32_t* __restrict__ ninc, double2* __restrict__ e) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const double* Y = Yall + (int64_t)(r / per_freq) * 5 * K;
    const double2* vr = v + (int64_t)r * Nvec;
    const int m = free_nodes[i];
    double2 acc = vr[5 * K + m];
    for (int q = 0; q < 2; ++q) {
        const int code = ninc[2 * (int64_t)m + q];
        if (code < 0) continue;
        const int vx = code / 6, f = code - 6 * (code / 6);
        for (int a = 0; a < 5; ++a) {
            const double fl = c_fluxd[a][f];
            if (fl == 0) continue;
            const double yi = fl / Y[a * K + vx];
            const double2 c = vr[a * K + vx];
            acc.x -= yi * c.x;
            acc.y -= yi * c.y;
        }
    }
    e[(int64_t)r * nf + i] = acc;
}

// Preconditioner, second half (Eq. 15): a = Y^{-1}(c + A_F^T b); potentials:
// b on free nodes, the input value on fixed nodes (identity rows of Kt).
__global__ void k_prec_post_vox(const double2* __restrict__ v, double2* __restrict__ out, int64_t Nvec, int64_t K,
                                const double* __restrict__ Yall, int per_freq, const int32_t* __restrict__ node,
                                const int32_t* __restrict__ free_id, const double2* __restrict__ b, int nf) {
    const int r = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 5 * K) return;
    const double* Y = Yall + (int64_t)(r / per_freq) * 5 * K;
    const int a = (int)(t / K);
    const int64_t vx = t - a * K;
    const double2* vr = v + (int64_t)r * Nvec;
    double2 s = vr[t];
    for (int f = 0; f < 6; ++f) {
        const double fl = c_fluxd[a][f];
        if (fl == 0) continue;
        const int id = free_id[node[vx * 6 + f]];
        if (id < 0) continue;
        const double2 bb = b[(int64_t)r * nf + id];
        s.x += fl * bb.x;
        s.y += fl * bb.y;
    }
    const double yi = 1.0 / Y[t];
    s.x *= yi;
    s.y *= yi;
    out[(int64_t)r * Nvec + t] = s;
}

__global__ void k_prec_post_node(const double2* __restrict__ v, double2* __restrict__ out, int64_t Nvec, int64_t K,
                                 int64_t M, const int32_t* __restrict__ free_id, const double2* __restrict__ b, int nf) {
    const int r = blockIdx.y;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int id = free_id[m];
    out[(int64_t)r * Nvec + 5 * K + m] = id >= 0 ? b[(int64_t)r * nf + id] : v[(int64_t)r * Nvec + 5 * K + m];
}

// ------------------------------------------------------------------ Arnoldi bookkeeping on the device
// One thread per right-hand side r (nb <= a few hundred). H is column-major per r,
// H[r][i + k (m + 1)]; cs, sn [r][m]; g [r][m + 1]. Complex arithmetic in double2.
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Column k of the Hessenberg matrix from the two Gram-Schmidt passes (h1 + h2, and the norm of
// the new vector below the diagonal), the earlier rotations applied to it, a new rotation that
// zeroes its sub-diagonal entry, the rotated right-hand side g, the scale 1/||w|| of the next
// basis vector, and the count of right-hand sides still above their tolerance (*active).
__global__ void k_arnoldi_givens(double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ sn,
                                 double2* __restrict__ g, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 const double2* __restrict__ hn2, int k, int m, int nb, const double* __restrict__ tol,
                                 const double* __restrict__ beta0, const int* __restrict__ done, double* __restrict__ scl,
                                 int* __restrict__ active) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nb) return;
    double2* Hr = H + (size_t)r * (m + 1) * m + (size_t)k * (m + 1);
    const double hn = sqrt(fmax(hn2[r].x, 0.0));
    for (int i = 0; i <= k; ++i) Hr[i] = zadd(h1[(size_t)r * (k + 1) + i], h2[(size_t)r * (k + 1) + i]);
    Hr[k + 1] = make_double2(hn, 0.0);
    scl[r] = hn > 1e-300 * fmax(1.0, beta0[r]) ? 1.0 / hn : 0.0;
    const double2* csr = cs + (size_t)r * m;
    const double2* snr = sn + (size_t)r * m;
    for (int i = 0; i < k; ++i) {
        const double2 a = Hr[i], b = Hr[i + 1];
        Hr[i] = zadd(zmul(csr[i], a), zmul(snr[i], b));
        Hr[i + 1] = zsub(zmul(zconj(csr[i]), b), zmul(zconj(snr[i]), a));
    }
    // rotation [c s; -conj(s) conj(c)] with c = |a| / t, s = (a / |a|) conj(b) / t, t = hypot(|a|, |b|)
    const double2 a = Hr[k], b = Hr[k + 1];
    double2 c, sv;
    const double na = zabs(a), nbv = zabs(b);
    if (nbv == 0) { c = make_double2(1, 0); sv = make_double2(0, 0); }
    else if (na == 0) { c = make_double2(0, 0); sv = zscale(zconj(b), 1.0 / nbv); }
    else {
        const double t = hypot(na, nbv);
        c = make_double2(na / t, 0);
        sv = zscale(zmul(zscale(a, 1.0 / na), zconj(b)), 1.0 / t);
    }
    cs[(size_t)r * m + k] = c;
    sn[(size_t)r * m + k] = sv;
    Hr[k] = zadd(zmul(c, a), zmul(sv, b));
    Hr[k + 1] = make_double2(0, 0);
    double2* gr = g + (size_t)r * (m + 1);
    const double2 gk = gr[k];
    gr[k + 1] = zscale(zmul(zconj(sv), gk), -1.0);
    gr[k] = zmul(c, gk);
    if (!(done[r] || zabs(gr[k + 1]) <= tol[r] * beta0[r])) atomicAdd(active, 1);
}

// y from the upper-triangular system H[0..kk) y = g (zero for converged right-hand sides)
__global__ void k_arnoldi_backsolve(const double2* __restrict__ H, const double2* __restrict__ g, double2* __restrict__ y,
                                    int kk, int m, int nb, const int* __restrict__ done) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nb) return;
    const double2* Hr = H + (size_t)r * (m + 1) * m;
    const double2* gr = g + (size_t)r * (m + 1);
    double2* yr = y + (size_t)r * kk;
    for (int i = kk - 1; i >= 0; --i) {
        double2 t = done[r] ? make_double2(0, 0) : gr[i];
        for (int j = i + 1; j < kk; ++j) t = zsub(t, zmul(Hr[i + (size_t)j * (m + 1)], yr[j]));
        const double2 d = Hr[i + (size_t)i * (m + 1)];
        const double dd = d.x * d.x + d.y * d.y;
        yr[i] = dd > 0 && !done[r] ? zscale(zmul(t, zconj(d)), 1.0 / dd) : make_double2(0, 0);
    }
}

// ------------------------------------------------------------------ host driver
// Krylov storage: V[i][r][n] (i <= m) and Z[i][r][n] (i < m), so basis vector i
// of all nb right-hand sides is one contiguous nb x N block that the batched
// preconditioner and operator product consume directly.
struct SolveWork {
    int nb = 0, m = 0;
    int per_freq = 1;        // items of one frequency (= number of ports)
    int amg_dev = 1;         // Schur solves on the device
    int64_t N = 0;
    int nf = 0;
    DevBuf X, B, R, W, D, V, Z, T32a, T32b, part, hbuf, E, Bs, Yd, freeid, freenodes, scl, om;
    // Arnoldi bookkeeping on the device: Hessenberg columns, rotations, rotated right-hand
    // sides, the two Gram-Schmidt coefficient sets, ||w||^2, the least-squares solution,
    // per-right-hand-side tolerance, initial norm, converged flag and the active counts
    DevBuf Hh, Hcs, Hsn, Hg, Hh1, Hh2, Hn, Hy, Htol, Hb0, Hdone, Hact;
    int* pin = nullptr;                 // pinned host copies of the active count (two slots)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~SolveWork() {
        for (DevBuf* b : {&X, &B, &R, &W, &D, &V, &Z, &T32a, &T32b, &part, &hbuf, &E, &Bs, &Yd, &freeid, &freenodes,
                          &scl, &om, &Hh, &Hcs, &Hsn, &Hg, &Hh1, &Hh2, &Hn, &Hy, &Htol, &Hb0, &Hdone, &Hact})
            dev_free(*b);
        if (pin) cudaFreeHost(pin);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

static unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static int nblk_dots(int64_t N) { return (int)((N + DOT_THREADS * DOT_PER_THREAD - 1) / (DOT_THREADS * DOT_PER_THREAD)); }

// out[r][i] = V_i^H w_r for i < nv, left on the device (no synchronisation)
static void dots_dev(Handle* h, SolveWork& s, const double2* Vb, int64_t ldv, int nv, const double2* w, double2* out) {
    const int64_t N = s.N;
    const int nblk = nblk_dots(N);
    k_dots<<<dim3(nblk, s.nb), DOT_THREADS, 0, h->stream>>>(Vb, ldv, N, w, N, nv, N, static_cast<double2*>(s.part.p),
                                                            nblk);
    k_dots_reduce<<<dim3(nv, s.nb), 256, 0, h->stream>>>(static_cast<double2*>(s.part.p), nblk, nv, out);
}

// out_r = beta * out_r + sign * sum_i coef[r][i] * Vb_i,r with the coefficients on the device
static void lincomb_dev(Handle* h, SolveWork& s, double2* out, const double2* Vb, int nv, const double2* coef,
                        double beta, double sign) {
    k_lincomb<<<dim3(blocks_for(s.N), s.nb), 256, 0, h->stream>>>(out, s.N, Vb, (int64_t)s.nb * s.N, s.N, coef, nv, nv,
                                                                   beta, s.N, sign);
}

static int norms(Handle* h, SolveWork& s, const double2* w, std::vector<double>& out) {
    std::vector<cdbl> t;
    const int64_t N = s.N;
    const int nblk = nblk_dots(N);
    k_dots<<<dim3(nblk, s.nb), DOT_THREADS, 0, h->stream>>>(w, N, N, w, N, 1, N, static_cast<double2*>(s.part.p), nblk);
    k_dots_reduce<<<dim3(1, s.nb), 256, 0, h->stream>>>(static_cast<double2*>(s.part.p), nblk, 1,
                                                        static_cast<double2*>(s.hbuf.p));
    t.resize(s.nb);
    SVH_CUDA_TRY(h, cudaMemcpyAsync(t.data(), s.hbuf.p, t.size() * 16, cudaMemcpyDeviceToHost, h->stream));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    out.resize(s.nb);
    for (int r = 0; r < s.nb; ++r) out[r] = std::sqrt(std::max(t[r].real(), 0.0));
    return SVH_OK;
}

// out = P in (Eq. 13-15) for the nb contiguous vectors of `in`; S^{-1} on the host
static int apply_precond(Handle* h, SolveWork& s, const double2* in, double2* out) {
    const int64_t K = h->K, M = h->M, N = s.N;
    const int nf = s.nf;
    k_prec_pre<<<dim3(blocks_for(nf), s.nb), 256, 0, h->stream>>>(in, N, K, static_cast<double*>(s.Yd.p), s.per_freq,
                                                                     static_cast<int32_t*>(s.freenodes.p), nf,
                                                                     static_cast<int32_t*>(h->d_ninc.p),
                                                                     static_cast<double2*>(s.E.p));
    if (s.amg_dev) {
        if (int rc = precond_schur_solve_dev(h, s.nb, s.per_freq, s.E.p, s.Bs.p)) return rc;
    } else {
        std::vector<double> e((size_t)s.nb * nf * 2), b((size_t)s.nb * nf * 2);
        SVH_CUDA_TRY(h, cudaMemcpyAsync(e.data(), s.E.p, e.size() * 8, cudaMemcpyDeviceToHost, h->stream));
        SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        int rc = precond_schur_solve(h, s.nb, s.per_freq, e.data(), b.data());
        if (rc) return rc;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(s.Bs.p, b.data(), b.size() * 8, cudaMemcpyHostToDevice, h->stream));
    }
    k_prec_post_vox<<<dim3(blocks_for(5 * K), s.nb), 256, 0, h->stream>>>(
        in, out, N, K, static_cast<double*>(s.Yd.p), s.per_freq, static_cast<int32_t*>(h->d_node.p),
        static_cast<int32_t*>(s.freeid.p), static_cast<double2*>(s.Bs.p), nf);
    k_prec_post_node<<<dim3(blocks_for(M), s.nb), 256, 0, h->stream>>>(in, out, N, K, M,
                                                                        static_cast<int32_t*>(s.freeid.p),
                                                                        static_cast<double2*>(s.Bs.p), nf);
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

// y = Kt x (masked operator): FP64 product, or FP32 product with conversions
static int apply_op(Handle* h, SolveWork& s, double omega, const double2* x, double2* y, int prec, int masked = 1) {
    const int64_t n = (int64_t)s.nb * s.N;
    const double* dom = static_cast<const double*>(s.om.p);
    if (prec == SVH_FP64) return launch_matvec64(h, omega, s.nb, x, y, masked, dom);
    float2* a = static_cast<float2*>(s.T32a.p);
    float2* b = static_cast<float2*>(s.T32b.p);
    k_to32<<<blocks_for(n), 256, 0, h->stream>>>(x, a, n);
    int rc = launch_matvec32(h, omega, s.nb, a, b, masked, dom);
    if (rc) return rc;
    k_to64<<<blocks_for(n), 256, 0, h->stream>>>(b, y, n);
    return SVH_OK;
}

// Flexible GMRES(m) for Kt D = R with right preconditioning; D in s.D.
// Stops right-hand side r when its estimated residual is <= tol[r] * ||R_r||.
// Each Arnoldi step runs entirely on the device: preconditioner, product, two Gram-Schmidt
// passes, the norm, the Hessenberg column with its Givens rotation and the rotated residual
// (k_arnoldi_givens); per step the host reads one int, how many right-hand sides are still
// above their tolerance (a pinned copy behind an event), to stop the cycle. The restart's
// small least-squares solve is k_arnoldi_backsolve.
static int fgmres(Handle* h, SolveWork& s, double omega, int prec, const std::vector<double>& tol, int maxit,
                  int& iters_out) {
    const int nb = s.nb, m = s.m;
    const int64_t N = s.N, blk = (int64_t)nb * N;
    double2* V = static_cast<double2*>(s.V.p);
    double2* Z = static_cast<double2*>(s.Z.p);
    double2* W = static_cast<double2*>(s.W.p);
    double2* Dd = static_cast<double2*>(s.D.p);
    double2* Rr = static_cast<double2*>(s.R.p);
    double2* Hh = static_cast<double2*>(s.Hh.p);
    double2* Hg = static_cast<double2*>(s.Hg.p);
    double2* h1 = static_cast<double2*>(s.Hh1.p);
    double2* h2 = static_cast<double2*>(s.Hh2.p);
    double2* hn = static_cast<double2*>(s.Hn.p);
    int* act = static_cast<int*>(s.Hact.p);
    const unsigned tb = 128, nbk = (unsigned)((nb + tb - 1) / tb);
    SVH_CUDA_TRY(h, cudaMemsetAsync(Dd, 0, (size_t)blk * 16, h->stream));
    std::vector<double> beta0;
    int rc = norms(h, s, Rr, beta0);
    if (rc) return rc;
    SVH_CUDA_TRY(h, cudaMemcpyAsync(s.Htol.p, tol.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, h->stream));
    SVH_CUDA_TRY(h, cudaMemcpyAsync(s.Hb0.p, beta0.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, h->stream));
    // V_0 slot temporarily holds the current residual
    SVH_CUDA_TRY(h, cudaMemcpyAsync(V, Rr, (size_t)blk * 16, cudaMemcpyDeviceToDevice, h->stream));
    int it = 0;
    while (true) {
        std::vector<double> beta;
        if ((rc = norms(h, s, V, beta))) return rc;
        std::vector<int> done(nb);
        bool all = true;
        for (int r = 0; r < nb; ++r) {
            done[r] = beta[r] <= tol[r] * beta0[r] || beta0[r] == 0;
            all = all && done[r];
        }
        if (all || it >= maxit) break;
        std::vector<double> inv(nb);
        for (int r = 0; r < nb; ++r) inv[r] = beta[r] > 0 ? 1.0 / beta[r] : 0.0;
        std::vector<cdbl> g0((size_t)nb * (m + 1), 0.0);
        for (int r = 0; r < nb; ++r) g0[(size_t)r * (m + 1)] = beta[r];
        SVH_CUDA_TRY(h, cudaMemcpyAsync(s.scl.p, inv.data(), nb * 8, cudaMemcpyHostToDevice, h->stream));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(s.Hdone.p, done.data(), nb * 4, cudaMemcpyHostToDevice, h->stream));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(Hg, g0.data(), g0.size() * 16, cudaMemcpyHostToDevice, h->stream));
        k_scale<<<dim3(blocks_for(N), nb), 256, 0, h->stream>>>(V, N, V, N, static_cast<double*>(s.scl.p), N);
        int kk = 0;
        for (int k = 0; k < m && it < maxit; ++k) {
            double2* Vk = V + k * blk;
            double2* Zk = Z + k * blk;
            if ((rc = apply_precond(h, s, Vk, Zk))) return rc;
            if ((rc = apply_op(h, s, omega, Zk, W, prec))) return rc;
            // classical Gram-Schmidt, twice, with the coefficients kept on the device
            dots_dev(h, s, V, blk, k + 1, W, h1);
            lincomb_dev(h, s, W, V, k + 1, h1, 1.0, -1.0);
            dots_dev(h, s, V, blk, k + 1, W, h2);
            lincomb_dev(h, s, W, V, k + 1, h2, 1.0, -1.0);
            dots_dev(h, s, W, N, 1, W, hn);
            SVH_CUDA_TRY(h, cudaMemsetAsync(act + (k & 1), 0, sizeof(int), h->stream));
            k_arnoldi_givens<<<nbk, tb, 0, h->stream>>>(Hh, static_cast<double2*>(s.Hcs.p),
                                                        static_cast<double2*>(s.Hsn.p), Hg, h1, h2, hn, k, m, nb,
                                                        static_cast<double*>(s.Htol.p), static_cast<double*>(s.Hb0.p),
                                                        static_cast<int*>(s.Hdone.p), static_cast<double*>(s.scl.p),
                                                        act + (k & 1));
            k_scale<<<dim3(blocks_for(N), nb), 256, 0, h->stream>>>(V + (k + 1) * blk, N, W, N,
                                                                    static_cast<double*>(s.scl.p), N);
            SVH_CUDA_TRY(h, cudaMemcpyAsync(s.pin + (k & 1), act + (k & 1), sizeof(int), cudaMemcpyDeviceToHost,
                                            h->stream));
            SVH_CUDA_TRY(h, cudaEventRecord(s.ev[k & 1], h->stream));
            ++it;
            kk = k + 1;
            // the one value the host reads per step: how many right-hand sides are still above
            // their tolerance (a step costs a preconditioner apply, far longer than this wait)
            SVH_CUDA_TRY(h, cudaEventSynchronize(s.ev[k & 1]));
            if (s.pin[k & 1] == 0) break;
        }
        // y from the triangular systems; D += sum_i y_i Z_i
        k_arnoldi_backsolve<<<nbk, tb, 0, h->stream>>>(Hh, Hg, static_cast<double2*>(s.Hy.p), kk, m, nb,
                                                       static_cast<int*>(s.Hdone.p));
        lincomb_dev(h, s, Dd, Z, kk, static_cast<double2*>(s.Hy.p), 1.0, 1.0);
        // residual of the correction problem for the restart: V_0 <- R - Kt D
        if ((rc = apply_op(h, s, omega, Dd, W, prec))) return rc;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(V, Rr, (size_t)blk * 16, cudaMemcpyDeviceToDevice, h->stream));
        k_sub<<<blocks_for(blk), 256, 0, h->stream>>>(V, W, blk);
    }
    iters_out = it;
    SVH_CUDA_TRY(h, cudaGetLastError());
    return SVH_OK;
}

static int alloc_work(Handle* h, SolveWork& s, int nb, int m) {
    s.nb = nb;
    s.m = m;
    s.N = 5 * h->K + h->M;
    const size_t blk = (size_t)nb * s.N;
    int rc;
    if ((rc = dev_alloc(h, s.X, blk * 16)) || (rc = dev_alloc(h, s.B, blk * 16)) || (rc = dev_alloc(h, s.R, blk * 16)) ||
        (rc = dev_alloc(h, s.W, blk * 16)) || (rc = dev_alloc(h, s.D, blk * 16)) ||
        (rc = dev_alloc(h, s.V, (size_t)(m + 1) * blk * 16)) || (rc = dev_alloc(h, s.Z, (size_t)m * blk * 16)) ||
        (rc = dev_alloc(h, s.T32a, blk * 8)) || (rc = dev_alloc(h, s.T32b, blk * 8)) ||
        (rc = dev_alloc(h, s.part, (size_t)nblk_dots(s.N) * nb * (m + 1) * 16)) ||
        (rc = dev_alloc(h, s.hbuf, (size_t)nb * (m + 1) * 16)) || (rc = dev_alloc(h, s.scl, (size_t)nb * 8)) ||
        (rc = dev_alloc(h, s.Hh, (size_t)nb * (m + 1) * m * 16)) || (rc = dev_alloc(h, s.Hcs, (size_t)nb * m * 16)) ||
        (rc = dev_alloc(h, s.Hsn, (size_t)nb * m * 16)) || (rc = dev_alloc(h, s.Hg, (size_t)nb * (m + 1) * 16)) ||
        (rc = dev_alloc(h, s.Hh1, (size_t)nb * (m + 1) * 16)) || (rc = dev_alloc(h, s.Hh2, (size_t)nb * (m + 1) * 16)) ||
        (rc = dev_alloc(h, s.Hn, (size_t)nb * 16)) || (rc = dev_alloc(h, s.Hy, (size_t)nb * m * 16)) ||
        (rc = dev_alloc(h, s.Htol, (size_t)nb * 8)) || (rc = dev_alloc(h, s.Hb0, (size_t)nb * 8)) ||
        (rc = dev_alloc(h, s.Hdone, (size_t)nb * 4)) || (rc = dev_alloc(h, s.Hact, 2 * sizeof(int))))
        return rc;
    SVH_CUDA_TRY(h, cudaHostAlloc(reinterpret_cast<void**>(&s.pin), 2 * sizeof(int), cudaHostAllocDefault));
    for (cudaEvent_t& e : s.ev) SVH_CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return SVH_OK;
}

}  // namespace svh

using namespace svh;

extern "C" {

void svh_default_options(svh_options* o) {
    if (!o) return;
    o->restart = 50;
    o->max_iterations = 2000;
    o->max_refinements = 8;
    o->inner_precision = SVH_FP32;
    o->rre = 1e-8;
    o->amg_tol = 1e-8;
    o->amg_on_device = 1;
}

int svh_solve(svh_handle* hh, const double* omegas, int nfreq, const svh_options* opt_in, double* Zport,
              double* Lport, svh_stats* st) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    cudaError_t ce = cudaSetDevice(h->device);
    if (ce != cudaSuccess) return cuda_err(h, ce, "cudaSetDevice");
    if (!h->have_grid || !h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_solve: grid and kernels needed");
    const int np = (int)h->port_plus.size();
    if (np == 0) return set_err(h, SVH_ERR_STATE, "svh_solve: the grid has no ports");
    if (!omegas || nfreq <= 0 || !Zport) return set_err(h, SVH_ERR_ARG, "svh_solve: bad frequencies or output");
    svh_options opt;
    svh_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.restart < 1 || opt.restart > 500 || !(opt.rre > 0) || !(opt.amg_tol > 0) || opt.max_iterations < 1 ||
        opt.max_refinements < 1 || (opt.inner_precision != SVH_FP32 && opt.inner_precision != SVH_FP64) ||
        (opt.amg_on_device != 0 && opt.amg_on_device != 1))
        return set_err(h, SVH_ERR_ARG, "svh_solve: bad options");
    for (int f = 0; f < nfreq; ++f)
        if (!(omegas[f] > 0) || !std::isfinite(omegas[f])) return set_err(h, SVH_ERR_ARG, "svh_solve: omega must be > 0");
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t K = h->K, M = h->M, N = 5 * K + M;
    // every (frequency, port) pair is one item of the batch: item r = f * np + p
    const int nb = np * nfreq;
    SolveWork s;
    s.per_freq = np;
    s.amg_dev = opt.amg_on_device;
    int rc = alloc_work(h, s, nb, opt.restart);
    if (rc) return rc;
    // right-hand sides: b_I = A_T^T Phi_T with Phi = 1 on the plus nodes of port p (same at every frequency)
    std::vector<cdbl> bh((size_t)nb * N, 0.0);
    std::vector<uint8_t> plus(M);
    for (int j = 0; j < np; ++j) {
        std::fill(plus.begin(), plus.end(), 0);
        for (int32_t m : h->port_plus[j]) plus[m] = 1;
        for (int64_t v = 0; v < K; ++v)
            for (int a = 0; a < 5; ++a) {
                double acc = 0;
                for (int f = 0; f < 6; ++f)
                    if (plus[h->node[v * 6 + f]]) acc += kFluxH[a][f];
                for (int f = 0; f < nfreq; ++f) bh[((size_t)f * np + j) * N + a * K + v] = acc;
            }
    }
    SVH_CUDA_TRY(h, cudaMemcpyAsync(s.B.p, bh.data(), bh.size() * 16, cudaMemcpyHostToDevice, h->stream));
    std::vector<double> item_om(nb);
    for (int r = 0; r < nb; ++r) item_om[r] = omegas[r / np];
    if ((rc = dev_upload(h, s.om, item_om.data(), (size_t)nb * 8))) return rc;
    // preconditioners: one Schur complement and AMG hierarchy per frequency (Y depends on omega)
    const auto ts = std::chrono::steady_clock::now();
    if ((rc = precond_setup(h, omegas, nfreq, opt.amg_tol))) return rc;
    int nf = 0;
    const int* fn = precond_free_nodes(h, &nf);
    s.nf = nf;
    std::vector<int32_t> fid(M, -1);
    for (int i = 0; i < nf; ++i) fid[fn[i]] = i;
    std::vector<double> Yall((size_t)nfreq * 5 * K);
    for (int f = 0; f < nfreq; ++f) std::memcpy(Yall.data() + (size_t)f * 5 * K, precond_Y(h, f), (size_t)5 * K * 8);
    if ((rc = dev_upload(h, s.Yd, Yall.data(), Yall.size() * 8)) ||
        (rc = dev_upload(h, s.freenodes, fn, (size_t)std::max(nf, 1) * 4)) ||
        (rc = dev_upload(h, s.freeid, fid.data(), (size_t)M * 4)) ||
        (rc = dev_alloc(h, s.E, (size_t)nb * std::max(nf, 1) * 16)) ||
        (rc = dev_alloc(h, s.Bs, (size_t)nb * std::max(nf, 1) * 16)))
        return rc;
    const double setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
    int total_it = 0, total_ref = 0;
    int status = SVH_OK;
    std::vector<double> bnorm;
    if ((rc = norms(h, s, static_cast<double2*>(s.B.p), bnorm))) return rc;
    double2* X = static_cast<double2*>(s.X.p);
    double2* R = static_cast<double2*>(s.R.p);
    double2* W = static_cast<double2*>(s.W.p);
    const int64_t blk = (int64_t)nb * N;
    SVH_CUDA_TRY(h, cudaMemsetAsync(X, 0, blk * 16, h->stream));
    std::vector<double> rn;
    double rel = 1.0;
    for (int ref = 0; ref <= opt.max_refinements; ++ref) {
        // true residual with the FP64 product
        if ((rc = apply_op(h, s, omegas[0], X, W, SVH_FP64))) return rc;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(R, s.B.p, blk * 16, cudaMemcpyDeviceToDevice, h->stream));
        k_sub<<<blocks_for(blk), 256, 0, h->stream>>>(R, W, blk);
        if ((rc = norms(h, s, R, rn))) return rc;
        rel = 0;
        for (int r = 0; r < nb; ++r) rel = std::max(rel, bnorm[r] > 0 ? rn[r] / bnorm[r] : 0.0);
        if (rel <= opt.rre || ref == opt.max_refinements) break;
        std::vector<double> tol(nb);
        for (int r = 0; r < nb; ++r) {
            const double need = rn[r] > 0 ? 0.5 * opt.rre * bnorm[r] / rn[r] : 1.0;
            tol[r] = opt.inner_precision == SVH_FP64 ? need : std::max(need, 1e-5);
        }
        int its = 0;
        if ((rc = fgmres(h, s, omegas[0], opt.inner_precision, tol, opt.max_iterations, its))) return rc;
        total_it += its;
        ++total_ref;
        k_add<<<blocks_for(blk), 256, 0, h->stream>>>(X, static_cast<double2*>(s.D.p), blk);
    }
    if (rel > opt.rre) status = SVH_ERR_NOT_CONVERGED;
    // port admittance from the node rows of the unmasked product (A I)
    if ((rc = apply_op(h, s, omegas[0], X, W, SVH_FP64, 0))) return rc;
    std::vector<cdbl> w(blk);
    SVH_CUDA_TRY(h, cudaMemcpyAsync(w.data(), W, blk * 16, cudaMemcpyDeviceToHost, h->stream));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (int f = 0; f < nfreq; ++f) {
        std::vector<cdbl> Y((size_t)np * np);
        for (int j = 0; j < np; ++j)
            for (int p = 0; p < np; ++p) {
                cdbl acc = 0;
                for (int32_t m : h->port_plus[p]) acc += w[((size_t)f * np + j) * N + 5 * K + m];
                Y[(size_t)p * np + j] = acc;
            }
        // Z = Y^{-1} by Gauss-Jordan with partial pivoting
        std::vector<cdbl> A(Y), Zi((size_t)np * np, 0.0);
        for (int i = 0; i < np; ++i) Zi[(size_t)i * np + i] = 1.0;
        for (int c = 0; c < np; ++c) {
            int piv = c;
            for (int r = c + 1; r < np; ++r)
                if (std::abs(A[(size_t)r * np + c]) > std::abs(A[(size_t)piv * np + c])) piv = r;
            if (std::abs(A[(size_t)piv * np + c]) == 0) return set_err(h, SVH_ERR_SINGULAR, "svh_solve: singular port admittance");
            for (int k = 0; k < np; ++k) {
                std::swap(A[(size_t)c * np + k], A[(size_t)piv * np + k]);
                std::swap(Zi[(size_t)c * np + k], Zi[(size_t)piv * np + k]);
            }
            const cdbl d = A[(size_t)c * np + c];
            for (int k = 0; k < np; ++k) { A[(size_t)c * np + k] /= d; Zi[(size_t)c * np + k] /= d; }
            for (int r = 0; r < np; ++r) {
                if (r == c) continue;
                const cdbl fct = A[(size_t)r * np + c];
                if (fct == cdbl(0)) continue;
                for (int k = 0; k < np; ++k) {
                    A[(size_t)r * np + k] -= fct * A[(size_t)c * np + k];
                    Zi[(size_t)r * np + k] -= fct * Zi[(size_t)c * np + k];
                }
            }
        }
        for (int i = 0; i < np * np; ++i) {
            Zport[((size_t)f * np * np + i) * 2] = Zi[i].real();
            Zport[((size_t)f * np * np + i) * 2 + 1] = Zi[i].imag();
            // the port inductance L = Im(Z) / omega (Sec. II.A, the quantity of Sec. III's error)
            if (Lport) Lport[(size_t)f * np * np + i] = Zi[i].imag() / omegas[f];
        }
    }
    // keep the solutions of the last frequency (host) for svh_get_solution and the adjoint
    const int flast = nfreq - 1;
    h->last_x.resize((size_t)np * N * 2);
    SVH_CUDA_TRY(h, cudaMemcpyAsync(h->last_x.data(), X + (int64_t)flast * np * N, (size_t)np * N * 16,
                                    cudaMemcpyDeviceToHost, h->stream));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->last_nb = np;
    h->last_omega = omegas[flast];
    h->last_Z.assign(Zport + (size_t)flast * np * np * 2, Zport + (size_t)(flast + 1) * np * np * 2);
    if (st) {
        st->iterations = total_it;
        st->refinements = total_ref;
        st->amg_levels = precond_levels(h);
        st->amg_avg_iterations = precond_avg_iters(h);
        st->final_rre = rel;
        st->setup_seconds = setup_s;
        st->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() - setup_s;
    }
    if (status) set_err(h, status, "svh_solve: relative residual above rre after the refinement budget");
    return status;
}

int svh_get_solution(const svh_handle* hh, int port, double* x) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !x) return SVH_ERR_ARG;
    if (h->last_nb == 0) return SVH_ERR_STATE;
    if (port < 0 || port >= h->last_nb) return SVH_ERR_ARG;
    const int64_t N = 5 * h->K + h->M;
    std::memcpy(x, h->last_x.data() + (size_t)port * N * 2, (size_t)N * 16);
    return SVH_OK;
}

int svh_precond_apply(svh_handle* hh, double omega, int nb, const double* in, double* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !in || !out || nb <= 0 || !(omega > 0)) return SVH_ERR_ARG;
    int rc = precond_setup(h, &omega, 1, 1e-12);
    if (rc) return rc;
    return precond_apply_host(h, nb, in, out);
}

}  // extern "C"
