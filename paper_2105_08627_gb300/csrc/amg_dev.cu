// amg_dev.cu -- the Schur solves of the preconditioner on the device.
//
// Sec. II.C applies P = Q^{-1} through S = A Y^{-1} A^T; its solves
// b = S^{-1} e (Eq. 14) run by AMG-preconditioned conjugate gradients, the
// per-iteration cost the paper attributes to its host AMG. Here the hierarchy
// built on the host (amg.cpp: pairwise aggregation, Galerkin operators, l1
// row norms, Cholesky factor of the coarsest level) is copied to the device
// once per frequency, and the flexible CG with its K-cycle runs there:
//   * a complex right-hand side is two real systems; they travel together as
//     double2 (x: the real part's system, y: the imaginary part's) and every
//     scalar of the iteration is a double2, one value per real system;
//   * the K-cycle's Krylov acceleration always takes both inner steps (the
//     host version skips the second when the first reduced the residual 4x),
//     so nothing waits for the host; the 2 x 2 Galerkin combination falls back
//     to the first step when the second adds nothing; levels below 8000
//     unknowns take one plain cycle (their launches are latency-bound and
//     the two steps would double the visits of every level below);
//   * smoothing, residual and restriction are one kernel (pre), and
//     prolongation, residual and the second smoothing sweep another (post);
//     the right-hand side b - a1 w1 and the coarse correction c1 v1 + c2 v2
//     are formed inside the kernels that read them;
//   * dot products finish in the last block to complete, summing the block
//     partials in index order (results do not depend on block scheduling);
//   * the coarsest level is solved by its dense inverse (from the host
//     Cholesky factor): one matrix-vector product;
//   * the K-cycle is a preconditioner inside flexible CG, so it runs in FP32
//     (matrices, vectors and arithmetic; its dot products accumulate in
//     FP64), while the CG itself (S p, residuals, iterates) stays FP64: the
//     cycle's gathers move half the bytes and its arithmetic avoids the slow
//     FP64 units of this GPU.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "svh_internal.h"

namespace svh {

namespace {

constexpr int TPB = 256;
constexpr int kKrylovMinRows = 8000;   // levels below this size take one plain cycle

__device__ __forceinline__ double2 d2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return d2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return d2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul(double2 a, double2 b) { return d2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 scl(double s, double2 a) { return d2(s * a.x, s * a.y); }

// FP32 pairs: the K-cycle (a preconditioner inside flexible CG) runs in FP32
// data and arithmetic; its dot products accumulate in FP64
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fmul(float2 a, float2 b) { return f2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 fscl(float s, float2 a) { return f2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 tof(double2 a) { return f2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 dprod(float2 a, float2 b) {
    return d2((double)a.x * (double)b.x, (double)a.y * (double)b.y);
}

// a right-hand side read on the fly: b - coef * w (w may be null)
struct VRef {
    const float2* b;
    const float2* w;
    const double2* coef;   // [nrhs]
};

__device__ __forceinline__ float2 vget(const VRef& B, int64_t off, float2 cf) {
    float2 v = B.b[off];
    if (B.w) v = fsub(v, fmul(cf, B.w[off]));
    return v;
}

// the coarse correction read on the fly: v1 (plain) or c1 v1 + c2 v2
struct XRef {
    const float2* v1;
    const float2* v2;
    const double2* c1;     // [nrhs] or null (plain)
    const double2* c2;
};

// per-level scalar slots, each [nrhs] double2
enum { S_D11 = 0, S_G1, S_A1, S_C1, S_C2, NSLOT };
// top-level CG slots
enum { F_BETA = 0, F_PQ, F_PQOLD, F_ALPHA, F_RR, F_BB, F_ACTIVE, F_ITERS, NFSLOT };

// ---- thread layout
// Vectors are [row][rhs] (all right-hand sides of a row side by side). A
// kernel over `rows` units (rows, or aggregates for the restriction) gives
// each (unit, rhs) a group of G lanes: lane = (u * nrhs + rhs) * G + sub, with
// U = TPB / (G nrhs) units per block pass and the blocks striding over the
// unit blocks. A thread's rhs is fixed, so its dot-product terms accumulate in
// registers; the lanes of a row's groups read the same matrix entries (one
// transaction) and gather contiguous [rhs] values.
struct Lanes {
    int sub, rhs, uloc, U;
    bool live;   // this lane belongs to a (unit, rhs) slot
};

__device__ __forceinline__ Lanes lanes(int G, int nrhs) {
    Lanes l;
    const int per = G * nrhs;
    l.U = TPB / per;
    l.live = (int)threadIdx.x < l.U * per;
    l.sub = threadIdx.x % G;
    l.rhs = (threadIdx.x / G) % nrhs;
    l.uloc = threadIdx.x / per;
    return l;
}

// In-place tree sum of the rows of red[rows][W] (shared) into red[0][*], in a
// fixed order (deterministic); every thread of the block calls it.
__device__ void reduce_rows(double2* red, int rows, int W) {
    int st = 1;
    while (st < rows) st <<= 1;
    for (st >>= 1; st > 0; st >>= 1) {
        __syncthreads();
        for (int q = threadIdx.x; q < st * W; q += TPB) {
            const int u = q / W, c = q - u * W;
            if (u + st < rows) red[u * W + c] = add(red[u * W + c], red[(u + st) * W + c]);
        }
    }
    __syncthreads();
}

// Block sums of the ND per-thread values of each rhs (the leader lane, sub 0,
// of every (unit, rhs) slot), then the last block to finish sums the block
// partials; both sums are fixed-shape trees, so the results do not depend on
// scheduling. Returns true in the last block with tot[rhs * ND + k] (shared)
// filled; the other blocks return false.
template <int ND>
__device__ bool block_sums_last(const double2 (&val)[ND], int G, int nrhs, double2* part, unsigned* cnt,
                                double2* tot) {
    __shared__ double2 red[TPB * ND];
    __shared__ bool last;
    const int W = nrhs * ND, U = TPB / (G * nrhs);
    const int sub = threadIdx.x % G, rhs = (threadIdx.x / G) % nrhs, uloc = threadIdx.x / (G * nrhs);
    if (sub == 0 && uloc < U)
#pragma unroll
        for (int k = 0; k < ND; ++k) red[uloc * W + rhs * ND + k] = val[k];
    reduce_rows(red, U, W);
    for (int q = threadIdx.x; q < W; q += TPB) part[(int64_t)blockIdx.x * W + q] = red[q];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int R = TPB / W;   // rows of partial sums, each over the blocks b = row (mod R)
    if ((int)threadIdx.x < R * W) {
        const int row = threadIdx.x / W, c = threadIdx.x - row * W;
        double2 acc = d2(0, 0);
        for (unsigned b = row; b < gridDim.x; b += R) acc = add(acc, __ldcg(part + (int64_t)b * W + c));
        red[row * W + c] = acc;
    }
    reduce_rows(red, R, W);
    for (int q = threadIdx.x; q < W; q += TPB) tot[q] = red[q];
    __syncthreads();
    if (threadIdx.x == 0) *cnt = 0;   // ready for the next launch
    return true;
}

// Sparse rows are taken by groups of G lanes (G = 1 .. 32: one lane per
// (row, rhs) on the large fine levels, more on the small coarse levels with
// long Galerkin rows): lane `sub` takes the row's entries sub, sub + G, ...;
// the group's partial sums meet in one shuffle reduction after the loops
// (every lane reaches it, so the shuffles stay convergent).
template <int G, typename V>
__device__ __forceinline__ V group_sum(V v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o, G);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o, G);
    }
    return v;   // complete in the group's lane 0
}

__device__ __forceinline__ float2 xcget(const XRef& X, int64_t idx, float2 c1, float2 c2) {
    if (!X.c1) return X.v1[idx];
    return fadd(fmul(c1, X.v1[idx]), fmul(c2, X.v2[idx]));
}

// K-cycle, first half: x0 = b / l1 (one l1-Jacobi sweep from zero), the
// residual b - A x0 and its restriction to the aggregates (sum over each);
// one lane group per (aggregate, rhs).
template <int G>
__global__ void __launch_bounds__(TPB) k_kc_pre(int n, int nc, int nrhs, const int* __restrict__ rp,
                                                const int* __restrict__ ci, const float* __restrict__ v,
                                                const float* __restrict__ l1inv, const int* __restrict__ crp,
                                                const int* __restrict__ cidx, VRef B, float2* __restrict__ rc) {
    const Lanes L = lanes(G, nrhs);
    const float2 cf = B.w ? tof(B.coef[L.rhs]) : f2(0, 0);
    for (int64_t ub = blockIdx.x; ub * L.U < nc; ub += gridDim.x) {
        const int64_t c = ub * L.U + L.uloc;
        const bool act = L.live && c < nc;
        float2 s = f2(0, 0);
        if (act) {
            for (int p = crp[c]; p < crp[c + 1]; ++p) {
                const int i = cidx[p];
                if (L.sub == 0) s = fadd(s, vget(B, (int64_t)i * nrhs + L.rhs, cf));
                for (int q = rp[i] + L.sub; q < rp[i + 1]; q += G) {
                    const int j = ci[q];
                    s = fsub(s, fscl(v[q] * l1inv[j], vget(B, (int64_t)j * nrhs + L.rhs, cf)));
                }
            }
        }
        s = group_sum<G>(s);
        if (act && L.sub == 0) rc[c * nrhs + L.rhs] = s;
    }
}

// K-cycle, second half: x1 = b / l1 + P xc (coarse correction), then one more
// l1-Jacobi sweep x = x1 + (b - A x1) / l1; one lane group per (row, rhs).
template <int G>
__global__ void __launch_bounds__(TPB) k_kc_post(int n, int nrhs, const int* __restrict__ rp,
                                                 const int* __restrict__ ci, const float* __restrict__ v,
                                                 const float* __restrict__ l1inv, const int* __restrict__ agg, VRef B,
                                                 XRef XC, float2* __restrict__ X) {
    const Lanes L = lanes(G, nrhs);
    const float2 cf = B.w ? tof(B.coef[L.rhs]) : f2(0, 0);
    const float2 c1 = XC.c1 ? tof(XC.c1[L.rhs]) : f2(1, 1), c2 = XC.c2 ? tof(XC.c2[L.rhs]) : f2(0, 0);
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        const bool act = L.live && i < n;
        float2 ax = f2(0, 0);
        if (act) {
            for (int q = rp[i] + L.sub; q < rp[i + 1]; q += G) {
                const int j = ci[q];
                const int64_t jx = (int64_t)j * nrhs + L.rhs;
                const float2 xj = fadd(fscl(l1inv[j], vget(B, jx, cf)), xcget(XC, (int64_t)agg[j] * nrhs + L.rhs, c1, c2));
                ax = fadd(ax, fscl(v[q], xj));
            }
        }
        ax = group_sum<G>(ax);
        if (act && L.sub == 0) {
            const int64_t ix = i * nrhs + L.rhs;
            const float2 bi = vget(B, ix, cf);
            const float2 xi = fadd(fscl(l1inv[i], bi), xcget(XC, (int64_t)agg[i] * nrhs + L.rhs, c1, c2));
            X[ix] = fadd(xi, fscl(l1inv[i], fsub(bi, ax)));
        }
    }
}

// coarsest level: X = C^{-1} b, one warp per (row, rhs)
__global__ void k_dense(int n, int nrhs, const float* __restrict__ cinv, const float2* __restrict__ b,
                        float2* __restrict__ X) {
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)n * nrhs) return;
    const int row = (int)(w / nrhs), r = (int)(w % nrhs);
    const float* cr = cinv + (int64_t)row * n;
    float x = 0, y = 0;
    for (int j = lane; j < n; j += 32) {
        const float c = cr[j];
        const float2 bj = b[(int64_t)j * nrhs + r];
        x += c * bj.x;
        y += c * bj.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0) X[(int64_t)row * nrhs + r] = f2(x, y);
}

// w = A vin with dot products; MODE 1 (first Krylov step): d11 = v1.w,
// g1 = v1.b -> a1 = g1 / d11. MODE 2 (second): d12 = v1.w, d22 = v2.w,
// g2 = v2.b -> (c1, c2) minimising the A-norm of the error over span{v1, v2}.
template <int MODE, int G>
__global__ void __launch_bounds__(TPB) k_kc_spmv(int n, int nrhs, const int* __restrict__ rp,
                                                 const int* __restrict__ ci, const float* __restrict__ v,
                                                 const float2* __restrict__ vin, const float2* __restrict__ v1,
                                                 const float2* __restrict__ b, float2* __restrict__ w,
                                                 double2* part, unsigned* cnt, double2* sc) {
    constexpr int ND = MODE == 1 ? 2 : 3;
    __shared__ double2 tot[64 * ND];
    const Lanes L = lanes(G, nrhs);
    double2 val[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) val[k] = d2(0, 0);
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        const bool act = L.live && i < n;
        float2 ax = f2(0, 0);
        if (act)
            for (int q = rp[i] + L.sub; q < rp[i + 1]; q += G)
                ax = fadd(ax, fscl(v[q], vin[(int64_t)ci[q] * nrhs + L.rhs]));
        ax = group_sum<G>(ax);
        if (act && L.sub == 0) {
            const int64_t ix = i * nrhs + L.rhs;
            w[ix] = ax;
            const float2 vi = vin[ix], bi = b[ix];
            if (MODE == 1) {
                val[0] = add(val[0], dprod(vi, ax));
                val[1] = add(val[1], dprod(vi, bi));
            } else {
                val[0] = add(val[0], dprod(v1[ix], ax));
                val[1] = add(val[1], dprod(vi, ax));
                val[2] = add(val[2], dprod(vi, bi));
            }
        }
    }
    if (!block_sums_last<ND>(val, G, nrhs, part, cnt, tot)) return;
    for (int r = threadIdx.x; r < nrhs; r += TPB) {
        double2* s = sc;
        if (MODE == 1) {
            const double2 d11 = tot[r * ND], g1 = tot[r * ND + 1];
            s[S_D11 * nrhs + r] = d11;
            s[S_G1 * nrhs + r] = g1;
            s[S_A1 * nrhs + r] = d2(d11.x > 0 ? g1.x / d11.x : 0.0, d11.y > 0 ? g1.y / d11.y : 0.0);
        } else {
            const double2 d11 = s[S_D11 * nrhs + r], g1 = s[S_G1 * nrhs + r], a1 = s[S_A1 * nrhs + r];
            const double2 d12 = tot[r * ND], d22 = tot[r * ND + 1], g2 = tot[r * ND + 2];
            double c1[2], c2[2];
            const double D11[2] = {d11.x, d11.y}, G1[2] = {g1.x, g1.y}, A1[2] = {a1.x, a1.y};
            const double D12[2] = {d12.x, d12.y}, D22[2] = {d22.x, d22.y}, G2[2] = {g2.x, g2.y};
            for (int k = 0; k < 2; ++k) {
                const double det = D11[k] * D22[k] - D12[k] * D12[k];
                if (det > 1e-14 * D11[k] * D22[k] && D11[k] > 0 && D22[k] > 0) {
                    c1[k] = (G1[k] * D22[k] - G2[k] * D12[k]) / det;
                    c2[k] = (D11[k] * G2[k] - D12[k] * G1[k]) / det;
                } else {
                    c1[k] = A1[k];
                    c2[k] = 0.0;
                }
            }
            s[S_C1 * nrhs + r] = d2(c1[0], c1[1]);
            s[S_C2 * nrhs + r] = d2(c2[0], c2[1]);
        }
    }
}

// ---- top-level flexible CG on S (one lane per (row, rhs))
// r = e (e given as [rhs][n]), x = 0, bb = e.e; a system with bb = 0 starts (and stays) inactive
__global__ void __launch_bounds__(TPB) k_fcg_init(int n, int nrhs, const double2* __restrict__ e,
                                                  double2* __restrict__ x, double2* __restrict__ rr, double2* part,
                                                  unsigned* cnt, double2* fs) {
    __shared__ double2 tot[64];
    const Lanes L = lanes(1, nrhs);
    double2 val[1] = {d2(0, 0)};
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        if (L.live && i < n) {
            const double2 ei = e[(int64_t)L.rhs * n + i];
            rr[i * nrhs + L.rhs] = ei;
            x[i * nrhs + L.rhs] = d2(0, 0);
            val[0] = add(val[0], mul(ei, ei));
        }
    }
    if (!block_sums_last<1>(val, 1, nrhs, part, cnt, tot)) return;
    for (int r = threadIdx.x; r < nrhs; r += TPB) {
        fs[F_BB * nrhs + r] = tot[r];
        fs[F_RR * nrhs + r] = tot[r];
        fs[F_ACTIVE * nrhs + r] = d2(tot[r].x > 0 ? 1.0 : 0.0, tot[r].y > 0 ? 1.0 : 0.0);
        fs[F_ITERS * nrhs + r] = d2(0, 0);
        fs[F_BETA * nrhs + r] = d2(0, 0);
        fs[F_PQOLD * nrhs + r] = d2(0, 0);
    }
}

// beta = (z . q_old) / (p_old . q_old): the new direction is S-orthogonal to the previous one
__global__ void __launch_bounds__(TPB) k_fcg_beta(int n, int nrhs, const double2* __restrict__ z,
                                                  const double2* __restrict__ qold, double2* part, unsigned* cnt,
                                                  double2* fs) {
    __shared__ double2 tot[64];
    const Lanes L = lanes(1, nrhs);
    double2 val[1] = {d2(0, 0)};
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        if (L.live && i < n) val[0] = add(val[0], mul(z[i * nrhs + L.rhs], qold[i * nrhs + L.rhs]));
    }
    if (!block_sums_last<1>(val, 1, nrhs, part, cnt, tot)) return;
    for (int r = threadIdx.x; r < nrhs; r += TPB) {
        const double2 pq = fs[F_PQOLD * nrhs + r];
        fs[F_BETA * nrhs + r] = d2(pq.x > 0 ? tot[r].x / pq.x : 0.0, pq.y > 0 ? tot[r].y / pq.y : 0.0);
    }
}

// p = z - beta p_old (p = z on the first iteration)
__global__ void k_fcg_dir(int64_t total, int nrhs, const double2* __restrict__ z, const double2* __restrict__ pold,
                          double2* __restrict__ p, const double2* __restrict__ fs, int first) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= total) return;
    p[o] = first ? z[o] : sub2(z[o], mul(fs[F_BETA * nrhs + (int)(o % nrhs)], pold[o]));
}

// q = S p, pq = p.q, alpha = (p.r) / pq for the active systems (0 for the others)
template <int G>
__global__ void __launch_bounds__(TPB) k_fcg_spmv(int n, int nrhs, const int* __restrict__ rp,
                                                  const int* __restrict__ ci, const double* __restrict__ v,
                                                  const double2* __restrict__ p, const double2* __restrict__ rr,
                                                  double2* __restrict__ q, double2* part, unsigned* cnt, double2* fs) {
    __shared__ double2 tot[64 * 2];
    const Lanes L = lanes(G, nrhs);
    double2 val[2] = {d2(0, 0), d2(0, 0)};
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        const bool act = L.live && i < n;
        double2 ax = d2(0, 0);
        if (act)
            for (int k = rp[i] + L.sub; k < rp[i + 1]; k += G) ax = add(ax, scl(v[k], p[(int64_t)ci[k] * nrhs + L.rhs]));
        ax = group_sum<G>(ax);
        if (act && L.sub == 0) {
            const int64_t ix = i * nrhs + L.rhs;
            q[ix] = ax;
            const double2 pi = p[ix];
            val[0] = add(val[0], mul(pi, ax));
            val[1] = add(val[1], mul(pi, rr[ix]));
        }
    }
    if (!block_sums_last<2>(val, G, nrhs, part, cnt, tot)) return;
    for (int r = threadIdx.x; r < nrhs; r += TPB) {
        const double2 act = fs[F_ACTIVE * nrhs + r];
        const double2 pq = tot[r * 2], pr = tot[r * 2 + 1];
        fs[F_PQ * nrhs + r] = pq;
        fs[F_ALPHA * nrhs + r] =
            d2(act.x > 0 && pq.x > 0 ? pr.x / pq.x : 0.0, act.y > 0 && pq.y > 0 ? pr.y / pq.y : 0.0);
    }
}

// x += alpha p, r -= alpha q; rr = r.r; a system stays active while ||r|| > tol ||e||
__global__ void __launch_bounds__(TPB) k_fcg_update(int n, int nrhs, const double2* __restrict__ p,
                                                    const double2* __restrict__ q, double2* __restrict__ x,
                                                    double2* __restrict__ rr, double2* part, unsigned* cnt,
                                                    double2* fs, double tol2) {
    __shared__ double2 tot[64];
    const Lanes L = lanes(1, nrhs);
    const double2 alpha = fs[F_ALPHA * nrhs + L.rhs];
    double2 val[1] = {d2(0, 0)};
    for (int64_t ub = blockIdx.x; ub * L.U < n; ub += gridDim.x) {
        const int64_t i = ub * L.U + L.uloc;
        if (L.live && i < n) {
            const int64_t ix = i * nrhs + L.rhs;
            const double2 xi = add(x[ix], mul(alpha, p[ix]));
            const double2 ri = sub2(rr[ix], mul(alpha, q[ix]));
            x[ix] = xi;
            rr[ix] = ri;
            val[0] = add(val[0], mul(ri, ri));
        }
    }
    if (!block_sums_last<1>(val, 1, nrhs, part, cnt, tot)) return;
    for (int r = threadIdx.x; r < nrhs; r += TPB) {
        const double2 bb = fs[F_BB * nrhs + r], act = fs[F_ACTIVE * nrhs + r];
        double2 it = fs[F_ITERS * nrhs + r];
        it.x += act.x;
        it.y += act.y;
        fs[F_ITERS * nrhs + r] = it;
        fs[F_RR * nrhs + r] = tot[r];
        fs[F_ACTIVE * nrhs + r] = d2(act.x > 0 && tot[r].x > tol2 * bb.x ? 1.0 : 0.0,
                                     act.y > 0 && tot[r].y > tol2 * bb.y ? 1.0 : 0.0);
        fs[F_PQOLD * nrhs + r] = fs[F_PQ * nrhs + r];
    }
}

// the K-cycle's FP32 input (r) and FP64 output (z)
__global__ void k_to_f32(int64_t total, const double2* __restrict__ a, float2* __restrict__ b) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < total) b[o] = tof(a[o]);
}
__global__ void k_to_f64(int64_t total, const float2* __restrict__ a, double2* __restrict__ b) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < total) b[o] = d2(a[o].x, a[o].y);
}

// solution out in the caller's [rhs][n] layout
__global__ void k_fcg_out(int n, int nrhs, const double2* __restrict__ x, double2* __restrict__ b) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (int64_t)n * nrhs) return;
    const int64_t i = o / nrhs;
    const int r = (int)(o % nrhs);
    b[(int64_t)r * n + i] = x[o];
}

// ---- device copy of one hierarchy
struct DLevel {
    int n = 0, nc = 0;
    double per_row = 1, per_agg = 1;   // mean entries per row, and per aggregate (restriction)
    bool krylov = true;          // coarse solves on this level take the two Krylov steps
    DevBuf rp, ci, v, agg, crp, cidx;   // v: FP64 values (the top-level CG product, level 0)
    DevBuf vf, l1f;                      // FP32 values and l1 norms for the K-cycle
    DevBuf v1, w1, v2, w2, rc;           // FP32 [n][nrhs] (rc: [nc][nrhs])
    DevBuf sc, part, cnt;        // scalar slots, block partials, completion counters
};

struct DevAmg {
    std::vector<DLevel> lv;
    DevBuf cinv;                 // dense inverse of the coarsest operator
    int nrhs = 0;                // capacity of the workspaces
    DevBuf fx, fr, fz, fp, fq, fpo, fqo, fs, fpart, fcnt;   // top-level CG (FP64)
    DevBuf kr, kz;               // FP32 K-cycle input (r) and output (z)
    double2* host_fs = nullptr;  // pinned copy of the CG slots
    cudaGraphExec_t ge[2] = {nullptr, nullptr};   // one CG iteration per parity
    int graph_nrhs = 0;
    double graph_tol2 = 0;
    // the solver's own stream (graphs cannot be captured on the legacy
    // default stream a caller may use), ordered after / before the caller's
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ~DevAmg() {
        if (st) cudaStreamDestroy(st);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        for (cudaGraphExec_t g : ge)
            if (g) cudaGraphExecDestroy(g);
        for (DLevel& L : lv)
            for (DevBuf* b : {&L.rp, &L.ci, &L.v, &L.vf, &L.l1f, &L.agg, &L.crp, &L.cidx, &L.v1, &L.w1, &L.v2,
                              &L.w2, &L.rc, &L.sc, &L.part, &L.cnt})
                dev_free(*b);
        for (DevBuf* b : {&cinv, &fx, &fr, &fz, &fp, &fq, &fpo, &fqo, &fs, &fpart, &fcnt, &kr, &kz}) dev_free(*b);
        if (host_fs) cudaFreeHost(host_fs);
    }
};

unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

constexpr int kMaxGrid = 152 * 8;   // blocks of a grid-striding kernel (and block partials)
constexpr int kMaxRhs = 64;         // right-hand sides per solve (complex; 2 real systems each)

// launch shape of a kernel over `units` units of `per` entries for nrhs right-hand sides:
// G lanes per (unit, rhs) -- one while the (unit, rhs) slots alone fill the GPU
// (~160 K threads), more on the small coarse levels (long Galerkin rows), at most one
// per entry and G nrhs <= TPB -- and the grid (capped: the blocks stride)
struct Geo {
    int G;
    unsigned grid;
};
Geo geo(int64_t units, double per, int nrhs) {
    int g = 1;
    while (g < 32 && g < per && (int64_t)g * units * nrhs < 160000 && 2 * g * nrhs <= TPB) g *= 2;
    const int U = TPB / (g * nrhs);
    const int64_t blocks = (units + U - 1) / U;
    return {g, (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, kMaxGrid))};
}

template <typename T>
T* P(DevBuf& b) { return static_cast<T*>(b.p); }

int upload(Handle* h, DevAmg& D, const AmgView& A) {
    SVH_CUDA_TRY(h, cudaStreamCreateWithFlags(&D.st, cudaStreamNonBlocking));
    SVH_CUDA_TRY(h, cudaEventCreateWithFlags(&D.ev_in, cudaEventDisableTiming));
    SVH_CUDA_TRY(h, cudaEventCreateWithFlags(&D.ev_out, cudaEventDisableTiming));
    const int nl = (int)A.lv.size();
    D.lv.resize(nl);
    for (int l = 0; l < nl; ++l) {
        const AmgLevelView& V = A.lv[l];
        DLevel& L = D.lv[l];
        L.n = V.n;
        L.nc = l + 1 < nl ? V.nc : 0;
        const int nnz = V.rp[V.n];
        L.per_row = (double)nnz / std::max(1, V.n);
        // the K-cycle's two Krylov steps double the visits of every level below; on the
        // small levels (latency-bound launches) one cycle is cheaper overall
        L.krylov = V.n >= kKrylovMinRows;
        L.per_agg = L.nc > 0 ? (double)nnz / L.nc : 1;
        std::vector<float> inv(V.n), vf(V.v, V.v + nnz);
        for (int i = 0; i < V.n; ++i) inv[i] = (float)(1.0 / V.l1[i]);
        int rc;
        if ((rc = dev_upload(h, L.rp, V.rp, (size_t)(V.n + 1) * 4)) || (rc = dev_upload(h, L.ci, V.ci, (size_t)nnz * 4)) ||
            (rc = dev_upload(h, L.vf, vf.data(), (size_t)nnz * 4)) || (rc = dev_upload(h, L.l1f, inv.data(), inv.size() * 4)))
            return rc;
        if (l == 0 && (rc = dev_upload(h, L.v, V.v, (size_t)nnz * 8))) return rc;
        if (L.nc > 0) {
            if ((rc = dev_upload(h, L.agg, V.agg, (size_t)V.n * 4)) ||
                (rc = dev_upload(h, L.crp, V.crp, (size_t)(L.nc + 1) * 4)) ||
                (rc = dev_upload(h, L.cidx, V.cidx, (size_t)V.n * 4)))
                return rc;
        }
    }
    // dense inverse of the coarsest operator from its Cholesky factor L (C = L L^T)
    const int n = A.nco;
    const double* Lf = A.chol;
    std::vector<double> inv((size_t)n * n), col(n);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {   // forward: L y = e_j
            double s = i == j ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= Lf[(size_t)i * n + k] * col[k];
            col[i] = s / Lf[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {   // backward: L^T x = y
            double s = col[i];
            for (int k = i + 1; k < n; ++k) s -= Lf[(size_t)k * n + i] * col[k];
            col[i] = s / Lf[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] = col[i];
    }
    std::vector<float> invf(inv.begin(), inv.end());
    return dev_upload(h, D.cinv, invf.data(), invf.size() * 4);
}

int ensure_work(Handle* h, DevAmg& D, int nrhs) {
    if (D.nrhs >= nrhs) return SVH_OK;
    for (cudaGraphExec_t& g : D.ge)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    D.graph_nrhs = 0;
    int rc;
    for (DLevel& L : D.lv) {
        const size_t vb = (size_t)nrhs * L.n * 8;
        if ((rc = dev_alloc(h, L.v1, vb)) || (rc = dev_alloc(h, L.w1, vb)) || (rc = dev_alloc(h, L.v2, vb)) ||
            (rc = dev_alloc(h, L.w2, vb)) || (rc = dev_alloc(h, L.rc, (size_t)nrhs * (L.nc > 0 ? L.nc : 1) * 8)) ||
            (rc = dev_alloc(h, L.sc, (size_t)NSLOT * nrhs * 16)) ||
            (rc = dev_alloc(h, L.part, (size_t)nrhs * kMaxGrid * 3 * 16)) || (rc = dev_alloc(h, L.cnt, 4)))
            return rc;
        SVH_CUDA_TRY(h, cudaMemsetAsync(L.cnt.p, 0, 4, D.st));
        SVH_CUDA_TRY(h, cudaMemsetAsync(L.sc.p, 0, (size_t)NSLOT * nrhs * 16, D.st));
    }
    const size_t vb = (size_t)nrhs * D.lv[0].n * 16;
    if ((rc = dev_alloc(h, D.fx, vb)) || (rc = dev_alloc(h, D.fr, vb)) || (rc = dev_alloc(h, D.fz, vb)) ||
        (rc = dev_alloc(h, D.fp, vb)) || (rc = dev_alloc(h, D.fq, vb)) || (rc = dev_alloc(h, D.fpo, vb)) ||
        (rc = dev_alloc(h, D.fqo, vb)) || (rc = dev_alloc(h, D.fs, (size_t)NFSLOT * nrhs * 16)) ||
        (rc = dev_alloc(h, D.fpart, (size_t)nrhs * kMaxGrid * 2 * 16)) || (rc = dev_alloc(h, D.fcnt, 4)) ||
        (rc = dev_alloc(h, D.kr, (size_t)nrhs * D.lv[0].n * 8)) || (rc = dev_alloc(h, D.kz, (size_t)nrhs * D.lv[0].n * 8)))
        return rc;
    SVH_CUDA_TRY(h, cudaMemsetAsync(D.fcnt.p, 0, 4, D.st));
    if (D.host_fs) cudaFreeHost(D.host_fs);
    D.host_fs = nullptr;
    SVH_CUDA_TRY(h, cudaMallocHost(&D.host_fs, (size_t)NFSLOT * nrhs * 16));
    D.nrhs = nrhs;
    return SVH_OK;
}

void kcycle(Handle* h, DevAmg& D, int l, VRef B, float2* X, int nrhs);

template <int G>
void launch_pre(DLevel& L, VRef B, int nrhs, unsigned grid, cudaStream_t s) {
    k_kc_pre<G><<<grid, TPB, 0, s>>>(L.n, L.nc, nrhs, P<int>(L.rp), P<int>(L.ci), P<float>(L.vf), P<float>(L.l1f),
                                     P<int>(L.crp), P<int>(L.cidx), B, P<float2>(L.rc));
}

template <int G>
void launch_post(DLevel& L, VRef B, XRef XC, float2* X, int nrhs, unsigned grid, cudaStream_t s) {
    k_kc_post<G><<<grid, TPB, 0, s>>>(L.n, nrhs, P<int>(L.rp), P<int>(L.ci), P<float>(L.vf), P<float>(L.l1f),
                                      P<int>(L.agg), B, XC, X);
}

template <int MODE, int G>
void launch_spmv_kc(DLevel& L, const float2* vin, const float2* v1, const float2* b, float2* w, int nrhs,
                    unsigned grid, cudaStream_t s) {
    k_kc_spmv<MODE, G><<<grid, TPB, 0, s>>>(L.n, nrhs, P<int>(L.rp), P<int>(L.ci), P<float>(L.vf), vin, v1, b, w,
                                            P<double2>(L.part), P<unsigned>(L.cnt), P<double2>(L.sc));
}

template <int MODE>
void spmv_kc(DLevel& L, const float2* vin, const float2* v1, const float2* b, float2* w, int nrhs,
             cudaStream_t s) {
    const Geo q = geo(L.n, L.per_row, nrhs);
    switch (q.G) {
        case 1: launch_spmv_kc<MODE, 1>(L, vin, v1, b, w, nrhs, q.grid, s); break;
        case 2: launch_spmv_kc<MODE, 2>(L, vin, v1, b, w, nrhs, q.grid, s); break;
        case 4: launch_spmv_kc<MODE, 4>(L, vin, v1, b, w, nrhs, q.grid, s); break;
        case 8: launch_spmv_kc<MODE, 8>(L, vin, v1, b, w, nrhs, q.grid, s); break;
        case 16: launch_spmv_kc<MODE, 16>(L, vin, v1, b, w, nrhs, q.grid, s); break;
        default: launch_spmv_kc<MODE, 32>(L, vin, v1, b, w, nrhs, q.grid, s); break;
    }
}

template <int G>
void launch_fcg_spmv(DLevel& L0, const double2* p, const double2* r, double2* q, DevAmg& D, int nrhs, unsigned grid,
                     cudaStream_t s) {
    k_fcg_spmv<G><<<grid, TPB, 0, s>>>(L0.n, nrhs, P<int>(L0.rp), P<int>(L0.ci), P<double>(L0.v), p, r, q,
                                       P<double2>(D.fpart), P<unsigned>(D.fcnt), P<double2>(D.fs));
}

void dense(DevAmg& D, const float2* b, float2* X, int nrhs, cudaStream_t s) {
    const int n = D.lv.back().n;
    const int64_t warps = (int64_t)n * nrhs;
    k_dense<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(n, nrhs, P<float>(D.cinv), b, X);
}

// two Krylov steps on level l with the level-l cycle as preconditioner; the
// result is c1 v1 + c2 v2 of this level (read by the caller's post kernel),
// or v1 alone on the coarsest level
void coarse_krylov(Handle* h, DevAmg& D, int l, const float2* b, int nrhs) {
    DLevel& L = D.lv[l];
    cudaStream_t s = D.st;
    if (l + 1 == (int)D.lv.size()) {
        dense(D, b, P<float2>(L.v1), nrhs, s);
        return;
    }
    if (!L.krylov) {   // small level: one cycle, no Krylov acceleration (result in v1)
        kcycle(h, D, l, VRef{b, nullptr, nullptr}, P<float2>(L.v1), nrhs);
        return;
    }
    kcycle(h, D, l, VRef{b, nullptr, nullptr}, P<float2>(L.v1), nrhs);
    spmv_kc<1>(L, P<float2>(L.v1), nullptr, b, P<float2>(L.w1), nrhs, s);
    kcycle(h, D, l, VRef{b, P<float2>(L.w1), P<double2>(L.sc) + S_A1 * nrhs}, P<float2>(L.v2), nrhs);
    spmv_kc<2>(L, P<float2>(L.v2), P<float2>(L.v1), b, P<float2>(L.w2), nrhs, s);
}

// X ~= A_l^{-1} B (zero initial guess), l below the coarsest level
void kcycle(Handle* h, DevAmg& D, int l, VRef B, float2* X, int nrhs) {
    DLevel& L = D.lv[l];
    DLevel& C = D.lv[l + 1];
    cudaStream_t s = D.st;
    const Geo qa = geo(L.nc, L.per_agg, nrhs);
    switch (qa.G) {
        case 1: launch_pre<1>(L, B, nrhs, qa.grid, s); break;
        case 2: launch_pre<2>(L, B, nrhs, qa.grid, s); break;
        case 4: launch_pre<4>(L, B, nrhs, qa.grid, s); break;
        case 8: launch_pre<8>(L, B, nrhs, qa.grid, s); break;
        case 16: launch_pre<16>(L, B, nrhs, qa.grid, s); break;
        default: launch_pre<32>(L, B, nrhs, qa.grid, s); break;
    }
    coarse_krylov(h, D, l + 1, P<float2>(L.rc), nrhs);
    XRef XC{P<float2>(C.v1), P<float2>(C.v2), nullptr, nullptr};
    if (l + 2 < (int)D.lv.size() && C.krylov) {
        XC.c1 = P<double2>(C.sc) + S_C1 * nrhs;
        XC.c2 = P<double2>(C.sc) + S_C2 * nrhs;
    }
    const Geo qr = geo(L.n, L.per_row, nrhs);
    switch (qr.G) {
        case 1: launch_post<1>(L, B, XC, X, nrhs, qr.grid, s); break;
        case 2: launch_post<2>(L, B, XC, X, nrhs, qr.grid, s); break;
        case 4: launch_post<4>(L, B, XC, X, nrhs, qr.grid, s); break;
        case 8: launch_post<8>(L, B, XC, X, nrhs, qr.grid, s); break;
        case 16: launch_post<16>(L, B, XC, X, nrhs, qr.grid, s); break;
        default: launch_post<32>(L, B, XC, X, nrhs, qr.grid, s); break;
    }
}

}  // namespace

void amg_dev_destroy(void* d) { delete static_cast<DevAmg*>(d); }

// b = S^{-1} e on the device for nb complex right-hand sides e[rhs][nf]
// (double2, device); right-hand side r belongs to frequency r / per_freq.
int precond_schur_solve_dev(Handle* h, int nb, int per_freq, const void* e_dev, void* b_dev) {
    if (per_freq < 1 || per_freq > kMaxRhs)
        return set_err(h, SVH_ERR_ARG, "preconditioner: the device AMG takes 1 to 64 right-hand sides per frequency");
    const int nfreq = nb / per_freq;
    for (int f = 0; f < nfreq; ++f) {
        void*& slot = precond_dev(h, f);
        AmgView A;
        if (int rc = precond_view(h, f, A)) return rc;
        if (!slot) {
            DevAmg* D = new DevAmg();
            int rc = upload(h, *D, A);
            if (rc) { delete D; return rc; }
            slot = D;
        }
        DevAmg& D = *static_cast<DevAmg*>(slot);
        const int nrhs = per_freq;
        if (int rc = ensure_work(h, D, nrhs)) return rc;
        const int n = D.lv[0].n;
        DLevel& L0 = D.lv[0];
        cudaStream_t s = D.st;
        SVH_CUDA_TRY(h, cudaEventRecord(D.ev_in, h->stream));   // e is ready on the caller's stream
        SVH_CUDA_TRY(h, cudaStreamWaitEvent(s, D.ev_in, 0));
        const double2* e = static_cast<const double2*>(e_dev) + (int64_t)f * per_freq * n;
        double2* x = P<double2>(D.fx);
        double2* r = P<double2>(D.fr);
        double2* fs = P<double2>(D.fs);
        const unsigned g1 = geo(n, 1, nrhs).grid;       // one lane per (row, rhs), grid-striding
        const Geo gs = geo(n, L0.per_row, nrhs);         // the level-0 product
        k_fcg_init<<<g1, TPB, 0, s>>>(n, nrhs, e, x, r, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs);
        const double tol2 = A.tol * A.tol;
        // iteration `it` uses (p, q) = (fp, fq) when it is even, (fpo, fqo) when
        // odd; iterations after the first are replayed from one CUDA graph per
        // parity (about a hundred small launches each), captured on first use
        auto iteration = [&](int it) {
            double2 *p = P<double2>(D.fp), *q = P<double2>(D.fq), *po = P<double2>(D.fpo), *qo = P<double2>(D.fqo);
            if (it & 1) { std::swap(p, po); std::swap(q, qo); }
            double2* z = P<double2>(D.fz);
            // z = K-cycle(r) in FP32 (a preconditioner: flexible CG keeps the iteration in FP64)
            const int64_t tot = (int64_t)n * nrhs;
            float2 *kr = P<float2>(D.kr), *kz = P<float2>(D.kz);
            k_to_f32<<<nblk(tot), TPB, 0, s>>>(tot, r, kr);
            if (D.lv.size() == 1) {
                dense(D, kr, kz, nrhs, s);
            } else {
                kcycle(h, D, 0, VRef{kr, nullptr, nullptr}, kz, nrhs);
            }
            k_to_f64<<<nblk(tot), TPB, 0, s>>>(tot, kz, z);
            if (it > 0)
                k_fcg_beta<<<g1, TPB, 0, s>>>(n, nrhs, z, qo, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs);
            k_fcg_dir<<<nblk((int64_t)n * nrhs), TPB, 0, s>>>((int64_t)n * nrhs, nrhs, z, po, p, fs, it == 0);
            switch (gs.G) {
                case 1: launch_fcg_spmv<1>(L0, p, r, q, D, nrhs, gs.grid, s); break;
                case 2: launch_fcg_spmv<2>(L0, p, r, q, D, nrhs, gs.grid, s); break;
                case 4: launch_fcg_spmv<4>(L0, p, r, q, D, nrhs, gs.grid, s); break;
                case 8: launch_fcg_spmv<8>(L0, p, r, q, D, nrhs, gs.grid, s); break;
                case 16: launch_fcg_spmv<16>(L0, p, r, q, D, nrhs, gs.grid, s); break;
                default: launch_fcg_spmv<32>(L0, p, r, q, D, nrhs, gs.grid, s); break;
            }
            k_fcg_update<<<g1, TPB, 0, s>>>(n, nrhs, p, q, x, r, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs, tol2);
        };
        if (D.graph_nrhs != nrhs || D.graph_tol2 != tol2) {
            for (int k = 0; k < 2; ++k)
                if (D.ge[k]) { cudaGraphExecDestroy(D.ge[k]); D.ge[k] = nullptr; }
            D.graph_nrhs = 0;
        }
        int it = 0;
        bool done = false;
        while (!done) {
            if (it >= A.maxit) return set_err(h, SVH_ERR_NOT_CONVERGED, "preconditioner: device AMG-CG did not converge");
            if (it == 0) {
                iteration(0);
            } else {
                cudaGraphExec_t& ge = D.ge[it & 1];
                if (!ge) {
                    cudaGraph_t gr = nullptr;
                    SVH_CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                    iteration(it);
                    SVH_CUDA_TRY(h, cudaStreamEndCapture(s, &gr));
                    cudaError_t ce = cudaGraphInstantiate(&ge, gr, 0);
                    cudaGraphDestroy(gr);
                    if (ce != cudaSuccess) { ge = nullptr; return cuda_err(h, ce, "cudaGraphInstantiate"); }
                    D.graph_nrhs = nrhs;
                    D.graph_tol2 = tol2;
                }
                SVH_CUDA_TRY(h, cudaGraphLaunch(ge, s));
            }
            ++it;
            SVH_CUDA_TRY(h, cudaGetLastError());
            SVH_CUDA_TRY(h, cudaMemcpyAsync(D.host_fs, fs, (size_t)NFSLOT * nrhs * 16, cudaMemcpyDeviceToHost, s));
            SVH_CUDA_TRY(h, cudaStreamSynchronize(s));
            done = true;
            for (int k = 0; k < nrhs; ++k) {
                const double2 a = D.host_fs[F_ACTIVE * nrhs + k];
                if (a.x > 0 || a.y > 0) done = false;
            }
        }
        double iters = 0;
        for (int k = 0; k < nrhs; ++k) {
            const double2 c = D.host_fs[F_ITERS * nrhs + k];
            iters += c.x + c.y;
        }
        precond_count(h, f, 2 * nrhs, (long long)iters);
        k_fcg_out<<<nblk((int64_t)n * nrhs), TPB, 0, s>>>(n, nrhs, x,
                                                          static_cast<double2*>(b_dev) + (int64_t)f * per_freq * n);
        SVH_CUDA_TRY(h, cudaEventRecord(D.ev_out, s));              // the caller's stream waits for b
        SVH_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, D.ev_out, 0));
    }
    return SVH_OK;
}

}  // namespace svh
