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
//     Cholesky factor): one matrix-vector product.
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

// a right-hand side read on the fly: b - coef * w (w may be null)
struct VRef {
    const double2* b;
    const double2* w;
    const double2* coef;   // [nrhs]
};

__device__ __forceinline__ double2 vget(const VRef& B, int64_t off, double2 cf) {
    double2 v = B.b[off];
    if (B.w) v = sub2(v, mul(cf, B.w[off]));
    return v;
}

// the coarse correction read on the fly: v1 (plain) or c1 v1 + c2 v2
struct XRef {
    const double2* v1;
    const double2* v2;
    const double2* c1;     // [nrhs] or null (plain)
    const double2* c2;
};

// per-level scalar slots, each [nrhs] double2
enum { S_D11 = 0, S_G1, S_A1, S_C1, S_C2, NSLOT };
// top-level CG slots
enum { F_BETA = 0, F_PQ, F_PQOLD, F_ALPHA, F_RR, F_BB, F_ACTIVE, F_ITERS, NFSLOT };

// Block-wide sums of ND double2 values; the last block to finish (per
// right-hand side, blockIdx.y) then sums all block partials in index order and
// returns true with the totals in tot (valid in every thread of that block).
template <int ND>
__device__ bool block_sums_last(double2 (&val)[ND], double2* part, unsigned* cnt, double2 (&tot)[ND]) {
    __shared__ double2 sh[TPB / 32][ND];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nblk = gridDim.x;
    double2* pr = part + (int64_t)blockIdx.y * nblk * ND;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        double x = val[k].x, y = val[k].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if (lane == 0) sh[warp][k] = d2(x, y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < ND; ++k) {
            double2 s = sh[0][k];
            for (int w = 1; w < TPB / 32; ++w) s = add(s, sh[w][k]);
            pr[(int64_t)blockIdx.x * ND + k] = s;
        }
        __threadfence();
        const unsigned t = atomicAdd(cnt + blockIdx.y, 1u);
        last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double2 acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = d2(0, 0);
    for (int b = threadIdx.x; b < nblk; b += TPB)
#pragma unroll
        for (int k = 0; k < ND; ++k) acc[k] = add(acc[k], __ldcg(pr + (int64_t)b * ND + k));
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        double x = acc[k].x, y = acc[k].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        if (lane == 0) sh[warp][k] = d2(x, y);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        double2 s = sh[0][k];
        for (int w = 1; w < TPB / 32; ++w) s = add(s, sh[w][k]);
        tot[k] = s;
    }
    if (threadIdx.x == 0) cnt[blockIdx.y] = 0;   // ready for the next launch
    return true;
}

// Sparse rows are processed by groups of G lanes (G = 1 .. 32: one lane per
// row on the large fine levels, more on the small coarse levels with long
// Galerkin rows): lane `sub` of a group takes the row's entries
// sub, sub + G, ...; the group's partial sums meet in one shuffle reduction
// after the loops (every lane reaches it, so the shuffles stay convergent).
template <int G>
__device__ __forceinline__ double2 group_sum(double2 v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o, G);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o, G);
    }
    return v;   // complete in the group's lane 0
}

// K-cycle, first half: x0 = b / l1 (one l1-Jacobi sweep from zero), the
// residual b - A x0 and its restriction to the aggregates (sum over each);
// one group per aggregate.
template <int G>
__global__ void __launch_bounds__(TPB) k_kc_pre(int n, int nc, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const double* __restrict__ v, const double* __restrict__ l1inv,
                                                const int* __restrict__ crp, const int* __restrict__ cidx, VRef B,
                                                double2* __restrict__ rc) {
    const int r = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(t / G), sub = (int)(t % G);
    const int64_t off = (int64_t)r * n;
    const double2 cf = B.w ? B.coef[r] : d2(0, 0);
    double2 s = d2(0, 0);
    if (c < nc) {
        for (int p = crp[c]; p < crp[c + 1]; ++p) {
            const int i = cidx[p];
            if (sub == 0) s = add(s, vget(B, off + i, cf));
            for (int q = rp[i] + sub; q < rp[i + 1]; q += G) {
                const int j = ci[q];
                s = sub2(s, scl(v[q] * l1inv[j], vget(B, off + j, cf)));
            }
        }
    }
    s = group_sum<G>(s);
    if (c < nc && sub == 0) rc[(int64_t)r * nc + c] = s;
}

__device__ __forceinline__ double2 xcget(const XRef& X, int64_t off, int r) {
    if (!X.c1) return X.v1[off];
    return add(mul(X.c1[r], X.v1[off]), mul(X.c2[r], X.v2[off]));
}

// K-cycle, second half: x1 = b / l1 + P xc (coarse correction), then one more
// l1-Jacobi sweep x = x1 + (b - A x1) / l1; one group per row.
template <int G>
__global__ void __launch_bounds__(TPB) k_kc_post(int n, int nc, const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ v, const double* __restrict__ l1inv,
                                                 const int* __restrict__ agg, VRef B, XRef XC,
                                                 double2* __restrict__ X) {
    const int r = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const int64_t off = (int64_t)r * n, offc = (int64_t)r * nc;
    const double2 cf = B.w ? B.coef[r] : d2(0, 0);
    double2 ax = d2(0, 0);
    if (i < n) {
        for (int q = rp[i] + sub; q < rp[i + 1]; q += G) {
            const int j = ci[q];
            const double2 xj = add(scl(l1inv[j], vget(B, off + j, cf)), xcget(XC, offc + agg[j], r));
            ax = add(ax, scl(v[q], xj));
        }
    }
    ax = group_sum<G>(ax);
    if (i < n && sub == 0) {
        const double2 bi = vget(B, off + i, cf);
        const double2 xi = add(scl(l1inv[i], bi), xcget(XC, offc + agg[i], r));
        X[off + i] = add(xi, scl(l1inv[i], sub2(bi, ax)));
    }
}

// coarsest level: X = C^{-1} b, one warp per row
__global__ void k_dense(int n, const double* __restrict__ cinv, const double2* __restrict__ b,
                        double2* __restrict__ X) {
    const int r = blockIdx.y;
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double* cr = cinv + (int64_t)row * n;
    const double2* br = b + (int64_t)r * n;
    double x = 0, y = 0;
    for (int j = lane; j < n; j += 32) {
        const double c = cr[j];
        const double2 bj = br[j];
        x += c * bj.x;
        y += c * bj.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0) X[(int64_t)r * n + row] = d2(x, y);
}

// w = A vin with dot products; MODE 1 (first Krylov step): d11 = v1.w,
// g1 = v1.b -> a1 = g1 / d11. MODE 2 (second): d12 = v1.w, d22 = v2.w,
// g2 = v2.b -> (c1, c2) minimising the A-norm of the error over span{v1, v2}.
template <int MODE, int G>
__global__ void __launch_bounds__(TPB) k_kc_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ v, const double2* __restrict__ vin,
                                                 const double2* __restrict__ v1, const double2* __restrict__ b,
                                                 double2* __restrict__ w, double2* part, unsigned* cnt, double2* sc,
                                                 int nrhs) {
    const int r = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const int64_t off = (int64_t)r * n;
    constexpr int ND = MODE == 1 ? 2 : 3;
    double2 val[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) val[k] = d2(0, 0);
    double2 ax = d2(0, 0);
    if (i < n)
        for (int q = rp[i] + sub; q < rp[i + 1]; q += G) ax = add(ax, scl(v[q], vin[off + ci[q]]));
    ax = group_sum<G>(ax);
    if (i < n && sub == 0) {
        w[off + i] = ax;
        const double2 vi = vin[off + i], bi = b[off + i];
        if (MODE == 1) {
            val[0] = mul(vi, ax);
            val[1] = mul(vi, bi);
        } else {
            val[0] = mul(v1[off + i], ax);
            val[1] = mul(vi, ax);
            val[2] = mul(vi, bi);
        }
    }
    double2 tot[ND];
    if (!block_sums_last<ND>(val, part, cnt, tot)) return;
    if (threadIdx.x != 0) return;
    double2* s = sc;
    if (MODE == 1) {
        const double2 d11 = tot[0], g1 = tot[1];
        s[S_D11 * nrhs + r] = d11;
        s[S_G1 * nrhs + r] = g1;
        s[S_A1 * nrhs + r] = d2(d11.x > 0 ? g1.x / d11.x : 0.0, d11.y > 0 ? g1.y / d11.y : 0.0);
    } else {
        const double2 d11 = s[S_D11 * nrhs + r], g1 = s[S_G1 * nrhs + r], a1 = s[S_A1 * nrhs + r];
        const double2 d12 = tot[0], d22 = tot[1], g2 = tot[2];
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

// ---- top-level flexible CG on S
// r = e, x = 0, bb = e.e; a system with bb = 0 starts (and stays) inactive
__global__ void __launch_bounds__(TPB) k_fcg_init(int n, const double2* __restrict__ e, double2* __restrict__ x,
                                                  double2* __restrict__ rr, double2* part, unsigned* cnt, double2* fs,
                                                  int nrhs) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t off = (int64_t)r * n;
    double2 val[1] = {d2(0, 0)};
    if (i < n) {
        const double2 ei = e[off + i];
        rr[off + i] = ei;
        x[off + i] = d2(0, 0);
        val[0] = mul(ei, ei);
    }
    double2 tot[1];
    if (!block_sums_last<1>(val, part, cnt, tot)) return;
    if (threadIdx.x != 0) return;
    fs[F_BB * nrhs + r] = tot[0];
    fs[F_RR * nrhs + r] = tot[0];
    fs[F_ACTIVE * nrhs + r] = d2(tot[0].x > 0 ? 1.0 : 0.0, tot[0].y > 0 ? 1.0 : 0.0);
    fs[F_ITERS * nrhs + r] = d2(0, 0);
    fs[F_BETA * nrhs + r] = d2(0, 0);
    fs[F_PQOLD * nrhs + r] = d2(0, 0);
}

// beta = (z . q_old) / (p_old . q_old): the new direction is S-orthogonal to the previous one
__global__ void __launch_bounds__(TPB) k_fcg_beta(int n, const double2* __restrict__ z,
                                                  const double2* __restrict__ qold, double2* part, unsigned* cnt,
                                                  double2* fs, int nrhs) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t off = (int64_t)r * n;
    double2 val[1] = {d2(0, 0)};
    if (i < n) val[0] = mul(z[off + i], qold[off + i]);
    double2 tot[1];
    if (!block_sums_last<1>(val, part, cnt, tot)) return;
    if (threadIdx.x != 0) return;
    const double2 pq = fs[F_PQOLD * nrhs + r];
    fs[F_BETA * nrhs + r] = d2(pq.x > 0 ? tot[0].x / pq.x : 0.0, pq.y > 0 ? tot[0].y / pq.y : 0.0);
}

// p = z - beta p_old (p = z on the first iteration)
__global__ void k_fcg_dir(int64_t n, const double2* __restrict__ z, const double2* __restrict__ pold,
                          double2* __restrict__ p, const double2* __restrict__ fs, int nrhs, int first) {
    const int r = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = r * n + i;
    p[o] = first ? z[o] : sub2(z[o], mul(fs[F_BETA * nrhs + r], pold[o]));
}

// q = S p, pq = p.q, alpha = (p.r) / pq for the active systems (0 for the others)
template <int G>
__global__ void __launch_bounds__(TPB) k_fcg_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                  const double* __restrict__ v, const double2* __restrict__ p,
                                                  const double2* __restrict__ rr, double2* __restrict__ q,
                                                  double2* part, unsigned* cnt, double2* fs, int nrhs) {
    const int r = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const int64_t off = (int64_t)r * n;
    double2 val[2] = {d2(0, 0), d2(0, 0)};
    double2 ax = d2(0, 0);
    if (i < n)
        for (int k = rp[i] + sub; k < rp[i + 1]; k += G) ax = add(ax, scl(v[k], p[off + ci[k]]));
    ax = group_sum<G>(ax);
    if (i < n && sub == 0) {
        q[off + i] = ax;
        const double2 pi = p[off + i];
        val[0] = mul(pi, ax);
        val[1] = mul(pi, rr[off + i]);
    }
    double2 tot[2];
    if (!block_sums_last<2>(val, part, cnt, tot)) return;
    if (threadIdx.x != 0) return;
    const double2 act = fs[F_ACTIVE * nrhs + r];
    const double2 pq = tot[0], pr = tot[1];
    fs[F_PQ * nrhs + r] = pq;
    fs[F_ALPHA * nrhs + r] = d2(act.x > 0 && pq.x > 0 ? pr.x / pq.x : 0.0, act.y > 0 && pq.y > 0 ? pr.y / pq.y : 0.0);
}

// x += alpha p, r -= alpha q; rr = r.r; a system stays active while ||r|| > tol ||e||
__global__ void __launch_bounds__(TPB) k_fcg_update(int n, const double2* __restrict__ p,
                                                    const double2* __restrict__ q, double2* __restrict__ x,
                                                    double2* __restrict__ rr, double2* part, unsigned* cnt,
                                                    double2* fs, int nrhs, double tol2) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t off = (int64_t)r * n;
    const double2 alpha = fs[F_ALPHA * nrhs + r];
    double2 val[1] = {d2(0, 0)};
    if (i < n) {
        const double2 xi = add(x[off + i], mul(alpha, p[off + i]));
        const double2 ri = sub2(rr[off + i], mul(alpha, q[off + i]));
        x[off + i] = xi;
        rr[off + i] = ri;
        val[0] = mul(ri, ri);
    }
    double2 tot[1];
    if (!block_sums_last<1>(val, part, cnt, tot)) return;
    if (threadIdx.x != 0) return;
    const double2 bb = fs[F_BB * nrhs + r], act = fs[F_ACTIVE * nrhs + r];
    double2 it = fs[F_ITERS * nrhs + r];
    it.x += act.x;
    it.y += act.y;
    fs[F_ITERS * nrhs + r] = it;
    fs[F_RR * nrhs + r] = tot[0];
    fs[F_ACTIVE * nrhs + r] = d2(act.x > 0 && tot[0].x > tol2 * bb.x ? 1.0 : 0.0,
                                 act.y > 0 && tot[0].y > tol2 * bb.y ? 1.0 : 0.0);
    fs[F_PQOLD * nrhs + r] = fs[F_PQ * nrhs + r];
}

// ---- device copy of one hierarchy
struct DLevel {
    int n = 0, nc = 0;
    int g = 1, gp = 1;           // lanes per row (SpMV kernels) and per aggregate (restriction)
    bool krylov = true;          // coarse solves on this level take the two Krylov steps
    DevBuf rp, ci, v, l1inv, agg, crp, cidx;
    DevBuf v1, w1, v2, w2, rc;   // [nrhs][n] (rc: [nrhs][nc])
    DevBuf sc, part, cnt;        // scalar slots, block partials, completion counters
};

struct DevAmg {
    std::vector<DLevel> lv;
    DevBuf cinv;                 // dense inverse of the coarsest operator
    int nrhs = 0;                // capacity of the workspaces
    DevBuf fx, fr, fz, fp, fq, fpo, fqo, fs, fpart, fcnt;   // top-level CG
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
            for (DevBuf* b : {&L.rp, &L.ci, &L.v, &L.l1inv, &L.agg, &L.crp, &L.cidx, &L.v1, &L.w1, &L.v2, &L.w2,
                              &L.rc, &L.sc, &L.part, &L.cnt})
                dev_free(*b);
        for (DevBuf* b : {&cinv, &fx, &fr, &fz, &fp, &fq, &fpo, &fqo, &fs, &fpart, &fcnt}) dev_free(*b);
        if (host_fs) cudaFreeHost(host_fs);
    }
};

unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// lanes per unit (row or aggregate) for `units` units of `per` entries on average:
// one lane per unit while the units alone fill the GPU (~160 K threads), more on
// the small coarse levels (whose Galerkin rows are long), at most one per entry
int lanes_for(int64_t units, double per) {
    int g = 1;
    while (g < 32 && g < per && (int64_t)g * units < 160000) g *= 2;
    return g;
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
        L.g = lanes_for(V.n, (double)nnz / std::max(1, V.n));
        // the K-cycle's two Krylov steps double the visits of every level below; on the
        // small levels (latency-bound launches) one cycle is cheaper overall
        L.krylov = V.n >= kKrylovMinRows;
        L.gp = L.nc > 0 ? lanes_for(L.nc, (double)nnz / L.nc) : 1;
        std::vector<double> inv(V.n);
        for (int i = 0; i < V.n; ++i) inv[i] = 1.0 / V.l1[i];
        int rc;
        if ((rc = dev_upload(h, L.rp, V.rp, (size_t)(V.n + 1) * 4)) || (rc = dev_upload(h, L.ci, V.ci, (size_t)nnz * 4)) ||
            (rc = dev_upload(h, L.v, V.v, (size_t)nnz * 8)) || (rc = dev_upload(h, L.l1inv, inv.data(), inv.size() * 8)))
            return rc;
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
    return dev_upload(h, D.cinv, inv.data(), inv.size() * 8);
}

int ensure_work(Handle* h, DevAmg& D, int nrhs) {
    if (D.nrhs >= nrhs) return SVH_OK;
    for (cudaGraphExec_t& g : D.ge)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    D.graph_nrhs = 0;
    int rc;
    for (DLevel& L : D.lv) {
        const size_t vb = (size_t)nrhs * L.n * 16;
        if ((rc = dev_alloc(h, L.v1, vb)) || (rc = dev_alloc(h, L.w1, vb)) || (rc = dev_alloc(h, L.v2, vb)) ||
            (rc = dev_alloc(h, L.w2, vb)) || (rc = dev_alloc(h, L.rc, (size_t)nrhs * (L.nc > 0 ? L.nc : 1) * 16)) ||
            (rc = dev_alloc(h, L.sc, (size_t)NSLOT * nrhs * 16)) ||
            (rc = dev_alloc(h, L.part, (size_t)nrhs * nblk((int64_t)L.n * L.g) * 3 * 16)) ||
            (rc = dev_alloc(h, L.cnt, (size_t)nrhs * 4)))
            return rc;
        SVH_CUDA_TRY(h, cudaMemsetAsync(L.cnt.p, 0, (size_t)nrhs * 4, D.st));
        SVH_CUDA_TRY(h, cudaMemsetAsync(L.sc.p, 0, (size_t)NSLOT * nrhs * 16, D.st));
    }
    const size_t vb = (size_t)nrhs * D.lv[0].n * 16;
    if ((rc = dev_alloc(h, D.fx, vb)) || (rc = dev_alloc(h, D.fr, vb)) || (rc = dev_alloc(h, D.fz, vb)) ||
        (rc = dev_alloc(h, D.fp, vb)) || (rc = dev_alloc(h, D.fq, vb)) || (rc = dev_alloc(h, D.fpo, vb)) ||
        (rc = dev_alloc(h, D.fqo, vb)) || (rc = dev_alloc(h, D.fs, (size_t)NFSLOT * nrhs * 16)) ||
        (rc = dev_alloc(h, D.fpart, (size_t)nrhs * std::max(nblk((int64_t)D.lv[0].n * D.lv[0].g), nblk(D.lv[0].n)) * 2 * 16)) ||
        (rc = dev_alloc(h, D.fcnt, (size_t)nrhs * 4)))
        return rc;
    SVH_CUDA_TRY(h, cudaMemsetAsync(D.fcnt.p, 0, (size_t)nrhs * 4, D.st));
    if (D.host_fs) cudaFreeHost(D.host_fs);
    D.host_fs = nullptr;
    SVH_CUDA_TRY(h, cudaMallocHost(&D.host_fs, (size_t)NFSLOT * nrhs * 16));
    D.nrhs = nrhs;
    return SVH_OK;
}

void kcycle(Handle* h, DevAmg& D, int l, VRef B, double2* X, int nrhs);

template <int G>
void launch_pre(DLevel& L, VRef B, int nrhs, cudaStream_t s) {
    k_kc_pre<G><<<dim3(nblk((int64_t)L.nc * G), nrhs), TPB, 0, s>>>(L.n, L.nc, P<int>(L.rp), P<int>(L.ci),
                                                                   P<double>(L.v), P<double>(L.l1inv), P<int>(L.crp),
                                                                   P<int>(L.cidx), B, P<double2>(L.rc));
}

template <int G>
void launch_post(DLevel& L, VRef B, XRef XC, double2* X, int nrhs, cudaStream_t s) {
    k_kc_post<G><<<dim3(nblk((int64_t)L.n * G), nrhs), TPB, 0, s>>>(L.n, L.nc, P<int>(L.rp), P<int>(L.ci),
                                                                    P<double>(L.v), P<double>(L.l1inv), P<int>(L.agg),
                                                                    B, XC, X);
}

template <int MODE, int G>
void launch_spmv_kc(DLevel& L, const double2* vin, const double2* v1, const double2* b, double2* w, int nrhs,
                    cudaStream_t s) {
    k_kc_spmv<MODE, G><<<dim3(nblk((int64_t)L.n * G), nrhs), TPB, 0, s>>>(
        L.n, P<int>(L.rp), P<int>(L.ci), P<double>(L.v), vin, v1, b, w, P<double2>(L.part), P<unsigned>(L.cnt),
        P<double2>(L.sc), nrhs);
}

template <int MODE>
void spmv_kc(DLevel& L, const double2* vin, const double2* v1, const double2* b, double2* w, int nrhs,
             cudaStream_t s) {
    switch (L.g) {
        case 1: launch_spmv_kc<MODE, 1>(L, vin, v1, b, w, nrhs, s); break;
        case 2: launch_spmv_kc<MODE, 2>(L, vin, v1, b, w, nrhs, s); break;
        case 4: launch_spmv_kc<MODE, 4>(L, vin, v1, b, w, nrhs, s); break;
        case 8: launch_spmv_kc<MODE, 8>(L, vin, v1, b, w, nrhs, s); break;
        case 16: launch_spmv_kc<MODE, 16>(L, vin, v1, b, w, nrhs, s); break;
        default: launch_spmv_kc<MODE, 32>(L, vin, v1, b, w, nrhs, s); break;
    }
}

template <int G>
void launch_fcg_spmv(DLevel& L0, const double2* p, const double2* r, double2* q, DevAmg& D, int nrhs,
                     cudaStream_t s) {
    k_fcg_spmv<G><<<dim3(nblk((int64_t)L0.n * G), nrhs), TPB, 0, s>>>(L0.n, P<int>(L0.rp), P<int>(L0.ci),
                                                                      P<double>(L0.v), p, r, q, P<double2>(D.fpart),
                                                                      P<unsigned>(D.fcnt), P<double2>(D.fs), nrhs);
}

// two Krylov steps on level l with the level-l cycle as preconditioner; the
// result is c1 v1 + c2 v2 of this level (read by the caller's post kernel),
// or v1 alone on the coarsest level
void coarse_krylov(Handle* h, DevAmg& D, int l, const double2* b, int nrhs) {
    DLevel& L = D.lv[l];
    cudaStream_t s = D.st;
    if (l + 1 == (int)D.lv.size()) {
        k_dense<<<dim3((L.n + 7) / 8, nrhs), 256, 0, s>>>(L.n, P<double>(D.cinv), b, P<double2>(L.v1));
        return;
    }
    if (!L.krylov) {   // small level: one cycle, no Krylov acceleration (result in v1)
        kcycle(h, D, l, VRef{b, nullptr, nullptr}, P<double2>(L.v1), nrhs);
        return;
    }
    kcycle(h, D, l, VRef{b, nullptr, nullptr}, P<double2>(L.v1), nrhs);
    spmv_kc<1>(L, P<double2>(L.v1), nullptr, b, P<double2>(L.w1), nrhs, s);
    kcycle(h, D, l, VRef{b, P<double2>(L.w1), P<double2>(L.sc) + S_A1 * nrhs}, P<double2>(L.v2), nrhs);
    spmv_kc<2>(L, P<double2>(L.v2), P<double2>(L.v1), b, P<double2>(L.w2), nrhs, s);
}

// X ~= A_l^{-1} B (zero initial guess), l below the coarsest level
void kcycle(Handle* h, DevAmg& D, int l, VRef B, double2* X, int nrhs) {
    DLevel& L = D.lv[l];
    DLevel& C = D.lv[l + 1];
    cudaStream_t s = D.st;
    switch (L.gp) {
        case 1: launch_pre<1>(L, B, nrhs, s); break;
        case 2: launch_pre<2>(L, B, nrhs, s); break;
        case 4: launch_pre<4>(L, B, nrhs, s); break;
        case 8: launch_pre<8>(L, B, nrhs, s); break;
        case 16: launch_pre<16>(L, B, nrhs, s); break;
        default: launch_pre<32>(L, B, nrhs, s); break;
    }
    coarse_krylov(h, D, l + 1, P<double2>(L.rc), nrhs);
    XRef XC{P<double2>(C.v1), P<double2>(C.v2), nullptr, nullptr};
    if (l + 2 < (int)D.lv.size() && C.krylov) {
        XC.c1 = P<double2>(C.sc) + S_C1 * nrhs;
        XC.c2 = P<double2>(C.sc) + S_C2 * nrhs;
    }
    switch (L.g) {
        case 1: launch_post<1>(L, B, XC, X, nrhs, s); break;
        case 2: launch_post<2>(L, B, XC, X, nrhs, s); break;
        case 4: launch_post<4>(L, B, XC, X, nrhs, s); break;
        case 8: launch_post<8>(L, B, XC, X, nrhs, s); break;
        case 16: launch_post<16>(L, B, XC, X, nrhs, s); break;
        default: launch_post<32>(L, B, XC, X, nrhs, s); break;
    }
}

}  // namespace

void amg_dev_destroy(void* d) { delete static_cast<DevAmg*>(d); }

// b = S^{-1} e on the device for nb complex right-hand sides e[rhs][nf]
// (double2, device); right-hand side r belongs to frequency r / per_freq.
int precond_schur_solve_dev(Handle* h, int nb, int per_freq, const void* e_dev, void* b_dev) {
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
        const unsigned g = nblk(n);
        k_fcg_init<<<dim3(g, nrhs), TPB, 0, s>>>(n, e, x, r, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs, nrhs);
        const double tol2 = A.tol * A.tol;
        // iteration `it` uses (p, q) = (fp, fq) when it is even, (fpo, fqo) when
        // odd; iterations after the first are replayed from one CUDA graph per
        // parity (about a hundred small launches each), captured on first use
        auto iteration = [&](int it) {
            double2 *p = P<double2>(D.fp), *q = P<double2>(D.fq), *po = P<double2>(D.fpo), *qo = P<double2>(D.fqo);
            if (it & 1) { std::swap(p, po); std::swap(q, qo); }
            double2* z = P<double2>(D.fz);
            if (D.lv.size() == 1) {
                k_dense<<<dim3((n + 7) / 8, nrhs), 256, 0, s>>>(n, P<double>(D.cinv), r, z);
            } else {
                kcycle(h, D, 0, VRef{r, nullptr, nullptr}, z, nrhs);
            }
            if (it > 0)
                k_fcg_beta<<<dim3(g, nrhs), TPB, 0, s>>>(n, z, qo, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs, nrhs);
            k_fcg_dir<<<dim3(g, nrhs), TPB, 0, s>>>(n, z, po, p, fs, nrhs, it == 0);
            switch (L0.g) {
                case 1: launch_fcg_spmv<1>(L0, p, r, q, D, nrhs, s); break;
                case 2: launch_fcg_spmv<2>(L0, p, r, q, D, nrhs, s); break;
                case 4: launch_fcg_spmv<4>(L0, p, r, q, D, nrhs, s); break;
                case 8: launch_fcg_spmv<8>(L0, p, r, q, D, nrhs, s); break;
                case 16: launch_fcg_spmv<16>(L0, p, r, q, D, nrhs, s); break;
                default: launch_fcg_spmv<32>(L0, p, r, q, D, nrhs, s); break;
            }
            k_fcg_update<<<dim3(g, nrhs), TPB, 0, s>>>(n, p, q, x, r, P<double2>(D.fpart), P<unsigned>(D.fcnt), fs,
                                                        nrhs, tol2);
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
        SVH_CUDA_TRY(h, cudaMemcpyAsync(static_cast<double2*>(b_dev) + (int64_t)f * per_freq * n, x,
                                        (size_t)nrhs * n * 16, cudaMemcpyDeviceToDevice, s));
        SVH_CUDA_TRY(h, cudaEventRecord(D.ev_out, s));              // the caller's stream waits for b
        SVH_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, D.ev_out, 0));
    }
    return SVH_OK;
}

}  // namespace svh
