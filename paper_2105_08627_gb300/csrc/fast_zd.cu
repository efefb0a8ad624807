// fast_zd.cu -- the z pass as a direct block-Toeplitz product (FP32; a tile
// variant of pass 3 of the product, for grids with few active planes).
//
// After the x and y transforms, each (kx, ky) point needs the z-cyclic
// convolution of its 5 bases' z-pencils with the 5 x 5 block kernel (Eq. 9).
// The circulant embedding is exact (Pz >= 2 Kz - 1 and every offset between
// active planes is below Kz), so the cyclic convolution equals the plain one:
//   Y_p(z) = sum_{z'} m_pq(z - z') X_q(z'),  m(dz) = sum_kz M(kz) e^{+2 pi i kz dz / Pz}
// with the transforms' conventions (forward e^-, inverse e+ unnormalised, the
// 1/(Px Py Pz) applied in the last pass). M(kz) is the block of
// block_multiply5; its entries are fixed combinations of the seven octant
// spectra, so m(dz) is the same combination of their z-space kernels
//   r_u(dz) = sum_kz s_u(kz) e^{+2 pi i kz dz / Pz}:
// real and even for the six z-even kernels, r_Sz(dz) = i rho(dz) with rho real
// and odd for S_z (its spectrum carries -i sign(kz)). The +-i factors of the
// S_z terms then cancel: g I_z + (+i I3) (2 s_z) becomes g I_z - 2 rho I3, and
// (+i I_z)(-2 s_z) becomes +2 rho I_z. For nza active planes this costs
// 17 nza^2 complex-by-real products per point (17 nonzero blocks), against
// 10 pencil transforms of Pz points and Pz block products for the FFT form.
#include <cuda_runtime.h>

#include <stdint.h>

#include "fastpass.cuh"

namespace svh {

// z-space kernels from the octant spectra: R[u][dz][ay][ax] = sum_az w_u[dz][az] S[u][az][ay][ax],
// w[0] (cosines, the z-even kernels) or w[1] (sines, S_z) in W[2][D][Hz]
__global__ void k_spec_to_zk(const float* __restrict__ S, float* __restrict__ R, const float* __restrict__ W,
                             int64_t plane, int Hz, int D) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= plane) return;
    const int u = blockIdx.y;
    const float* w = W + (u == 3 ? D * Hz : 0);
    float s[ZK_MAX_HZ];
#pragma unroll
    for (int az = 0; az < ZK_MAX_HZ; ++az) s[az] = az < Hz ? __ldg(S + ((int64_t)u * Hz + az) * plane + p) : 0.f;
    for (int d = 0; d < D; ++d) {
        float acc = 0.f;
#pragma unroll
        for (int az = 0; az < ZK_MAX_HZ; ++az)
            if (az < Hz) acc = fmaf(__ldg(w + d * Hz + az), s[az], acc);
        R[((int64_t)u * D + d) * plane + p] = acc;
    }
}

void launch_spec_to_zk(const float* S, float* R, const float* W, int Hx, int Hy, int Hz, int D, cudaStream_t s) {
    const int64_t plane = (int64_t)Hx * Hy;
    k_spec_to_zk<<<dim3((unsigned)((plane + 255) / 256), 7), 256, 0, s>>>(S, R, W, plane, Hz, D);
}

// One block per (32 kx, ky): thread (zi, lane) owns output plane zi of point
// kx0 + lane for all 5 bases. The point's z-space kernels at the D offsets are
// staged once in shared memory as the 7 values the block product uses (g, s_x
// and s_y with the x/y signs of the odd kernels folded in, 2 rho of S_z, and
// q_x + q_y, q_x - q_y, q_x + q_y + 4 q_z), so a thread keeps few registers
// and four blocks fit an SM. Each item's 5 x NZ input values of the 32 points
// travel by cp.async into a ring of ZD_DEPTH shared slots, ZD_DEPTH - 1 items
// ahead (one barrier per item), and the outputs go back in place (each thread
// stores exactly the values it copied).
constexpr int ZD_DEPTH = 3;
template <int NZ>
__global__ void __launch_bounds__(32 * NZ, 4) k_zdirect(const __grid_constant__ PassArgs a) {
    using C = float2;
    __shared__ C xs[ZD_DEPTH][5][NZ][32];
    __shared__ float rs[7][ZK_MAX_D][32];
    const int zi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kx = blockIdx.x * 32 + lane, ky = blockIdx.y;
    const int Px = a.Px, Py = a.Py, D = a.zkD;
    const bool ok = kx < Px;
    C* B2 = static_cast<C*>(a.B2);
    const int64_t P2 = (int64_t)Py * Px;
    const int64_t pt = (int64_t)ky * Px + kx;
    auto addr = [&](int b, int q) { return ((int64_t)(b * 5 + q) * NZ + zi) * P2 + pt; };
    auto issue = [&](int b) {
        if (b < a.nb && ok) {
#pragma unroll
            for (int q = 0; q < 5; ++q) cp_async8(&xs[b % ZD_DEPTH][q][zi][lane], B2 + addr(b, q));
        }
        cp_async_commit();
    };
#pragma unroll
    for (int b = 0; b < ZD_DEPTH - 1; ++b) issue(b);
    {
        const int kxx = min(kx, Px - 1);
        const int ax = min(kxx, Px - kxx), ay = min(ky, Py - ky);
        const float sgx = 2 * kxx <= Px ? 1.f : -1.f, sgy = 2 * ky <= Py ? 1.f : -1.f;
        const int64_t zplane = (int64_t)a.Hx * a.Hy, uplane = zplane * D;
        for (int d = zi; d < D; d += NZ) {
            const float* r = a.zk + (int64_t)d * zplane + (int64_t)ay * a.Hx + ax;
            const float qx = __ldg(r + 4 * uplane), qy = __ldg(r + 5 * uplane), qz = __ldg(r + 6 * uplane);
            rs[0][d][lane] = __ldg(r);
            rs[1][d][lane] = sgx * __ldg(r + uplane);
            rs[2][d][lane] = sgy * __ldg(r + 2 * uplane);
            rs[3][d][lane] = 2.f * __ldg(r + 3 * uplane);
            rs[4][d][lane] = qx + qy;
            rs[5][d][lane] = qx - qy;
            rs[6][d][lane] = qx + qy + 4.f * qz;
        }
    }
    // this plane's offsets to the others: kernel row |dz| and the sign of S_z's odd kernel
    int roff[NZ];
    float rsg[NZ];
    {
        const int z0 = __ldg(a.zlist + zi);
#pragma unroll
        for (int zj = 0; zj < NZ; ++zj) {
            const int dz = z0 - __ldg(a.zlist + zj);
            roff[zj] = (dz < 0 ? -dz : dz) * 32 + lane;
            rsg[zj] = dz < 0 ? -1.f : 1.f;
        }
    }
    const float* rsf = &rs[0][0][0];
    constexpr int RU = ZK_MAX_D * 32;   // stride between the 7 kernel rows of rs
    for (int b = 0; b < a.nb; ++b) {
        const int cur = b % ZD_DEPTH;
        cp_async_wait<ZD_DEPTH - 2>();
        __syncthreads();   // item b has landed for every thread; every thread is done with item b - 1
        issue(b + ZD_DEPTH - 1);
        C Yx = make_float2(0.f, 0.f), Yy = Yx, Yz = Yx, Y2 = Yx, Y3 = Yx;
#pragma unroll
        for (int zj = 0; zj < NZ; ++zj) {
            const float* r = rsf + roff[zj];
            const float g = r[0], sx = r[RU], sy = r[2 * RU], rz = rsg[zj] * r[3 * RU];
            const float qs = r[4 * RU], qd = r[5 * RU], q3 = r[6 * RU];
            const C Ix = xs[cur][0][zj][lane], Iy = xs[cur][1][zj][lane], Iz = xs[cur][2][zj][lane];
            const C I2 = xs[cur][3][zj][lane], I3 = xs[cur][4][zj][lane];
            // -i (I2 + I3) sx, -i (I3 - I2) sy: (-i v) = (v.y, -v.x)
            const float px = I2.x + I3.x, py = I2.y + I3.y, mx = I3.x - I2.x, my = I3.y - I2.y;
            Yx.x = fmaf(g, Ix.x, fmaf(sx, py, Yx.x));
            Yx.y = fmaf(g, Ix.y, fmaf(-sx, px, Yx.y));
            Yy.x = fmaf(g, Iy.x, fmaf(sy, my, Yy.x));
            Yy.y = fmaf(g, Iy.y, fmaf(-sy, mx, Yy.y));
            Yz.x = fmaf(g, Iz.x, fmaf(-rz, I3.x, Yz.x));
            Yz.y = fmaf(g, Iz.y, fmaf(-rz, I3.y, Yz.y));
            // +i v = (-v.y, v.x): Y2 += sx (i Ix) - sy (i Iy) + qs I2 + qd I3
            Y2.x = fmaf(-sx, Ix.y, fmaf(sy, Iy.y, fmaf(qs, I2.x, fmaf(qd, I3.x, Y2.x))));
            Y2.y = fmaf(sx, Ix.x, fmaf(-sy, Iy.x, fmaf(qs, I2.y, fmaf(qd, I3.y, Y2.y))));
            // Y3 += sx (i Ix) + sy (i Iy) + 2 rho Iz + qd I2 + (qs + 4 qz) I3
            Y3.x = fmaf(-sx, Ix.y, fmaf(-sy, Iy.y, fmaf(rz, Iz.x, fmaf(qd, I2.x, fmaf(q3, I3.x, Y3.x)))));
            Y3.y = fmaf(sx, Ix.x, fmaf(sy, Iy.x, fmaf(rz, Iz.y, fmaf(qd, I2.y, fmaf(q3, I3.y, Y3.y)))));
        }
        if (ok) {
            B2[addr(b, 0)] = Yx;
            B2[addr(b, 1)] = Yy;
            B2[addr(b, 2)] = Yz;
            B2[addr(b, 3)] = Y2;
            B2[addr(b, 4)] = Y3;
        }
    }
    cp_async_wait<0>();
}

template <int NZ>
static void run_zdirect(const PassArgs& a, cudaStream_t s) {
    k_zdirect<NZ><<<dim3((unsigned)((a.Px + 31) / 32), (unsigned)a.Py), 32 * NZ, 0, s>>>(a);
}

bool launch_z_direct(const PassArgs& a, cudaStream_t s) {
    if (!a.zk || a.zkD <= 0) return false;
    if (a.zkD > ZK_MAX_D) return false;
    switch (a.nza) {
        case 1: run_zdirect<1>(a, s); return true;
        case 2: run_zdirect<2>(a, s); return true;
        case 3: run_zdirect<3>(a, s); return true;
        case 4: run_zdirect<4>(a, s); return true;
        case 5: run_zdirect<5>(a, s); return true;
        case 6: run_zdirect<6>(a, s); return true;
        case 7: run_zdirect<7>(a, s); return true;
        case 8: run_zdirect<8>(a, s); return true;
        default: return false;
    }
}

}  // namespace svh
