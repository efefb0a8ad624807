// svh_api.cpp -- C ABI entry points: handle, voxel grid and face nodes, kernel
// spectra (circulant embedding and transform of Eq. 9), Tucker-SVD
// (Algorithm 1) and the matvec front end.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "svh_internal.h"

namespace svh {

int set_err(Handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_err(Handle* h, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(h, SVH_ERR_OOM, std::string(what) + ": out of device memory");
    }
    return set_err(h, SVH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void prof_at(Handle* h, int p, int end, cudaStream_t s) {
    if (!h->prof_on || h->prof_calls >= h->prof_max) return;
    cudaEventRecord(h->prof_ev[((size_t)h->prof_calls * SVH_NPASS + p) * 2 + end], s);
}

static void prof_release(Handle* h) {
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
    h->prof_on = false;
    h->prof_max = h->prof_calls = 0;
}

void dev_free(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int dev_alloc(Handle* h, DevBuf& b, size_t bytes) {
    dev_free(b);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return cuda_err(h, e, "cudaMalloc");
    }
    b.bytes = bytes;
    return SVH_OK;
}

int dev_upload(Handle* h, DevBuf& b, const void* src, size_t bytes) {
    int rc = dev_alloc(h, b, bytes);
    if (rc) return rc;
    if (bytes) {
        SVH_CUDA_TRY(h, cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, h->stream));
        SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return SVH_OK;
}

static bool smooth(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// FFT size for K voxels: 2K when it has only factors 2, 3, 5, 7, else the
// smallest such size >= 2K - 1 (the circulant needs P >= 2K - 1, Eq. 9).
static int fft_size(int K) {
    if (smooth(2 * K)) return 2 * K;
    int n = 2 * K - 1;
    while (!smooth(n)) ++n;
    return n;
}

// Default padded size of an axis: any P >= 2K - 1 embeds the convolution
// exactly, so take the smallest size that has size-specialised kernels (x, y:
// 16 .. 1024; z: 8 .. 48), else the smallest 2,3,5,7-smooth size (2K first).
static int default_fft_size(int K, bool zaxis) {
    static const int xy[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
    static const int zz[] = {8, 12, 16, 24, 32, 48};
    if (zaxis) {
        for (int p : zz)
            if (p >= 2 * K - 1) return p;
    } else {
        for (int p : xy)
            if (p >= 2 * K - 1) return p;
    }
    return fft_size(K);
}

static FftPlanHost make_plan(int N) {
    FftPlanHost p;
    p.N = N;
    int n = N;
    while (n % 8 == 0) { p.R.push_back(8); n /= 8; }
    while (n % 4 == 0) { p.R.push_back(4); n /= 4; }
    while (n % 2 == 0) { p.R.push_back(2); n /= 2; }
    for (int r : {3, 5, 7})
        while (n % r == 0) { p.R.push_back(r); n /= r; }
    return p;
}

static void free_kernels(Handle* h) {
    dev_free(h->d_spec32);
    dev_free(h->d_zk32);
    dev_free(h->d_zkw);
    h->zk_D = 0;
    h->zk_version = -1;
    dev_free(h->d_spec64);
    for (int i = 0; i < 3; ++i) { dev_free(h->d_tw32[i]); dev_free(h->d_tw64[i]); }
    for (int u = 0; u < 7; ++u) {
        dev_free(h->d_tk_core[u]);
        dev_free(h->d_tk_core_zk[u]);
        for (int i = 0; i < 3; ++i) dev_free(h->d_tk_F[u][i]);
        h->tucker_on[u] = false;
        h->tk[u] = Tucker();
    }
    dev_free(h->d_tk_w1);
    dev_free(h->d_tk_probs);
    h->tk_zk_D = 0;
    ++h->tk_version;
    h->have_kernels = false;
    h->toep.clear();
    h->spec.clear();
}

static void free_all(Handle* h) {
    free_kernels(h);
    prof_release(h);
    precond_free(h);
    for (DevBuf* b : {&h->d_vidx, &h->d_rows, &h->d_rinfo, &h->d_vx, &h->d_rowmask, &h->d_zlist, &h->d_node,
                      &h->d_ninc, &h->d_free, &h->d_lam, &h->d_sig0, &h->d_B1, &h->d_B2, &h->d_xin, &h->d_yout,
                      &h->d_omegas, &h->d_status})
        dev_free(*b);
}

// ------------------------------------------------------------------ spectra
// Octant spectrum of a circulant built from kernel values T(d), 0 <= d < K, and
// their parity extension T(-d) = +-T(d): along an even axis the transform of
// C[i] = T(i), C[P-i] = T(-i) is T(0) + 2 sum_d T(d) cos(2 pi k d / P); along
// the odd axis of S_a it is -2j sum_d T(d) sin(2 pi k d / P). The octant
// k_i <= P_i/2 holds every distinct value.
static void axis_matrix(std::vector<double>& c, int H, int K, int P, bool odd) {
    c.assign((size_t)H * K, 0.0);
    const double twopi = 6.283185307179586476925286766559;
    for (int k = 0; k < H; ++k)
        for (int d = 0; d < K; ++d) {
            long long m = ((long long)k * d) % P;
            double ang = twopi * (double)m / (double)P;
            c[(size_t)k * K + d] = odd ? (d == 0 ? 0.0 : 2.0 * std::sin(ang))
                                       : (d == 0 ? 1.0 : 2.0 * std::cos(ang));
        }
}

static void spectra_host(int Kx, int Ky, int Kz, int Px, int Py, int Pz, const double* toep, double* spec) {
    const int Hx = Px / 2 + 1, Hy = Py / 2 + 1, Hz = Pz / 2 + 1;
    const size_t Kt = (size_t)Kx * Ky * Kz, Ht = (size_t)Hx * Hy * Hz;
    std::vector<double> cx[2], cy[2], cz[2];
    for (int o = 0; o < 2; ++o) {
        axis_matrix(cx[o], Hx, Kx, Px, o == 1);
        axis_matrix(cy[o], Hy, Ky, Py, o == 1);
        axis_matrix(cz[o], Hz, Kz, Pz, o == 1);
    }
    std::vector<double> A((size_t)Kz * Ky * Hx), B((size_t)Kz * Hy * Hx);
    for (int u = 0; u < 7; ++u) {
        const bool ox = (u == 1), oy = (u == 2), oz = (u == 3);
        const double* T = toep + u * Kt;
        const double* mx = cx[ox].data();
        const double* my = cy[oy].data();
        const double* mz = cz[oz].data();
        // along x: A[dz][dy][kx] = sum_dx T[dz][dy][dx] mx[kx][dx]
#pragma omp parallel for schedule(static)
        for (long long r = 0; r < (long long)Kz * Ky; ++r) {
            const double* row = T + r * Kx;
            double* out = A.data() + r * Hx;
            for (int k = 0; k < Hx; ++k) {
                const double* m = mx + (size_t)k * Kx;
                double s = 0;
                for (int d = 0; d < Kx; ++d) s += m[d] * row[d];
                out[k] = s;
            }
        }
        // along y: B[dz][ky][kx] = sum_dy A[dz][dy][kx] my[ky][dy]
#pragma omp parallel for schedule(static) collapse(2)
        for (int dz = 0; dz < Kz; ++dz)
            for (int ky = 0; ky < Hy; ++ky) {
                double* out = B.data() + ((size_t)dz * Hy + ky) * Hx;
                for (int k = 0; k < Hx; ++k) out[k] = 0;
                for (int dy = 0; dy < Ky; ++dy) {
                    double c = my[(size_t)ky * Ky + dy];
                    const double* in = A.data() + ((size_t)dz * Ky + dy) * Hx;
                    for (int k = 0; k < Hx; ++k) out[k] += c * in[k];
                }
            }
        // along z: S[kz][ky][kx] = sum_dz B[dz][ky][kx] mz[kz][dz]
        double* S = spec + u * Ht;
#pragma omp parallel for schedule(static)
        for (int kz = 0; kz < Hz; ++kz) {
            double* out = S + (size_t)kz * Hy * Hx;
            for (size_t i = 0; i < (size_t)Hy * Hx; ++i) out[i] = 0;
            for (int dz = 0; dz < Kz; ++dz) {
                double c = mz[(size_t)kz * Kz + dz];
                const double* in = B.data() + (size_t)dz * Hy * Hx;
                for (size_t i = 0; i < (size_t)Hy * Hx; ++i) out[i] += c * in[i];
            }
        }
    }
}

static void compute_spectra(Handle* h) {
    h->spec.assign((size_t)7 * h->Hx * h->Hy * h->Hz, 0.0);
    spectra_host(h->Kx, h->Ky, h->Kz, h->Px, h->Py, h->Pz, h->toep.data(), h->spec.data());
}

// Face-node numbering (Sec. II.A): scanning voxels in raster order and faces
// in the order -x,+x,-y,+y,-z,+z, a face takes the next id when first met.
// node[v*6+f] receives the ids; ninc[2m], ninc[2m+1] the codes v*6+f of the
// (at most two) voxel faces at node m (-1 if absent). Returns M.
static int64_t number_faces(int Kx, int Ky, int Kz, const std::vector<int32_t>& vox,
                            std::vector<int32_t>& node, std::vector<int32_t>& ninc) {
    const int64_t K = (int64_t)vox.size();
    std::vector<int32_t> fxs((size_t)(Kx + 1) * Ky * Kz, -1), fys((size_t)Kx * (Ky + 1) * Kz, -1),
        fzs((size_t)Kx * Ky * (Kz + 1), -1);
    node.assign(K * 6, -1);
    ninc.clear();
    ninc.reserve(K * 8);
    int64_t M = 0;
    for (int64_t v = 0; v < K; ++v) {
        int64_t g = vox[v];
        int x = (int)(g % Kx), y = (int)((g / Kx) % Ky), z = (int)(g / ((int64_t)Kx * Ky));
        int32_t* slot[6] = {
            &fxs[((size_t)z * Ky + y) * (Kx + 1) + x], &fxs[((size_t)z * Ky + y) * (Kx + 1) + x + 1],
            &fys[((size_t)z * (Ky + 1) + y) * Kx + x], &fys[((size_t)z * (Ky + 1) + y + 1) * Kx + x],
            &fzs[((size_t)z * Ky + y) * Kx + x], &fzs[((size_t)(z + 1) * Ky + y) * Kx + x]};
        for (int f = 0; f < 6; ++f) {
            if (*slot[f] < 0) {
                *slot[f] = (int32_t)M++;
                ninc.push_back(-1);
                ninc.push_back(-1);
            }
            int32_t m = *slot[f];
            node[v * 6 + f] = m;
            int32_t code = (int32_t)(v * 6 + f);
            if (ninc[2 * m] < 0) ninc[2 * m] = code;
            else ninc[2 * m + 1] = code;
        }
    }
    return M;
}

static int install_kernels(Handle* h) {
    compute_spectra(h);
    const size_t Ht = (size_t)h->Hx * h->Hy * h->Hz;
    int rc = dev_upload(h, h->d_spec64, h->spec.data(), 7 * Ht * sizeof(double));
    if (rc) return rc;
    std::vector<float> s32(h->spec.begin(), h->spec.end());
    rc = dev_upload(h, h->d_spec32, s32.data(), 7 * Ht * sizeof(float));
    ++h->spec_version;
    h->spec32_tk_version = -1;
    if (rc) return rc;
    const int P[3] = {h->Px, h->Py, h->Pz};
    const double twopi = 6.283185307179586476925286766559;
    for (int a = 0; a < 3; ++a) {
        h->plan[a] = make_plan(P[a]);
        std::vector<double> t64(2 * P[a]);
        std::vector<float> t32(2 * P[a]);
        for (int m = 0; m < P[a]; ++m) {
            double ang = twopi * (double)m / (double)P[a];
            t64[2 * m] = std::cos(ang);
            t64[2 * m + 1] = -std::sin(ang);
            t32[2 * m] = (float)t64[2 * m];
            t32[2 * m + 1] = (float)t64[2 * m + 1];
        }
        rc = dev_upload(h, h->d_tw64[a], t64.data(), t64.size() * sizeof(double));
        if (rc) return rc;
        rc = dev_upload(h, h->d_tw32[a], t32.data(), t32.size() * sizeof(float));
        if (rc) return rc;
    }
    for (int u = 0; u < 7; ++u) h->tucker_on[u] = false;
    h->kernel_mode = SVH_KERNELS_RESIDENT;
    h->have_kernels = true;
    return SVH_OK;
}

// ------------------------------------------------------------------ Tucker-SVD (Algorithm 1)
// Left singular vectors of the mode unfolding X (D rows), given its transpose
// as D columns of length m (cols[p * m + r]): Householder QR of the tall
// matrix [cols] = Q R (rows padded with zeros to at least D), then one-sided
// (Hestenes) Jacobi on R, R V = U Sigma, whose accumulated rotations V are
// the right singular vectors of R, i.e. the left singular vectors of X =
// R^T Q^T. Both steps are backward stable, so the singular values are accurate
// to ~ eps sigma_max (a Gram matrix would carry eps ||X||^2 instead). Pairs of
// columns are rotated in round-robin order, disjoint pairs in parallel.
// V: row-major D x D with the vectors as columns; w: sigma^2.
static void svd_left_vectors(std::vector<double>& cols, int m, int D, std::vector<double>& V, std::vector<double>& w) {
    // Householder QR, column by column
    for (int j = 0; j < D; ++j) {
        double* x = cols.data() + (size_t)j * m;
        double nx = 0;
        for (int i = j; i < m; ++i) nx += x[i] * x[i];
        nx = std::sqrt(nx);
        if (nx == 0) continue;
        const double alpha = x[j] > 0 ? -nx : nx;
        std::vector<double> v(x + j, x + m);
        v[0] -= alpha;
        double vn2 = 0;
        for (double e : v) vn2 += e * e;
        if (vn2 == 0) continue;
#pragma omp parallel for schedule(static) if (D - j > 16)
        for (int k = j + 1; k < D; ++k) {
            double* y = cols.data() + (size_t)k * m + j;
            double sdot = 0;
            for (size_t i = 0; i < v.size(); ++i) sdot += v[i] * y[i];
            const double f = 2.0 * sdot / vn2;
            for (size_t i = 0; i < v.size(); ++i) y[i] -= f * v[i];
        }
        x[j] = alpha;
        for (int i = j + 1; i < m; ++i) x[i] = 0.0;
    }
    // A = R (column-major, D x D), V = I
    std::vector<double> A((size_t)D * D, 0.0), Vc((size_t)D * D, 0.0);
    for (int j = 0; j < D; ++j) {
        for (int i = 0; i <= j; ++i) A[(size_t)j * D + i] = cols[(size_t)j * m + i];
        Vc[(size_t)j * D + j] = 1.0;
    }
    const int mm = D + (D & 1);
    std::vector<int> order(mm);
    std::iota(order.begin(), order.end(), 0);
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < mm - 1; ++round) {
#pragma omp parallel for schedule(static) reduction(+ : rotated) if (D > 64)
            for (int k = 0; k < mm / 2; ++k) {
                int p = order[k], q = order[mm - 1 - k];
                if (p > q) std::swap(p, q);
                if (q >= D) continue;   // dummy partner
                double* ap = A.data() + (size_t)p * D;
                double* aq = A.data() + (size_t)q * D;
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < D; ++i) {
                    al += ap[i] * ap[i];
                    be += aq[i] * aq[i];
                    ga += ap[i] * aq[i];
                }
                if (std::fabs(ga) <= 1e-15 * std::sqrt(al * be) || ga == 0) continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                double* vp = Vc.data() + (size_t)p * D;
                double* vq = Vc.data() + (size_t)q * D;
                for (int i = 0; i < D; ++i) {
                    const double a0 = ap[i], a1 = aq[i];
                    ap[i] = c * a0 - sn * a1;
                    aq[i] = sn * a0 + c * a1;
                    const double v0 = vp[i], v1 = vq[i];
                    vp[i] = c * v0 - sn * v1;
                    vq[i] = sn * v0 + c * v1;
                }
                ++rotated;
            }
            const int last = order[mm - 1];
            for (int k = mm - 1; k > 1; --k) order[k] = order[k - 1];
            order[1] = last;
        }
        if (!rotated) break;
    }
    V.assign((size_t)D * D, 0.0);
    w.assign(D, 0.0);
    for (int k = 0; k < D; ++k) {
        double s2 = 0;
        for (int i = 0; i < D; ++i) {
            s2 += A[(size_t)k * D + i] * A[(size_t)k * D + i];
            V[(size_t)i * D + k] = Vc[(size_t)k * D + i];
        }
        w[k] = s2;
    }
}

// mode-i product with F^T (projection), tensor stored [D3][D2][D1] (mode 1 fastest)
static std::vector<double> project(const std::vector<double>& X, const int dims[3], int mode,
                                   const std::vector<double>& F, int r) {
    int out_dims[3] = {dims[0], dims[1], dims[2]};
    out_dims[mode] = r;
    std::vector<double> Y((size_t)out_dims[0] * out_dims[1] * out_dims[2], 0.0);
    const int D1 = dims[0], D2 = dims[1], D3 = dims[2];
    const int O1 = out_dims[0], O2 = out_dims[1];
#pragma omp parallel for schedule(static)
    for (int c = 0; c < out_dims[2]; ++c)
        for (int b = 0; b < out_dims[1]; ++b)
            for (int a = 0; a < out_dims[0]; ++a) {
                double s = 0;
                if (mode == 0)
                    for (int i = 0; i < D1; ++i) s += F[(size_t)i * r + a] * X[((size_t)c * D2 + b) * D1 + i];
                else if (mode == 1)
                    for (int i = 0; i < D2; ++i) s += F[(size_t)i * r + b] * X[((size_t)c * D2 + i) * D1 + a];
                else
                    for (int i = 0; i < D3; ++i) s += F[(size_t)i * r + c] * X[((size_t)i * D2 + b) * D1 + a];
                Y[((size_t)c * O2 + b) * O1 + a] = s;
            }
    return Y;
}

static void tucker_svd(const double* O, const int dims[3], double tol, Tucker& out) {
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    double norm2 = 0;
    for (size_t i = 0; i < n; ++i) norm2 += O[i] * O[i];
    const double thr2 = tol * tol / 3.0 * norm2;
    std::vector<double> C(O, O + n);
    int cdims[3] = {dims[0], dims[1], dims[2]};
    for (int mode = 0; mode < 3; ++mode) {
        const int D = dims[mode];
        // left singular vectors of the mode-i unfolding of the ORIGINAL tensor (Algorithm 1)
        const int D1 = dims[0], D2 = dims[1], D3 = dims[2];
        const size_t R = n / D;
        const int m = (int)std::max<size_t>(R, (size_t)D);
        std::vector<double> cols((size_t)D * m, 0.0);   // column p: the entries with index p along this mode
#pragma omp parallel for schedule(static)
        for (int p = 0; p < D; ++p) {
            double* col = cols.data() + (size_t)p * m;
            if (mode == 0) {
                for (size_t r = 0; r < (size_t)D2 * D3; ++r) col[r] = O[r * D1 + p];
            } else if (mode == 1) {
                for (int c = 0; c < D3; ++c)
                    for (int a = 0; a < D1; ++a) col[(size_t)c * D1 + a] = O[((size_t)c * D2 + p) * D1 + a];
            } else {
                for (size_t r = 0; r < (size_t)D1 * D2; ++r) col[r] = O[(size_t)p * D1 * D2 + r];
            }
        }
        std::vector<double> V, w;
        svd_left_vectors(cols, m, D, V, w);
        std::vector<int> idx(D);
        std::iota(idx.begin(), idx.end(), 0);
        std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
        // Rank: smallest d whose discarded part of the unfolding, measured as
        // ||(I - U_d U_d^T) O_(i)||_F^2 = sum_{r >= d} ||u_r^T O_(i)||^2 with the
        // rows u_r^T O_(i) computed from O itself, is <= thr2. (The Gram
        // eigenvalues alone carry round-off of eps ||O||^2, the size of thr2
        // when tol ~ 1e-8; the residual form keeps the bound exact.)
        std::vector<double> rown(D, 0.0);
#pragma omp parallel for schedule(dynamic)
        for (int r = 0; r < D; ++r) {
            const int k = idx[r];
            double acc = 0;
            if (mode == 0) {
                for (size_t t = 0; t < (size_t)D2 * D3; ++t) {
                    double s = 0;
                    for (int p = 0; p < D1; ++p) s += V[(size_t)p * D + k] * O[t * D1 + p];
                    acc += s * s;
                }
            } else if (mode == 1) {
                for (int c = 0; c < D3; ++c)
                    for (int a = 0; a < D1; ++a) {
                        double s = 0;
                        for (int p = 0; p < D2; ++p) s += V[(size_t)p * D + k] * O[((size_t)c * D2 + p) * D1 + a];
                        acc += s * s;
                    }
            } else {
                for (size_t t = 0; t < (size_t)D1 * D2; ++t) {
                    double s = 0;
                    for (int p = 0; p < D3; ++p) s += V[(size_t)p * D + k] * O[(size_t)p * D1 * D2 + t];
                    acc += s * s;
                }
            }
            rown[r] = acc;
        }
        int d = D;
        double tail = 0;
        for (int r = D - 1; r >= 1; --r) {
            tail += rown[r];
            if (tail <= thr2) d = r;
            else break;
        }
        std::vector<double> F((size_t)D * d);
        for (int i = 0; i < D; ++i)
            for (int k = 0; k < d; ++k) F[(size_t)i * d + k] = V[(size_t)i * D + idx[k]];
        C = project(C, cdims, mode, F, d);
        cdims[mode] = d;
        out.F[mode] = F;
        out.d[mode] = d;
    }
    out.core = C;
}

static int upload_tucker(Handle* h, int u) {
    const int rc = upload_tucker_device(h, u);
    if (rc) return rc;
    h->tucker_on[u] = true;
    ++h->tk_version;
    return SVH_OK;
}

}  // namespace svh

using namespace svh;

#define HCHECK(h)                                   \
    do {                                            \
        if (!(h)) return SVH_ERR_ARG;               \
        cudaError_t e__ = cudaSetDevice((h)->device); \
        if (e__ != cudaSuccess) return cuda_err((h), e__, "cudaSetDevice"); \
    } while (0)

extern "C" {

int svh_create(svh_handle** out, int device, void* stream) {
    if (!out) return SVH_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return SVH_ERR_CUDA;
    }
    Handle* h = new (std::nothrow) Handle();
    if (!h) return SVH_ERR_OOM;
    h->device = device;
    h->stream = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess) {
        delete h;
        return SVH_ERR_CUDA;
    }
    *out = reinterpret_cast<svh_handle*>(h);
    return SVH_OK;
}

int svh_destroy(svh_handle* hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (cudaStream_t st : {h->aux, h->cpy_in, h->cpy_out})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (cudaEvent_t e : {h->ev_fork, h->ev_spec, h->ev_done, h->ev_x})
        if (e) cudaEventDestroy(e);
    for (int j = 0; j < kHostChunks; ++j) {
        if (h->ev_in[j]) cudaEventDestroy(h->ev_in[j]);
        if (h->ev_out[j]) cudaEventDestroy(h->ev_out[j]);
    }
    free_all(h);
    if (h->tsvd) tsvd_free(h->tsvd);
    delete h;
    return SVH_OK;
}

const char* svh_last_error(const svh_handle* hh) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h) return "null handle";
    return h->err.c_str();
}

int svh_set_stream(svh_handle* hh, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return SVH_OK;
}

int svh_setup_grid(svh_handle* hh, int Kx, int Ky, int Kz, double dx, const uint8_t* occ,
                   const double* lambda, const double* sigma0, const svh_port* ports, int nports) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (Kx <= 0 || Ky <= 0 || Kz <= 0 || !(dx > 0) || !occ || !lambda || !sigma0 || nports < 0 ||
        (nports > 0 && !ports))
        return set_err(h, SVH_ERR_ARG, "svh_setup_grid: bad sizes or null arrays");
    if ((int64_t)Kx * Ky * Kz > (int64_t)1 << 31)
        return set_err(h, SVH_ERR_ARG, "svh_setup_grid: grid too large");
    free_all(h);
    h->have_grid = false;
    h->Kx = Kx; h->Ky = Ky; h->Kz = Kz; h->dx = dx;
    const int64_t Kt = (int64_t)Kx * Ky * Kz;
    std::vector<int32_t> gidx(Kt, -1);
    h->vox.clear();
    for (int64_t i = 0; i < Kt; ++i)
        if (occ[i]) {
            if (!(lambda[i] > 0) || !(sigma0[i] >= 0) || !std::isfinite(lambda[i]) || !std::isfinite(sigma0[i]))
                return set_err(h, SVH_ERR_ARG, "svh_setup_grid: lambda must be > 0 and sigma0 >= 0 on voxels");
            gidx[i] = (int32_t)h->vox.size();
            h->vox.push_back((int32_t)i);
        }
    const int64_t K = (int64_t)h->vox.size();
    if (K == 0) return set_err(h, SVH_ERR_ARG, "svh_setup_grid: no voxels");
    h->K = K;
    h->lam.resize(K);
    h->sig0.resize(K);
    for (int64_t v = 0; v < K; ++v) { h->lam[v] = lambda[h->vox[v]]; h->sig0[v] = sigma0[h->vox[v]]; }
    // face nodes, first-appearance order over voxels and faces -x,+x,-y,+y,-z,+z
    std::vector<int32_t> ninc;
    const int64_t M = number_faces(Kx, Ky, Kz, h->vox, h->node, ninc);
    h->M = M;
    // ports
    h->fixed.assign(M, 0);
    h->port_plus.clear();
    h->port_minus.clear();
    for (int p = 0; p < nports; ++p) {
        for (int side = 0; side < 2; ++side) {
            int n = side == 0 ? ports[p].n_plus : ports[p].n_minus;
            const int32_t* faces = side == 0 ? ports[p].plus : ports[p].minus;
            if (n <= 0 || !faces) return set_err(h, SVH_ERR_ARG, "svh_setup_grid: empty port terminal");
            std::vector<int32_t> nodes;
            for (int i = 0; i < n; ++i) {
                int64_t code = faces[i];
                int64_t cell = code / 6;
                int f = (int)(code % 6);
                if (code < 0 || cell >= Kt || gidx[cell] < 0)
                    return set_err(h, SVH_ERR_ARG, "svh_setup_grid: port face on an empty voxel");
                nodes.push_back(h->node[(int64_t)gidx[cell] * 6 + f]);
            }
            std::sort(nodes.begin(), nodes.end());
            nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
            for (int32_t m : nodes) h->fixed[m] = 1;
            (side == 0 ? h->port_plus : h->port_minus).push_back(nodes);
        }
    }
    // floating islands (no terminal): fix the -x node of their first voxel
    std::vector<int32_t> parent(K);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t a) {
        while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
        return a;
    };
    for (int64_t m = 0; m < M; ++m)
        if (ninc[2 * m + 1] >= 0) {
            int32_t a = find(ninc[2 * m] / 6), b = find(ninc[2 * m + 1] / 6);
            if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
    std::vector<uint8_t> has_term(K, 0);
    for (int64_t v = 0; v < K; ++v)
        for (int f = 0; f < 6; ++f)
            if (h->fixed[h->node[v * 6 + f]]) has_term[find((int32_t)v)] = 1;
    h->gauge.clear();
    for (int64_t v = 0; v < K; ++v)
        if (find((int32_t)v) == v && !has_term[v]) {
            h->gauge.push_back(h->node[v * 6 + 0]);
            h->fixed[h->node[v * 6 + 0]] = 1;
        }
    // active planes and rows
    h->zlist.clear();
    h->rows.clear();
    std::vector<uint8_t> zact(Kz, 0);
    for (int64_t v = 0; v < K; ++v) zact[h->vox[v] / ((int64_t)Kx * Ky)] = 1;
    for (int z = 0; z < Kz; ++z)
        if (zact[z]) h->zlist.push_back(z);
    const int nza = (int)h->zlist.size();
    std::vector<int32_t> vidx((size_t)nza * Ky * Kx, -1);
    std::vector<uint8_t> rowmask((size_t)nza * Ky, 0);
    for (int zi = 0; zi < nza; ++zi) {
        int z = h->zlist[zi];
        for (int y = 0; y < Ky; ++y)
            for (int x = 0; x < Kx; ++x) {
                int32_t v = gidx[((int64_t)z * Ky + y) * Kx + x];
                vidx[((size_t)zi * Ky + y) * Kx + x] = v;
                if (v >= 0) rowmask[(size_t)zi * Ky + y] = 1;
            }
        for (int y = 0; y < Ky; ++y)
            if (rowmask[(size_t)zi * Ky + y]) h->rows.push_back(zi * Ky + y);
    }
    // voxels are numbered in cell order (x fastest): each active row's voxels are one range
    std::vector<int32_t> rinfo(2 * h->rows.size()), vx(K);
    for (size_t i = 0; i < h->rows.size(); ++i) {
        const int32_t* vr = vidx.data() + (size_t)h->rows[i] * Kx;
        int32_t first = -1, count = 0;
        for (int x = 0; x < Kx; ++x)
            if (vr[x] >= 0) {
                if (first < 0) first = vr[x];
                if (vr[x] != first + count) return set_err(h, SVH_ERR_STATE, "svh_setup_grid: voxel order");
                ++count;
            }
        rinfo[2 * i] = first;
        rinfo[2 * i + 1] = count;
    }
    for (int64_t v = 0; v < K; ++v) vx[v] = (int32_t)(h->vox[v] % Kx);
    h->Px = default_fft_size(Kx, false); h->Py = default_fft_size(Ky, false); h->Pz = default_fft_size(Kz, true);
    h->Hx = h->Px / 2 + 1; h->Hy = h->Py / 2 + 1; h->Hz = h->Pz / 2 + 1;
    std::vector<uint8_t> freem(M);
    for (int64_t m = 0; m < M; ++m) freem[m] = h->fixed[m] ? 0 : 1;
    int rc;
    if ((rc = dev_upload(h, h->d_vidx, vidx.data(), vidx.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_rows, h->rows.data(), h->rows.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_rinfo, rinfo.data(), rinfo.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_vx, vx.data(), vx.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_rowmask, rowmask.data(), rowmask.size()))) return rc;
    if ((rc = dev_upload(h, h->d_zlist, h->zlist.data(), h->zlist.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_node, h->node.data(), h->node.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_ninc, ninc.data(), ninc.size() * 4))) return rc;
    if ((rc = dev_upload(h, h->d_free, freem.data(), freem.size()))) return rc;
    if ((rc = dev_upload(h, h->d_lam, h->lam.data(), K * 8))) return rc;
    if ((rc = dev_upload(h, h->d_sig0, h->sig0.data(), K * 8))) return rc;
    if (!h->d_status.p) {
        const int32_t zero = 0;
        if ((rc = dev_upload(h, h->d_status, &zero, 4))) return rc;
    }
    if ((rc = matvec_streams(h))) return rc;
    h->have_grid = true;
    return SVH_OK;
}

int svh_set_fft_sizes(svh_handle* hh, int Px, int Py, int Pz) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_set_fft_sizes: no grid");
    if (Px < 2 * h->Kx - 1 || Py < 2 * h->Ky - 1 || Pz < 2 * h->Kz - 1 || !smooth(Px) || !smooth(Py) || !smooth(Pz))
        return set_err(h, SVH_ERR_ARG, "svh_set_fft_sizes: need P_i >= 2K_i - 1 with factors 2,3,5,7");
    free_kernels(h);
    h->Px = Px; h->Py = Py; h->Pz = Pz;
    h->Hx = Px / 2 + 1; h->Hy = Py / 2 + 1; h->Hz = Pz / 2 + 1;
    return SVH_OK;
}

int svh_get_grid_info(const svh_handle* hh, svh_grid_info* info) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !info) return SVH_ERR_ARG;
    if (!h->have_grid) return SVH_ERR_STATE;
    info->Kx = h->Kx; info->Ky = h->Ky; info->Kz = h->Kz;
    info->Px = h->Px; info->Py = h->Py; info->Pz = h->Pz;
    info->Hx = h->Hx; info->Hy = h->Hy; info->Hz = h->Hz;
    info->K = h->K; info->M = h->M; info->N = 5 * h->K + h->M;
    info->nports = (int32_t)h->port_plus.size();
    int32_t nf = 0;
    for (uint8_t f : h->fixed) nf += f;
    info->n_fixed_nodes = nf;
    info->n_active_planes = (int32_t)h->zlist.size();
    info->n_active_rows = (int32_t)h->rows.size();
    info->dx = h->dx;
    return SVH_OK;
}

int svh_get_nodes(const svh_handle* hh, int32_t* node) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !node) return SVH_ERR_ARG;
    if (!h->have_grid) return SVH_ERR_STATE;
    std::memcpy(node, h->node.data(), h->node.size() * 4);
    return SVH_OK;
}

int svh_load_toeplitz(svh_handle* hh, const double* T) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!T) return set_err(h, SVH_ERR_ARG, "svh_load_toeplitz: null");
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_load_toeplitz: call svh_setup_grid first");
    const size_t n = (size_t)7 * h->Kx * h->Ky * h->Kz;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(T[i])) return set_err(h, SVH_ERR_ARG, "svh_load_toeplitz: non-finite value");
    free_kernels(h);
    h->toep.assign(T, T + n);
    return install_kernels(h);
}

int svh_generate_toeplitz(svh_handle* hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_generate_toeplitz: call svh_setup_grid first");
    free_kernels(h);
    std::vector<double> T;
    int rc = generate_toeplitz_device(h, T);
    if (rc) return rc;
    h->toep.swap(T);
    return install_kernels(h);
}

int svh_get_toeplitz(const svh_handle* hh, double* T) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !T) return SVH_ERR_ARG;
    if (!h->have_kernels || h->toep.empty()) return SVH_ERR_STATE;
    std::memcpy(T, h->toep.data(), h->toep.size() * sizeof(double));
    return SVH_OK;
}

int svh_get_spectra(const svh_handle* hh, double* S) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !S) return SVH_ERR_ARG;
    if (!h->have_kernels) return SVH_ERR_STATE;
    std::memcpy(S, h->spec.data(), h->spec.size() * sizeof(double));
    return SVH_OK;
}

int svh_get_spectra32(svh_handle* hh, float* S) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!S) return set_err(h, SVH_ERR_ARG, "svh_get_spectra32: null output");
    if (!h->have_kernels || !h->d_spec32.p) return set_err(h, SVH_ERR_STATE, "svh_get_spectra32: no kernels");
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    SVH_CUDA_TRY(h, cudaMemcpy(S, h->d_spec32.p, (size_t)7 * h->Hx * h->Hy * h->Hz * sizeof(float),
                               cudaMemcpyDeviceToHost));
    return SVH_OK;
}

int svh_load_tucker(svh_handle* hh, int u, int d1, int d2, int d3, const double* core,
                    const double* F1, const double* F2, const double* F3) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_load_tucker: load kernels first");
    if (u < 0 || u > 6 || d1 <= 0 || d2 <= 0 || d3 <= 0 || d1 > h->Hx || d2 > h->Hy || d3 > h->Hz ||
        !core || !F1 || !F2 || !F3)
        return set_err(h, SVH_ERR_ARG, "svh_load_tucker: bad kernel id, ranks or arrays");
    Tucker& t = h->tk[u];
    t.d[0] = d1; t.d[1] = d2; t.d[2] = d3;
    t.core.assign(core, core + (size_t)d1 * d2 * d3);
    t.F[0].assign(F1, F1 + (size_t)h->Hx * d1);
    t.F[1].assign(F2, F2 + (size_t)h->Hy * d2);
    t.F[2].assign(F3, F3 + (size_t)h->Hz * d3);
    return upload_tucker(h, u);
}

int svh_tucker_compress(svh_handle* hh, double tol, int32_t* ranks) {
    return svh_tucker_compress_on(hh, tol, ranks, 1);
}

int svh_tucker_compress_on(svh_handle* hh, double tol, int32_t* ranks, int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_tucker_compress: load kernels first");
    if (!(tol > 0) || tol >= 1) return set_err(h, SVH_ERR_ARG, "svh_tucker_compress: need 0 < tol < 1");
    const int dims[3] = {h->Hx, h->Hy, h->Hz};
    const size_t Ht = (size_t)h->Hx * h->Hy * h->Hz;
    // the device routine takes the QR of each unfolding's transpose, which needs it tall
    if (h->Hx > h->Hy * h->Hz || h->Hy > h->Hx * h->Hz || h->Hz > h->Hx * h->Hy) on_device = 0;
    for (int u = 0; u < 7; ++u) {
        if (on_device) {
            Tucker t;
            if (int rc = tucker_svd_device(h, u, tol, t)) return rc;
            h->tk[u] = t;
        } else {
            tucker_svd(h->spec.data() + u * Ht, dims, tol, h->tk[u]);
        }
        int rc = upload_tucker(h, u);
        if (rc) return rc;
        if (ranks)
            for (int i = 0; i < 3; ++i) ranks[u * 3 + i] = h->tk[u].d[i];
    }
    return SVH_OK;
}

int svh_get_tucker(const svh_handle* hh, int u, int32_t* d, double* core, double* F1, double* F2, double* F3) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || u < 0 || u > 6 || !d) return SVH_ERR_ARG;
    if (!h->tucker_on[u]) return SVH_ERR_STATE;
    const Tucker& t = h->tk[u];
    for (int i = 0; i < 3; ++i) d[i] = t.d[i];
    if (core) std::memcpy(core, t.core.data(), t.core.size() * 8);
    if (F1) std::memcpy(F1, t.F[0].data(), t.F[0].size() * 8);
    if (F2) std::memcpy(F2, t.F[1].data(), t.F[1].size() * 8);
    if (F3) std::memcpy(F3, t.F[2].data(), t.F[2].size() * 8);
    return SVH_OK;
}

int svh_set_kernel_mode(svh_handle* hh, int mode) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (mode != SVH_KERNELS_RESIDENT && mode != SVH_KERNELS_TUCKER_REBUILD)
        return set_err(h, SVH_ERR_ARG, "svh_set_kernel_mode: unknown mode");
    if (mode == SVH_KERNELS_TUCKER_REBUILD)
        for (int u = 0; u < 7; ++u)
            if (!h->tucker_on[u])
                return set_err(h, SVH_ERR_STATE, "svh_set_kernel_mode: every kernel needs Tucker data");
    h->kernel_mode = mode;
    return SVH_OK;
}

int svh_rebuild_spectra(svh_handle* hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_rebuild_spectra: no kernels");
    return launch_tucker_rebuild(h, h->stream);
}

int svh_matvec(svh_handle* hh, double omega, int nb, const void* x, void* y, int precision) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_grid || !h->have_kernels)
        return set_err(h, SVH_ERR_STATE, "svh_matvec: grid and kernels must be set up first");
    if (!(omega > 0) || !std::isfinite(omega) || nb <= 0 || !x || !y || (precision != SVH_FP32 && precision != SVH_FP64))
        return set_err(h, SVH_ERR_ARG, "svh_matvec: bad omega, nb, pointers or precision");
    const size_t bytes = (size_t)nb * (5 * h->K + h->M) * (precision == SVH_FP32 ? 8 : 16);
    const char* xc = static_cast<const char*>(x);
    const char* yc = static_cast<const char*>(y);
    if (xc < yc + bytes && yc < xc + bytes) return set_err(h, SVH_ERR_ARG, "svh_matvec: x and y overlap");
    return precision == SVH_FP32 ? launch_matvec32(h, omega, nb, x, y, 0) : launch_matvec64(h, omega, nb, x, y, 0);
}

int svh_get_device_status(svh_handle* hh, int32_t* status, int clear) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!status) return SVH_ERR_ARG;
    *status = 0;
    if (!h->d_status.p) return SVH_OK;
    SVH_CUDA_TRY(h, cudaMemcpyAsync(status, h->d_status.p, 4, cudaMemcpyDeviceToHost, h->stream));
    if (clear) SVH_CUDA_TRY(h, cudaMemsetAsync(h->d_status.p, 0, 4, h->stream));
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SVH_OK;
}

int svh_autotune(svh_handle* hh, int nb, int32_t* variants, double* ms) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_grid || !h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_autotune: grid and kernels needed");
    if (nb <= 0) return set_err(h, SVH_ERR_ARG, "svh_autotune: nb must be positive");
    return autotune(h, nb, variants, ms);
}

int svh_set_pass_variant(svh_handle* hh, int pass, int variant) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_set_pass_variant: no grid");
    return set_pass_variant(h, pass, variant);
}

int svh_get_pass_variants(const svh_handle* hh, int32_t* counts, int32_t* chosen) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    if (!h->have_grid) return SVH_ERR_STATE;
    get_pass_variants(h, counts, chosen);
    return SVH_OK;
}

int svh_matvec_omegas(svh_handle* hh, const double* omegas, int nb, const void* x, void* y, int precision) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->have_grid || !h->have_kernels)
        return set_err(h, SVH_ERR_STATE, "svh_matvec_omegas: grid and kernels must be set up first");
    if (!omegas || nb <= 0 || !x || !y || (precision != SVH_FP32 && precision != SVH_FP64))
        return set_err(h, SVH_ERR_ARG, "svh_matvec_omegas: bad arguments");
    for (int b = 0; b < nb; ++b)
        if (!(omegas[b] > 0) || !std::isfinite(omegas[b])) return set_err(h, SVH_ERR_ARG, "svh_matvec_omegas: omega must be > 0");
    const size_t bytes = (size_t)nb * (5 * h->K + h->M) * (precision == SVH_FP32 ? 8 : 16);
    const char* xc = static_cast<const char*>(x);
    const char* yc = static_cast<const char*>(y);
    if (xc < yc + bytes && yc < xc + bytes) return set_err(h, SVH_ERR_ARG, "svh_matvec_omegas: x and y overlap");
    if (h->d_omegas.bytes < (size_t)nb * 8) { int rc = dev_alloc(h, h->d_omegas, (size_t)nb * 8); if (rc) return rc; }
    SVH_CUDA_TRY(h, cudaMemcpyAsync(h->d_omegas.p, omegas, (size_t)nb * 8, cudaMemcpyHostToDevice, h->stream));
    const double* dom = static_cast<const double*>(h->d_omegas.p);
    return precision == SVH_FP32 ? launch_matvec32(h, omegas[0], nb, x, y, 0, dom)
                                 : launch_matvec64(h, omegas[0], nb, x, y, 0, dom);
}

int svh_matvec_host(svh_handle* hh, double omega, int nb, const void* x, void* y, int precision) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!x || !y || nb <= 0 || (precision != SVH_FP32 && precision != SVH_FP64))
        return set_err(h, SVH_ERR_ARG, "svh_matvec_host: bad arguments");
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_matvec_host: no grid");
    if (!h->have_kernels) return set_err(h, SVH_ERR_STATE, "svh_matvec_host: grid and kernels must be set up first");
    if (!(omega > 0) || !std::isfinite(omega)) return set_err(h, SVH_ERR_ARG, "svh_matvec_host: omega must be > 0");
    const size_t item = (size_t)(5 * h->K + h->M) * (precision == SVH_FP32 ? 8 : 16);
    const size_t bytes = (size_t)nb * item;
    int rc;
    if (h->d_xin.bytes < bytes && (rc = dev_alloc(h, h->d_xin, bytes))) return rc;
    if (h->d_yout.bytes < bytes && (rc = dev_alloc(h, h->d_yout, bytes))) return rc;
    // The items go in up to kHostChunks chunks: every chunk is copied in on cpy_in as early as
    // the link allows, multiplied on the handle's stream once its copy has landed, and copied out
    // on cpy_out while the next chunk is multiplied, so only the first chunk's input copy and the
    // last chunk's output copy add to the product's time. The first chunk's product runs the
    // Tucker restore (rebuild mode), forked before its input copy so that the two overlap; the
    // later chunks reuse the restored kernels.
    const int nch = std::min(nb, kHostChunks);
    char* xd = static_cast<char*>(h->d_xin.p);
    char* yd = static_cast<char*>(h->d_yout.p);
    const char* xh = static_cast<const char*>(x);
    char* yh = static_cast<char*>(y);
    if ((rc = matvec_prefork(h))) return rc;   // creates the copy streams too
    SVH_CUDA_TRY(h, cudaEventRecord(h->ev_in[0], h->stream));   // the caller's earlier work on the stream
    SVH_CUDA_TRY(h, cudaStreamWaitEvent(h->cpy_in, h->ev_in[0], 0));
    int first[kHostChunks + 1];
    for (int j = 0; j <= nch; ++j) first[j] = (int)((int64_t)nb * j / nch);
    for (int j = 0; j < nch; ++j) {
        const size_t off = (size_t)first[j] * item, len = (size_t)(first[j + 1] - first[j]) * item;
        SVH_CUDA_TRY(h, cudaMemcpyAsync(xd + off, xh + off, len, cudaMemcpyHostToDevice, h->cpy_in));
        SVH_CUDA_TRY(h, cudaEventRecord(h->ev_in[j], h->cpy_in));
    }
    for (int j = 0; j < nch && !rc; ++j) {
        const size_t off = (size_t)first[j] * item, len = (size_t)(first[j + 1] - first[j]) * item;
        const int nbj = first[j + 1] - first[j];
        SVH_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_in[j], 0));
        if (j == 0) {
            if ((rc = matvec_mark_input_ready(h))) break;
            rc = precision == SVH_FP32 ? launch_matvec32(h, omega, nbj, xd + off, yd + off, 0)
                                       : launch_matvec64(h, omega, nbj, xd + off, yd + off, 0);
        } else {
            rc = launch_matvec_reuse(h, omega, nbj, xd + off, yd + off, precision);
        }
        if (rc) break;
        SVH_CUDA_TRY(h, cudaEventRecord(h->ev_out[j], h->stream));
        SVH_CUDA_TRY(h, cudaStreamWaitEvent(h->cpy_out, h->ev_out[j], 0));
        SVH_CUDA_TRY(h, cudaMemcpyAsync(yh + off, yd + off, len, cudaMemcpyDeviceToHost, h->cpy_out));
    }
    h->preforked = false;   // consumed by the first product (or left over by a failed call)
    cudaError_t e1 = cudaStreamSynchronize(h->cpy_in);
    cudaError_t e2 = cudaStreamSynchronize(h->cpy_out);
    cudaError_t e3 = cudaStreamSynchronize(h->stream);
    if (rc) return rc;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return cuda_err(h, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "svh_matvec_host");
    return SVH_OK;
}

int svh_profile_begin(svh_handle* hh, int max_calls) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (max_calls <= 0 || max_calls > 100000) return set_err(h, SVH_ERR_ARG, "svh_profile_begin: bad max_calls");
    prof_release(h);
    h->prof_ev.resize((size_t)max_calls * SVH_NPASS * 2);
    for (auto& e : h->prof_ev) SVH_CUDA_TRY(h, cudaEventCreate(&e));
    h->prof_max = max_calls;
    h->prof_calls = 0;
    h->prof_on = true;
    return SVH_OK;
}

int svh_profile_end(svh_handle* hh, double* ms, int* ncalls) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    HCHECK(h);
    if (!h->prof_on || !ms || !ncalls) return set_err(h, SVH_ERR_STATE, "svh_profile_end: not profiling");
    SVH_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (h->aux) SVH_CUDA_TRY(h, cudaStreamSynchronize(h->aux));
    for (int p = 0; p < SVH_NPASS; ++p) ms[p] = 0.0;
    for (int c = 0; c < h->prof_calls; ++c)
        for (int p = 0; p < SVH_NPASS; ++p) {
            float t = 0.f;
            SVH_CUDA_TRY(h, cudaEventElapsedTime(&t, h->prof_ev[((size_t)c * SVH_NPASS + p) * 2],
                                                 h->prof_ev[((size_t)c * SVH_NPASS + p) * 2 + 1]));
            ms[p] += t;
        }
    *ncalls = h->prof_calls;
    prof_release(h);
    return SVH_OK;
}

int svh_host_face_nodes(int Kx, int Ky, int Kz, const uint8_t* occ, int64_t* K_out, int64_t* M_out,
                        int32_t* node) {
    if (Kx <= 0 || Ky <= 0 || Kz <= 0 || !occ || !K_out || !M_out) return SVH_ERR_ARG;
    const int64_t Kt = (int64_t)Kx * Ky * Kz;
    std::vector<int32_t> vox;
    for (int64_t i = 0; i < Kt; ++i)
        if (occ[i]) vox.push_back((int32_t)i);
    std::vector<int32_t> nd, ninc;
    *M_out = number_faces(Kx, Ky, Kz, vox, nd, ninc);
    *K_out = (int64_t)vox.size();
    if (node) std::memcpy(node, nd.data(), nd.size() * 4);
    return SVH_OK;
}

int svh_host_spectra(int Kx, int Ky, int Kz, int Px, int Py, int Pz, const double* T, double* S) {
    if (Kx <= 0 || Ky <= 0 || Kz <= 0 || !T || !S || Px < 2 * Kx - 1 || Py < 2 * Ky - 1 || Pz < 2 * Kz - 1)
        return SVH_ERR_ARG;
    spectra_host(Kx, Ky, Kz, Px, Py, Pz, T, S);
    return SVH_OK;
}

int svh_host_tucker_svd(const double* O, int D1, int D2, int D3, double tol, int32_t* d, double* core,
                        double* F1, double* F2, double* F3) {
    if (!O || D1 <= 0 || D2 <= 0 || D3 <= 0 || !(tol > 0) || !d || !core || !F1 || !F2 || !F3) return SVH_ERR_ARG;
    const int dims[3] = {D1, D2, D3};
    Tucker t;
    tucker_svd(O, dims, tol, t);
    for (int i = 0; i < 3; ++i) d[i] = t.d[i];
    std::memcpy(core, t.core.data(), t.core.size() * 8);
    std::memcpy(F1, t.F[0].data(), t.F[0].size() * 8);
    std::memcpy(F2, t.F[1].data(), t.F[1].size() * 8);
    std::memcpy(F3, t.F[2].data(), t.F[2].size() * 8);
    return SVH_OK;
}

}  // extern "C"
