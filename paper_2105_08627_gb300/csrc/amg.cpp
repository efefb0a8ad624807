// amg.cpp -- host aggregation AMG for the Schur complement of the sparse preconditioner.
//
// Sec. II.C: the preconditioner P = Q^{-1}, Q = [Y, -A^T; A, 0] with
// Y = diag(|Z_kk|) (Eq. 12-13), is applied through the Schur complement
// S = A Y^{-1} A^T (real, symmetric positive definite on the free nodes):
// e = d - A Y^{-1} c, b = S^{-1} e (Eq. 14), a = Y^{-1}(c + A^T b) (Eq. 15).
// S^{-1} e is computed here by flexible conjugate gradients preconditioned
// with an aggregation-based algebraic multigrid K-cycle, the method the paper
// takes from AGMG (written here from the published idea, not from that code):
//   * aggregation: two passes of pairwise matching -- each node is paired
//     with its unpaired neighbour of strongest coupling |a_ij| (at least
//     beta = 0.25 of its strongest one), so aggregates hold up to 4 nodes;
//     S is not an M-matrix (the linear bases couple face nodes with positive
//     weights), so the strength test uses magnitudes;
//   * coarse operator: Galerkin P^T A P with P the aggregate indicator;
//   * smoother: l1-Jacobi (x += (b - A x) / sum_j |a_ij|), one sweep before
//     and after the coarse correction, parallel over rows;
//   * K-cycle: the coarse correction is itself accelerated by two steps of
//     flexible CG preconditioned by the next level's cycle;
//   * coarsest level (<= 400 unknowns): dense Cholesky.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "svh_internal.h"

namespace svh {

struct Csr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

struct AmgLevel {
    Csr A;
    std::vector<double> l1;      // l1 row norms (smoother)
    std::vector<int> agg;        // fine -> coarse index
    std::vector<int> crp, cidx;  // coarse index -> its fine indices (CSR), for a parallel restriction
    int nc = 0;
};

// per-solve scratch of the cycle, one set per level (solves on one hierarchy
// may run concurrently, each with its own workspace)
struct AmgWork {
    struct Lv { std::vector<double> r, rc, xc, v1, w1, rr, v2, w2; };
    std::vector<Lv> lv;
};

struct Amg {
    std::vector<AmgLevel> lv;
    std::vector<double> chol;    // dense Cholesky factor of the coarsest operator (row-major, lower)
    int nco = 0;
};

static void spmv(const Csr& A, const double* x, double* y) {
#pragma omp parallel for schedule(static) if (A.n > 20000)
    for (int i = 0; i < A.n; ++i) {
        double s = 0;
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) s += A.v[p] * x[A.ci[p]];
        y[i] = s;
    }
}

// one pass of pairwise matching on A: returns the number of groups and fills grp.
// A node left alone (all its strong neighbours already matched) then joins the
// group of its strongest neighbour, so every pass at least halves the count.
static int pairwise(const Csr& A, std::vector<int>& grp) {
    const int n = A.n;
    grp.assign(n, -1);
    std::vector<double> strongest(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double m = 0;
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
            if (A.ci[p] != i) m = std::max(m, std::fabs(A.v[p]));
        strongest[i] = m;
    }
    int ng = 0;
    const double beta = 0.25;
    std::vector<int> size;
    for (int i = 0; i < n; ++i) {
        if (grp[i] >= 0) continue;
        int best = -1;
        double bv = 0;
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            const int j = A.ci[p];
            if (j == i || grp[j] >= 0) continue;
            const double c = std::fabs(A.v[p]);
            if (c >= beta * strongest[i] && c > 0 && c > bv) { bv = c; best = j; }
        }
        grp[i] = ng;
        size.push_back(1);
        if (best >= 0) { grp[best] = ng; size[ng] = 2; }
        ++ng;
    }
    // singletons join their strongest neighbour's group
    std::vector<int> target(ng);
    for (int g = 0; g < ng; ++g) target[g] = g;
    for (int i = 0; i < n; ++i) {
        const int g = grp[i];
        if (size[g] != 1) continue;
        int best = -1;
        double bv = 0;
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            const int j = A.ci[p];
            if (j == i) continue;
            const double c = std::fabs(A.v[p]);
            if (c > bv && size[grp[j]] >= 2) { bv = c; best = j; }
        }
        if (best >= 0) target[g] = grp[best];
    }
    std::vector<int> newid(ng, -1);
    int nn = 0;
    for (int i = 0; i < n; ++i) {
        const int t = target[grp[i]];
        if (newid[t] < 0) newid[t] = nn++;
        grp[i] = newid[t];
    }
    return nn;
}

// Galerkin product P^T A P for the indicator prolongation of `agg`
static Csr galerkin(const Csr& A, const std::vector<int>& agg, int nc) {
    std::vector<std::vector<std::pair<int, double>>> rows(nc);
    for (int i = 0; i < A.n; ++i) {
        const int I = agg[i];
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) rows[I].push_back({agg[A.ci[p]], A.v[p]});
    }
    Csr C;
    C.n = nc;
    C.rp.assign(nc + 1, 0);
    for (int I = 0; I < nc; ++I) {
        auto& r = rows[I];
        std::sort(r.begin(), r.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        int last = -1;
        for (auto& e : r) {
            if (e.first != last) {
                C.ci.push_back(e.first);
                C.v.push_back(e.second);
                last = e.first;
            } else {
                C.v.back() += e.second;
            }
        }
        C.rp[I + 1] = (int)C.ci.size();
    }
    return C;
}

static void l1norms(AmgLevel& L) {
    L.l1.assign(L.A.n, 0.0);
    for (int i = 0; i < L.A.n; ++i) {
        double s = 0;
        for (int p = L.A.rp[i]; p < L.A.rp[i + 1]; ++p) s += std::fabs(L.A.v[p]);
        L.l1[i] = s > 0 ? s : 1.0;
    }
}

static bool amg_setup(const Csr& S, Amg& amg) {
    amg.lv.clear();
    AmgLevel L0;
    L0.A = S;
    amg.lv.push_back(std::move(L0));
    while (true) {
        AmgLevel& L = amg.lv.back();
        l1norms(L);
        if (L.A.n <= 400) break;
        std::vector<int> g1, g2;
        const int n1 = pairwise(L.A, g1);
        Csr A1 = galerkin(L.A, g1, n1);
        const int n2 = pairwise(A1, g2);
        if (n2 > 0.85 * L.A.n) break;   // coarsening stalled: stop here
        L.agg.resize(L.A.n);
        for (int i = 0; i < L.A.n; ++i) L.agg[i] = g2[g1[i]];
        L.nc = n2;
        L.crp.assign(n2 + 1, 0);
        for (int i = 0; i < L.A.n; ++i) L.crp[L.agg[i] + 1]++;
        for (int c = 0; c < n2; ++c) L.crp[c + 1] += L.crp[c];
        L.cidx.resize(L.A.n);
        {
            std::vector<int> pos(L.crp.begin(), L.crp.end() - 1);
            for (int i = 0; i < L.A.n; ++i) L.cidx[pos[L.agg[i]]++] = i;
        }
        AmgLevel next;
        next.A = galerkin(L.A, L.agg, n2);
        amg.lv.push_back(std::move(next));
    }
    // dense Cholesky of the coarsest operator
    const Csr& C = amg.lv.back().A;
    const int n = C.n;
    amg.nco = n;
    if (std::getenv("SVH_DEBUG_AMG")) {
        for (const auto& L : amg.lv) std::fprintf(stderr, "amg level n=%d nnz=%zu\n", L.A.n, L.A.ci.size());
    }
    if (n > 3000) {
        if (std::getenv("SVH_DEBUG_AMG")) std::fprintf(stderr, "amg coarsening stalled at n=%d\n", n);
        return false;
    }
    std::vector<double> D((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int p = C.rp[i]; p < C.rp[i + 1]; ++p) D[(size_t)i * n + C.ci[p]] = C.v[p];
    for (int j = 0; j < n; ++j) {
        double s = D[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= D[(size_t)j * n + k] * D[(size_t)j * n + k];
        if (!(s > 0)) {
            if (std::getenv("SVH_DEBUG_AMG")) std::fprintf(stderr, "amg coarsest Cholesky pivot %d = %g\n", j, s);
            return false;
        }
        const double d = std::sqrt(s);
        D[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = D[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= D[(size_t)i * n + k] * D[(size_t)j * n + k];
            D[(size_t)i * n + j] = t / d;
        }
    }
    amg.chol.swap(D);
    return true;
}

static void coarse_solve(const Amg& amg, const double* b, double* x) {
    const int n = amg.nco;
    const double* L = amg.chol.data();
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

static double dotp(const double* a, const double* b, int n) {
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void kcycle(const Amg& amg, AmgWork& wk, int l, const double* b, double* x);

// size the workspace for this hierarchy (hierarchies of different frequencies
// differ in their coarse levels, so every level's sizes are checked)
static void work_init(const Amg& amg, AmgWork& wk) {
    bool ok = wk.lv.size() == amg.lv.size();
    for (size_t l = 0; ok && l < amg.lv.size(); ++l)
        ok = wk.lv[l].r.size() == (size_t)amg.lv[l].A.n && wk.lv[l].rc.size() == (size_t)amg.lv[l].nc;
    if (ok) return;
    wk.lv.assign(amg.lv.size(), AmgWork::Lv());
    for (size_t l = 0; l < amg.lv.size(); ++l) {
        const int n = amg.lv[l].A.n, nc = amg.lv[l].nc;
        auto& w = wk.lv[l];
        w.r.assign(n, 0); w.rc.assign(nc, 0); w.xc.assign(nc, 0);
        w.v1.assign(n, 0); w.w1.assign(n, 0); w.rr.assign(n, 0); w.v2.assign(n, 0); w.w2.assign(n, 0);
    }
}

// Two steps of flexible CG on level l with the level-l cycle as
// preconditioner: the K-cycle's Krylov acceleration of the coarse solve.
static void coarse_krylov(const Amg& amg, AmgWork& wk, int l, const double* b, double* x) {
    const AmgLevel& L = amg.lv[l];
    const Csr& A = L.A;
    const int n = A.n;
    if (l == (int)amg.lv.size() - 1) {
        kcycle(amg, wk, l, b, x);
        return;
    }
    auto& W = wk.lv[l];
    double* v1 = W.v1.data();
    double* w1 = W.w1.data();
    double* r = W.rr.data();
    double* v2 = W.v2.data();
    double* w2 = W.w2.data();
    kcycle(amg, wk, l, b, v1);
    spmv(A, v1, w1);
    const double d11 = dotp(v1, w1, n);
    const double g1 = dotp(v1, b, n);
    if (!(d11 > 0)) { std::fill(x, x + n, 0.0); return; }
    const double a1 = g1 / d11;
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) r[i] = b[i] - a1 * w1[i];
    const double nr = std::sqrt(dotp(r, r, n)), nb = std::sqrt(dotp(b, b, n));
    if (nr <= 0.25 * nb) {   // one step already reduced the residual enough
#pragma omp parallel for schedule(static) if (n > 20000)
        for (int i = 0; i < n; ++i) x[i] = a1 * v1[i];
        return;
    }
    kcycle(amg, wk, l, r, v2);
    spmv(A, v2, w2);
    // minimise the A-norm of the error over span{v1, v2} (2 x 2 Galerkin system)
    const double d12 = dotp(v1, w2, n), d22 = dotp(v2, w2, n);
    const double g2 = dotp(v2, b, n);
    const double det = d11 * d22 - d12 * d12;
    double c1 = a1, c2 = 0.0;
    if (det > 1e-14 * d11 * d22) {
        c1 = (g1 * d22 - g2 * d12) / det;
        c2 = (d11 * g2 - d12 * g1) / det;
    }
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) x[i] = c1 * v1[i] + c2 * v2[i];
}

// K-cycle with zero initial guess: x ~= A_l^{-1} b. One l1-Jacobi sweep,
// coarse correction by coarse_krylov on level l+1, one l1-Jacobi sweep.
static void kcycle(const Amg& amg, AmgWork& wk, int l, const double* b, double* x) {
    const AmgLevel& L = amg.lv[l];
    const int n = L.A.n;
    if (l == (int)amg.lv.size() - 1) {
        coarse_solve(amg, b, x);
        return;
    }
    double* r = wk.lv[l].r.data();
    double* rc = wk.lv[l].rc.data();
    double* xc = wk.lv[l].xc.data();
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) x[i] = b[i] / L.l1[i];
    spmv(L.A, x, r);
#pragma omp parallel for schedule(static) if (L.nc > 20000)
    for (int c = 0; c < L.nc; ++c) {
        double s = 0;
        for (int p = L.crp[c]; p < L.crp[c + 1]; ++p) s += b[L.cidx[p]] - r[L.cidx[p]];
        rc[c] = s;
    }
    coarse_krylov(amg, wk, l + 1, rc, xc);
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) x[i] += xc[L.agg[i]];
    spmv(L.A, x, r);
#pragma omp parallel for schedule(static) if (n > 20000)
    for (int i = 0; i < n; ++i) x[i] += (b[i] - r[i]) / L.l1[i];
}

// Flexible CG (the K-cycle is not a fixed linear operator) for S x = b, x0 = 0;
// each new direction is S-orthogonalised against the previous one.
// Returns iterations, or -1 if not converged.
static int pcg(const Csr& S, const Amg& amg, AmgWork& wk, const double* b, double* x, double tol, int maxit) {
    work_init(amg, wk);
    const int n = S.n;
    std::vector<double> r(b, b + n), z(n), p(n), q(n), pold(n), qold(n);
    std::fill(x, x + n, 0.0);
    const double nb = std::sqrt(dotp(r.data(), r.data(), n));
    if (nb == 0) return 0;
    double pq_old = 0;
    for (int it = 1; it <= maxit; ++it) {
        kcycle(amg, wk, 0, r.data(), z.data());
        p = z;
        if (it > 1) {
            const double beta = dotp(z.data(), qold.data(), n) / pq_old;
#pragma omp parallel for schedule(static) if (n > 20000)
            for (int i = 0; i < n; ++i) p[i] -= beta * pold[i];
        }
        spmv(S, p.data(), q.data());
        const double pq = dotp(p.data(), q.data(), n);
        const double alpha = dotp(p.data(), r.data(), n) / pq;
#pragma omp parallel for schedule(static) if (n > 20000)
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        if (std::sqrt(dotp(r.data(), r.data(), n)) <= tol * nb) return it;
        pold.swap(p);
        qold.swap(q);
        pq_old = pq;
    }
    return -1;
}

// ------------------------------------------------------------------ preconditioner state on a handle
struct Precond {
    double omega = 0;
    std::vector<double> Yd;       // [5K] |Z_kk|
    std::vector<int> free_id;     // node -> free index or -1
    std::vector<int> free_nodes;  // free index -> node
    Csr S;
    Amg amg;
    double tol = 1e-8;
    int maxit = 500;
    long long pcg_calls = 0, pcg_iters = 0;
    void* dev = nullptr;          // device copy of the hierarchy (amg_dev.cu)
    ~Precond() { if (dev) amg_dev_destroy(dev); }
};

static const double kFlux[5][6] = {
    {-1, 1, 0, 0, 0, 0}, {0, 0, -1, 1, 0, 0}, {0, 0, 0, 0, -1, 1}, {0.5, 0.5, -0.5, -0.5, 0, 0}, {0.5, 0.5, 0.5, 0.5, -1, -1}};
static const double kSbeta[5] = {1.0, 1.0, 1.0, 1.0 / 6.0, 0.5};

// one Precond per frequency of the current solve (h->precond points to this)
struct PrecondSet {
    std::vector<Precond*> f;
    ~PrecondSet() { for (Precond* p : f) delete p; }
};

void precond_free(Handle* h) {
    delete static_cast<PrecondSet*>(h->precond);
    h->precond = nullptr;
}

static Precond* P_at(Handle* h, int fi) { return static_cast<PrecondSet*>(h->precond)->f[fi]; }

// Y = |diag Z| (Eq. 12) at omega: two-fluid diagonal plus the Green self term
// j omega mu dx T_bb(0) (G00(0) for x, y, z; Qx+Qy for 2D; Qx+Qy+4Qz for 3D).
static int precond_setup_one(Handle* h, double omega, double tol, Precond*& out) {
    Precond* P = new Precond();
    P->omega = omega;
    P->tol = tol;
    const double mu = 4e-7 * 3.14159265358979323846;
    const int64_t K = h->K, M = h->M, Kt = (int64_t)h->Kx * h->Ky * h->Kz;
    const double* T = h->toep.data();
    const double t0[7] = {T[0], T[Kt], T[2 * Kt], T[3 * Kt], T[4 * Kt], T[5 * Kt], T[6 * Kt]};
    const double self[5] = {t0[0], t0[0], t0[0], t0[4] + t0[5], t0[4] + t0[5] + 4 * t0[6]};
    P->Yd.resize(5 * K);
    for (int64_t v = 0; v < K; ++v) {
        const double lm = h->lam[v], s0 = h->sig0[v];
        const double wml2 = omega * mu * lm * lm, tt = s0 * wml2, den = 1 + tt * tt;
        const double ca = s0 * wml2 * wml2 / den, cb = omega * mu * (lm * lm / den);
        for (int a = 0; a < 5; ++a) {
            const double re = ca * kSbeta[a] / h->dx;
            const double im = cb * kSbeta[a] / h->dx + omega * mu * h->dx * self[a];
            P->Yd[a * K + v] = std::sqrt(re * re + im * im);
        }
    }
    P->free_id.assign(M, -1);
    for (int64_t m = 0; m < M; ++m)
        if (!h->fixed[m]) {
            P->free_id[m] = (int)P->free_nodes.size();
            P->free_nodes.push_back((int)m);
        }
    const int nf = (int)P->free_nodes.size();
    // S = A_F Y^-1 A_F^T, row by row: row m couples the nodes of the voxels at m
    std::vector<std::vector<std::pair<int, double>>> rows(nf);
    for (int64_t v = 0; v < K; ++v) {
        const int32_t* nd = &h->node[v * 6];
        for (int a = 0; a < 5; ++a) {
            const double yi = 1.0 / P->Yd[a * K + v];
            for (int f1 = 0; f1 < 6; ++f1) {
                if (kFlux[a][f1] == 0) continue;
                const int r = P->free_id[nd[f1]];
                if (r < 0) continue;
                for (int f2 = 0; f2 < 6; ++f2) {
                    if (kFlux[a][f2] == 0) continue;
                    const int c = P->free_id[nd[f2]];
                    if (c < 0) continue;
                    rows[r].push_back({c, kFlux[a][f1] * kFlux[a][f2] * yi});
                }
            }
        }
    }
    Csr& S = P->S;
    S.n = nf;
    S.rp.assign(nf + 1, 0);
    for (int r = 0; r < nf; ++r) {
        auto& e = rows[r];
        std::sort(e.begin(), e.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        int last = -1;
        for (auto& q : e) {
            if (q.first != last) { S.ci.push_back(q.first); S.v.push_back(q.second); last = q.first; }
            else S.v.back() += q.second;
        }
        S.rp[r + 1] = (int)S.ci.size();
        std::vector<std::pair<int, double>>().swap(e);
    }
    if (!amg_setup(S, P->amg)) {
        delete P;
        return set_err(h, SVH_ERR_SINGULAR, "preconditioner: coarsest Schur operator not positive definite "
                                            "(a conductor without terminal or gauge?)");
    }
    out = P;
    return SVH_OK;
}

int precond_setup(Handle* h, const double* omegas, int nfreq, double tol) {
    if (!h->have_grid || !h->have_kernels) return set_err(h, SVH_ERR_STATE, "preconditioner: grid and kernels needed");
    precond_free(h);
    PrecondSet* set = new PrecondSet();
    h->precond = set;
    for (int f = 0; f < nfreq; ++f) {
        Precond* P = nullptr;
        int rc = precond_setup_one(h, omegas[f], tol, P);
        if (rc) return rc;
        set->f.push_back(P);
    }
    return SVH_OK;
}

// b = S^{-1} e for nb complex right-hand sides given on the free nodes
// (interleaved re, im; e[rhs][nf]); right-hand side r belongs to frequency
// r / per_freq. Real and imaginary parts are two real solves.
int precond_schur_solve(Handle* h, int nb, int per_freq, const double* e, double* b) {
    const int nf = P_at(h, 0)->S.n;
    const int ntask = 2 * nb;   // real and imaginary parts of every right-hand side
    const int nthreads = omp_get_max_threads();
    // many independent solves: one per thread (inner loops serial); few: inner loops parallel
    const bool outer = ntask >= 4 && nthreads > 1;
    std::vector<int> status(ntask, 0);
    std::vector<long long> iters(ntask, 0);
    auto one = [&](int t, AmgWork& wk, std::vector<double>& re, std::vector<double>& xr) {
        const int r = t >> 1, part = t & 1;
        Precond* P = P_at(h, r / per_freq);
        for (int i = 0; i < nf; ++i) re[i] = e[((size_t)r * nf + i) * 2 + part];
        const int it = pcg(P->S, P->amg, wk, re.data(), xr.data(), P->tol, P->maxit);
        status[t] = it < 0;
        iters[t] = it;
        for (int i = 0; i < nf; ++i) b[((size_t)r * nf + i) * 2 + part] = xr[i];
    };
    if (outer) {
#pragma omp parallel
        {
            AmgWork wk;
            std::vector<double> re(nf), xr(nf);
#pragma omp for schedule(dynamic, 1)
            for (int t = 0; t < ntask; ++t) one(t, wk, re, xr);
        }
    } else {
        AmgWork wk;
        std::vector<double> re(nf), xr(nf);
        for (int t = 0; t < ntask; ++t) one(t, wk, re, xr);
    }
    for (int t = 0; t < ntask; ++t) {
        if (status[t]) return set_err(h, SVH_ERR_NOT_CONVERGED, "preconditioner: AMG-PCG did not converge");
        Precond* P = P_at(h, (t >> 1) / per_freq);
        P->pcg_calls++;
        P->pcg_iters += iters[t];
    }
    return SVH_OK;
}

const double* precond_Y(Handle* h, int fi) { return P_at(h, fi)->Yd.data(); }
int precond_nfreq(Handle* h) { return h->precond ? (int)static_cast<PrecondSet*>(h->precond)->f.size() : 0; }
int precond_view(Handle* h, int fi, AmgView& out) {
    if (!h->precond || fi < 0 || fi >= precond_nfreq(h)) return set_err(h, SVH_ERR_STATE, "preconditioner: not set up");
    const Precond* P = P_at(h, fi);
    out.lv.clear();
    for (const AmgLevel& L : P->amg.lv) {
        AmgLevelView v;
        v.n = L.A.n;
        v.nc = L.nc;
        v.rp = L.A.rp.data();
        v.ci = L.A.ci.data();
        v.v = L.A.v.data();
        v.l1 = L.l1.data();
        v.agg = L.agg.data();
        v.crp = L.crp.data();
        v.cidx = L.cidx.data();
        out.lv.push_back(v);
    }
    out.chol = P->amg.chol.data();
    out.nco = P->amg.nco;
    out.tol = P->tol;
    out.maxit = P->maxit;
    return SVH_OK;
}
void*& precond_dev(Handle* h, int fi) { return P_at(h, fi)->dev; }
void precond_count(Handle* h, int fi, long long calls, long long iters) {
    Precond* P = P_at(h, fi);
    P->pcg_calls += calls;
    P->pcg_iters += iters;
}
const int* precond_free_nodes(Handle* h, int* nf) {
    Precond* P = P_at(h, 0);
    *nf = (int)P->free_nodes.size();
    return P->free_nodes.data();
}
int precond_levels(Handle* h) { return h->precond ? (int)P_at(h, 0)->amg.lv.size() : 0; }
double precond_avg_iters(Handle* h) {
    if (!h->precond) return 0.0;
    long long c = 0, it = 0;
    for (Precond* P : static_cast<PrecondSet*>(h->precond)->f) { c += P->pcg_calls; it += P->pcg_iters; }
    return c ? (double)it / c : 0.0;
}

// host reference of the whole preconditioner apply (Eq. 13-15) for nb vectors of length N
int precond_apply_host(Handle* h, int nb, const double* in, double* out) {
    Precond* P = P_at(h, 0);
    const int64_t K = h->K, M = h->M, N = 5 * K + M;
    const int nf = P->S.n;
    std::vector<double> e((size_t)nb * nf * 2), bsol((size_t)nb * nf * 2);
    for (int r = 0; r < nb; ++r) {
        const double* c = in + (size_t)r * N * 2;
        double* ee = e.data() + (size_t)r * nf * 2;
        for (int i = 0; i < nf; ++i) {
            const int m = P->free_nodes[i];
            ee[2 * i] = c[(5 * K + m) * 2];
            ee[2 * i + 1] = c[(5 * K + m) * 2 + 1];
        }
        for (int64_t v = 0; v < K; ++v)
            for (int a = 0; a < 5; ++a) {
                const double yi = 1.0 / P->Yd[a * K + v];
                const double cr = c[(a * K + v) * 2] * yi, ci = c[(a * K + v) * 2 + 1] * yi;
                for (int f = 0; f < 6; ++f) {
                    const int id = P->free_id[h->node[v * 6 + f]];
                    if (kFlux[a][f] == 0 || id < 0) continue;
                    ee[2 * id] -= kFlux[a][f] * cr;
                    ee[2 * id + 1] -= kFlux[a][f] * ci;
                }
            }
    }
    int rc = precond_schur_solve(h, nb, nb, e.data(), bsol.data());
    if (rc) return rc;
    for (int r = 0; r < nb; ++r) {
        const double* c = in + (size_t)r * N * 2;
        double* o = out + (size_t)r * N * 2;
        const double* bb = bsol.data() + (size_t)r * nf * 2;
        for (int64_t m = 0; m < M; ++m) {   // fixed nodes: identity
            o[(5 * K + m) * 2] = c[(5 * K + m) * 2];
            o[(5 * K + m) * 2 + 1] = c[(5 * K + m) * 2 + 1];
        }
        for (int i = 0; i < nf; ++i) {
            o[(5 * K + P->free_nodes[i]) * 2] = bb[2 * i];
            o[(5 * K + P->free_nodes[i]) * 2 + 1] = bb[2 * i + 1];
        }
        for (int64_t v = 0; v < K; ++v)
            for (int a = 0; a < 5; ++a) {
                double sr = c[(a * K + v) * 2], si = c[(a * K + v) * 2 + 1];
                for (int f = 0; f < 6; ++f) {
                    const int id = P->free_id[h->node[v * 6 + f]];
                    if (kFlux[a][f] == 0 || id < 0) continue;
                    sr += kFlux[a][f] * bb[2 * id];
                    si += kFlux[a][f] * bb[2 * id + 1];
                }
                const double yi = 1.0 / P->Yd[a * K + v];
                o[(a * K + v) * 2] = sr * yi;
                o[(a * K + v) * 2 + 1] = si * yi;
            }
    }
    return SVH_OK;
}

}  // namespace svh

using namespace svh;

extern "C" int svh_host_amg_solve(int n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                                  const double* b, double* x, double tol, int maxit, int32_t* iters,
                                  int32_t* levels) {
    if (n <= 0 || !rowptr || !colidx || !vals || !b || !x || !(tol > 0) || maxit <= 0) return SVH_ERR_ARG;
    Csr S;
    S.n = n;
    S.rp.assign(rowptr, rowptr + n + 1);
    S.ci.assign(colidx, colidx + rowptr[n]);
    S.v.assign(vals, vals + rowptr[n]);
    Amg amg;
    if (!amg_setup(S, amg)) return SVH_ERR_SINGULAR;
    AmgWork wk;
    const int it = pcg(S, amg, wk, b, x, tol, maxit);
    if (iters) *iters = it;
    if (levels) *levels = (int)amg.lv.size();
    return it < 0 ? SVH_ERR_NOT_CONVERGED : SVH_OK;
}

// S x = b for nrhs complex right-hand sides (b, x: [nrhs][n] interleaved
// re, im; real and imaginary parts are separate real systems) by the device
// AMG-CG on a hierarchy built here (the solver of svh_solve's preconditioner).
extern "C" int svh_device_amg_solve(int n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                                    const double* b, double* x, int nrhs, double tol, int maxit, int32_t* iters,
                                    int32_t* levels) {
    if (n <= 0 || nrhs <= 0 || !rowptr || !colidx || !vals || !b || !x || !(tol > 0) || maxit <= 0) return SVH_ERR_ARG;
    Handle h;
    if (cudaGetDevice(&h.device) != cudaSuccess) return SVH_ERR_CUDA;
    PrecondSet* set = new PrecondSet();
    h.precond = set;
    Precond* P = new Precond();
    set->f.push_back(P);
    P->tol = tol;
    P->maxit = maxit;
    P->S.n = n;
    P->S.rp.assign(rowptr, rowptr + n + 1);
    P->S.ci.assign(colidx, colidx + rowptr[n]);
    P->S.v.assign(vals, vals + rowptr[n]);
    int rc = SVH_OK;
    DevBuf de, dx;
    if (!amg_setup(P->S, P->amg)) rc = SVH_ERR_SINGULAR;
    const size_t bytes = (size_t)nrhs * n * 16;
    if (!rc) rc = dev_upload(&h, de, b, bytes);
    if (!rc) rc = dev_alloc(&h, dx, bytes);
    if (!rc) rc = precond_schur_solve_dev(&h, nrhs, nrhs, de.p, dx.p);
    if (!rc && cudaMemcpy(x, dx.p, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SVH_ERR_CUDA;
    if (iters) *iters = P->pcg_calls ? (int32_t)(P->pcg_iters / P->pcg_calls) : 0;
    if (levels) *levels = (int32_t)P->amg.lv.size();
    dev_free(de);
    dev_free(dx);
    precond_free(&h);
    return rc;
}
