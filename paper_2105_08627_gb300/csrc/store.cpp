// store.cpp -- Algorithm 2: the install-time store of Tucker-compressed unit
// Toeplitz tensors, cropped to a structure's grid at set-up.
//
// Algorithm 2 computes the Toeplitz tensors once for a large domain, keeps
// their Tucker cores and factors (Algorithm 1) on disk, and at each set-up
// restores them (Eq. 10), takes the leading K_x x K_y x K_z block and scales
// it. The unit kernels here are dimensionless (every block of Z is
// j omega mu dx T_u, with the dx scale applied inside the product), so the
// crop needs no scaling factor; a store therefore serves every voxel size.
// Cropping the restored tensor equals restoring with the leading K_i rows of
// each factor, so only those rows are used.
//
// File layout (host byte order, doubles): 8-byte magic "SVHTST01", int32
// Kx, Ky, Kz, int32 0, double tol; then for each of the 7 kernels: int32 d1,
// d2, d3, int32 0, core[d3][d2][d1], F1[Kx][d1], F2[Ky][d2], F3[Kz][d3].
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "svh_internal.h"

namespace svh {
namespace {

const char kMagic[8] = {'S', 'V', 'H', 'T', 'S', 'T', '0', '1'};

struct StoreKernel {
    int d[3] = {0, 0, 0};
    std::vector<double> core, F[3];
};

struct FileCloser {
    void operator()(std::FILE* f) const { if (f) std::fclose(f); }
};
using File = std::unique_ptr<std::FILE, FileCloser>;

int write_store(const char* path, int Kx, int Ky, int Kz, const double* T, double tol) {
    const int K[3] = {Kx, Ky, Kz};
    const size_t Kt = (size_t)Kx * Ky * Kz;
    File f(std::fopen(path, "wb"));
    if (!f) return SVH_ERR_ARG;
    const int32_t hdr[4] = {Kx, Ky, Kz, 0};
    bool ok = std::fwrite(kMagic, 1, 8, f.get()) == 8 && std::fwrite(hdr, 4, 4, f.get()) == 4 &&
              std::fwrite(&tol, 8, 1, f.get()) == 1;
    std::vector<double> core(Kt), F1((size_t)Kx * Kx), F2((size_t)Ky * Ky), F3((size_t)Kz * Kz);
    for (int u = 0; ok && u < 7; ++u) {
        int32_t d[4] = {0, 0, 0, 0};
        const int rc = svh_host_tucker_svd(T + u * Kt, Kx, Ky, Kz, tol, d, core.data(), F1.data(), F2.data(),
                                           F3.data());
        if (rc != SVH_OK) return rc;
        const size_t nc = (size_t)d[0] * d[1] * d[2];
        ok = std::fwrite(d, 4, 4, f.get()) == 4 && std::fwrite(core.data(), 8, nc, f.get()) == nc &&
             std::fwrite(F1.data(), 8, (size_t)K[0] * d[0], f.get()) == (size_t)K[0] * d[0] &&
             std::fwrite(F2.data(), 8, (size_t)K[1] * d[1], f.get()) == (size_t)K[1] * d[1] &&
             std::fwrite(F3.data(), 8, (size_t)K[2] * d[2], f.get()) == (size_t)K[2] * d[2];
    }
    return ok ? SVH_OK : SVH_ERR_ARG;
}

// reads the store and restores the leading Kx x Ky x Kz block of each kernel into T[7][Kz][Ky][Kx]
int read_store(const char* path, int Kx, int Ky, int Kz, double* T, int32_t* ranks) {
    File f(std::fopen(path, "rb"));
    if (!f) return SVH_ERR_ARG;
    char magic[8];
    int32_t hdr[4];
    double tol = 0;
    if (std::fread(magic, 1, 8, f.get()) != 8 || std::memcmp(magic, kMagic, 8) != 0 ||
        std::fread(hdr, 4, 4, f.get()) != 4 || std::fread(&tol, 8, 1, f.get()) != 1)
        return SVH_ERR_ARG;
    const int S[3] = {hdr[0], hdr[1], hdr[2]};
    if (S[0] <= 0 || S[1] <= 0 || S[2] <= 0 || Kx > S[0] || Ky > S[1] || Kz > S[2]) return SVH_ERR_ARG;
    const int K[3] = {Kx, Ky, Kz};
    const size_t Kt = (size_t)Kx * Ky * Kz;
    for (int u = 0; u < 7; ++u) {
        int32_t d[4];
        if (std::fread(d, 4, 4, f.get()) != 4) return SVH_ERR_ARG;
        for (int i = 0; i < 3; ++i)
            if (d[i] <= 0 || d[i] > S[i]) return SVH_ERR_ARG;
        StoreKernel k;
        for (int i = 0; i < 3; ++i) k.d[i] = d[i];
        const size_t nc = (size_t)d[0] * d[1] * d[2];
        k.core.resize(nc);
        if (std::fread(k.core.data(), 8, nc, f.get()) != nc) return SVH_ERR_ARG;
        for (int i = 0; i < 3; ++i) {
            k.F[i].resize((size_t)S[i] * d[i]);
            if (std::fread(k.F[i].data(), 8, k.F[i].size(), f.get()) != k.F[i].size()) return SVH_ERR_ARG;
        }
        if (ranks)
            for (int i = 0; i < 3; ++i) ranks[u * 3 + i] = d[i];
        // Eq. 10 with the leading K_i rows of each factor (rows are indexed k * d_i + c)
        const int d1 = d[0], d2 = d[1], d3 = d[2];
        std::vector<double> A1((size_t)d3 * d2 * Kx), A2((size_t)d3 * Ky * Kx);
#pragma omp parallel for schedule(static)
        for (int cb = 0; cb < d3 * d2; ++cb)
            for (int x = 0; x < Kx; ++x) {
                double s = 0;
                const double* c = k.core.data() + (size_t)cb * d1;
                const double* fr = k.F[0].data() + (size_t)x * d1;
                for (int a = 0; a < d1; ++a) s += c[a] * fr[a];
                A1[(size_t)cb * Kx + x] = s;
            }
#pragma omp parallel for schedule(static)
        for (int c3 = 0; c3 < d3; ++c3)
            for (int y = 0; y < Ky; ++y) {
                double* out = A2.data() + ((size_t)c3 * Ky + y) * Kx;
                for (int x = 0; x < Kx; ++x) out[x] = 0;
                const double* fr = k.F[1].data() + (size_t)y * d2;
                for (int b = 0; b < d2; ++b) {
                    const double w = fr[b];
                    const double* in = A1.data() + ((size_t)c3 * d2 + b) * Kx;
                    for (int x = 0; x < Kx; ++x) out[x] += w * in[x];
                }
            }
        double* Tu = T + u * Kt;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < Kz; ++z) {
            double* out = Tu + (size_t)z * Ky * Kx;
            for (size_t i = 0; i < (size_t)Ky * Kx; ++i) out[i] = 0;
            const double* fr = k.F[2].data() + (size_t)z * d3;
            for (int c3 = 0; c3 < d3; ++c3) {
                const double w = fr[c3];
                const double* in = A2.data() + (size_t)c3 * Ky * Kx;
                for (size_t i = 0; i < (size_t)Ky * Kx; ++i) out[i] += w * in[i];
            }
        }
    }
    (void)K;
    return SVH_OK;
}

}  // namespace
}  // namespace svh

using namespace svh;

extern "C" int svh_toeplitz_store_write(const char* path, int Kx, int Ky, int Kz, const double* T, double tol) {
    if (!path || Kx <= 0 || Ky <= 0 || Kz <= 0 || !(tol > 0)) return SVH_ERR_ARG;
    if (T) return write_store(path, Kx, Ky, Kz, T, tol);
    // generate the unit tensors on the current device (the quadrature of svh_generate_toeplitz)
    Handle h;
    if (cudaGetDevice(&h.device) != cudaSuccess) return SVH_ERR_CUDA;
    h.Kx = Kx;
    h.Ky = Ky;
    h.Kz = Kz;
    std::vector<double> Tg;
    const int rc = generate_toeplitz_device(&h, Tg);
    if (rc) return rc;
    return write_store(path, Kx, Ky, Kz, Tg.data(), tol);
}

extern "C" int svh_toeplitz_store_read(const char* path, int Kx, int Ky, int Kz, double* T, int32_t* ranks) {
    if (!path || !T || Kx <= 0 || Ky <= 0 || Kz <= 0) return SVH_ERR_ARG;
    return read_store(path, Kx, Ky, Kz, T, ranks);
}

extern "C" int svh_load_toeplitz_store(svh_handle* hh, const char* path) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !path) return SVH_ERR_ARG;
    if (!h->have_grid) return set_err(h, SVH_ERR_STATE, "svh_load_toeplitz_store: call svh_setup_grid first");
    std::vector<double> T((size_t)7 * h->Kx * h->Ky * h->Kz);
    const int rc = read_store(path, h->Kx, h->Ky, h->Kz, T.data(), nullptr);
    if (rc) return set_err(h, rc, "svh_load_toeplitz_store: unreadable store, or a grid larger than the store's");
    return svh_load_toeplitz(hh, T.data());
}
