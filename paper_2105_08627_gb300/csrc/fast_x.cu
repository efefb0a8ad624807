// fast_x.cu -- launchers of the size-specialised x passes (see fastpass.cuh).
#include <algorithm>
#include <type_traits>

#include "fastpass.cuh"

namespace svh {

template <typename T, int N1, int N2, bool INV, int NT>
static void run_x(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    static_assert(NT % N2 == 0, "threads per block must be a multiple of N2");
    constexpr int L = NT / N2;
    const size_t sm = (size_t)(N1 * N2 + L * N2 * (N1 + 1)) * sizeof(C);
    cudaFuncSetAttribute(k_xrow<T, N1, N2, INV, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned grid = (unsigned)((a.nlines + L - 1) / L);
    k_xrow<T, N1, N2, INV, NT><<<grid, NT, sm, s>>>(a);
}

// inverse + epilogue, grouped by (item, row): NT threads = 5 bases x (NT / (5 N2)) rows x N2
template <typename T, int N1, int N2, int NT>
static void run_xinv(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int L = NT / N2;
    constexpr int G = L / 5;
    const size_t step1 = (size_t)L * N2 * (N1 + 1);
    const size_t keep = (size_t)L * (a.Kx + 1);
    const size_t sm = (size_t)(N1 * N2 + std::max(step1, keep)) * sizeof(C);
    cudaFuncSetAttribute(k_xinv_grouped<T, N1, N2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int64_t groups = (int64_t)a.nb * a.nrows;
    k_xinv_grouped<T, N1, N2, NT><<<(unsigned)((groups + G - 1) / G), NT, sm, s>>>(a);
}

// Tile variants (FP32; a.var selects one, the autotuner times them):
// row pass (forward, and inverse sizes without a grouped kernel):
//   0: N1 x N2 split, 256 threads; 1: 512 threads; 2: 128 threads;
//   3: transposed split N2 x N1, 256 threads (where both factors suit);
// grouped inverse: 0: 320 threads (4 item-rows x 5 bases per 16-point
//   column set), 1: 640 threads, 2: 160 threads.
// FP64 has variant 0 only (128 threads; grouped inverse 320).
template <typename T, bool INV, int N1, int N2, bool SWAP>
static bool run_x_size(const PassArgs& a, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        switch (a.var) {
            case 1: run_x<T, N1, N2, INV, 512>(a, s); return true;
            case 2: run_x<T, N1, N2, INV, 128>(a, s); return true;
            case 3:
                if constexpr (SWAP) { run_x<T, N2, N1, INV, 256>(a, s); return true; }
                break;
            default: break;
        }
        run_x<T, N1, N2, INV, 256>(a, s);
    } else {
        run_x<T, N1, N2, INV, 128>(a, s);
    }
    return true;
}

template <typename T, int N1, int N2>
static bool run_xinv_size(const PassArgs& a, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (a.var == 1) { run_xinv<T, N1, N2, 640>(a, s); return true; }
        if (a.var == 2) { run_xinv<T, N1, N2, 160>(a, s); return true; }
    }
    run_xinv<T, N1, N2, 320>(a, s);
    return true;
}

template <typename T, bool INV>
static bool dispatch_x(const PassArgs& a, cudaStream_t s) {
    if (INV) {
        switch (a.Px) {
            case 16: return run_xinv_size<T, 4, 4>(a, s);
            case 32: return run_xinv_size<T, 8, 4>(a, s);
            case 64: return run_xinv_size<T, 8, 8>(a, s);
            case 128: return run_xinv_size<T, 16, 8>(a, s);
            case 256: return run_xinv_size<T, 16, 16>(a, s);
            case 512: return run_xinv_size<T, 32, 16>(a, s);
            case 1024: return run_xinv_size<T, 32, 32>(a, s);
            default: break;
        }
    }
    switch (a.Px) {
        case 16: return run_x_size<T, INV, 4, 4, false>(a, s);
        case 32: return run_x_size<T, INV, 8, 4, true>(a, s);
        case 48: return run_x_size<T, INV, 12, 4, false>(a, s);
        case 64: return run_x_size<T, INV, 8, 8, false>(a, s);
        case 96: return run_x_size<T, INV, 12, 8, false>(a, s);
        case 128: return run_x_size<T, INV, 16, 8, true>(a, s);
        case 192: return run_x_size<T, INV, 24, 8, false>(a, s);
        case 256: return run_x_size<T, INV, 16, 16, false>(a, s);
        case 384: return run_x_size<T, INV, 24, 16, false>(a, s);
        case 512: return run_x_size<T, INV, 32, 16, true>(a, s);
        case 768: return run_x_size<T, INV, 48, 16, false>(a, s);
        case 1024: return run_x_size<T, INV, 32, 32, false>(a, s);
        default: return false;
    }
}

int x_fast_variants(int Px, bool inv, bool fp32) {
    if (!fp32) return 1;
    const bool grouped = Px == 16 || Px == 32 || Px == 64 || Px == 128 || Px == 256 || Px == 512 || Px == 1024;
    if (inv && grouped) return 3;
    switch (Px) {
        case 32: case 128: case 512: return 4;
        case 16: case 48: case 64: case 96: case 192: case 256: case 384: case 768: case 1024: return 3;
        default: return 0;
    }
}

template <typename T> bool launch_x_fast(const PassArgs& a, bool inv, cudaStream_t s) {
    return inv ? dispatch_x<T, true>(a, s) : dispatch_x<T, false>(a, s);
}
template bool launch_x_fast<float>(const PassArgs&, bool, cudaStream_t);
template bool launch_x_fast<double>(const PassArgs&, bool, cudaStream_t);

}  // namespace svh
