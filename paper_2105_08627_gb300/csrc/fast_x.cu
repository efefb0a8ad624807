// fast_x.cu -- launchers of the size-specialised x passes (see fastpass.cuh).
#include <algorithm>

#include "fastpass.cuh"

namespace svh {

template <typename T, int N1, int N2, bool INV>
static void run_x(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int NT = sizeof(T) == 4 ? 256 : 128;
    constexpr int L = NT / N2;
    const size_t sm = (size_t)(N1 * N2 + L * N2 * (N1 + 1)) * sizeof(C);
    cudaFuncSetAttribute(k_xrow<T, N1, N2, INV, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned grid = (unsigned)((a.nlines + L - 1) / L);
    k_xrow<T, N1, N2, INV, NT><<<grid, NT, sm, s>>>(a);
}

// inverse + epilogue, grouped by (item, row): 320 threads = 5 bases x (64 / N2) rows x N2
template <typename T, int N1, int N2>
static void run_xinv(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int NT = 320;
    constexpr int L = NT / N2;
    constexpr int G = L / 5;
    const size_t step1 = (size_t)L * N2 * (N1 + 1);
    const size_t keep = (size_t)L * (a.Kx + 1);
    const size_t sm = (size_t)(N1 * N2 + std::max(step1, keep)) * sizeof(C);
    cudaFuncSetAttribute(k_xinv_grouped<T, N1, N2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int64_t groups = (int64_t)a.nb * a.nrows;
    k_xinv_grouped<T, N1, N2, NT><<<(unsigned)((groups + G - 1) / G), NT, sm, s>>>(a);
}

template <typename T, bool INV>
static bool dispatch_x(const PassArgs& a, cudaStream_t s) {
    if (INV) {
        switch (a.Px) {
            case 16: run_xinv<T, 4, 4>(a, s); return true;
            case 32: run_xinv<T, 8, 4>(a, s); return true;
            case 64: run_xinv<T, 8, 8>(a, s); return true;
            case 128: run_xinv<T, 16, 8>(a, s); return true;
            case 256: run_xinv<T, 16, 16>(a, s); return true;
            case 512: run_xinv<T, 32, 16>(a, s); return true;
            case 1024: run_xinv<T, 32, 32>(a, s); return true;
            default: break;
        }
    }
    switch (a.Px) {
        case 16: run_x<T, 4, 4, INV>(a, s); return true;
        case 32: run_x<T, 8, 4, INV>(a, s); return true;
        case 48: run_x<T, 12, 4, INV>(a, s); return true;
        case 64: run_x<T, 8, 8, INV>(a, s); return true;
        case 96: run_x<T, 12, 8, INV>(a, s); return true;
        case 128: run_x<T, 16, 8, INV>(a, s); return true;
        case 192: run_x<T, 24, 8, INV>(a, s); return true;
        case 256: run_x<T, 16, 16, INV>(a, s); return true;
        case 384: run_x<T, 24, 16, INV>(a, s); return true;
        case 512: run_x<T, 32, 16, INV>(a, s); return true;
        case 768: run_x<T, 48, 16, INV>(a, s); return true;
        case 1024: run_x<T, 32, 32, INV>(a, s); return true;
        default: return false;
    }
}

template <typename T> bool launch_x_fast(const PassArgs& a, bool inv, cudaStream_t s) {
    return inv ? dispatch_x<T, true>(a, s) : dispatch_x<T, false>(a, s);
}
template bool launch_x_fast<float>(const PassArgs&, bool, cudaStream_t);
template bool launch_x_fast<double>(const PassArgs&, bool, cudaStream_t);

}  // namespace svh
