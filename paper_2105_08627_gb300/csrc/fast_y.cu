// fast_y.cu -- launchers of the size-specialised y passes (see fastpass.cuh).
//
// Tile variants (FP32; the autotuner times them, a.var selects one):
//   0: the default split N = N1 x N2 with 256 threads per block,
//   1: the same split with 512 threads (twice the kx columns per block),
//   2: the same split with 128 threads,
//   3: the transposed split N2 x N1 with 256 threads (sizes where both
//      factors suit the pruned first and second stages; elsewhere 3 runs 0),
//   4: the cp.async-staged persistent kernel k_ycol_async, 8 kx columns per tile (sizes >= 256;
//      4-column tiles, more blocks per SM, measured slower).
// FP64 has variant 0 only (128 threads).
#include <algorithm>
#include <type_traits>

#include "fastpass.cuh"

namespace svh {

template <typename T, int N1, int N2, bool INV, int NT>
static void run_y(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    static_assert(NT % N2 == 0, "threads per block must be a multiple of N2");
    constexpr int TB = NT / N2;
    const size_t sm = (size_t)(N1 * N2) * (1 + TB) * sizeof(C);
    cudaFuncSetAttribute(k_ycol_fast<T, N1, N2, INV, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + TB - 1) / TB, a.nza, a.nb * 5);
    k_ycol_fast<T, N1, N2, INV, NT><<<grid, NT, sm, s>>>(a);
}

// variant 4: the cp.async-staged persistent kernel (FP32), as many blocks as fit an SM
template <int N1, int N2, bool INV, int NT>
static void run_y_async(const PassArgs& a, cudaStream_t s) {
    constexpr int TB = NT / N2;
    constexpr int N = N1 * N2;
    // forward: room for the planes' active-row bits when they take at most 4 KB
    const int wpp = (a.Ky + 31) / 32;
    const int rbw = (!INV && (size_t)a.nza * wpp * 4 <= 4096) ? wpp : 0;
    const size_t sm = (size_t)(N + (INV ? N : N / 2) * TB + N * TB) * sizeof(float2) + (size_t)a.nza * rbw * 4;
    cudaFuncSetAttribute(k_ycol_async<N1, N2, INV, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ycol_async<N1, N2, INV, NT>, NT, sm);
    const int ntiles = ((a.Px + TB - 1) / TB) * a.nza * a.nb * 5;
    const int grid = std::max(1, std::min(ntiles, std::max(1, sms) * std::max(1, per_sm)));
    k_ycol_async<N1, N2, INV, NT><<<grid, NT, sm, s>>>(a, ntiles, rbw);
}

// N1 x N2 default split; SWAP: the transposed split is a variant too
template <typename T, bool INV, int N1, int N2, bool SWAP>
static bool run_y_size(const PassArgs& a, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        switch (a.var) {
            case 1: run_y<T, N1, N2, INV, 512>(a, s); return true;
            case 2: run_y<T, N1, N2, INV, 128>(a, s); return true;
            case 3:
                if constexpr (SWAP) { run_y<T, N2, N1, INV, 256>(a, s); return true; }
                break;
            case 4:
                // (whole 16-byte column pairs: Px a multiple of the 8-column tile)
                if constexpr (N1 * N2 >= 256 && N2 <= 64)
                    if (a.Px % 8 == 0) { run_y_async<N1, N2, INV, 8 * N2>(a, s); return true; }
                break;
            default: break;
        }
        run_y<T, N1, N2, INV, 256>(a, s);
    } else {
        run_y<T, N1, N2, INV, 128>(a, s);
    }
    return true;
}

template <typename T, bool INV>
static bool dispatch_y(const PassArgs& a, cudaStream_t s) {
    switch (a.Py) {
        case 16: return run_y_size<T, INV, 4, 4, false>(a, s);
        case 32: return run_y_size<T, INV, 8, 4, true>(a, s);
        case 48: return run_y_size<T, INV, 12, 4, false>(a, s);
        case 64: return run_y_size<T, INV, 8, 8, false>(a, s);
        case 96: return run_y_size<T, INV, 12, 8, false>(a, s);
        case 128: return run_y_size<T, INV, 16, 8, true>(a, s);
        case 192: return run_y_size<T, INV, 24, 8, false>(a, s);
        case 256: return run_y_size<T, INV, 16, 16, false>(a, s);
        case 384: return run_y_size<T, INV, 24, 16, false>(a, s);
        case 512: return run_y_size<T, INV, 32, 16, true>(a, s);
        case 768: return run_y_size<T, INV, 48, 16, false>(a, s);
        case 1024: return run_y_size<T, INV, 32, 32, false>(a, s);
        default: return false;
    }
}

int y_fast_variants(int Py, bool fp32) {
    if (!fp32) return 1;
    switch (Py) {   // 4: the cp.async-staged kernel (sizes >= 256; where 3 has no transposed split it runs 0)
        case 256: case 384: case 512: case 768: case 1024: return 5;
        case 32: case 128: return 4;
        case 16: case 48: case 64: case 96: case 192: return 3;
        default: return 0;
    }
}

template <typename T> bool launch_y_fast(const PassArgs& a, bool inv, cudaStream_t s) {
    return inv ? dispatch_y<T, true>(a, s) : dispatch_y<T, false>(a, s);
}
template bool launch_y_fast<float>(const PassArgs&, bool, cudaStream_t);
template bool launch_y_fast<double>(const PassArgs&, bool, cudaStream_t);

}  // namespace svh
