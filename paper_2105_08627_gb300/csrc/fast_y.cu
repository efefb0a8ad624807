// fast_y.cu -- launchers of the size-specialised y passes (see fastpass.cuh).
#include "fastpass.cuh"

namespace svh {

template <typename T, int N1, int N2, bool INV>
static void run_y(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int NT = sizeof(T) == 4 ? 256 : 128;
    constexpr int TB = NT / N2;
    const size_t sm = (size_t)(N1 * N2) * (1 + TB) * sizeof(C);
    cudaFuncSetAttribute(k_ycol_fast<T, N1, N2, INV, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + TB - 1) / TB, a.nza, a.nb * 5);
    k_ycol_fast<T, N1, N2, INV, NT><<<grid, NT, sm, s>>>(a);
}

template <typename T, bool INV>
static bool dispatch_y(const PassArgs& a, cudaStream_t s) {
    switch (a.Py) {
        case 16: run_y<T, 4, 4, INV>(a, s); return true;
        case 32: run_y<T, 8, 4, INV>(a, s); return true;
        case 48: run_y<T, 12, 4, INV>(a, s); return true;
        case 64: run_y<T, 8, 8, INV>(a, s); return true;
        case 96: run_y<T, 12, 8, INV>(a, s); return true;
        case 128: run_y<T, 16, 8, INV>(a, s); return true;
        case 192: run_y<T, 24, 8, INV>(a, s); return true;
        case 256: run_y<T, 16, 16, INV>(a, s); return true;
        case 384: run_y<T, 24, 16, INV>(a, s); return true;
        case 512: run_y<T, 32, 16, INV>(a, s); return true;
        case 768: run_y<T, 48, 16, INV>(a, s); return true;
        case 1024: run_y<T, 32, 32, INV>(a, s); return true;
        default: return false;
    }
}

template <typename T> bool launch_y_fast(const PassArgs& a, bool inv, cudaStream_t s) {
    return inv ? dispatch_y<T, true>(a, s) : dispatch_y<T, false>(a, s);
}
template bool launch_y_fast<float>(const PassArgs&, bool, cudaStream_t);
template bool launch_y_fast<double>(const PassArgs&, bool, cudaStream_t);

}  // namespace svh
