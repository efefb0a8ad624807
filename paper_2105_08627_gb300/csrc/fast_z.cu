// fast_z.cu -- launchers of the size-specialised z pass (see fastpass.cuh).
#include "fastpass.cuh"

namespace svh {

template <typename T, int PZ>
static void run_z(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    const size_t sm = (size_t)5 * PZ * 32 * sizeof(C) + (size_t)7 * PZ * 32 * sizeof(T);
    cudaFuncSetAttribute(k_zpass_fast<T, PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + 31) / 32, a.Py);
    if (a.zcontig && 2 * a.nza <= PZ) {
        cudaFuncSetAttribute(k_zpass_half<T, PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_zpass_half<T, PZ><<<grid, 160, sm, s>>>(a);
        return;
    }
    k_zpass_fast<T, PZ><<<grid, 160, sm, s>>>(a);
}

template <typename T> bool launch_z_fast(const PassArgs& a, cudaStream_t s) {
    switch (a.Pz) {
        case 8: run_z<T, 8>(a, s); return true;
        case 12: run_z<T, 12>(a, s); return true;
        case 16: run_z<T, 16>(a, s); return true;
        case 24: run_z<T, 24>(a, s); return true;
        case 32: run_z<T, 32>(a, s); return true;
        case 48: run_z<T, 48>(a, s); return true;
        default: return false;
    }
}
template bool launch_z_fast<float>(const PassArgs&, cudaStream_t);
template bool launch_z_fast<double>(const PassArgs&, cudaStream_t);

}  // namespace svh
