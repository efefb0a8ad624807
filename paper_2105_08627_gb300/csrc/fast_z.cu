// fast_z.cu -- launchers of the size-specialised z pass (see fastpass.cuh).
#include "fastpass.cuh"

namespace svh {

template <typename T, int PZ>
static void run_z(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    const size_t sm = (size_t)5 * PZ * 32 * sizeof(C) + (size_t)7 * PZ * 32 * sizeof(T);
    cudaFuncSetAttribute(k_zpass_fast<T, PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + 31) / 32, a.Py);
    // variant 0: the pruned kernel when the active planes are contiguous; 1: the full one
    if (a.var == 0 && a.zcontig && 2 * a.nza <= PZ) {
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
int z_fast_variants(int Pz, bool fp32) {
    (void)fp32;
    return z_fast_size(Pz) ? 2 : 0;
}
bool z_fast_size(int Pz) {
    return Pz == 8 || Pz == 12 || Pz == 16 || Pz == 24 || Pz == 32 || Pz == 48;
}
template bool launch_z_fast<float>(const PassArgs&, cudaStream_t);
template bool launch_z_fast<double>(const PassArgs&, cudaStream_t);

}  // namespace svh
