// fast_z.cu -- launchers of the size-specialised z pass (see fastpass.cuh).
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "fastpass.cuh"

namespace svh {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA view of B2 for k_zpass_tma: floats [nb 5 nza][Py][2 Px], box {64, 1, 5 nza}
static bool b2_tensor_map(const PassArgs& a, CUtensorMap* m) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !a.B2 || a.Px % 2 || 5 * a.nza > 256) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * a.Px, (cuuint64_t)a.Py, (cuuint64_t)a.nb * 5 * a.nza};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * a.Px * sizeof(float), (cuuint64_t)2 * a.Px * a.Py * sizeof(float)};
    const cuuint32_t box[3] = {64, 1, (cuuint32_t)(5 * a.nza)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.B2, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int PZ>
static bool run_z_tma(const PassArgs& a, cudaStream_t s) {
    CUtensorMap m;
    if (!a.status || !b2_tensor_map(a, &m)) return false;
    const size_t sm = (size_t)2 * 5 * a.nza * 32 * sizeof(float2) + (size_t)5 * PZ * 32 * sizeof(float2) +
                      (size_t)7 * PZ * 32 * sizeof(float) + 2 * sizeof(uint64_t) + 128;
    cudaFuncSetAttribute(k_zpass_tma<PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + 31) / 32, a.Py);
    k_zpass_tma<PZ><<<grid, 160, sm, s>>>(a, m);
    return true;
}

template <typename T, int PZ>
static void run_z(const PassArgs& a, cudaStream_t s) {
    using C = typename CT<T>::type;
    const size_t sm = (size_t)5 * PZ * 32 * sizeof(C) + (size_t)7 * PZ * 32 * sizeof(T);
    cudaFuncSetAttribute(k_zpass_fast<T, PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((a.Px + 31) / 32, a.Py);
    // variant 0: the pruned kernel when the active planes are contiguous; 1: the full
    // one; 2: the pruned kernel with TMA-staged boxes (FP32); 4: pencils split over two
    // threads (FP32, fast_zs.cu); other choices fall back to 0 or 1
    if constexpr (std::is_same<T, float>::value) {
        if (a.var == 2 && a.zcontig && 2 * a.nza <= PZ && run_z_tma<PZ>(a, s)) return;
        if (a.var == 4 && launch_z_split(a, s)) return;   // 3 is the direct z pass (fast_zd.cu)
        if ((a.var == 5 || a.var == 6) && launch_z_split16(a, s, a.var == 5)) return;
    }
    if (a.var != 1 && a.zcontig && 2 * a.nza <= PZ) {
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
    return z_fast_size(Pz) ? (fp32 ? 3 : 2) : 0;
}
bool z_fast_size(int Pz) {
    return Pz == 8 || Pz == 12 || Pz == 16 || Pz == 24 || Pz == 32 || Pz == 48;
}
template bool launch_z_fast<float>(const PassArgs&, cudaStream_t);
template bool launch_z_fast<double>(const PassArgs&, cudaStream_t);

}  // namespace svh
