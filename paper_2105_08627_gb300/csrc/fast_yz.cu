// fast_yz.cu -- launcher of the fused x / yz / x path (see fused.cuh).
#include <algorithm>

#include "fused.cuh"

namespace svh {

namespace {

template <int N1, int N2, int NTX>
void run_xfwd_t(const PassArgs& a, cudaStream_t s) {
    constexpr int L = NTX / N2;
    const size_t sm = (size_t)(N1 * N2 + L * (N2 * (N1 + 1) + 1)) * sizeof(float2);
    cudaFuncSetAttribute(k_xfwd_t<N1, N2, NTX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_xfwd_t<N1, N2, NTX><<<(unsigned)((a.nlines + L - 1) / L), NTX, sm, s>>>(a);
}

template <int N1, int N2, int NTX>
void run_xinv_t(const PassArgs& a, cudaStream_t s) {
    constexpr int L = NTX / N2;
    constexpr int G = L / 5;
    const size_t sm = (size_t)(N1 * N2 + L * (N2 * (N1 + 1) + 1)) * sizeof(float2);
    cudaFuncSetAttribute(k_xinv_t<N1, N2, NTX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int64_t groups = (int64_t)a.nb * a.nrows;
    k_xinv_t<N1, N2, NTX><<<(unsigned)((groups + G - 1) / G), NTX, sm, s>>>(a);
}

// x passes on B1T: sizes with a split whose factors suit both pruned stages
bool x_t_size(int Px) { return Px == 64 || Px == 128 || Px == 256 || Px == 512 || Px == 1024; }

void run_x_t(const PassArgs& a, bool inv, cudaStream_t s) {
    switch (a.Px) {
        case 64: inv ? run_xinv_t<8, 8, 320>(a, s) : run_xfwd_t<8, 8, 256>(a, s); break;
        case 128: inv ? run_xinv_t<16, 8, 320>(a, s) : run_xfwd_t<16, 8, 256>(a, s); break;
        case 256: inv ? run_xinv_t<16, 16, 640>(a, s) : run_xfwd_t<16, 16, 256>(a, s); break;
        case 512: inv ? run_xinv_t<32, 16, 640>(a, s) : run_xfwd_t<32, 16, 256>(a, s); break;
        default: inv ? run_xinv_t<32, 32, 640>(a, s) : run_xfwd_t<32, 32, 256>(a, s); break;
    }
}

// returns false (nothing launched) when the shared memory does not fit
template <int NY1, int NY2, int PZ>
bool run_yz(const PassArgs& a, size_t limit, cudaStream_t s, bool dry) {
    size_t sm = yz_smem_bytes<NY1, NY2, PZ, 640>(a.nza);
    if (sm <= limit) {
        if (!dry) {
            cudaFuncSetAttribute(k_yz_fused<NY1, NY2, PZ, 640>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_yz_fused<NY1, NY2, PZ, 640><<<dim3(a.Px, a.nb), 640, sm, s>>>(a);
        }
        return true;
    }
    sm = yz_smem_bytes<NY1, NY2, PZ, 320>(a.nza);
    if (sm <= limit) {
        if (!dry) {
            cudaFuncSetAttribute(k_yz_fused<NY1, NY2, PZ, 320>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_yz_fused<NY1, NY2, PZ, 320><<<dim3(a.Px, a.nb), 320, sm, s>>>(a);
        }
        return true;
    }
    return false;
}

template <int NY1, int NY2>
bool run_yz_pz(const PassArgs& a, size_t limit, cudaStream_t s, bool dry) {
    switch (a.Pz) {
        case 8: return run_yz<NY1, NY2, 8>(a, limit, s, dry);
        case 16: return run_yz<NY1, NY2, 16>(a, limit, s, dry);
        case 24: return run_yz<NY1, NY2, 24>(a, limit, s, dry);
        case 32: return run_yz<NY1, NY2, 32>(a, limit, s, dry);
        default: return false;
    }
}

bool run_yz_any(const PassArgs& a, size_t limit, cudaStream_t s, bool dry) {
    switch (a.Py) {
        case 128: return run_yz_pz<8, 16>(a, limit, s, dry);
        case 256: return run_yz_pz<16, 16>(a, limit, s, dry);
        case 512: return run_yz_pz<16, 32>(a, limit, s, dry);
        default: return false;
    }
}

}  // namespace

// The fused path (FP32): x forward onto B1T, one fused y/z/y kernel, x
// inverse + epilogue from B1T. Needs contiguous active planes (shifted z
// pencils), spectra resident in a.spec and the slab in shared memory.
bool fused_path_ok(const PassArgs& a, size_t smem_limit) {
    if (!a.zcontig || 2 * a.nza > a.Pz || !x_t_size(a.Px)) return false;
    return run_yz_any(a, smem_limit, nullptr, true);
}

void launch_x_t(const PassArgs& a, bool inv, cudaStream_t s) { run_x_t(a, inv, s); }

void launch_yz(const PassArgs& a, size_t smem_limit, cudaStream_t s) { run_yz_any(a, smem_limit, s, false); }

}  // namespace svh
