// Instantiations of the fused particle pass in 3D, both forms.
#include "pic_gpp3d.cuh"
#include "pic_launch.h"

namespace pic {

namespace {

// FP32 form, l <= 2: four blocks per SM (at most 128 registers; the staged stage of four blocks
// fits in shared memory and the extra warps hide latency); higher orders keep their registers
template <int L, int KT>
__global__ void __launch_bounds__(128, (L <= 2 ? 4 : 1)) k_gpp3d_f32(const __grid_constant__ RunDev rd)
{
    extern __shared__ __align__(16) float sf3[];
    tile_3d<L, KT, float>(rd, blockIdx.x, sf3);
}

template <int L, int KT>
__global__ void __launch_bounds__(128) k_gpp3d_f64(const __grid_constant__ RunDev rd)
{
    tile_3d<L, KT, double>(rd, blockIdx.x);
}

template <int L, int KT>
cudaError_t go(const RunDev &rd, cudaStream_t st)
{
    if (rd.prec == 1) {  // FP32 form
        const size_t smem = stage3d_bytes(rd);
        cudaError_t e = cudaFuncSetAttribute(k_gpp3d_f32<L, KT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gpp3d_f32<L, KT><<<(unsigned)rd.ntiles, 128, smem, st>>>(rd);
    } else {
        k_gpp3d_f64<L, KT><<<(unsigned)rd.ntiles, 128, 0, st>>>(rd);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gpp3d(const RunDev &rd, int kt, cudaStream_t st)
{
    const bool wide = kt > rd.l + 1;
    switch (rd.l) {
    case 1: return wide ? go<1, 3>(rd, st) : go<1, 2>(rd, st);
    case 2: return wide ? go<2, 4>(rd, st) : go<2, 3>(rd, st);
    case 3: return wide ? go<3, 5>(rd, st) : go<3, 4>(rd, st);
    case 4: return wide ? go<4, 6>(rd, st) : go<4, 5>(rd, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t gpp3d_smem_bytes(const RunDev &rd)
{
    return rd.prec == 1 ? stage3d_bytes(rd) : 0;
}

}  // namespace pic
