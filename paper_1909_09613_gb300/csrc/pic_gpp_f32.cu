// Instantiations of the fused particle pass, float arithmetic.
#include "pic_gpp_kernels.cuh"
#include "pic_launch.h"

namespace pic {

namespace {

template <int L, int KT, bool DET>
__global__ void __launch_bounds__(256, 2) k_gpp2d(const __grid_constant__ RunDev rd)
{
    extern __shared__ __align__(16) char smem[];
    tile_2d<L, KT, float, DET>(rd, smem, blockIdx.x);
}

template <int L, int KT>
cudaError_t go(const RunDev &rd, cudaStream_t st)
{
    const size_t smem = stage2d_bytes<float>(rd.reg_nodes, rd.l, true, rd.det != 0);
    auto k = rd.det ? k_gpp2d<L, KT, true> : k_gpp2d<L, KT, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)rd.ntiles, 256, smem, st>>>(rd);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gpp_f32(const RunDev &rd, int kt, cudaStream_t st)
{
    if (rd.dim != 2) return launch_gpp3d(rd, kt, st);
    const bool wide = kt > rd.l + 1;
    switch (rd.l) {
    case 1: return wide ? go<1, 3>(rd, st) : go<1, 2>(rd, st);
    case 2: return wide ? go<2, 4>(rd, st) : go<2, 3>(rd, st);
    case 3: return wide ? go<3, 5>(rd, st) : go<3, 4>(rd, st);
    case 4: return wide ? go<4, 6>(rd, st) : go<4, 5>(rd, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t gpp_smem_bytes_f32(const RunDev &rd)
{
    return rd.dim == 2 ? stage2d_bytes<float>(rd.reg_nodes, rd.l, true, rd.det != 0)
                       : gpp3d_smem_bytes(rd);
}

// Dynamic shared memory a work item of this run needs in the batched kernel: the copy of the
// run descriptor (tables included) and a stage without its own tables.
size_t gpp_batch_smem_bytes_f32(const RunDev &rd)
{
    if (rd.dim != 2) return 0;
    return (sizeof(RunDev) + 15) / 16 * 16 + stage2d_bytes<float>(rd.reg_nodes, rd.l, false);
}

}  // namespace pic
