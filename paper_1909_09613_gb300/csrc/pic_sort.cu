// Tile sort of one species' particle store (single-run launches).
//
// Two orders, both grouping particles by tile (tiles and cells in a tile numbered x-fastest);
// rank = the particle's rank among the particles of its cell in the previous order:
//  * cell-major (FP32 form): by (tile, cell, rank).  A warp's 32 consecutive particles sit in
//    one cell or two neighbouring ones: shared-memory gathers broadcast, and the warp's
//    Esirkepov currents are summed in registers before they reach shared memory.
//  * slot-major (FP64 form): by (tile, rank, cell).  A tile runs through groups holding one
//    particle of every cell with more than `rank` particles, so a warp's lanes sit in 32
//    different cells and their per-lane shared-memory atomics do not collide.
// Both orders are stable and a pure function of the cells of the previous order: the same on
// every run, whatever the order in which the atomics of the counting stage were served.
//
//   1. count    : tile-major cell key per particle, its count and a provisional place
//   2. tile_sum : particles per tile;  scan: exclusive scan over tiles -> tile_start
//   3. layout   : one CTA per tile; first position of every cell (cell-major) and, for the
//                 slot-major order, the position of every (cell, rank)
//   4. place    : every particle index at its provisional cell-major position
//   5. scatter  : per cell-major position, the rank of its particle in its cell (indices below
//                 it in the cell's segment); the particle is copied to the position of that
//                 rank in the other buffer
#include "pic_launch.h"
#include "pic_sort_dev.cuh"

namespace pic {

namespace {

constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) k_count(const __grid_constant__ RunDev rd, int s)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < rd.sp[s].n) sort_count_one(rd, s, p);
}

__global__ void k_tile_sum(const __grid_constant__ RunDev rd)
{
    sort_tile_sum_block(rd, blockIdx.x);
}

__global__ void k_scan(const int64_t *cnt, int64_t *start, int64_t nt)
{
    sort_scan_block(cnt, start, nt);
}

__global__ void k_layout(const __grid_constant__ RunDev rd, const int64_t *tile_start)
{
    sort_layout_block(rd, tile_start, blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) k_place(const __grid_constant__ RunDev rd, int s)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < rd.sp[s].n) sort_place_one(rd, p);
}

__global__ void __launch_bounds__(kBlock) k_scatter(const __grid_constant__ RunDev rd, int s,
                                                    void *d0, void *d1, void *d2, void *m0,
                                                    void *m1, void *m2, int32_t *dcell)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rd.sp[s].n) return;
    void *dp[3] = {d0, d1, d2};
    void *dm[3] = {m0, m1, m2};
    sort_scatter_one(rd, s, r, dp, dm, dcell);
}

}  // namespace

cudaError_t launch_sort(const RunDev &rd, int s, int64_t *tile_start, void *const *dst_pos,
                        void *const *dst_mom, int32_t *dst_cell, cudaStream_t st)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    const int64_t nkeys = rd.ntiles * TC;
    cudaError_t e = cudaMemsetAsync(rd.sc.cnt, 0, nkeys * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t n = rd.sp[s].n;
    if (n > 0) k_count<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(rd, s);
    const int tb = ((TC + 31) / 32) * 32;
    k_tile_sum<<<(unsigned)rd.ntiles, tb, 0, st>>>(rd);
    k_scan<<<1, 1024, 0, st>>>(rd.sc.tile_count, tile_start, rd.ntiles);
    k_layout<<<(unsigned)rd.ntiles, tb, 0, st>>>(rd, tile_start);
    if (n > 0) k_place<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(rd, s);
    if (n > 0)
        k_scatter<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(
            rd, s, dst_pos[0], dst_pos[1], dst_pos[2], dst_mom[0], dst_mom[1], dst_mom[2],
            dst_cell);
    return cudaGetLastError();
}

}  // namespace pic
