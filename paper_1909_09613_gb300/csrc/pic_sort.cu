// Tile sort of one species' particle store.
//
// Two orders, both grouping particles by tile (tiles and cells in a tile numbered x-fastest);
// slot = the particle's rank among the particles of its cell:
//  * cell-major (FP32 form): by (tile, cell, slot).  A warp's 32 consecutive particles sit in
//    one cell or two neighbouring ones: shared-memory gathers broadcast, and the warp's
//    Esirkepov currents are summed in registers before they reach shared memory.
//  * slot-major (FP64 form): by (tile, slot, cell).  A tile runs through groups holding one
//    particle of every cell with more than `slot` particles, so a warp's lanes sit in 32
//    different cells and their per-lane shared-memory atomics do not collide.
// The cell at every position is fixed by the cell counts; which of a cell's particles takes
// which slot is decided by atomics and is not reproducible.
//
//   1. k_count   : tile-major cell key per particle, slot = atomicAdd(count[key], 1)
//   2. k_tile_sum: particles per tile;  k_scan: exclusive scan over tiles -> tile_start
//   3. k_layout  : one CTA per tile; first position of every cell (cell-major) and, for the
//                  slot-major order, the position of every (cell, slot)
//   4. k_scatter : copy every particle to its position in the other buffer
#include "pic_launch.h"

namespace pic {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ void cell_coords(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                            int c[3])
{
    if (rd.prec == 1) {
        const int cc = sp.cell[p];
        c[0] = cc % rd.n[0];
        c[1] = (cc / rd.n[0]) % rd.n[1];
        c[2] = cc / (rd.n[0] * rd.n[1]);
    } else {
        c[2] = 0;
        for (int a = 0; a < rd.dim; ++a) c[a] = (int)floor(((const double *)sp.pos[a])[p]);
    }
}

__device__ __forceinline__ int tile_major_key(const RunDev &rd, const int c[3])
{
    const int ti = c[0] / rd.tile[0], tj = c[1] / rd.tile[1], tk = c[2] / rd.tile[2];
    const int tile = (tk * rd.ntile[1] + tj) * rd.ntile[0] + ti;
    const int local = ((c[2] - tk * rd.tile[2]) * rd.tile[1] + (c[1] - tj * rd.tile[1])) * rd.tile[0]
                      + (c[0] - ti * rd.tile[0]);
    return tile * (rd.tile[0] * rd.tile[1] * rd.tile[2]) + local;
}

__global__ void __launch_bounds__(kBlock) k_count(const __grid_constant__ RunDev rd, int s,
                                                  SortScratch sc)
{
    const SpeciesDev &sp = rd.sp[s];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= sp.n) return;
    int c[3];
    cell_coords(rd, sp, p, c);
    const int key = tile_major_key(rd, c);
    sc.key[p] = key;
    sc.slot[p] = atomicAdd(sc.cnt + key, 1);
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive block scan of one int per thread (blockDim.x <= 1024); *total gets the sum
__device__ int block_excl_scan(int v, int *total)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        int x = (lane < nw) ? wsum[lane] : 0;
        const int xi = warp_incl_scan(x);
        wsum[lane] = xi - x;
        if (lane == nw - 1) *total = xi;
    }
    __syncthreads();
    const int r = wsum[w] + inc - v;
    __syncthreads();
    return r;
}

// particles per tile (one CTA per tile, TC threads)
__global__ void k_tile_sum(const __grid_constant__ RunDev rd, SortScratch sc)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    const int64_t t = blockIdx.x;
    __shared__ int tot;
    int v = 0;
    for (int c = threadIdx.x; c < TC; c += blockDim.x) v += sc.cnt[t * TC + c];
    int dummy = block_excl_scan(v, &tot);
    (void)dummy;
    __syncthreads();
    if (threadIdx.x == 0) sc.tile_count[t] = tot;
}

// exclusive scan of tile_count[0..nt) into tile_start[0..nt] (single CTA, chunked)
__global__ void k_scan(const int64_t *cnt, int64_t *start, int64_t nt)
{
    __shared__ int64_t carry;
    __shared__ int64_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < nt; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = (i < nt) ? cnt[i] : 0;
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t tt = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += tt;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            int64_t x = (lane < nw) ? wsum[lane] : 0;
            int64_t xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t tt = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += tt;
            }
            wsum[lane] = xi - x;
        }
        __syncthreads();
        const int64_t excl = carry + wsum[w] + inc - v;
        if (i < nt) start[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[nt] = carry;
}

// One CTA per tile with TC threads (one per cell of the tile).
__global__ void k_layout(const __grid_constant__ RunDev rd, SortScratch sc,
                         const int64_t *tile_start, int slot_major)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    const int64_t t = blockIdx.x;
    const int c = threadIdx.x;
    __shared__ int tot;
    __shared__ int maxc;
    const int cnt = (c < TC) ? sc.cnt[t * TC + c] : 0;
    if (threadIdx.x == 0) maxc = 0;
    __syncthreads();
    if (cnt > 0) atomicMax(&maxc, cnt);
    const int first = block_excl_scan(cnt, &tot);
    const int64_t base = tile_start[t];
    if (c < TC) sc.cell_first[t * TC + c] = (int32_t)(base + first);
    if (!slot_major) return;
    __syncthreads();
    const int ms = maxc;
    int goff = 0;
    for (int s = 0; s < ms; ++s) {
        const int flag = (cnt > s) ? 1 : 0;
        const int rank = block_excl_scan(flag, &tot);
        if (flag) sc.pos[base + first + s] = (int32_t)(base + goff + rank);
        goff += tot;
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void mv(const void *src, void *dst, int64_t p, int64_t q)
{
    ((T *)dst)[q] = ((const T *)src)[p];
}

__global__ void __launch_bounds__(kBlock) k_scatter(const __grid_constant__ RunDev rd, int s,
                                                    SortScratch sc, void *d0, void *d1, void *d2,
                                                    void *m0, void *m1, void *m2, int32_t *dcell,
                                                    int slot_major)
{
    const SpeciesDev &sp = rd.sp[s];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= sp.n) return;
    const int64_t r = (int64_t)sc.cell_first[sc.key[p]] + sc.slot[p];
    const int64_t q = slot_major ? (int64_t)sc.pos[r] : r;
    void *dp[3] = {d0, d1, d2};
    void *dm[3] = {m0, m1, m2};
    if (rd.prec == 1) {
        dcell[q] = sp.cell[p];
        for (int a = 0; a < rd.dim; ++a) mv<float>(sp.pos[a], dp[a], p, q);
        for (int a = 0; a < 3; ++a) mv<float>(sp.mom[a], dm[a], p, q);
    } else {
        for (int a = 0; a < rd.dim; ++a) mv<double>(sp.pos[a], dp[a], p, q);
        for (int a = 0; a < 3; ++a) mv<double>(sp.mom[a], dm[a], p, q);
    }
}

}  // namespace

cudaError_t launch_sort(const RunDev &rd, int s, const SortScratch &sc, int64_t *tile_start,
                        void *const *dst_pos, void *const *dst_mom, int32_t *dst_cell,
                        cudaStream_t st)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    const int64_t nkeys = rd.ntiles * TC;
    cudaError_t e = cudaMemsetAsync(sc.cnt, 0, nkeys * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t n = rd.sp[s].n;
    if (n > 0) k_count<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(rd, s, sc);
    const int tb = ((TC + 31) / 32) * 32;
    k_tile_sum<<<(unsigned)rd.ntiles, tb, 0, st>>>(rd, sc);
    k_scan<<<1, 1024, 0, st>>>(sc.tile_count, tile_start, rd.ntiles);
    const int slot_major = rd.slot_major;
    k_layout<<<(unsigned)rd.ntiles, tb, 0, st>>>(rd, sc, tile_start, slot_major);
    if (n > 0)
        k_scatter<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(
            rd, s, sc, dst_pos[0], dst_pos[1], dst_pos[2], dst_mom[0], dst_mom[1], dst_mom[2],
            dst_cell, slot_major);
    return cudaGetLastError();
}

}  // namespace pic
