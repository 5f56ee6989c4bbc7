// Device bodies of the tile sort, shared by the single-run launches (pic_sort.cu) and the
// batched launches (pic_batch.cu).  See pic_sort.cu for the two orders and the stages.
#pragma once
#include "pic_common.cuh"

namespace pic {

__device__ __forceinline__ void sort_cell_coords(const RunDev &rd, const SpeciesDev &sp,
                                                 int64_t p, int c[3])
{
    if (rd.prec == 1) {
        const int cc = sp.cell[p];
        c[0] = cc % rd.n[0];
        c[1] = (cc / rd.n[0]) % rd.n[1];
        c[2] = cc / (rd.n[0] * rd.n[1]);
    } else {
        c[2] = 0;
        // positions are kept in [0, n); the clamp only keeps a non-finite one inside the grid
        for (int a = 0; a < rd.dim; ++a)
            c[a] = min(max((int)floor(((const double *)sp.pos[a])[p]), 0), rd.n[a] - 1);
    }
}

__device__ __forceinline__ int sort_tile_major_key(const RunDev &rd, const int c[3])
{
    const int ti = c[0] / rd.tile[0], tj = c[1] / rd.tile[1], tk = c[2] / rd.tile[2];
    const int tile = (tk * rd.ntile[1] + tj) * rd.ntile[0] + ti;
    const int local = ((c[2] - tk * rd.tile[2]) * rd.tile[1] + (c[1] - tj * rd.tile[1])) * rd.tile[0]
                      + (c[0] - ti * rd.tile[0]);
    return tile * (rd.tile[0] * rd.tile[1] * rd.tile[2]) + local;
}

__device__ __forceinline__ int sort_warp_incl_scan(int v)
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
__device__ __forceinline__ int sort_block_excl_scan(int v, int *total)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = sort_warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        const int x = (lane < nw) ? wsum[lane] : 0;
        const int xi = sort_warp_incl_scan(x);
        wsum[lane] = xi - x;
        if (lane == nw - 1) *total = xi;
    }
    __syncthreads();
    const int r = wsum[w] + inc - v;
    __syncthreads();
    return r;
}

// 1. tile-major cell key of particle p, the particle count of every key, and a provisional
//    place among the particles of its key (taken from an atomic, so not reproducible; stage 5
//    replaces it by the particle's rank in the previous order)
__device__ __forceinline__ void sort_count_one(const RunDev &rd, int s, int64_t p)
{
    const SpeciesDev &sp = rd.sp[s];
    int c[3];
    sort_cell_coords(rd, sp, p, c);
    const int key = sort_tile_major_key(rd, c);
    rd.sc.key[p] = key;
    // lanes with the same key (neighbours in a sorted store) take consecutive slots from one
    // atomic of their leader instead of contending for the counter one by one
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(rd.sc.cnt + key, __popc(same));
    base = __shfl_sync(same, base, leader);
    rd.sc.slot[p] = base + __popc(same & ((1u << lane) - 1u));
}

// 2. particles of tile t (block-wide, one thread per cell of the tile)
__device__ __forceinline__ void sort_tile_sum_block(const RunDev &rd, int64_t t)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    __shared__ int tot;
    int v = 0;
    for (int c = threadIdx.x; c < TC; c += blockDim.x) v += rd.sc.cnt[t * TC + c];
    (void)sort_block_excl_scan(v, &tot);
    __syncthreads();
    if (threadIdx.x == 0) rd.sc.tile_count[t] = tot;
}

// 3. exclusive scan of tile_count[0..nt) into start[0..nt] (block-wide, chunked)
__device__ __forceinline__ void sort_scan_block(const int64_t *cnt, int64_t *start, int64_t nt)
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
            const int64_t x = (lane < nw) ? wsum[lane] : 0;
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

// 4. first position of every cell of tile t and, slot-major, of every (cell, slot)
//    (block-wide with at least TC threads)
__device__ __forceinline__ void sort_layout_block(const RunDev &rd, const int64_t *tile_start,
                                                  int64_t t)
{
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    const int c = threadIdx.x;
    __shared__ int tot;
    __shared__ int maxc;
    const int cnt = (c < TC) ? rd.sc.cnt[t * TC + c] : 0;
    if (threadIdx.x == 0) maxc = 0;
    __syncthreads();
    if (cnt > 0) atomicMax(&maxc, cnt);
    const int first = sort_block_excl_scan(cnt, &tot);
    const int64_t base = tile_start[t];
    if (c < TC) rd.sc.cell_first[t * TC + c] = (int32_t)(base + first);
    if (!rd.slot_major) return;
    __syncthreads();
    const int ms = maxc;
    int goff = 0;
    for (int s = 0; s < ms; ++s) {
        const int flag = (cnt > s) ? 1 : 0;
        const int rank = sort_block_excl_scan(flag, &tot);
        if (flag) rd.sc.pos[base + first + s] = (int32_t)(base + goff + rank);
        goff += tot;
        __syncthreads();
    }
}

// 5. the index of particle p at its provisional place in its cell's segment of the cell-major
//    order (the segment of key k is cell_first[k] .. cell_first[k] + cnt[k] - 1)
__device__ __forceinline__ void sort_place_one(const RunDev &rd, int64_t p)
{
    const int k = rd.sc.key[p];
    rd.sc.idx[(int64_t)rd.sc.cell_first[k] + rd.sc.slot[p]] = (int32_t)p;
}

// 6. cell-major position r: the particle p placed there by stage 5 is moved to the position of
//    its rank among the particles of its cell in the previous order (the number of indices
//    below p in the segment), which makes the order stable and the same on every run: sorted
//    by (tile, cell, previous index), or in the slot-major order by (tile, rank, cell).  The
//    threads of a warp usually share a segment, so its loads are broadcasts; the cost grows
//    with the square of a cell's occupancy.
__device__ __forceinline__ void sort_scatter_one(const RunDev &rd, int s, int64_t r,
                                                 void *const *dp, void *const *dm, int32_t *dcell)
{
    const SpeciesDev &sp = rd.sp[s];
    const int32_t p = rd.sc.idx[r];
    const int k = rd.sc.key[p];
    const int64_t first = rd.sc.cell_first[k];
    const int m = rd.sc.cnt[k];
    const int32_t *seg = rd.sc.idx + first;
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (__ldg(seg + j) < p) ? 1 : 0;
    const int64_t rr = first + rank;
    const int64_t q = rd.slot_major ? (int64_t)rd.sc.pos[rr] : rr;
    if (rd.prec == 1) {
        dcell[q] = sp.cell[p];
        for (int a = 0; a < rd.dim; ++a) ((float *)dp[a])[q] = ((const float *)sp.pos[a])[p];
        for (int a = 0; a < 3; ++a) ((float *)dm[a])[q] = ((const float *)sp.mom[a])[p];
    } else {
        for (int a = 0; a < rd.dim; ++a) ((double *)dp[a])[q] = ((const double *)sp.pos[a])[p];
        for (int a = 0; a < 3; ++a) ((double *)dm[a])[q] = ((const double *)sp.mom[a])[p];
    }
}

}  // namespace pic
