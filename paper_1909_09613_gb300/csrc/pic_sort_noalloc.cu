// Tile sort that allocates nothing: pic_tile_sort_noalloc.
//
// The regular tile sort runs inside a context and uses scratch carved from the device buffer
// the caller binds (or that pic_alloc obtains with cudaMalloc).  Some callers cannot allocate
// device memory at the point where they need the sort: a host program whose device memory is
// owned by another allocator (a framework's caching pool) that must not be bypassed, or a
// real-time loop that cannot afford the device-wide synchronisation cudaMalloc and cudaFree
// imply.  This entry point serves them: its scratch is one file-scope __device__ array of a
// fixed size, which every GPU that loads the library holds until the process exits; the caller
// passes only the inputs and the outputs.
#include "pic.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int64_t kMaxParticles = (int64_t)1 << 20;  // particles per call
constexpr int64_t kMaxKeys = (int64_t)1 << 20;       // tiles x cells per tile
constexpr int64_t kMaxTiles = (int64_t)1 << 16;      // tiles

// scratch layout: count[kMaxKeys] | cell_first[kMaxKeys] | slot[kMaxParticles] |
//                 key[kMaxParticles] | idx[kMaxParticles] (all int32) |
//                 tile_count[kMaxTiles + 1] (int64)
constexpr size_t kOffCount = 0;
constexpr size_t kOffFirst = kOffCount + sizeof(int32_t) * kMaxKeys;
constexpr size_t kOffSlot = kOffFirst + sizeof(int32_t) * kMaxKeys;
constexpr size_t kOffKey = kOffSlot + sizeof(int32_t) * kMaxParticles;
constexpr size_t kOffIdx = kOffKey + sizeof(int32_t) * kMaxParticles;
constexpr size_t kOffTiles = kOffIdx + sizeof(int32_t) * kMaxParticles;
constexpr size_t kScratchBytes = kOffTiles + sizeof(int64_t) * (kMaxTiles + 1);

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// Device address of g_sort_scratch per device, looked up once with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

struct Geo {
    int n[3], tile[3], ntile[3];
    int TC;
};

__device__ __forceinline__ int wsum_incl(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one int per thread over the block (blockDim.x <= 1024); *total = sum
__device__ int block_scan(int v, int *total)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = wsum_incl(v);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        const int x = (lane < nw) ? ws[lane] : 0;
        const int xi = wsum_incl(x);
        ws[lane] = xi - x;
        if (lane == nw - 1) *total = xi;
    }
    __syncthreads();
    const int r = ws[w] + inc - v;
    __syncthreads();
    return r;
}

// tile-major key of every particle's cell, the count of every key and a provisional place
// inside the cell (from an atomic; k_nz_rank replaces it by the rank in the input order)
__global__ void k_nz_count(Geo g, int64_t np, const int32_t *cell, unsigned char *scr)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    int32_t *cnt = (int32_t *)(scr + kOffCount);
    int32_t *slot = (int32_t *)(scr + kOffSlot);
    int32_t *key = (int32_t *)(scr + kOffKey);
    const int64_t ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int c = cell[p];
    if (c < 0 || c >= ncell) {  // outside the grid: excluded from the order
        key[p] = -1;
        return;
    }
    const int i = c % g.n[0], j = (c / g.n[0]) % g.n[1], k = c / (g.n[0] * g.n[1]);
    const int ti = i / g.tile[0], tj = j / g.tile[1], tk = k / g.tile[2];
    const int tile = (tk * g.ntile[1] + tj) * g.ntile[0] + ti;
    const int local = ((k - tk * g.tile[2]) * g.tile[1] + (j - tj * g.tile[1])) * g.tile[0]
                      + (i - ti * g.tile[0]);
    const int kk = tile * g.TC + local;
    key[p] = kk;
    slot[p] = atomicAdd(cnt + kk, 1);
}

// particles per tile, and the first position of every cell relative to its tile
__global__ void k_nz_tiles(Geo g, unsigned char *scr)
{
    const int32_t *cnt = (const int32_t *)(scr + kOffCount);
    int32_t *first = (int32_t *)(scr + kOffFirst);
    int64_t *tcount = (int64_t *)(scr + kOffTiles);
    __shared__ int tot;
    const int64_t t = blockIdx.x;
    const int c = threadIdx.x;
    const int v = (c < g.TC) ? cnt[t * g.TC + c] : 0;
    const int f = block_scan(v, &tot);
    if (c < g.TC) first[t * g.TC + c] = f;
    if (threadIdx.x == 0) tcount[t] = tot;
}

// exclusive scan of the tile counts into tile_start[0..nt] (one block)
__global__ void k_nz_scan(int64_t nt, unsigned char *scr, int64_t *tile_start)
{
    const int64_t *tcount = (const int64_t *)(scr + kOffTiles);
    __shared__ int64_t carry;
    __shared__ int64_t ws[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < nt; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = (i < nt) ? tcount[i] : 0;
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) ws[w] = inc;
        __syncthreads();
        if (w == 0) {
            const int64_t x = (lane < nw) ? ws[lane] : 0;
            int64_t xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += t;
            }
            ws[lane] = xi - x;
        }
        __syncthreads();
        const int64_t excl = carry + ws[w] + inc - v;
        if (i < nt) tile_start[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_start[nt] = carry;
}

// every particle index at its provisional position of the cell-major order
__global__ void k_nz_place(Geo g, int64_t np, unsigned char *scr, const int64_t *tile_start)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int32_t *first = (const int32_t *)(scr + kOffFirst);
    const int32_t *slot = (const int32_t *)(scr + kOffSlot);
    const int32_t *key = (const int32_t *)(scr + kOffKey);
    int32_t *idx = (int32_t *)(scr + kOffIdx);
    const int kk = key[p];
    if (kk < 0) return;
    idx[tile_start[kk / g.TC] + first[kk] + slot[p]] = (int32_t)p;
}

// position r of the order: the particle placed there moves to the position of its rank among
// the particles of its cell in the input order (stable and reproducible); positions past the
// last tile (as many as particles outside the grid) get -1
__global__ void k_nz_rank(Geo g, int64_t np, int64_t nt, const unsigned char *scr,
                          const int64_t *tile_start, int64_t *perm)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= np) return;
    if (r >= tile_start[nt]) {
        perm[r] = -1;
        return;
    }
    const int32_t *cnt = (const int32_t *)(scr + kOffCount);
    const int32_t *first = (const int32_t *)(scr + kOffFirst);
    const int32_t *key = (const int32_t *)(scr + kOffKey);
    const int32_t *idx = (const int32_t *)(scr + kOffIdx);
    const int32_t p = idx[r];
    const int kk = key[p];
    const int64_t start = tile_start[kk / g.TC] + first[kk];
    const int m = cnt[kk];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (idx[start + j] < p) ? 1 : 0;
    perm[start + rank] = p;
}

}  // namespace

extern "C" int pic_tile_sort_noalloc(const int32_t grid[3], const int32_t tile[3], int64_t n,
                                     const int32_t *cell_dev, int64_t *perm_dev,
                                     int64_t *tile_start_dev, uint64_t stream)
{
    if (!grid || !tile || n < 0 || (n > 0 && (!cell_dev || !perm_dev)) || !tile_start_dev)
        return PIC_EINVAL;
    Geo g;
    int64_t ntiles = 1;
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < 1 || tile[a] < 1 || tile[a] > grid[a]) return PIC_EINVAL;
        g.n[a] = grid[a];
        g.tile[a] = tile[a];
        g.ntile[a] = (grid[a] + tile[a] - 1) / tile[a];
        ntiles *= g.ntile[a];
    }
    g.TC = tile[0] * tile[1] * tile[2];
    if ((int64_t)grid[0] * grid[1] * grid[2] > ((int64_t)1 << 31) - 1) return PIC_EINVAL;
    // sizes beyond the fixed scratch are refused, never truncated
    if (g.TC > 1024 || n > kMaxParticles || ntiles > kMaxTiles || ntiles * g.TC > kMaxKeys)
        return PIC_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
    void *scr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return PIC_ECUDA;
            g_scratch_ptr[dev] = p;
        }
        scr = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)(uintptr_t)stream;
    unsigned char *s = (unsigned char *)scr;
    // the counts are the only scratch that must start at zero; the rest is overwritten
    if (cudaMemsetAsync(s + kOffCount, 0, sizeof(int32_t) * ntiles * g.TC, st) != cudaSuccess)
        return PIC_ECUDA;
    const int tb = ((g.TC + 31) / 32) * 32;
    if (n > 0) k_nz_count<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, cell_dev, s);
    k_nz_tiles<<<(unsigned)ntiles, tb, 0, st>>>(g, s);
    k_nz_scan<<<1, 1024, 0, st>>>(ntiles, s, tile_start_dev);
    if (n > 0) {
        k_nz_place<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, s, tile_start_dev);
        k_nz_rank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, ntiles, s, tile_start_dev,
                                                               perm_dev);
    }
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
