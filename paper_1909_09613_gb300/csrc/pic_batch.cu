// Batched form: many independent 2D runs of uneven size (FP32 precision form) advanced together.
//
// One step of the whole batch is a fixed sequence of launches, captured once in a CUDA graph
// and replayed: a plan kernel decides on the device which runs are due for a tile sort; the
// batched sort kernels sort only those runs (one block table per stage covers every run);
// the current of every run is cleared; ONE persistent gather-push-deposit kernel (one CTA per
// SM slot) pulls (run, tile) work items, heaviest first, from a device counter and processes
// them with the same tile code as a single run; three batched Yee launches finish the step.
// Nothing on the host changes between steps, so the captured graph stays valid.
#include "pic.h"
#include "pic_gpp_kernels.cuh"
#include "pic_grid_dev.cuh"
#include "pic_launch.h"
#include "pic_sort_dev.cuh"

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

using namespace pic;

// access to a context's descriptor (pic_api.cu)
namespace pic {
RunDev *ctx_rundev(pic_ctx *c);
void ctx_after_batch(pic_ctx *c, const RunDev &dev_copy, int age, int64_t steps);
int ctx_kt(const pic_ctx *c);
int ctx_prepare_batch(pic_ctx *c);
int ctx_sort_interval(const pic_ctx *c);
int ctx_age(const pic_ctx *c);
cudaStream_t ctx_stream(const pic_ctx *c);
bool ctx_bound(const pic_ctx *c);
}  // namespace pic

namespace {

constexpr int kBlock = 256;
// elements per thread of the per-particle, per-key and per-cell stages: fewer, fuller blocks
// (the blocks of runs that are not due for a sort exit at once, and there are many of them)
constexpr int kPartPer = 8, kKeyPer = 8, kCellPer = 4;

struct RunState {
    int age, interval, due, kt;
};

struct BlockMap {
    int run;
    int block;  // block index inside the run's range
};

// ---- plan: which runs sort this step ----
__global__ void k_b_plan(int n, RunState *st, int *counter)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) *counter = 0;
    if (r >= n) return;
    RunState s = st[r];
    s.due = s.age >= s.interval ? 1 : 0;
    if (s.due) s.age = 0;
    s.age += 1;
    st[r] = s;
}

// ---- batched sort stages (each skips runs that are not due) ----
__global__ void __launch_bounds__(kBlock) k_b_zero_cnt(const RunDev *runs, const RunState *st,
                                                       const BlockMap *bm)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    const RunDev &rd = runs[m.run];
    const int64_t nk = rd.ntiles * rd.tile[0] * rd.tile[1] * rd.tile[2];
    int32_t *cnt = rd.sc.cnt;
    for (int k = 0; k < kKeyPer; ++k) {
        const int64_t i = ((int64_t)m.block * kKeyPer + k) * blockDim.x + threadIdx.x;
        if (i < nk) cnt[i] = 0;
    }
}

__global__ void __launch_bounds__(kBlock) k_b_count(const RunDev *runs, const RunState *st,
                                                    const BlockMap *bm, int s)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    const RunDev &rd = runs[m.run];
    const int64_t n = rd.sp[s].n;
    for (int k = 0; k < kPartPer; ++k) {
        const int64_t p = ((int64_t)m.block * kPartPer + k) * blockDim.x + threadIdx.x;
        if (p < n) sort_count_one(rd, s, p);
    }
}

__global__ void k_b_tile_sum(const RunDev *runs, const RunState *st, const BlockMap *bm)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    sort_tile_sum_block(runs[m.run], m.block);
}

__global__ void k_b_scan(const RunDev *runs, const RunState *st, int s)
{
    const int r = blockIdx.x;
    if (!st[r].due) return;
    const RunDev &rd = runs[r];
    sort_scan_block(rd.sc.tile_count, rd.sp[s].tile_start, rd.ntiles);
}

__global__ void k_b_layout(const RunDev *runs, const RunState *st, const BlockMap *bm, int s)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    const RunDev &rd = runs[m.run];
    sort_layout_block(rd, rd.sp[s].tile_start, m.block);
}

__global__ void __launch_bounds__(kBlock) k_b_place(const RunDev *runs, const RunState *st,
                                                    const BlockMap *bm, int s)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    const RunDev &rd = runs[m.run];
    const int64_t n = rd.sp[s].n;
    for (int k = 0; k < kPartPer; ++k) {
        const int64_t p = ((int64_t)m.block * kPartPer + k) * blockDim.x + threadIdx.x;
        if (p < n) sort_place_one(rd, p);
    }
}

// one thread per cell-major position r of the run's species (the same range as its particles)
__global__ void __launch_bounds__(kBlock) k_b_scatter(const RunDev *runs, const RunState *st,
                                                      const BlockMap *bm, int s)
{
    const BlockMap m = bm[blockIdx.x];
    if (!st[m.run].due) return;
    const RunDev &rd = runs[m.run];
    const SpeciesDev &sp = rd.sp[s];
    for (int k = 0; k < kPartPer; ++k) {
        const int64_t r = ((int64_t)m.block * kPartPer + k) * blockDim.x + threadIdx.x;
        if (r < sp.n) sort_scatter_one(rd, s, r, sp.pos_alt, sp.mom_alt, sp.cell_alt);
    }
}

// the sorted buffers become the current ones
__global__ void k_b_swap(RunDev *runs, const RunState *st, int n, int s)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || !st[r].due) return;
    SpeciesDev &sp = runs[r].sp[s];
    for (int a = 0; a < 3; ++a) {
        void *t = sp.pos[a]; sp.pos[a] = sp.pos_alt[a]; sp.pos_alt[a] = t;
        t = sp.mom[a]; sp.mom[a] = sp.mom_alt[a]; sp.mom_alt[a] = t;
    }
    int32_t *c = sp.cell; sp.cell = sp.cell_alt; sp.cell_alt = c;
}

// ---- current cleared, Yee updates ----
__global__ void __launch_bounds__(kBlock) k_b_zero_j(const RunDev *runs, const BlockMap *bm)
{
    const BlockMap m = bm[blockIdx.x];
    const RunDev &rd = runs[m.run];
    double *j0 = rd.F[6], *j1 = rd.F[7], *j2 = rd.F[8];
    for (int k = 0; k < kCellPer; ++k) {
        const int64_t c = ((int64_t)m.block * kCellPer + k) * blockDim.x + threadIdx.x;
        if (c < rd.ncell) {
            j0[c] = 0.0;
            j1[c] = 0.0;
            j2[c] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_b_yee_b(const RunDev *runs, const BlockMap *bm,
                                                    int shadow)
{
    const BlockMap m = bm[blockIdx.x];
    const RunDev &rd = runs[m.run];
    for (int k = 0; k < kCellPer; ++k) {
        const int64_t c = ((int64_t)m.block * kCellPer + k) * blockDim.x + threadIdx.x;
        if (c < rd.ncell) yee_b_cell(rd, c, 0.5 * rd.dt, shadow);
    }
}

__global__ void __launch_bounds__(kBlock) k_b_yee_e(const RunDev *runs, const BlockMap *bm)
{
    const BlockMap m = bm[blockIdx.x];
    const RunDev &rd = runs[m.run];
    for (int k = 0; k < kCellPer; ++k) {
        const int64_t c = ((int64_t)m.block * kCellPer + k) * blockDim.x + threadIdx.x;
        if (c < rd.ncell) yee_e_cell(rd, c, 1);
    }
}

// ---- the persistent gather-push-deposit kernel over all runs' tiles ----
template <int L, int KT>
__device__ __forceinline__ bool try_tile(const RunDev &rd, int kt, char *smem, int64_t tile)
{
    if (rd.l != L || kt != KT) return false;
    tile_2d<L, KT, float>(rd, smem, tile, rd.tt);  // the descriptor copy holds the tables
    return true;
}

__global__ void __launch_bounds__(256, 2) k_b_gpp(const RunDev *runs, const RunState *st,
                                              const int2 *items, int nitems, int *counter)
{
    extern __shared__ __align__(16) char smem_all[];
    // the run descriptor is copied next to the tile stage so that the particle loop reads it
    // from shared memory (stores to the particle arrays cannot alias it)
    RunDev *rds = (RunDev *)smem_all;
    char *smem = smem_all + ((sizeof(RunDev) + 15) / 16) * 16;
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= nitems) return;
        const int2 w = items[it];
        const int kt = st[w.x].kt;
        for (int i = threadIdx.x; i < (int)(sizeof(RunDev) / sizeof(int)); i += blockDim.x)
            ((int *)rds)[i] = ((const int *)(runs + w.x))[i];
        __syncthreads();
        const RunDev &rd = *rds;
        // every run in a batch uses the wide integer-node stencil (l + 2 nodes; the extra
        // weight is zero when c dt <= dx/2), so two instances cover the batch
        if (!(try_tile<2, 4>(rd, kt, smem, w.y) || try_tile<3, 5>(rd, kt, smem, w.y)))
            set_err(rd.err, 1);
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct pic_batch {
    int n;
    std::vector<pic_ctx *> ctx;
    cudaStream_t stream;
    bool own_stream;   // the runs use the legacy default stream, which cannot be captured
    // host-side tables
    std::vector<BlockMap> bm_part[PIC_NSP_MAX], bm_cell, bm_key, bm_tile;
    std::vector<int2> items;
    int nsp;
    int max_tc;
    size_t smem;
    // device memory
    char *base;
    size_t bytes;
    bool owns;
    RunDev *d_runs;
    RunState *d_state;
    BlockMap *d_bm_part[PIC_NSP_MAX], *d_bm_cell, *d_bm_key, *d_bm_tile;
    int2 *d_items;
    int *d_counter;
    // graph of one step
    cudaGraphExec_t exec;
    bool have_graph;
    cudaEvent_t ev0, ev1;
    bool timing;
    double gpp_ms;
    int64_t steps_since_sync;
    int64_t launches;  // kernels per step
};

namespace {

template <typename T>
size_t table_bytes(const std::vector<T> &v) { return align_up(std::max<size_t>(v.size(), 1) * sizeof(T), 256); }

// Launch sequence of one batch step on b->stream (also used while capturing).
cudaError_t enqueue_step(pic_batch *b)
{
    cudaStream_t st = b->stream;
    int64_t nl = 0;
    k_b_plan<<<(b->n + 127) / 128, 128, 0, st>>>(b->n, b->d_state, b->d_counter);
    ++nl;
    if (!b->bm_key.empty()) {
        k_b_zero_cnt<<<(unsigned)b->bm_key.size(), kBlock, 0, st>>>(b->d_runs, b->d_state, b->d_bm_key);
        ++nl;
    }
    const int tb = ((b->max_tc + 31) / 32) * 32;
    for (int s = 0; s < b->nsp; ++s) {
        if (s > 0 && !b->bm_key.empty()) {
            k_b_zero_cnt<<<(unsigned)b->bm_key.size(), kBlock, 0, st>>>(b->d_runs, b->d_state, b->d_bm_key);
            ++nl;
        }
        if (!b->bm_part[s].empty()) {
            k_b_count<<<(unsigned)b->bm_part[s].size(), kBlock, 0, st>>>(b->d_runs, b->d_state,
                                                                         b->d_bm_part[s], s);
            ++nl;
        }
        k_b_tile_sum<<<(unsigned)b->bm_tile.size(), tb, 0, st>>>(b->d_runs, b->d_state, b->d_bm_tile);
        k_b_scan<<<b->n, 1024, 0, st>>>(b->d_runs, b->d_state, s);
        k_b_layout<<<(unsigned)b->bm_tile.size(), tb, 0, st>>>(b->d_runs, b->d_state, b->d_bm_tile, s);
        nl += 3;
        if (!b->bm_part[s].empty()) {
            k_b_place<<<(unsigned)b->bm_part[s].size(), kBlock, 0, st>>>(b->d_runs, b->d_state,
                                                                         b->d_bm_part[s], s);
            ++nl;
            k_b_scatter<<<(unsigned)b->bm_part[s].size(), kBlock, 0, st>>>(b->d_runs, b->d_state,
                                                                           b->d_bm_part[s], s);
            ++nl;
        }
        k_b_swap<<<(b->n + 127) / 128, 128, 0, st>>>(b->d_runs, b->d_state, b->n, s);
        ++nl;
    }
    k_b_zero_j<<<(unsigned)b->bm_cell.size(), kBlock, 0, st>>>(b->d_runs, b->d_bm_cell);
    ++nl;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_gpp, 256, b->smem);
    const int grid = std::max(1, std::min<int>((int)b->items.size(), sms * std::max(per_sm, 1)));
    if (b->timing) cudaEventRecord(b->ev0, st);
    k_b_gpp<<<grid, 256, b->smem, st>>>(b->d_runs, b->d_state, b->d_items, (int)b->items.size(),
                                         b->d_counter);
    if (b->timing) cudaEventRecord(b->ev1, st);
    ++nl;
    k_b_yee_b<<<(unsigned)b->bm_cell.size(), kBlock, 0, st>>>(b->d_runs, b->d_bm_cell, 0);
    k_b_yee_e<<<(unsigned)b->bm_cell.size(), kBlock, 0, st>>>(b->d_runs, b->d_bm_cell);
    k_b_yee_b<<<(unsigned)b->bm_cell.size(), kBlock, 0, st>>>(b->d_runs, b->d_bm_cell, 1);
    nl += 3;
    b->launches = nl;
    return cudaGetLastError();
}

void push_blocks(std::vector<BlockMap> &v, int run, int64_t count, int per)
{
    const int64_t nb = (count + per - 1) / per;
    for (int64_t i = 0; i < nb; ++i) v.push_back({run, (int)i});
}

}  // namespace

extern "C" {

int pic_batch_create(pic_ctx *const *runs, int n, pic_batch **out)
{
    if (!runs || n <= 0 || !out) return PIC_EINVAL;
    *out = nullptr;
    pic_batch *b = new (std::nothrow) pic_batch;
    if (!b) return PIC_ENOMEM;
    b->n = n;
    b->ctx.assign(runs, runs + n);
    b->stream = ctx_stream(runs[0]);
    b->own_stream = false;
    b->nsp = ctx_rundev(runs[0])->nsp;
    b->max_tc = 1;
    b->smem = 0;
    b->base = nullptr;
    b->bytes = 0;
    b->owns = false;
    b->have_graph = false;
    b->timing = false;
    b->gpp_ms = 0.0;
    b->steps_since_sync = 0;
    b->launches = 0;
    std::vector<std::pair<int64_t, int2>> work;
    for (int r = 0; r < n; ++r) {
        pic_ctx *c = runs[r];
        if (!c || !ctx_bound(c)) { delete b; return PIC_ESTATE; }
        const RunDev &rd = *ctx_rundev(c);
        if (rd.dim != 2 || rd.prec != PIC_FP32_MIXED || rd.nsp != b->nsp || rd.l < 2 || rd.l > 3
            || rd.det || ctx_stream(c) != b->stream) {
            delete b;
            return PIC_EINVAL;
        }
        const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
        b->max_tc = std::max(b->max_tc, TC);
        b->smem = std::max(b->smem, stage2d_bytes<float>(rd.reg_nodes, rd.l, false));
        for (int s = 0; s < b->nsp; ++s) push_blocks(b->bm_part[s], r, rd.sp[s].n, kBlock * kPartPer);
        push_blocks(b->bm_cell, r, rd.ncell, kBlock * kCellPer);
        push_blocks(b->bm_key, r, rd.ntiles * TC, kBlock * kKeyPer);
        for (int64_t t = 0; t < rd.ntiles; ++t) b->bm_tile.push_back({r, (int)t});
        int64_t np = 0;
        for (int s = 0; s < b->nsp; ++s) np += rd.sp[s].n;
        const int64_t per_tile = rd.ntiles > 0 ? np / rd.ntiles : 0;
        for (int64_t t = 0; t < rd.ntiles; ++t) work.push_back({per_tile, make_int2(r, (int)t)});
    }
    // heaviest work items first (longest-processing-time order for the dynamic scheduler)
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<int64_t, int2> &a, const std::pair<int64_t, int2> &c) {
                         return a.first > c.first;
                     });
    for (auto &w : work) b->items.push_back(w.second);
    b->smem += ((sizeof(RunDev) + 15) / 16) * 16;
    if (b->smem > 227 * 1024) { delete b; return PIC_EINVAL; }
    if (b->stream == 0) {
        // a blocking stream is ordered with the legacy default stream the runs use
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault) != cudaSuccess) {
            delete b;
            return PIC_ECUDA;
        }
        b->own_stream = true;
    }
    *out = b;
    return PIC_OK;
}

int pic_batch_footprint(const pic_batch *b, size_t *bytes)
{
    if (!b || !bytes) return PIC_EINVAL;
    size_t s = align_up(b->n * sizeof(RunDev), 256) + align_up(b->n * sizeof(RunState), 256);
    for (int i = 0; i < b->nsp; ++i) s += table_bytes(b->bm_part[i]);
    s += table_bytes(b->bm_cell) + table_bytes(b->bm_key) + table_bytes(b->bm_tile);
    s += table_bytes(b->items) + 256 + 256;
    *bytes = s;
    return PIC_OK;
}

int pic_batch_bind_memory(pic_batch *b, void *dev, size_t bytes)
{
    if (!b || !dev) return PIC_EINVAL;
    size_t need = 0;
    pic_batch_footprint(b, &need);
    if (bytes < need) return PIC_ENOMEM;
    char *p = (char *)align_up((size_t)dev, 256);
    auto take = [&](size_t nb) { char *r = p; p += align_up(nb, 256); return r; };
    b->base = (char *)dev;
    b->bytes = bytes;
    b->d_runs = (RunDev *)take(b->n * sizeof(RunDev));
    b->d_state = (RunState *)take(b->n * sizeof(RunState));
    for (int i = 0; i < b->nsp; ++i) b->d_bm_part[i] = (BlockMap *)take(table_bytes(b->bm_part[i]));
    b->d_bm_cell = (BlockMap *)take(table_bytes(b->bm_cell));
    b->d_bm_key = (BlockMap *)take(table_bytes(b->bm_key));
    b->d_bm_tile = (BlockMap *)take(table_bytes(b->bm_tile));
    b->d_items = (int2 *)take(table_bytes(b->items));
    b->d_counter = (int *)take(sizeof(int));
    for (int r = 0; r < b->n; ++r) {
        const int e = ctx_prepare_batch(b->ctx[r]);
        if (e != PIC_OK) return e;
    }
    // descriptors and tables
    std::vector<RunDev> rds(b->n);
    std::vector<RunState> sts(b->n);
    for (int r = 0; r < b->n; ++r) {
        rds[r] = *ctx_rundev(b->ctx[r]);
        sts[r].age = ctx_age(b->ctx[r]);
        sts[r].interval = ctx_sort_interval(b->ctx[r]);
        sts[r].due = 0;
        sts[r].kt = ctx_rundev(b->ctx[r])->l + 2;
    }
    cudaStream_t st = b->stream;
    auto up = [&](void *dst, const void *src, size_t nb) {
        return nb == 0 || cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    bool ok = up(b->d_runs, rds.data(), rds.size() * sizeof(RunDev))
              && up(b->d_state, sts.data(), sts.size() * sizeof(RunState));
    for (int i = 0; i < b->nsp && ok; ++i)
        ok = up(b->d_bm_part[i], b->bm_part[i].data(), b->bm_part[i].size() * sizeof(BlockMap));
    ok = ok && up(b->d_bm_cell, b->bm_cell.data(), b->bm_cell.size() * sizeof(BlockMap))
         && up(b->d_bm_key, b->bm_key.data(), b->bm_key.size() * sizeof(BlockMap))
         && up(b->d_bm_tile, b->bm_tile.data(), b->bm_tile.size() * sizeof(BlockMap))
         && up(b->d_items, b->items.data(), b->items.size() * sizeof(int2));
    if (!ok || cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
    if (cudaFuncSetAttribute(k_b_gpp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem)
        != cudaSuccess)
        return PIC_ECUDA;
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
        return PIC_ECUDA;
    return PIC_OK;
}

int pic_batch_alloc(pic_batch *b)
{
    if (!b) return PIC_EINVAL;
    size_t need = 0;
    pic_batch_footprint(b, &need);
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) return PIC_ENOMEM;
    const int r = pic_batch_bind_memory(b, p, need);
    if (r != PIC_OK) { cudaFree(p); return r; }
    b->owns = true;
    return PIC_OK;
}

int pic_batch_step(pic_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return PIC_EINVAL;
    if (!b->base) return PIC_ESTATE;
    if (!b->have_graph) {
        cudaGraph_t g;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return PIC_ECUDA;
        }
        const cudaError_t e = enqueue_step(b);
        if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || e != cudaSuccess) {
            cudaGetLastError();
            return PIC_ECUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return PIC_ECUDA;
        b->have_graph = true;
    }
    for (int i = 0; i < nsteps; ++i)
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return PIC_ECUDA;
    b->steps_since_sync += nsteps;
    return PIC_OK;
}

// Time of the persistent particle kernel in one replayed step (ms): runs one step with event
// records around it (outside the captured graph).
int pic_batch_time_gpp(pic_batch *b, double *ms)
{
    if (!b || !ms) return PIC_EINVAL;
    if (!b->base) return PIC_ESTATE;
    b->timing = true;
    const cudaError_t e = enqueue_step(b);
    b->timing = false;
    if (e != cudaSuccess) return PIC_ECUDA;
    b->steps_since_sync += 1;
    if (cudaEventSynchronize(b->ev1) != cudaSuccess) return PIC_ECUDA;
    float f = 0.0f;
    if (cudaEventElapsedTime(&f, b->ev0, b->ev1) != cudaSuccess) return PIC_ECUDA;
    *ms = f;
    return PIC_OK;
}

int pic_batch_info(const pic_batch *b, int64_t *work_items, int64_t *launches_per_step)
{
    if (!b) return PIC_EINVAL;
    if (work_items) *work_items = (int64_t)b->items.size();
    if (launches_per_step) *launches_per_step = b->launches;
    return PIC_OK;
}

// Write the device-side run state (buffer swaps of the sorts, sort ages, step counts) back
// into the contexts.  Syncs.
int pic_batch_sync(pic_batch *b)
{
    if (!b) return PIC_EINVAL;
    if (!b->base) return PIC_ESTATE;
    std::vector<RunDev> rds(b->n);
    std::vector<RunState> sts(b->n);
    if (cudaMemcpyAsync(rds.data(), b->d_runs, b->n * sizeof(RunDev), cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess
        || cudaMemcpyAsync(sts.data(), b->d_state, b->n * sizeof(RunState), cudaMemcpyDeviceToHost,
                           b->stream) != cudaSuccess
        || cudaStreamSynchronize(b->stream) != cudaSuccess)
        return PIC_ECUDA;
    for (int r = 0; r < b->n; ++r) ctx_after_batch(b->ctx[r], rds[r], sts[r].age, b->steps_since_sync);
    b->steps_since_sync = 0;
    int32_t err = 0;
    for (int r = 0; r < b->n; ++r) {
        int32_t e = 0;
        if (cudaMemcpy(&e, rds[r].err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
        err |= e;
    }
    if (err & PIC_ERR_NONFINITE) return PIC_ENAN;
    if (err & PIC_ERR_OUTSIDE_TILE) return PIC_EOVERFLOW;
    return PIC_OK;
}

void pic_batch_destroy(pic_batch *b)
{
    if (!b) return;
    if (b->base) {
        cudaStreamSynchronize(b->stream);
        if (b->steps_since_sync) pic_batch_sync(b);
        cudaEventDestroy(b->ev0);
        cudaEventDestroy(b->ev1);
    }
    if (b->have_graph) cudaGraphExecDestroy(b->exec);
    if (b->owns && b->base) cudaFree(b->base);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
