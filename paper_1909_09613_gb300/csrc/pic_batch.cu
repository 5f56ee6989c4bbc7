// Batched form: many independent 2D runs of uneven size (FP32 precision form) advanced together.
//
// One step of the whole batch is a fixed sequence of launches, captured once in a CUDA graph
// and replayed: a plan kernel decides on the device which runs are due for a tile sort; the
// batched sort kernels sort only those runs; the current of every run is cleared; ONE
// persistent gather-push-deposit kernel (one CTA per SM slot) pulls (run, tile) work items,
// heaviest first, from a device counter and processes them with the same tile code as a single
// run; three batched Yee launches finish the step.
//
// Every launch has a fixed grid and walks device-resident tables (run descriptors, per-stage
// block maps, work items) whose lengths it reads from device memory.  The captured graph
// therefore does not depend on which runs the batch holds: pic_batch_set_runs replaces the
// runs between steps by writing the old runs' device state back and uploading new tables, and
// the same graph keeps serving (a set larger than the tables' capacity needs a new batch).
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
// threads of the per-tile sort stages: one per cell of the largest tile a run may have
constexpr int kTileThreads = 1024;
// work items of a split tile: at most kPartMax, each of at least kPartMin particles
constexpr int kPartMax = 8;
constexpr int64_t kPartMin = 2048;

struct RunState {
    int age, interval, due, kt;
};

struct BlockMap {
    int run;
    int block;  // block index inside the run's range
};

// Lengths of the device tables, read by every stage (the graph never changes with them), and
// the number of runs due for a tile sort this step (written by k_b_plan).
struct Counts {
    int runs;
    int cell, items;
    int due;
};

// ---- plan: which runs sort this step ----
// One block: every run's sort age advances, and the runs due for a sort are listed in run
// order (a block scan of the due flags), for the sort stages to walk.
__global__ void __launch_bounds__(1024) k_b_plan(Counts *cn, RunState *st, int *due, int *counter)
{
    __shared__ int tot;
    if (threadIdx.x == 0) *counter = 0;
    const int n = cn->runs;
    int base = 0;
    for (int r0 = 0; r0 < n; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        int flag = 0;
        if (r < n) {
            RunState s = st[r];
            s.due = s.age >= s.interval ? 1 : 0;
            if (s.due) s.age = 0;
            s.age += 1;
            st[r] = s;
            flag = s.due;
        }
        const int pos = sort_block_excl_scan(flag, &tot);
        if (flag) due[base + pos] = r;
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) cn->due = base;
}

// ---- batched sort stages: each walks the due runs only.  Work block e of the d-th due run
// goes to CUDA block (e + 97 d) mod gridDim, so that the few work blocks of small runs spread
// over the grid instead of queueing on its first blocks. ----
__device__ __forceinline__ int64_t part_blocks(int64_t n)
{
    return (n + kBlock * kPartPer - 1) / (kBlock * kPartPer);
}

// first work block of due run d that this CUDA block takes
__device__ __forceinline__ int64_t first_block(int d)
{
    const int shift = (int)((97ll * d) % gridDim.x);
    return (blockIdx.x + gridDim.x - shift) % gridDim.x;
}

__global__ void __launch_bounds__(kBlock) k_b_zero_cnt(const Counts *cn, const RunDev *runs,
                                                       const int *due)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        const int64_t nk = rd.ntiles * rd.tile[0] * rd.tile[1] * rd.tile[2];
        int32_t *cnt = rd.sc.cnt;
        const int64_t nb = (nk + kBlock * kKeyPer - 1) / (kBlock * kKeyPer);
        for (int64_t e = first_block(d); e < nb; e += gridDim.x)
            for (int k = 0; k < kKeyPer; ++k) {
                const int64_t i = (e * kKeyPer + k) * blockDim.x + threadIdx.x;
                if (i < nk) cnt[i] = 0;
            }
    }
}

__global__ void __launch_bounds__(kBlock) k_b_count(const Counts *cn, const RunDev *runs,
                                                    const int *due, int s)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        const int64_t n = rd.sp[s].n;
        for (int64_t e = first_block(d); e < part_blocks(n); e += gridDim.x)
            for (int k = 0; k < kPartPer; ++k) {
                const int64_t p = (e * kPartPer + k) * blockDim.x + threadIdx.x;
                if (p < n) sort_count_one(rd, s, p);
            }
    }
}

// block-wide stages: the loop indices are uniform over the block, so every thread takes part
// in the block's barriers and scans
__global__ void __launch_bounds__(kTileThreads) k_b_tile_sum(const Counts *cn, const RunDev *runs,
                                                             const int *due)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        for (int64_t t = first_block(d); t < rd.ntiles; t += gridDim.x) {
            sort_tile_sum_block(rd, t);
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(1024) k_b_scan(const Counts *cn, const RunDev *runs,
                                                 const int *due, int s)
{
    for (int d = blockIdx.x; d < cn->due; d += gridDim.x) {
        const RunDev &rd = runs[due[d]];
        sort_scan_block(rd.sc.tile_count, rd.sp[s].tile_start, rd.ntiles);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTileThreads) k_b_layout(const Counts *cn, const RunDev *runs,
                                                           const int *due, int s)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        for (int64_t t = first_block(d); t < rd.ntiles; t += gridDim.x) {
            sort_layout_block(rd, rd.sp[s].tile_start, t);
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_b_place(const Counts *cn, const RunDev *runs,
                                                    const int *due, int s)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        const int64_t n = rd.sp[s].n;
        for (int64_t e = first_block(d); e < part_blocks(n); e += gridDim.x)
            for (int k = 0; k < kPartPer; ++k) {
                const int64_t p = (e * kPartPer + k) * blockDim.x + threadIdx.x;
                if (p < n) sort_place_one(rd, p);
            }
    }
}

// one thread per cell-major position r of the run's species (the same range as its particles)
__global__ void __launch_bounds__(kBlock) k_b_scatter(const Counts *cn, const RunDev *runs,
                                                      const int *due, int s)
{
    const int nd = cn->due;
    for (int d = 0; d < nd; ++d) {
        const RunDev &rd = runs[due[d]];
        const SpeciesDev &sp = rd.sp[s];
        for (int64_t e = first_block(d); e < part_blocks(sp.n); e += gridDim.x)
            for (int k = 0; k < kPartPer; ++k) {
                const int64_t r = (e * kPartPer + k) * blockDim.x + threadIdx.x;
                if (r < sp.n) sort_scatter_one(rd, s, r, sp.pos_alt, sp.mom_alt, sp.cell_alt);
            }
    }
}

// the sorted buffers become the current ones
__global__ void k_b_swap(const Counts *cn, RunDev *runs, const int *due, int s)
{
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < cn->due; d += gridDim.x * blockDim.x) {
        SpeciesDev &sp = runs[due[d]].sp[s];
        for (int a = 0; a < 3; ++a) {
            void *t = sp.pos[a]; sp.pos[a] = sp.pos_alt[a]; sp.pos_alt[a] = t;
            t = sp.mom[a]; sp.mom[a] = sp.mom_alt[a]; sp.mom_alt[a] = t;
        }
        int32_t *c = sp.cell; sp.cell = sp.cell_alt; sp.cell_alt = c;
    }
}

// ---- current cleared, Yee updates ----
__global__ void __launch_bounds__(kBlock) k_b_zero_j(const Counts *cn, const RunDev *runs,
                                                     const BlockMap *bm)
{
    for (int b = blockIdx.x; b < cn->cell; b += gridDim.x) {
        const BlockMap m = bm[b];
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
}

__global__ void __launch_bounds__(kBlock) k_b_yee_b(const Counts *cn, const RunDev *runs,
                                                    const BlockMap *bm, int shadow)
{
    for (int b = blockIdx.x; b < cn->cell; b += gridDim.x) {
        const BlockMap m = bm[b];
        const RunDev &rd = runs[m.run];
        for (int k = 0; k < kCellPer; ++k) {
            const int64_t c = ((int64_t)m.block * kCellPer + k) * blockDim.x + threadIdx.x;
            if (c < rd.ncell) yee_b_cell(rd, c, 0.5 * rd.dt, shadow);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_b_yee_e(const Counts *cn, const RunDev *runs,
                                                    const BlockMap *bm)
{
    for (int b = blockIdx.x; b < cn->cell; b += gridDim.x) {
        const BlockMap m = bm[b];
        const RunDev &rd = runs[m.run];
        for (int k = 0; k < kCellPer; ++k) {
            const int64_t c = ((int64_t)m.block * kCellPer + k) * blockDim.x + threadIdx.x;
            if (c < rd.ncell) yee_e_cell(rd, c, 1);
        }
    }
}

// ---- the persistent gather-push-deposit kernel over all runs' tiles ----
template <int L, int KT>
__device__ __forceinline__ bool try_tile(const RunDev &rd, int kt, char *smem, int tile,
                                         const int *split)
{
    if (rd.l != L || kt != KT) return false;
    tile_2d<L, KT, float>(rd, smem, tile, rd.tt, split);  // the descriptor copy holds the tables
    return true;
}

__global__ void __launch_bounds__(256, 2) k_b_gpp(const Counts *cn, const RunDev *runs,
                                              const RunState *st, const int4 *items, int *counter)
{
    extern __shared__ __align__(16) char smem_all[];
    // the run descriptor is copied next to the tile stage so that the particle loop reads it
    // from shared memory (stores to the particle arrays cannot alias it)
    RunDev *rds = (RunDev *)smem_all;
    char *smem = smem_all + ((sizeof(RunDev) + 15) / 16) * 16;
    __shared__ int item;
    __shared__ int4 work;  // run, tile, part, parts
    const int nitems = cn->items;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            item = atomicAdd(counter, 1);
            if (item < nitems) work = items[item];
        }
        __syncthreads();
        const int it = item;
        if (it >= nitems) return;
        const int2 w = make_int2(work.x, work.y);
        const int kt = st[w.x].kt;
        for (int i = threadIdx.x; i < (int)(sizeof(RunDev) / sizeof(int)); i += blockDim.x)
            ((int *)rds)[i] = ((const int *)(runs + w.x))[i];
        __syncthreads();
        const RunDev &rd = *rds;
        // every run in a batch uses the wide integer-node stencil (l + 2 nodes; the extra
        // weight is zero when c dt <= dx/2), so two instances cover the batch
        if (!(try_tile<2, 4>(rd, kt, smem, w.y, &work.z) || try_tile<3, 5>(rd, kt, smem, w.y, &work.z)))
            set_err(rd.err, 1);
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void push_blocks(std::vector<BlockMap> &v, int run, int64_t count, int per)
{
    const int64_t nb = (count + per - 1) / per;
    for (int64_t i = 0; i < nb; ++i) v.push_back({run, (int)i});
}

}  // namespace

struct pic_batch {
    int n;                          // runs the batch holds now
    std::vector<pic_ctx *> ctx;
    cudaStream_t stream;      // where the batch's steps run (captured)
    cudaStream_t run_stream;  // the runs' own stream (every run of a set must share it)
    bool own_stream;   // the runs use the legacy default stream, which cannot be captured
    int nsp;
    size_t smem;       // dynamic shared memory of the persistent kernel (fixed by the graph)
    // table capacities (entries; the work items are one per tile) and the current tables
    int cap_runs;
    int64_t cap_cell, cap_tile;
    std::vector<BlockMap> bm_cell;
    std::vector<int4> items;
    // device memory
    char *base;
    size_t bytes;
    bool owns;
    Counts *d_counts;
    RunDev *d_runs;
    RunState *d_state;
    int *d_due;        // runs due for a sort this step (k_b_plan)
    BlockMap *d_bm_cell;
    int4 *d_items;
    int *d_counter;
    // launch shapes and the graph of one step
    int grid_runs, grid_scan, grid_stage, grid_tile, grid_gpp;
    cudaGraphExec_t exec;
    bool have_graph;
    cudaEvent_t ev0, ev1;
    bool timing;
    int64_t steps_since_sync;
    int64_t launches;  // kernels per step
    int ctas_per_sm;   // cap on the persistent kernel's CTAs per SM (0: none)
};

namespace {

template <typename T>
size_t cap_bytes(int64_t entries) { return align_up((size_t)std::max<int64_t>(entries, 1) * sizeof(T), 256); }

// Tables of a set of runs (validated: 2D, FP32 form, l = 2 or 3, not deterministic, the batch's
// species count and stream), and the shared memory its work items need.
struct Tables {
    std::vector<BlockMap> cell;
    std::vector<int4> items;
    size_t smem = 0;
};

int build_tables(pic_ctx *const *runs, int n, int nsp, cudaStream_t stream, Tables &t)
{
    std::vector<std::pair<int64_t, int4>> work;
    std::vector<pic_ctx *> seen(runs, runs + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return PIC_EINVAL;  // twice
    for (int r = 0; r < n; ++r) {
        pic_ctx *c = runs[r];
        if (!c || !ctx_bound(c)) return PIC_ESTATE;
        const RunDev &rd = *ctx_rundev(c);
        if (rd.dim != 2 || rd.prec != PIC_FP32_MIXED || rd.nsp != nsp || rd.l < 2 || rd.l > 3
            || rd.det || ctx_stream(c) != stream)
            return PIC_EINVAL;
        const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
        if (TC > kTileThreads) return PIC_EINVAL;
        t.smem = std::max(t.smem, stage2d_bytes<float>(rd.reg_nodes, rd.l, false));
        push_blocks(t.cell, r, rd.ncell, kBlock * kCellPer);
        int64_t np = 0;
        for (int s = 0; s < nsp; ++s) np += rd.sp[s].n;
        const int64_t per_tile = rd.ntiles > 0 ? np / rd.ntiles : 0;
        for (int64_t i = 0; i < rd.ntiles; ++i) work.push_back({per_tile, make_int4(r, (int)i, 0, 1)});
    }
    // A set of few particles leaves most CTA slots of the persistent kernel idle while the
    // heaviest tiles take the whole step: split every tile that holds more than the average
    // load of a slot (and more than kPartMin particles) into up to kPartMax items that share
    // its particles.
    {
        int dev_id = 0, sms = 0;
        if (cudaGetDevice(&dev_id) != cudaSuccess
            || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess)
            return PIC_ECUDA;
        int64_t total = 0;
        for (const auto &w : work) total += w.first;
        const int64_t share = std::max<int64_t>(total / (2 * (int64_t)std::max(sms, 1)), kPartMin);
        std::vector<std::pair<int64_t, int4>> split;
        for (const auto &w : work) {
            const int parts = (int)std::min<int64_t>(kPartMax, std::max<int64_t>(1, (w.first + share - 1) / share));
            for (int k = 0; k < parts; ++k)
                split.push_back({w.first / parts, make_int4(w.second.x, w.second.y, k, parts)});
        }
        work.swap(split);
    }
    // heaviest work items first (longest-processing-time order for the dynamic scheduler)
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<int64_t, int4> &a, const std::pair<int64_t, int4> &c) {
                         return a.first > c.first;
                     });
    for (auto &w : work) t.items.push_back(w.second);
    t.smem += ((sizeof(RunDev) + 15) / 16) * 16;
    return PIC_OK;
}

bool tables_fit(const pic_batch *b, const Tables &t, int n)
{
    return !(n > b->cap_runs || (int64_t)t.cell.size() > b->cap_cell
             || (int64_t)t.items.size() > b->cap_tile || t.smem > b->smem);
}

// Launch sequence of one batch step on b->stream (also used while capturing).  Every grid is
// fixed by the capacities; the kernels read the table lengths from d_counts.
cudaError_t enqueue_step(pic_batch *b)
{
    cudaStream_t st = b->stream;
    const Counts *cn = b->d_counts;
    int64_t nl = 0;
    k_b_plan<<<1, 1024, 0, st>>>(b->d_counts, b->d_state, b->d_due, b->d_counter);
    ++nl;
    for (int s = 0; s < b->nsp; ++s) {
        k_b_zero_cnt<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_due);
        k_b_count<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_due, s);
        k_b_tile_sum<<<b->grid_tile, kTileThreads, 0, st>>>(cn, b->d_runs, b->d_due);
        k_b_scan<<<b->grid_scan, 1024, 0, st>>>(cn, b->d_runs, b->d_due, s);
        k_b_layout<<<b->grid_tile, kTileThreads, 0, st>>>(cn, b->d_runs, b->d_due, s);
        k_b_place<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_due, s);
        k_b_scatter<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_due, s);
        k_b_swap<<<b->grid_runs, 128, 0, st>>>(cn, b->d_runs, b->d_due, s);
        nl += 8;
    }
    k_b_zero_j<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_bm_cell);
    ++nl;
    if (b->timing) cudaEventRecord(b->ev0, st);
    k_b_gpp<<<b->grid_gpp, 256, b->smem, st>>>(cn, b->d_runs, b->d_state, b->d_items, b->d_counter);
    if (b->timing) cudaEventRecord(b->ev1, st);
    ++nl;
    k_b_yee_b<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_bm_cell, 0);
    k_b_yee_e<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_bm_cell);
    k_b_yee_b<<<b->grid_stage, kBlock, 0, st>>>(cn, b->d_runs, b->d_bm_cell, 1);
    nl += 3;
    b->launches = nl;
    return cudaGetLastError();
}

// Write the device-side state of the batch's current runs (buffer swaps of the sorts, sort
// ages, step counts) back into their contexts.  Syncs.  Returns the latched error bits.
int write_back(pic_batch *b, int32_t *err_out)
{
    int32_t err = 0;
    if (b->n > 0) {
        std::vector<RunDev> rds(b->n);
        std::vector<RunState> sts(b->n);
        if (cudaMemcpyAsync(rds.data(), b->d_runs, b->n * sizeof(RunDev), cudaMemcpyDeviceToHost,
                            b->stream) != cudaSuccess
            || cudaMemcpyAsync(sts.data(), b->d_state, b->n * sizeof(RunState),
                               cudaMemcpyDeviceToHost, b->stream) != cudaSuccess
            || cudaStreamSynchronize(b->stream) != cudaSuccess)
            return PIC_ECUDA;
        for (int r = 0; r < b->n; ++r)
            ctx_after_batch(b->ctx[r], rds[r], sts[r].age, b->steps_since_sync);
        for (int r = 0; r < b->n; ++r) {
            int32_t e = 0;
            if (cudaMemcpy(&e, rds[r].err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess)
                return PIC_ECUDA;
            err |= e;
        }
    }
    b->steps_since_sync = 0;
    if (err_out) *err_out = err;
    return PIC_OK;
}

// Upload the descriptors, states and tables of a run set (already validated and fitting the
// capacities) and make it the batch's current set.
int upload(pic_batch *b, pic_ctx *const *runs, int n, Tables &t)
{
    for (int r = 0; r < n; ++r) {
        const int e = ctx_prepare_batch(runs[r]);
        if (e != PIC_OK) return e;
    }
    std::vector<RunDev> rds(n);
    std::vector<RunState> sts(n);
    for (int r = 0; r < n; ++r) {
        rds[r] = *ctx_rundev(runs[r]);
        sts[r].age = ctx_age(runs[r]);
        sts[r].interval = ctx_sort_interval(runs[r]);
        sts[r].due = 0;
        sts[r].kt = ctx_rundev(runs[r])->l + 2;
    }
    Counts cn;
    std::memset(&cn, 0, sizeof(cn));
    cn.runs = n;
    cn.cell = (int)t.cell.size();
    cn.items = (int)t.items.size();
    cudaStream_t st = b->stream;
    auto up = [&](void *dst, const void *src, size_t nb) {
        return nb == 0 || cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    bool ok = up(b->d_runs, rds.data(), rds.size() * sizeof(RunDev))
              && up(b->d_state, sts.data(), sts.size() * sizeof(RunState))
              && up(b->d_counts, &cn, sizeof(cn));
    ok = ok && up(b->d_bm_cell, t.cell.data(), t.cell.size() * sizeof(BlockMap))
         && up(b->d_items, t.items.data(), t.items.size() * sizeof(int4));
    // the host vectors are released on return: wait for the copies
    if (!ok || cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
    b->n = n;
    b->ctx.assign(runs, runs + n);
    b->bm_cell.swap(t.cell);
    b->items.swap(t.items);
    b->steps_since_sync = 0;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_create(pic_ctx *const *runs, int n, pic_batch **out)
{
    if (!runs || n <= 0 || !out || !runs[0]) return PIC_EINVAL;
    *out = nullptr;
    if (!ctx_bound(runs[0])) return PIC_ESTATE;
    pic_batch *b = new (std::nothrow) pic_batch;
    if (!b) return PIC_ENOMEM;
    b->n = 0;
    b->stream = ctx_stream(runs[0]);
    b->run_stream = b->stream;
    b->own_stream = false;
    b->nsp = ctx_rundev(runs[0])->nsp;
    b->base = nullptr;
    b->bytes = 0;
    b->owns = false;
    b->have_graph = false;
    b->timing = false;
    b->steps_since_sync = 0;
    b->launches = 0;
    b->ctas_per_sm = 0;
    Tables t;
    const int e = build_tables(runs, n, b->nsp, b->stream, t);
    if (e != PIC_OK) { delete b; return e; }
    if (t.smem > 227 * 1024) { delete b; return PIC_EINVAL; }
    // capacities of the initial set (pic_batch_reserve raises them before binding)
    b->smem = t.smem;
    b->cap_runs = n;
    b->cap_cell = (int64_t)t.cell.size();
    b->cap_tile = (int64_t)t.items.size();
    // the initial set, uploaded by pic_batch_bind_memory
    b->ctx.assign(runs, runs + n);
    b->bm_cell.swap(t.cell);
    b->items.swap(t.items);
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

int pic_batch_reserve(pic_batch *b, const pic_batch_capacity *cap)
{
    if (!b || !cap) return PIC_EINVAL;
    if (b->base) return PIC_ESTATE;  // the capacities size the bound memory
    if (cap->runs < 0 || cap->cells < 0 || cap->tiles < 0 || cap->stage_bytes > 227 * 1024
        || cap->ctas_per_sm < 0)
        return PIC_EINVAL;
    b->ctas_per_sm = cap->ctas_per_sm;
    b->cap_runs = std::max(b->cap_runs, (int)cap->runs);
    b->cap_cell = std::max<int64_t>(b->cap_cell, cap->cells / (kBlock * kCellPer) + cap->runs);
    b->cap_tile = std::max<int64_t>(b->cap_tile, cap->tiles);
    b->smem = std::max(b->smem, std::min(cap->stage_bytes, (size_t)227 * 1024));
    return PIC_OK;
}

int pic_batch_footprint(const pic_batch *b, size_t *bytes)
{
    if (!b || !bytes) return PIC_EINVAL;
    size_t s = align_up(sizeof(Counts), 256);
    s += cap_bytes<RunDev>(b->cap_runs) + cap_bytes<RunState>(b->cap_runs)
         + cap_bytes<int>(b->cap_runs);
    s += cap_bytes<BlockMap>(b->cap_cell) + cap_bytes<int4>(b->cap_tile) + 256 + 256;
    *bytes = s;
    return PIC_OK;
}

int pic_batch_bind_memory(pic_batch *b, void *dev, size_t bytes)
{
    if (!b || !dev) return PIC_EINVAL;
    if (b->base) return PIC_ESTATE;
    size_t need = 0;
    pic_batch_footprint(b, &need);
    if (bytes < need) return PIC_ENOMEM;
    char *p = (char *)align_up((size_t)dev, 256);
    auto take = [&](size_t nb) { char *r = p; p += align_up(nb, 256); return r; };
    b->bytes = bytes;
    b->d_counts = (Counts *)take(sizeof(Counts));
    b->d_runs = (RunDev *)take(cap_bytes<RunDev>(b->cap_runs));
    b->d_state = (RunState *)take(cap_bytes<RunState>(b->cap_runs));
    b->d_due = (int *)take(cap_bytes<int>(b->cap_runs));
    b->d_bm_cell = (BlockMap *)take(cap_bytes<BlockMap>(b->cap_cell));
    b->d_items = (int4 *)take(cap_bytes<int4>(b->cap_tile));
    b->d_counter = (int *)take(sizeof(int));
    // launch shapes, fixed for the life of the batch (and of its graph)
    int dev_id = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev_id) != cudaSuccess
        || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess)
        return PIC_ECUDA;
    // the attribute is the function's limit, shared by every batch: set it to the largest the
    // device allows beside the kernel's static shared memory, so that no batch lowers it under
    // another batch's captured graph
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_id) != cudaSuccess
        || cudaFuncGetAttributes(&fa, k_b_gpp) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ECUDA;
    }
    const int maxdyn = optin - (int)fa.sharedSizeBytes;
    if (maxdyn < (int)b->smem) return PIC_EINVAL;
    if (cudaFuncSetAttribute(k_b_gpp, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn)
        != cudaSuccess) {
        cudaGetLastError();
        return PIC_ECUDA;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_gpp, 256, b->smem);
    auto clampg = [](int64_t want, int64_t cap) { return (int)std::max<int64_t>(1, std::min(want, cap)); };
    b->grid_runs = clampg((b->cap_runs + 127) / 128, 1 << 20);
    b->grid_scan = clampg(b->cap_runs, sms);
    b->grid_stage = (int)sms * 8;
    b->grid_tile = (int)sms * 2;
    if (b->ctas_per_sm > 0) per_sm = std::min(per_sm, b->ctas_per_sm);
    b->grid_gpp = clampg(b->cap_tile, (int64_t)sms * std::max(per_sm, 1));
    b->base = (char *)dev;
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
        return PIC_ECUDA;
    Tables t;
    t.cell.swap(b->bm_cell);
    t.items.swap(b->items);
    std::vector<pic_ctx *> runs = b->ctx;
    return upload(b, runs.data(), (int)runs.size(), t);
}

int pic_batch_alloc(pic_batch *b)
{
    if (!b) return PIC_EINVAL;
    size_t need = 0;
    pic_batch_footprint(b, &need);
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) return PIC_ENOMEM;
    const int r = pic_batch_bind_memory(b, p, need);
    if (r != PIC_OK) { cudaFree(p); b->base = nullptr; return r; }
    b->owns = true;
    return PIC_OK;
}

int pic_batch_set_runs(pic_batch *b, pic_ctx *const *runs, int n)
{
    if (!b || n < 0 || (n > 0 && !runs)) return PIC_EINVAL;
    if (!b->base) return PIC_ESTATE;
    Tables t;
    int e = build_tables(runs, n, b->nsp, b->run_stream, t);
    if (e != PIC_OK) return e;
    if (!tables_fit(b, t, n)) return PIC_ENOMEM;
    int32_t err = 0;
    e = write_back(b, &err);
    if (e != PIC_OK) return e;
    return upload(b, runs, n, t);
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

// Time of the persistent particle kernel in one step (ms): runs one step with event records
// around it (outside the captured graph).
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
    int32_t err = 0;
    const int e = write_back(b, &err);
    if (e != PIC_OK) return e;
    if (err & PIC_ERR_NONFINITE) return PIC_ENAN;
    if (err & PIC_ERR_OUTSIDE_TILE) return PIC_EOVERFLOW;
    return PIC_OK;
}

void pic_batch_destroy(pic_batch *b)
{
    if (!b) return;
    if (b->base) {
        cudaStreamSynchronize(b->stream);
        if (b->steps_since_sync) write_back(b, nullptr);
        cudaEventDestroy(b->ev0);
        cudaEventDestroy(b->ev1);
    }
    if (b->have_graph) cudaGraphExecDestroy(b->exec);
    if (b->owns && b->base) cudaFree(b->base);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
