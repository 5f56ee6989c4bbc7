// C-ABI of libpic (declared in include/pic.h): context management, device memory layout,
// particle loading and read-back, the step loop, and diagnostics.
#include "pic.h"
#include "pic_launch.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace pic;

namespace pic {
cudaError_t launch_gpp_f32(const RunDev &rd, int kt, cudaStream_t st);
cudaError_t launch_gpp_f64(const RunDev &rd, int kt, cudaStream_t st);
size_t gpp_smem_bytes_f32(const RunDev &rd);
size_t gpp_batch_smem_bytes_f32(const RunDev &rd);
size_t gpp_smem_bytes_f64(const RunDev &rd);
}  // namespace pic

struct pic_ctx {
    RunDev rd;                 // device-side descriptor (pointers filled on bind)
    int kt;                    // nodes of the integer-node stencil (max over axes)
    int sort_interval;
    int age;                   // steps since the last sort
    int64_t step;
    cudaStream_t stream;
    int64_t cap[PIC_MAX_SPECIES];
    bool loaded[PIC_MAX_SPECIES];
    // memory
    char *base;
    size_t bytes;
    bool owns;
    void *bufA[PIC_MAX_SPECIES][7];   // current store: pos[3], mom[3], cell
    void *bufB[PIC_MAX_SPECIES][7];   // sort target
    int64_t *tile_start[PIC_MAX_SPECIES];
    double *wc[PIC_MAX_SPECIES];      // FP64 2D weight cache (see SpeciesDev::wc)
    bool wc_valid[PIC_MAX_SPECIES];   // the cache holds the weights of the current store
    SortScratch sc;
    char *staging;
    size_t staging_bytes;
    double *diag_out;
    double *rho;
    // charge-conservation diagnostics: rho of the previous pic_diag (continuity residual) and
    // the Gauss residual recorded by the first step after a load or field set (drift)
    double *rho_prev;
    double *gref;
    bool rho_prev_valid;
    int64_t rho_prev_step;
    bool gref_valid;
    unsigned long long *jlo;  // FP64 deterministic run: low fixed-point words of J (3 ncell)
    int32_t *err;
    size_t smem;
    // timing of the particle pass: a ring of event pairs, drained when it fills
    cudaEvent_t ev0[64], ev1[64];
    bool have_events;
    // host loads: copies of the next chunk (copy_stream) overlap the packing of the previous
    // one (stream), the two halves of the staging buffer alternating
    cudaStream_t copy_stream;
    cudaEvent_t ev_ready, ev_copied[2], ev_packed[2];
    bool have_copy;
    int ev_pending;
    double gpp_ms;
    int64_t gpp_launches;
    int64_t kernel_launches;   // every kernel this context has launched
};

namespace {

// particles per host<->device staging chunk (load and read-back)
constexpr int64_t kChunk = (int64_t)1 << 22;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t staging_size(const RunDev &rd, int64_t capmax)
{
    const int64_t m = std::min<int64_t>(std::max<int64_t>(capmax, 1), kChunk);
    return align_up((size_t)m * ((rd.dim + 3) * sizeof(double) + sizeof(int64_t)) + 4 * 256, 256);
}

int pos_bytes(const pic_ctx *c) { return c->rd.prec == PIC_FP32_MIXED ? 4 : 8; }

// FP64 2D, l <= 3: 2 (l + 1) cached B-spline weights per particle of capacity (SpeciesDev::wc)
size_t weight_cache_bytes(const pic_ctx *c, int s)
{
    if (c->rd.prec != PIC_FP64 || c->rd.dim != 2 || c->rd.l > 3) return 0;
    return (size_t)c->cap[s] * 2 * (c->rd.l + 1) * sizeof(double);
}

int particle_bytes(const pic_ctx *c)
{
    const int d = c->rd.dim;
    return c->rd.prec == PIC_FP32_MIXED ? 4 + 4 * d + 12 : 8 * d + 24;
}

// Node offsets (relative to a particle's cell) that the stencils of one axis can touch.
void axis_reach(int l, const TTable &tt, int kt, int *lo, int *hi)
{
    const double eps = 1e-9;
    auto fl = [](double v) { return (int)std::floor(v); };
    const double hl = 0.5 * l;
    const int wh_lo = fl(-hl), wh_hi = fl(1.0 - eps - hl) + l;
    const double R = tt.Rint + tt.Rfrac;
    const int t_lo = fl(-R) + 1, t_hi = fl(1.0 - eps - R) + 1 + kt - 1;
    const double h0 = 0.5 * (l - 1);
    const int d_lo = fl(-h0) - 1, d_hi = fl(1.0 - eps - h0) + l + 1;
    *lo = -std::min(wh_lo, std::min(t_lo, d_lo));
    *hi = std::max(wh_hi, std::max(t_hi, d_hi));
}

void refresh_species_ptrs(pic_ctx *c)
{
    for (int s = 0; s < c->rd.nsp; ++s) {
        SpeciesDev &sp = c->rd.sp[s];
        for (int a = 0; a < 3; ++a) {
            sp.pos[a] = c->bufA[s][a];
            sp.mom[a] = c->bufA[s][3 + a];
        }
        sp.cell = (int32_t *)c->bufA[s][6];
        sp.tile_start = c->tile_start[s];
        for (int a = 0; a < 3; ++a) {
            sp.pos_alt[a] = c->bufB[s][a];
            sp.mom_alt[a] = c->bufB[s][3 + a];
        }
        sp.cell_alt = (int32_t *)c->bufB[s][6];
        sp.wc = c->wc[s];
        sp.wc_stride = c->cap[s];
        sp.wc_mode = c->wc[s] ? (c->wc_valid[s] ? 2 : 1) : 0;
    }
    c->rd.sc = c->sc;
}

int latched_status(pic_ctx *c)
{
    int32_t e = 0;
    if (cudaMemcpyAsync(&e, c->err, sizeof(e), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return PIC_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    if (e & PIC_ERR_NONFINITE) return PIC_ENAN;
    if (e & PIC_ERR_OUTSIDE_TILE) return PIC_EOVERFLOW;
    if (e & PIC_ERR_TIMEOUT) return PIC_ETIMEOUT;
    return PIC_OK;
}

int sort_species(pic_ctx *c, int s)
{
    RunDev rd = c->rd;
    refresh_species_ptrs(c);
    rd = c->rd;
    cudaError_t e = launch_sort(rd, s, c->tile_start[s], c->bufB[s], c->bufB[s] + 3,
                                (int32_t *)c->bufB[s][6], c->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    c->kernel_launches += rd.sp[s].n > 0 ? 6 : 3;
    for (int i = 0; i < 7; ++i) std::swap(c->bufA[s][i], c->bufB[s][i]);
    c->wc_valid[s] = false;  // the weight cache follows the old order
    refresh_species_ptrs(c);
    return PIC_OK;
}

// Add the elapsed time of the pending event pairs to gpp_ms (waits for the last one).
void drain_events(pic_ctx *c)
{
    if (!c->have_events || c->ev_pending == 0) return;
    if (cudaEventSynchronize(c->ev1[c->ev_pending - 1]) == cudaSuccess) {
        for (int i = 0; i < c->ev_pending; ++i) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, c->ev0[i], c->ev1[i]) == cudaSuccess) c->gpp_ms += ms;
        }
    }
    c->ev_pending = 0;
}

int sort_all(pic_ctx *c)
{
    for (int s = 0; s < c->rd.nsp; ++s) {
        const int r = sort_species(c, s);
        if (r != PIC_OK) return r;
    }
    c->age = 0;
    return PIC_OK;
}

// Species constants of a load (charge, mass, weight and the derived per-step factors).
void set_species(pic_ctx *c, int species, double q, double m, double w, int64_t n)
{
    // the particles change: the charge-conservation references no longer apply
    c->gref_valid = false;
    c->rho_prev_valid = false;
    SpeciesDev &sp = c->rd.sp[species];
    const RunDev &rd = c->rd;
    const double vc = rd.dx[0] * rd.dx[1] * (rd.dim == 3 ? rd.dx[2] : 1.0);
    sp.q = q;
    sp.m = m;
    sp.w = w;
    sp.qmdt_half = 0.5 * q * rd.dt / m;
    for (int a = 0; a < 3; ++a) sp.kx[a] = -q * w * rd.dx[a] / (vc * rd.dt);
    sp.kz = q * w / vc;
    sp.n = n;
    refresh_species_ptrs(c);
}

// After the particle store of a species is written: tile-sort it and mark it loaded.
int finish_load(pic_ctx *c, int species)
{
    // the loaded species is sorted now; the shared sort age keeps counting the steps since the
    // other species were sorted (resetting it could let them drift past the staged halo
    // before the next automatic sort)
    const int r = sort_species(c, species);
    if (r != PIC_OK) return r;
    c->loaded[species] = true;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    return PIC_OK;
}

uint64_t sm64_mix_host(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Key of the SplitMix64 stream named by (seed, ids...), the schedule documented in pic.h.
uint64_t stream_key(uint64_t seed, uint64_t a, uint64_t b, uint64_t d)
{
    const uint64_t G = 0x9E3779B97F4A7C15ull;
    uint64_t k = sm64_mix_host(seed + G);
    k = sm64_mix_host(k ^ ((a + 1) * G));
    k = sm64_mix_host(k ^ ((b + 1) * G));
    k = sm64_mix_host(k ^ ((d + 1) * G));
    return k;
}

// Fixed-point scale of a deterministic run: s = the largest bound of one particle's
// contribution to one node over the species, |q w dx_a / (V_c dt)| for J_a (the Esirkepov
// prefix sums and form factors are at most 1 in magnitude) and |q w / V_c| for the
// out-of-plane current (|v| < 1).
void set_det_scale(pic_ctx *c)
{
    RunDev &rd = c->rd;
    double sc = 0.0;
    for (int s = 0; s < rd.nsp; ++s) {
        const SpeciesDev &sp = rd.sp[s];
        for (int a = 0; a < 3; ++a) sc = std::max(sc, std::fabs(sp.kx[a]));
        sc = std::max(sc, std::fabs(sp.kz));
    }
    if (!(sc > 0.0) || !std::isfinite(sc)) sc = 1.0;
    rd.det_scale = sc;
    rd.det_inv32 = (float)(std::ldexp(1.0, 40) / sc);
    rd.det_inv64 = std::ldexp(1.0, 31) / sc;
}

// Record G = D.E - rho of the current state as the reference of the Gauss-residual drift.
int capture_gauss_ref(pic_ctx *c)
{
    if (c->gref_valid) return PIC_OK;
    refresh_species_ptrs(c);
    if (launch_gauss_ref(c->rd, c->rho, c->gref, c->diag_out, c->stream) != cudaSuccess)
        return PIC_ECUDA;
    c->kernel_launches += 2;
    for (int s = 0; s < c->rd.nsp; ++s) c->kernel_launches += c->rd.sp[s].n > 0 ? 1 : 0;
    c->gref_valid = true;
    return PIC_OK;
}

int load_common(pic_ctx *c, int species, double q, double m, double w, int64_t n,
                const double *x, const double *u, bool on_device)
{
    if (!c || !c->base) return c ? PIC_ESTATE : PIC_EINVAL;
    if (species < 0 || species >= c->rd.nsp || n < 0 || n > c->cap[species]) return PIC_EINVAL;
    if (!(m > 0.0) || !(w >= 0.0) || (n > 0 && (!x || !u))) return PIC_EINVAL;
    set_species(c, species, q, m, w, n);
    const int d = c->rd.dim;
    // page-locked host arrays the device can address (cudaHostAlloc / cudaHostRegister) are read
    // by the packing kernel in place, over the host link, without the staging copies
    const double *xd = nullptr, *ud = nullptr;
    if (!on_device && n > 0) {
        cudaPointerAttributes ax, au;
        int dev = -1;
        // the device pointers are this device's (memory pinned through another device's
        // context takes the staging path)
        if (cudaGetDevice(&dev) == cudaSuccess
            && cudaPointerGetAttributes(&ax, x) == cudaSuccess && ax.type == cudaMemoryTypeHost
            && ax.devicePointer && ax.device == dev
            && cudaPointerGetAttributes(&au, u) == cudaSuccess
            && au.type == cudaMemoryTypeHost && au.devicePointer && au.device == dev) {
            xd = (const double *)ax.devicePointer;
            ud = (const double *)au.devicePointer;
        }
        cudaGetLastError();  // a pageable pointer is not an error here
    }
    if (on_device || xd) {
        if (launch_pack(c->rd, species, on_device ? x : xd, n, on_device ? u : ud, n, n, 0,
                        c->stream) != cudaSuccess)
            return PIC_ECUDA;
        if (n > 0) c->kernel_launches += 1;
    } else if (n > 0) {
        // host arrays go through the two halves of the staging buffer in turn: the copies of
        // chunk k (copy_stream) overlap the packing of chunk k - 1 (stream)
        if (!c->have_copy) {
            bool ok = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
            const unsigned fl = cudaEventDisableTiming;
            ok = ok && cudaEventCreateWithFlags(&c->ev_ready, fl) == cudaSuccess;
            for (int b = 0; b < 2; ++b)
                ok = ok && cudaEventCreateWithFlags(&c->ev_copied[b], fl) == cudaSuccess
                     && cudaEventCreateWithFlags(&c->ev_packed[b], fl) == cudaSuccess;
            if (!ok) return PIC_ECUDA;
            c->have_copy = true;
        }
        const int64_t ch = std::min<int64_t>(kChunk / 2, (int64_t)(c->staging_bytes / (2 * (d + 3) * sizeof(double))));
        if (ch < 1) return PIC_ENOMEM;
        // the staging buffer may still be in use by earlier work on the context's stream
        if (cudaEventRecord(c->ev_ready, c->stream) != cudaSuccess
            || cudaStreamWaitEvent(c->copy_stream, c->ev_ready, 0) != cudaSuccess)
            return PIC_ECUDA;
        int k = 0;
        for (int64_t p0 = 0; p0 < n; p0 += ch, ++k) {
            const int b = k & 1;
            const int64_t mc = std::min(ch, n - p0);
            double *sx = (double *)c->staging + (size_t)b * (d + 3) * ch;
            double *su = sx + (size_t)d * mc;
            if (k >= 2 && cudaStreamWaitEvent(c->copy_stream, c->ev_packed[b], 0) != cudaSuccess)
                return PIC_ECUDA;
            for (int a = 0; a < d; ++a)
                if (cudaMemcpyAsync(sx + (size_t)a * mc, x + (size_t)a * n + p0, mc * sizeof(double),
                                    cudaMemcpyHostToDevice, c->copy_stream) != cudaSuccess)
                    return PIC_ECUDA;
            for (int a = 0; a < 3; ++a)
                if (cudaMemcpyAsync(su + (size_t)a * mc, u + (size_t)a * n + p0, mc * sizeof(double),
                                    cudaMemcpyHostToDevice, c->copy_stream) != cudaSuccess)
                    return PIC_ECUDA;
            if (cudaEventRecord(c->ev_copied[b], c->copy_stream) != cudaSuccess
                || cudaStreamWaitEvent(c->stream, c->ev_copied[b], 0) != cudaSuccess)
                return PIC_ECUDA;
            if (launch_pack(c->rd, species, sx, mc, su, mc, mc, p0, c->stream) != cudaSuccess) return PIC_ECUDA;
            if (cudaEventRecord(c->ev_packed[b], c->stream) != cudaSuccess) return PIC_ECUDA;
            c->kernel_launches += 1;
        }
    }
    return finish_load(c, species);
}

}  // namespace

extern "C" {

const char *pic_strerror(int s)
{
    switch (s) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument";
    case PIC_ENOMEM: return "not enough device memory bound";
    case PIC_ECFL: return "time step violates the Courant limit or the one-cell-per-step bound";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_EOVERFLOW: return "a particle left the staged region of its tile";
    case PIC_ETIMEOUT: return "a bounded device wait gave up";
    case PIC_ENAN: return "non-finite value in fields or particles";
    case PIC_ESTATE: return "call out of order (no device memory bound)";
    default: return "unknown status";
    }
}

int pic_create(const int32_t grid[3], const double dx[3], double dt, int spline_order, int scheme,
               const pic_options *opt, pic_ctx **out)
{
    if (!grid || !dx || !out) return PIC_EINVAL;
    *out = nullptr;
    if (spline_order < 1 || spline_order > 4) return PIC_EINVAL;
    if (scheme != PIC_SCHEME_MC && scheme != PIC_SCHEME_WT) return PIC_EINVAL;
    if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1) return PIC_EINVAL;
    const int dim = grid[2] > 1 ? 3 : 2;
    const int64_t ncell = (int64_t)grid[0] * grid[1] * grid[2];
    if (ncell > (int64_t)1 << 30) return PIC_EINVAL;
    for (int a = 0; a < dim; ++a)
        if (!(dx[a] > 0.0) || !std::isfinite(dx[a])) return PIC_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return PIC_EINVAL;
    for (int a = 0; a < dim; ++a)
        if (dt / dx[a] >= 1.0) return PIC_ECFL;  // the one-cell-per-step bound of the move
    pic_options o;
    std::memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.solver != PIC_SOLVER_YEE && o.solver != PIC_SOLVER_M4) return PIC_EINVAL;
    // Courant limit of App. C: (c dt)^2 sum_i A_i sin^2(k_i dx_i/2)/dx_i^2 < 1 for every k; the
    // maximum over k sits at a corner of the Brillouin zone (each k_i dx_i in {0, pi}).
    {
        double worst = 0.0;
        for (int mask = 1; mask < (1 << dim); ++mask) {
            double sum = 0.0;
            for (int a = 0; a < dim; ++a) {
                if (!(mask >> a & 1)) continue;
                double A = 1.0;
                if (o.solver == PIC_SOLVER_M4) {
                    for (int b = 0; b < dim; ++b) {
                        const double r = dt / dx[b];
                        const double coef = (b == a) ? (r * r - 1.0) / 12.0 : r * r / 12.0;
                        if (mask >> b & 1) A -= 4.0 * coef;  // 1 - cos(pi) = 2
                    }
                }
                sum += A / (dx[a] * dx[a]);
            }
            worst = std::max(worst, dt * dt * sum);
        }
        if (!(worst < 1.0)) return PIC_ECFL;
    }
    if (o.n_species <= 0) o.n_species = 2;
    if (o.n_species > PIC_MAX_SPECIES) return PIC_EINVAL;
    if (o.precision != PIC_FP64 && o.precision != PIC_FP32_MIXED) return PIC_EINVAL;
    if (o.deterministic != 0 && o.deterministic != 1) return PIC_EINVAL;

    pic_ctx *c = new (std::nothrow) pic_ctx;
    if (!c) return PIC_ENOMEM;
    std::memset(c, 0, sizeof(*c));
    RunDev &rd = c->rd;
    rd.dim = dim;
    rd.l = spline_order;
    rd.scheme = scheme;
    rd.prec = o.precision;
    rd.ncell = ncell;
    rd.det = o.deterministic;
    for (int a = 0; a < 3; ++a) {
        rd.n[a] = grid[a];
        rd.dx[a] = (a < dim) ? dx[a] : 1.0;
        rd.dtt[a] = (a < dim) ? dt / rd.dx[a] : 0.0;
    }
    rd.dt = dt;
    rd.m4 = o.solver == PIC_SOLVER_M4 ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            const double r = (b < dim) ? dt / rd.dx[b] : 0.0;
            rd.beta[a][b] = (rd.m4 && a != b && a < dim && b < dim) ? r * r / 12.0 : 0.0;
        }
        const double r = (a < dim) ? dt / rd.dx[a] : 0.0;
        rd.delta[a] = (rd.m4 && a < dim) ? (r * r - 1.0) / 12.0 : 0.0;
    }
    for (int a = 0; a < 3; ++a) rd.idx[a] = 1.0 / rd.dx[a];
    rd.div_n0 = make_fastdiv(rd.n[0]);
    rd.div_n01 = make_fastdiv(rd.n[0] * rd.n[1]);
    // tiles
    // default tiles (measured on the 2048x1024 cubic workload: the FP32 form is 2% faster with
    // 64x8 than with 32x8, the FP64 form the same with both); a deterministic FP32 run keeps
    // 64-bit words in its shared current tile and takes 32x8 so that two CTAs share an SM.  3D
    // (256x64x64 quadratic pair plasma, 8 per cell, ms per step): the FP32 form 1.95 with 16x4x2
    // against 2.15 with 8x4x4 (a warp's 32 cells span 16 nodes of two rows, fewer L2 sectors per
    // reduction of its deposit), the FP64 form 13.1 with either
    const bool f32 = rd.prec == PIC_FP32_MIXED && !rd.det;
    const int deft[2][3] = {{f32 ? 64 : 32, 8, 1}, {f32 ? 16 : 8, 4, f32 ? 2 : 4}};
    for (int a = 0; a < 3; ++a) {
        int t = o.tile[a] > 0 ? o.tile[a] : deft[dim - 2][a];
        if (a >= dim) t = 1;
        t = std::min(t, rd.n[a]);
        rd.tile[a] = t;
        rd.ntile[a] = (rd.n[a] + t - 1) / t;
    }
    if ((int64_t)rd.tile[0] * rd.tile[1] * rd.tile[2] > 1024) { delete c; return PIC_EINVAL; }
    rd.ntiles = (int64_t)rd.ntile[0] * rd.ntile[1] * rd.ntile[2];
    // interpolation tables
    c->kt = 0;
    for (int a = 0; a < 3; ++a) {
        if (a >= dim) { build_ttable(spline_order, PIC_SCHEME_MC, 0.5, &rd.tt[a]); continue; }
        if (!build_ttable(spline_order, scheme, rd.dtt[a], &rd.tt[a])) { delete c; return PIC_ECFL; }
        c->kt = std::max(c->kt, rd.tt[a].K);
    }
    // sort interval and staged region
    double dmax = 0.0;
    for (int a = 0; a < dim; ++a) dmax = std::max(dmax, rd.dtt[a]);
    // default sort interval: particles stay within the staged halo until the next sort --
    // 2 cells in 2D, 1 cell in the FP32 3D form (whose tile stage would not fit in shared memory
    // with more), and 8 steps for the FP64 3D form, which reads its fields through L1
    int K = o.sort_interval;
    if (K <= 0) {
        if (dim == 2) K = (int)std::floor(2.0 / dmax) + 1;
        else if (o.precision == PIC_FP32_MIXED) K = (int)std::floor(1.0 / dmax) + 1;
        else K = 8;
    }
    c->sort_interval = std::max(1, K);
    int64_t nodes = 1;
    for (int a = 0; a < 3; ++a) {
        if (a >= dim) { rd.pre[a] = 0; rd.post[a] = 0; rd.reg[a] = 1; rd.drift[a] = 0; continue; }
        int lo, hi;
        // the halo covers the wide integer-node stencil (l + 2 nodes) so that the run can
        // also be advanced by the batched kernel, which uses that stencil for every run
        axis_reach(spline_order, rd.tt[a], std::max(c->kt, spline_order + 2), &lo, &hi);
        const int D = (int)std::ceil((c->sort_interval - 1) * rd.dtt[a] - 1e-12);
        rd.drift[a] = std::max(D, 0);
        rd.pre[a] = rd.drift[a] + lo;
        rd.post[a] = rd.drift[a] + hi;
        rd.reg[a] = rd.tile[a] + rd.pre[a] + rd.post[a];
        // an even row stride keeps every even node of a staged row 8-byte aligned (the FP32
        // deposit adds neighbouring x nodes in pairs)
        if (a == 0 && (rd.reg[0] & 1)) { rd.post[0] += 1; rd.reg[0] += 1; }
        nodes *= rd.reg[a];
    }
    rd.reg_nodes = nodes;
    // padded FP32 current of the 3D FP32 form: the Esirkepov window of a particle in cell c
    // spans nodes c - jp_lo .. c + l + 1 - (l - 1) / 2 along every axis
    rd.jp_lo = 0;
    for (int a = 0; a < 3; ++a) rd.jp[a] = rd.n[a];
    if (dim == 3 && rd.prec == PIC_FP32_MIXED && !rd.det) {
        const int lo = (spline_order - 1) / 2 + 1 + (spline_order % 2 == 0 ? 1 : 0);
        const int hi = spline_order + 1 - (spline_order - 1) / 2;
        rd.jp_lo = lo;
        for (int a = 0; a < 3; ++a) rd.jp[a] = rd.n[a] + lo + hi;
        // x rows of a multiple of 4 nodes with at least 3 spare ones: a window row is added as
        // aligned node pairs from the even node at or below its first node (4-wide groups,
        // which this padding would also allow, measured 1% slower)
        rd.jp[0] = (rd.jp[0] + 3 + 3) / 4 * 4;
    }
    rd.jp_nodes = (int64_t)rd.jp[0] * rd.jp[1] * rd.jp[2];
    // Tile order.  The FP32 form sums the currents of a warp's lanes through shared memory when
    // their windows lie in a few neighbouring cells of a row: cell-major order gives that, and
    // measured on a GB300 (512x256 pair plasma, FP32 particle kernel, ns per particle, cell-major
    // vs slot-major) it is the faster one from 4 particles of a species per cell up for odd l,
    // whose lanes of one row share their y window (cubic: 4 per species 0.102 vs 0.135, 8 per
    // species 0.075 vs 0.123), and from 6 up for even l (quadratic: 4 per species 0.132 vs
    // 0.096, 6 per species 0.092 vs 0.090, 8 per species 0.083 vs 0.086); below that (and in
    // the FP64 form, which deposits per lane) the slot-major order puts the lanes of a warp in
    // different cells for per-lane shared atomics.  3D (FP32 current by paired L2 reductions,
    // no warp frame): cell-major from 4 per species for every l (256x64x64, quadratic, 4 per
    // species, ms per step: 1.54 cell-major against 1.61 slot-major with 16x4x2 tiles).
    {
        int64_t capmax = 0;
        for (int s = 0; s < o.n_species; ++s) capmax = std::max(capmax, (int64_t)o.capacity[s]);
        const int64_t per_cell_min = (dim == 3 || (spline_order & 1)) ? 4 : 6;
        const bool dense = rd.ncell > 0 && capmax >= per_cell_min * rd.ncell;
        if (o.tile_order < PIC_ORDER_AUTO || o.tile_order > PIC_ORDER_SLOT) { delete c; return PIC_EINVAL; }
        const bool cell = o.tile_order == PIC_ORDER_AUTO ? dense : o.tile_order == PIC_ORDER_CELL;
        rd.slot_major = (rd.prec == PIC_FP32_MIXED && cell) ? 0 : 1;
    }
    rd.nsp = o.n_species;
    for (int s = 0; s < o.n_species; ++s) {
        if (o.capacity[s] < 0 || o.capacity[s] >= ((int64_t)1 << 31)) { delete c; return PIC_EINVAL; }
        c->cap[s] = o.capacity[s];
    }
    c->stream = (cudaStream_t)(uintptr_t)o.stream;
    c->smem = 0;
    if (dim == 2 || rd.prec == PIC_FP32_MIXED) {
        c->smem = rd.prec == PIC_FP32_MIXED ? gpp_smem_bytes_f32(rd) : gpp_smem_bytes_f64(rd);
        if (c->smem > 227 * 1024) { delete c; return PIC_EINVAL; }
    }
    *out = c;
    return PIC_OK;
}

// The 3D FP32 form (not deterministic) sums its current in an FP32 buffer (RunDev::J32).
static bool uses_j32(const RunDev &rd)
{
    return rd.dim == 3 && rd.prec == PIC_FP32_MIXED && !rd.det;
}

int pic_footprint(const pic_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return PIC_EINVAL;
    const RunDev &rd = c->rd;
    const size_t A = 256;
    size_t b = 0;
    b += 9 * align_up(rd.ncell * sizeof(double), A);                           // F
    if (rd.prec == PIC_FP32_MIXED) b += 6 * align_up(rd.ncell * sizeof(float), A);  // Fs
    const int pb = particle_bytes(c);
    int64_t capmax = 0, captot = 0;
    for (int s = 0; s < rd.nsp; ++s) {
        capmax = std::max(capmax, c->cap[s]);
        captot += c->cap[s];
    }
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    for (int s = 0; s < rd.nsp; ++s) b += align_up((size_t)c->cap[s] * pb + 7 * A, A);  // current stores
    for (int s = 0; s < rd.nsp; ++s) b += align_up((rd.ntiles + 1) * sizeof(int64_t), A);           // tile_start
    for (int s = 0; s < rd.nsp; ++s) b += align_up(weight_cache_bytes(c, s), A);                  // wc
    // sort targets and sort scratch
    for (int s = 0; s < rd.nsp; ++s) b += align_up((size_t)c->cap[s] * pb + 7 * A, A);
    b += 2 * align_up(rd.ntiles * TC * sizeof(int32_t), A);
    b += 4 * align_up((size_t)capmax * sizeof(int32_t), A);
    b += align_up((rd.ntiles + 1) * sizeof(int64_t), A);
    b += staging_size(rd, capmax);                // host<->device staging (chunked)
    b += 3 * align_up(rd.ncell * sizeof(double), A);  // rho, rho_prev, gref
    if (rd.det && rd.prec == PIC_FP64) b += 3 * align_up(rd.ncell * sizeof(double), A);  // jlo
    if (uses_j32(rd)) b += align_up(3 * rd.jp_nodes * sizeof(float), A);                // J32
    b += 2 * A;                                   // diag out, err
    b += A;                                       // base alignment slack
    (void)captot;
    *bytes = b;
    return PIC_OK;
}

int pic_bind_memory(pic_ctx *c, void *dev, size_t bytes)
{
    if (!c || !dev) return PIC_EINVAL;
    size_t need = 0;
    pic_footprint(c, &need);
    if (bytes < need) return PIC_ENOMEM;
    RunDev &rd = c->rd;
    const size_t A = 256;
    char *p = (char *)align_up((size_t)dev, A);
    auto take = [&](size_t n) { char *r = p; p += align_up(n, A); return r; };
    c->base = (char *)dev;
    c->bytes = bytes;
    for (int f = 0; f < 9; ++f) rd.F[f] = (double *)take(rd.ncell * sizeof(double));
    for (int f = 0; f < 6; ++f) rd.Fs[f] = rd.prec == PIC_FP32_MIXED ? (float *)take(rd.ncell * sizeof(float)) : nullptr;
    const int pbs = pos_bytes(c);
    auto carve_store = [&](void **buf, int64_t cap, char *&q) {
        auto t2 = [&](size_t n) { char *r = q; q += align_up(n, A); return r; };
        for (int a = 0; a < 3; ++a) buf[a] = (a < rd.dim) ? t2((size_t)cap * pbs) : nullptr;
        for (int a = 0; a < 3; ++a) buf[3 + a] = t2((size_t)cap * pbs);
        buf[6] = rd.prec == PIC_FP32_MIXED ? t2((size_t)cap * sizeof(int32_t)) : nullptr;
    };
    const int pb = particle_bytes(c);
    for (int s = 0; s < rd.nsp; ++s) {
        char *q = p;
        carve_store(c->bufA[s], c->cap[s], q);
        take((size_t)c->cap[s] * pb + 7 * A);
    }
    for (int s = 0; s < rd.nsp; ++s) c->tile_start[s] = (int64_t *)take((rd.ntiles + 1) * sizeof(int64_t));
    for (int s = 0; s < rd.nsp; ++s) {
        const size_t wb = weight_cache_bytes(c, s);
        c->wc[s] = wb ? (double *)take(wb) : nullptr;
        c->wc_valid[s] = false;
    }
    int64_t capmax = 0;
    for (int s = 0; s < rd.nsp; ++s) capmax = std::max(capmax, c->cap[s]);
    const int TC = rd.tile[0] * rd.tile[1] * rd.tile[2];
    for (int s = 0; s < rd.nsp; ++s) {
        char *q = p;
        carve_store(c->bufB[s], c->cap[s], q);
        take((size_t)c->cap[s] * pb + 7 * A);
    }
    c->sc.cnt = (int32_t *)take(rd.ntiles * TC * sizeof(int32_t));
    c->sc.cell_first = (int32_t *)take(rd.ntiles * TC * sizeof(int32_t));
    c->sc.slot = (int32_t *)take((size_t)capmax * sizeof(int32_t));
    c->sc.key = (int32_t *)take((size_t)capmax * sizeof(int32_t));
    c->sc.idx = (int32_t *)take((size_t)capmax * sizeof(int32_t));
    c->sc.pos = (int32_t *)take((size_t)capmax * sizeof(int32_t));
    c->sc.tile_count = (int64_t *)take((rd.ntiles + 1) * sizeof(int64_t));
    c->staging_bytes = staging_size(rd, capmax);
    c->staging = take(c->staging_bytes);
    c->rho = (double *)take(rd.ncell * sizeof(double));
    c->rho_prev = (double *)take(rd.ncell * sizeof(double));
    c->gref = (double *)take(rd.ncell * sizeof(double));
    c->jlo = nullptr;
    for (int a = 0; a < 3; ++a) rd.Jlo[a] = nullptr;
    if (rd.det && rd.prec == PIC_FP64) {
        c->jlo = (unsigned long long *)take(3 * rd.ncell * sizeof(double));
        for (int a = 0; a < 3; ++a) rd.Jlo[a] = c->jlo + a * rd.ncell;
    }
    for (int a = 0; a < 3; ++a) rd.J32[a] = nullptr;
    if (uses_j32(rd)) {
        float *j = (float *)take(3 * rd.jp_nodes * sizeof(float));
        for (int a = 0; a < 3; ++a) rd.J32[a] = j + a * rd.jp_nodes;
    }
    c->rho_prev_valid = false;
    c->gref_valid = false;
    c->diag_out = (double *)take(8 * sizeof(double));
    c->err = (int32_t *)take(sizeof(int32_t));
    rd.err = c->err;
    if ((size_t)(p - (char *)dev) > bytes) return PIC_ENOMEM;
    for (int s = 0; s < rd.nsp; ++s) {
        rd.sp[s].n = 0;
        rd.sp[s].m = 1.0;
    }
    refresh_species_ptrs(c);
    cudaError_t e = cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream);
    for (int f = 0; f < 9 && e == cudaSuccess; ++f)
        e = cudaMemsetAsync(rd.F[f], 0, rd.ncell * sizeof(double), c->stream);
    for (int f = 0; f < 6 && e == cudaSuccess && rd.Fs[f]; ++f)
        e = cudaMemsetAsync(rd.Fs[f], 0, rd.ncell * sizeof(float), c->stream);
    for (int s = 0; s < rd.nsp && e == cudaSuccess; ++s)
        e = cudaMemsetAsync(c->tile_start[s], 0, (rd.ntiles + 1) * sizeof(int64_t), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    if (!c->have_events) {
        bool ok = true;
        for (int i = 0; i < 64; ++i)
            ok = ok && cudaEventCreate(&c->ev0[i]) == cudaSuccess && cudaEventCreate(&c->ev1[i]) == cudaSuccess;
        c->have_events = ok;
    }
    return PIC_OK;
}

int pic_alloc(pic_ctx *c)
{
    if (!c) return PIC_EINVAL;
    size_t need = 0;
    pic_footprint(c, &need);
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) return PIC_ENOMEM;
    const int r = pic_bind_memory(c, p, need);
    if (r != PIC_OK) { cudaFree(p); return r; }
    c->owns = true;
    return PIC_OK;
}

int pic_load_particles(pic_ctx *c, int species, double q, double m, double w, int64_t n,
                       const double *x, const double *u)
{
    return load_common(c, species, q, m, w, n, x, u, false);
}

int pic_load_particles_device(pic_ctx *c, int species, double q, double m, double w, int64_t n,
                              const double *x, const double *u)
{
    return load_common(c, species, q, m, w, n, x, u, true);
}

// Both drifting-plasma loaders: theta > 0 draws the co-moving momenta from the Juttner-Synge
// distribution (Sobol's method), else from N(0, u_th^2) per component.
static int load_drifting(pic_ctx *c, int species, double q, double m, double w, int64_t per_cell,
                         double gamma, double u_th, double theta, uint64_t seed, uint64_t run,
                         int pos_species)
{
    if (!c || !c->base) return c ? PIC_ESTATE : PIC_EINVAL;
    if (species < 0 || species >= c->rd.nsp || pos_species < 0 || per_cell < 0) return PIC_EINVAL;
    if (!(m > 0.0) || !(w >= 0.0) || !(gamma >= 1.0) || !(u_th >= 0.0) || !std::isfinite(gamma)
        || !std::isfinite(u_th) || !(theta >= 0.0) || !std::isfinite(theta))
        return PIC_EINVAL;
    if (per_cell > 0 && c->rd.ncell > c->cap[species] / per_cell) return PIC_EINVAL;
    const int64_t n = c->rd.ncell * per_cell;
    set_species(c, species, q, m, w, n);
    LoadKeys k;
    for (int a = 0; a < 3; ++a) {
        k.pos[a] = stream_key(seed, run, (uint64_t)pos_species, 10 + a);
        k.mom[2 * a] = stream_key(seed, run, (uint64_t)species, 20 + 2 * a);
        k.mom[2 * a + 1] = stream_key(seed, run, (uint64_t)species, 21 + 2 * a);
    }
    k.flip = stream_key(seed, run, (uint64_t)species, 30);
    for (int j = 0; j < 4; ++j) k.jut[j] = stream_key(seed, run, (uint64_t)species, 40 + j);
    k.dir[0] = stream_key(seed, run, (uint64_t)species, 44);
    k.dir[1] = stream_key(seed, run, (uint64_t)species, 45);
    if (launch_load_plasma(c->rd, species, k, per_cell, gamma, u_th, theta, n, c->stream)
        != cudaSuccess)
        return PIC_ECUDA;
    if (n > 0) c->kernel_launches += 1;
    const int r = finish_load(c, species);
    return r != PIC_OK ? r : latched_status(c);
}

int pic_load_drifting_plasma(pic_ctx *c, int species, double q, double m, double w,
                             int64_t per_cell, double gamma, double u_th, uint64_t seed,
                             uint64_t run, int pos_species)
{
    return load_drifting(c, species, q, m, w, per_cell, gamma, u_th, 0.0, seed, run, pos_species);
}

int pic_load_drifting_juttner(pic_ctx *c, int species, double q, double m, double w,
                              int64_t per_cell, double gamma, double theta, uint64_t seed,
                              uint64_t run, int pos_species)
{
    if (!(theta >= PIC_JUTTNER_MIN_THETA)) return PIC_EINVAL;
    return load_drifting(c, species, q, m, w, per_cell, gamma, 0.0, theta, seed, run, pos_species);
}

int pic_set_fields(pic_ctx *c, int comp, const double *host, size_t count)
{
    if (!c || !host || comp < 0 || comp > 5) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    if (count != (size_t)c->rd.ncell) return PIC_EINVAL;
    if (cudaMemcpyAsync(c->rd.F[comp], host, count * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
        return PIC_ECUDA;
    c->gref_valid = false;  // D.E changes: the drift is measured from the next step on
    if (c->rd.prec == PIC_FP32_MIXED) {
        if (launch_shadow(c->rd, c->stream) != cudaSuccess) return PIC_ECUDA;
        c->kernel_launches += 1;
    }
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_step(pic_ctx *c, int nsteps)
{
    if (!c || nsteps < 0) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    RunDev &rd = c->rd;
    const bool shadow = rd.prec == PIC_FP32_MIXED;
    drain_events(c);
    c->gpp_ms = 0.0;
    c->gpp_launches = 0;
    if (nsteps > 0) {
        const int r = capture_gauss_ref(c);
        if (r != PIC_OK) return r;
    }
    if (rd.det) set_det_scale(c);
    for (int it = 0; it < nsteps; ++it) {
        if (c->age >= c->sort_interval) {
            const int r = sort_all(c);
            if (r != PIC_OK) return r;
        }
        refresh_species_ptrs(c);
        if (rd.J32[0]) {  // F[6..8] are written whole from J32 after the particle pass
            if (cudaMemsetAsync(rd.J32[0], 0, 3 * rd.jp_nodes * sizeof(float), c->stream) != cudaSuccess)
                return PIC_ECUDA;
        } else {
            for (int a = 6; a < 9; ++a)
                if (cudaMemsetAsync(rd.F[a], 0, rd.ncell * sizeof(double), c->stream) != cudaSuccess)
                    return PIC_ECUDA;
        }
        if (c->jlo && cudaMemsetAsync(c->jlo, 0, 3 * rd.ncell * sizeof(double), c->stream) != cudaSuccess)
            return PIC_ECUDA;
        if (c->have_events) {
            if (c->ev_pending == 64) drain_events(c);
            cudaEventRecord(c->ev0[c->ev_pending], c->stream);
        }
        const cudaError_t e = rd.prec == PIC_FP32_MIXED ? launch_gpp_f32(rd, c->kt, c->stream)
                                                        : launch_gpp_f64(rd, c->kt, c->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
        if (c->have_events) cudaEventRecord(c->ev1[c->ev_pending++], c->stream);
        c->gpp_launches += 1;
        if (rd.det) {  // the fixed-point sums become the FP64 current
            if (launch_det_finish(rd, c->stream) != cudaSuccess) return PIC_ECUDA;
            c->kernel_launches += 1;
        } else if (rd.J32[0]) {  // the FP32 sums become the FP64 current
            if (launch_j32_finish(rd, c->stream) != cudaSuccess) return PIC_ECUDA;
            c->kernel_launches += 1;
        }
        for (int s = 0; s < rd.nsp; ++s) c->wc_valid[s] = c->wc[s] != nullptr;
        if (launch_yee_b(rd, 0.5 * rd.dt, false, c->stream) != cudaSuccess) return PIC_ECUDA;
        if (launch_yee_e(rd, shadow, c->stream) != cudaSuccess) return PIC_ECUDA;
        if (launch_yee_b(rd, 0.5 * rd.dt, shadow, c->stream) != cudaSuccess) return PIC_ECUDA;
        c->kernel_launches += 4;
        c->age += 1;
        c->step += 1;
    }
    return PIC_OK;
}

int pic_last_gpp_ms(pic_ctx *c, double *ms, int64_t *launches)
{
    if (!c || !ms) return PIC_EINVAL;
    drain_events(c);
    *ms = c->gpp_ms;
    if (launches) *launches = c->gpp_launches;
    return PIC_OK;
}

int pic_kernel_launches(const pic_ctx *c, int64_t *count)
{
    if (!c || !count) return PIC_EINVAL;
    *count = c->kernel_launches;
    return PIC_OK;
}

int pic_sort(pic_ctx *c)
{
    if (!c) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    return sort_all(c);
}

int pic_sync(pic_ctx *c)
{
    if (!c) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    return latched_status(c);
}

int pic_read_fields(pic_ctx *c, int comp, double *host, size_t count)
{
    if (!c || !host || comp < 0 || comp > 8) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    if (count != (size_t)c->rd.ncell) return PIC_EINVAL;
    if (cudaMemcpyAsync(host, c->rd.F[comp], count * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return PIC_ECUDA;
    return latched_status(c);
}

int pic_read_particles(pic_ctx *c, int species, double *x, double *u, int64_t *cell, int64_t n)
{
    if (!c || species < 0 || species >= c->rd.nsp) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    const RunDev &rd = c->rd;
    const int64_t np = rd.sp[species].n;
    if (n != np || (np > 0 && (!x || !u))) return PIC_EINVAL;
    if (np == 0) return latched_status(c);
    refresh_species_ptrs(c);
    const int d = rd.dim;
    for (int64_t p0 = 0; p0 < np; p0 += kChunk) {
        const int64_t m = std::min(kChunk, np - p0);
        double *sx = (double *)c->staging;
        double *su = sx + (size_t)d * m;
        int64_t *scell = (int64_t *)(su + (size_t)3 * m);
        if (launch_unpack(c->rd, species, sx, su, scell, m, p0, c->stream) != cudaSuccess) return PIC_ECUDA;
        c->kernel_launches += 1;
        for (int a = 0; a < d; ++a)
            if (cudaMemcpyAsync(x + (size_t)a * np + p0, sx + (size_t)a * m, m * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
                return PIC_ECUDA;
        for (int a = 0; a < 3; ++a)
            if (cudaMemcpyAsync(u + (size_t)a * np + p0, su + (size_t)a * m, m * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
                return PIC_ECUDA;
        if (cell && cudaMemcpyAsync(cell + p0, scell, m * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    c->stream) != cudaSuccess)
            return PIC_ECUDA;
        // the staging buffer is reused by the next chunk
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    }
    return latched_status(c);
}

int pic_read_tile_offsets(pic_ctx *c, int species, int64_t *offsets, int64_t count)
{
    if (!c || !offsets || species < 0 || species >= c->rd.nsp) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    if (count != c->rd.ntiles + 1) return PIC_EINVAL;
    if (cudaMemcpyAsync(offsets, c->tile_start[species], count * sizeof(int64_t),
                        cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return PIC_ECUDA;
    return latched_status(c);
}

int pic_tile_info(const pic_ctx *c, int32_t tile[3], int64_t *ntiles, int32_t *sort_interval,
                  int32_t *slot_major)
{
    if (c && slot_major) *slot_major = c->rd.slot_major;
    if (!c) return PIC_EINVAL;
    if (tile)
        for (int a = 0; a < 3; ++a) tile[a] = c->rd.tile[a];
    if (ntiles) *ntiles = c->rd.ntiles;
    if (sort_interval) *sort_interval = c->sort_interval;
    return PIC_OK;
}

int pic_smem_info(const pic_ctx *c, size_t *own_bytes, size_t *batched_bytes,
                  size_t *two_per_sm_bytes)
{
    if (!c) return PIC_EINVAL;
    if (own_bytes) *own_bytes = c->smem;
    if (batched_bytes)
        *batched_bytes = c->rd.prec == PIC_FP32_MIXED ? gpp_batch_smem_bytes_f32(c->rd) : 0;
    if (two_per_sm_bytes) {
        *two_per_sm_bytes = 0;
        int dev = 0, per_sm = 0, reserved = 0;
        if (cudaGetDevice(&dev) == cudaSuccess
            && cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)
                   == cudaSuccess
            && cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)
                   == cudaSuccess) {
            // two blocks of dynamic + static + reserved shared memory per SM; 64 bytes cover
            // the kernels' static shared variables
            const long v = (long)per_sm / 2 - reserved - 64;
            *two_per_sm_bytes = v > 0 ? (size_t)v : 0;
        } else {
            cudaGetLastError();  // no device: leave 0
        }
    }
    return PIC_OK;
}

int pic_diag(pic_ctx *c, pic_diag_t *out)
{
    if (!c || !out) return PIC_EINVAL;
    if (!c->base) return PIC_ESTATE;
    refresh_species_ptrs(c);
    const RunDev &rd = c->rd;
    const bool cont = c->rho_prev_valid && c->step == c->rho_prev_step + 1;
    if (launch_diag(rd, c->diag_out, c->rho, c->gref_valid ? c->gref : nullptr,
                    cont ? c->rho_prev : nullptr, c->stream) != cudaSuccess)
        return PIC_ECUDA;
    c->kernel_launches += 2 + 2 * rd.nsp;
    // this rho is the reference of the next call's continuity residual
    if (cudaMemcpyAsync(c->rho_prev, c->rho, rd.ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
        return PIC_ECUDA;
    c->rho_prev_valid = true;
    c->rho_prev_step = c->step;
    double h[6] = {0, 0, 0, 0, 0, 0};
    int32_t e = 0;
    if (cudaMemcpyAsync(h, c->diag_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return PIC_ECUDA;
    if (cudaMemcpyAsync(&e, c->err, sizeof(e), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return PIC_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
    const double vc = rd.dx[0] * rd.dx[1] * (rd.dim == 3 ? rd.dx[2] : 1.0);
    out->step = c->step;
    out->field_energy = 0.5 * h[0] * vc;
    out->kinetic_energy = h[1];
    double qt = 0.0;
    for (int s = 0; s < rd.nsp; ++s) qt += rd.sp[s].q * rd.sp[s].w * (double)rd.sp[s].n;
    out->total_charge = qt;
    out->max_gauss_residual = h[2];
    out->max_gauss_residual_drift = c->gref_valid ? h[3] : 0.0;
    out->max_continuity_residual = cont ? h[4] : std::nan("");
    out->error_flags = e;
    if (e & PIC_ERR_NONFINITE) return PIC_ENAN;
    if (e & PIC_ERR_OUTSIDE_TILE) return PIC_EOVERFLOW;
    return PIC_OK;
}

void pic_destroy(pic_ctx *c)
{
    if (!c) return;
    if (c->base) cudaStreamSynchronize(c->stream);
    if (c->have_events) {
        for (int i = 0; i < 64; ++i) {
            cudaEventDestroy(c->ev0[i]);
            cudaEventDestroy(c->ev1[i]);
        }
    }
    if (c->have_copy) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
        cudaEventDestroy(c->ev_ready);
        for (int b = 0; b < 2; ++b) {
            cudaEventDestroy(c->ev_copied[b]);
            cudaEventDestroy(c->ev_packed[b]);
        }
    }
    if (c->owns && c->base) cudaFree(c->base);
    delete c;
}

// Host evaluation of the per-axis integer-node weights that the kernels use (T_l for the WT
// scheme, W_l for MC): particle offset delta in [0,1) of its cell, dtt = c dt / dx.
// Fills w[0..*count-1] for nodes *base .. *base + *count - 1 relative to the cell.
int pic_axis_weights(int spline_order, int scheme, double dtt, double delta, double *w,
                     int *base, int *count)
{
    if (!w || !base || !count || !(delta >= 0.0 && delta < 1.0)) return PIC_EINVAL;
    TTable t;
    if (!build_ttable(spline_order, scheme, dtt, &t)) return PIC_EINVAL;
    *base = ttable_eval_host(&t, spline_order, delta, w);
    *count = t.K;
    return PIC_OK;
}

}  // extern "C"

namespace pic {

RunDev *ctx_rundev(pic_ctx *c)
{
    refresh_species_ptrs(c);
    return &c->rd;
}

void ctx_after_batch(pic_ctx *c, const RunDev &d, int age, int64_t steps)
{
    for (int s = 0; s < c->rd.nsp; ++s) {
        for (int a = 0; a < 3; ++a) {
            c->bufA[s][a] = d.sp[s].pos[a];
            c->bufB[s][a] = d.sp[s].pos_alt[a];
            c->bufA[s][3 + a] = d.sp[s].mom[a];
            c->bufB[s][3 + a] = d.sp[s].mom_alt[a];
        }
        c->bufA[s][6] = d.sp[s].cell;
        c->bufB[s][6] = d.sp[s].cell_alt;
        c->wc_valid[s] = false;
    }
    refresh_species_ptrs(c);
    c->age = age;
    c->step += steps;
}

int ctx_kt(const pic_ctx *c) { return c->kt; }
// before a batch takes the run over: record the Gauss-residual reference if a load or field
// set left it stale (the batch's steps do not), and wait for it
int ctx_prepare_batch(pic_ctx *c)
{
    const int r = capture_gauss_ref(c);
    if (r != PIC_OK) return r;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
int ctx_sort_interval(const pic_ctx *c) { return c->sort_interval; }
int ctx_age(const pic_ctx *c) { return c->age; }
cudaStream_t ctx_stream(const pic_ctx *c) { return c->stream; }
bool ctx_bound(const pic_ctx *c) { return c->base != nullptr; }

}  // namespace pic
