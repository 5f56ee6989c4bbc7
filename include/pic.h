/*
 * libpic -- GB300 (sm_103a) relativistic electromagnetic PIC step with the WT force
 * interpolation of Lu, Kilian, Guo, Li and Liang, "Time-step dependent force interpolation
 * scheme for suppressing numerical Cherenkov instability in relativistic particle-in-cell
 * simulations" (arXiv:1909.09613).
 *
 * One step (pic_step) = field gather at x^n from E^n, B^n (Sec. 2: Eq. interpolation-EB-real-mod
 * for the WT scheme, Eq. interpolation-EB-real-org for the momentum-conserving MC scheme) ->
 * relativistic Boris push u^{n-1/2} -> u^{n+1/2} (Sec. 1; equations of motion App. E) -> move
 * x^{n+1} = x^n + dt u/gamma -> Esirkepov charge-conserving current deposit J^{n+1/2} with the
 * B-spline form factor W_l (Sec. 1, Sec. 2 Eq. shape-real) -> periodic Yee update
 * B^{n+1/2}, E^{n+1}, B^{n+1} (Sec. 1 "staggered Yee grid"; App. C with A_i = 1, or the M4
 * modified-Faraday stencil of App. C selected by pic_options.solver).
 *
 * Units are the paper's dimensionless ones (App. E): c = 1, 4 pi absorbed, u = gamma v in units
 * of c, so du/dt = (q/m)(E + v x B), dE/dt = curl B - J, dB/dt = -curl E.
 *
 * Grid layout: periodic, nx x ny (x nz; nz = 1 means 2D).  Node (i, j, k) lives at linear index
 * (k*ny + j)*nx + i of every field array (x fastest).  The Yee components sit at
 *   E1 (i+1/2, j, k)  E2 (i, j+1/2, k)  E3 (i, j, k+1/2)
 *   B1 (i, j+1/2, k+1/2)  B2 (i+1/2, j, k+1/2)  B3 (i+1/2, j+1/2, k),  J with E,
 * the value for the node with integer parts (i, j, k) being stored at that node's index.
 *
 * Conventions:
 *   - every function returns PIC_OK (0) or a negative pic_status; no C++ exception crosses
 *     the boundary;
 *   - host pointers are owned by the caller and are only read/written during the call;
 *   - device work is issued on the context's stream (pic_options.stream); functions that
 *     return data to the host synchronise that stream;
 *   - asynchronous device errors (a particle found outside its tile's staged region, a
 *     non-finite value found by pic_diag) are latched in the context's error word, returned by
 *     pic_diag in error_flags and turned into PIC_EOVERFLOW / PIC_ENAN by the next syncing call;
 *   - a context must not be used from two host threads at once.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_MAX_SPECIES 4

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,    /* bad argument                                                   */
    PIC_ENOMEM = -2,    /* bound memory too small / allocation failed                     */
    PIC_ECFL = -3,      /* c dt violates the Yee Courant limit or the stencil range        */
    PIC_ECUDA = -4,     /* a CUDA runtime call failed                                      */
    PIC_EOVERFLOW = -5, /* a particle left the staged region of its tile (sort too rare)   */
    PIC_ETIMEOUT = -6,  /* a bounded device wait gave up                                   */
    PIC_ENAN = -7,      /* a non-finite field or particle value was found                  */
    PIC_ESTATE = -8     /* call out of order (e.g. no memory bound yet)                    */
} pic_status;

enum { PIC_SCHEME_MC = 0, PIC_SCHEME_WT = 1 };
enum { PIC_FP64 = 0, PIC_FP32_MIXED = 1 };
enum { PIC_SOLVER_YEE = 0, PIC_SOLVER_M4 = 1 };
enum { PIC_ORDER_AUTO = 0, PIC_ORDER_CELL = 1, PIC_ORDER_SLOT = 2 };

/* Error bits of pic_diag_t.error_flags. */
enum { PIC_ERR_OUTSIDE_TILE = 1, PIC_ERR_NONFINITE = 2, PIC_ERR_TIMEOUT = 4 };

typedef struct {
    int32_t tile[3];        /* cells per particle tile; 0 = library default                 */
    int32_t sort_interval;  /* steps between tile sorts; 0 = chosen from c dt and the halo   */
    int32_t precision;      /* PIC_FP64: FP64 positions/momenta/gather/push/deposit.
                               PIC_FP32_MIXED: int32 cell + FP32 in-cell offset, FP32 momenta,
                               FP32 gather/push and tile accumulation; FP64 Yee fields, FP64
                               global current and FP64 diagnostics (in 3D the current is summed
                               by FP32 L2 reductions into a padded FP32 buffer, whose periodic
                               images are added in FP64 after the particle pass)             */
    int32_t n_species;      /* species this context will hold (1..PIC_MAX_SPECIES)          */
    int64_t capacity[PIC_MAX_SPECIES]; /* max particles per species                         */
    uint64_t stream;        /* cudaStream_t to issue work on (0 = legacy default stream)    */
    int32_t solver;         /* PIC_SOLVER_YEE: Yee curl in Faraday's law; PIC_SOLVER_M4: the
                               modified Faraday stencil with fourth-order dispersion error of
                               App. C (beta_ij = (c dt/dx_j)^2/12, delta_i = ((c dt/dx_i)^2-1)/12,
                               Eq. Maxwell-A); Ampere's stencil is the Yee one in both        */
    int32_t tile_order;     /* order of the particles of a tile in the FP32 form:
                               PIC_ORDER_AUTO (0): cell-major when a species holds >= 4
                               (odd spline order) or >= 6 (even) particles per cell, else
                               slot-major; PIC_ORDER_CELL (1):
                               (tile, cell, slot), the warp deposits of neighbouring lanes are
                               summed through shared memory; PIC_ORDER_SLOT (2): (tile, slot,
                               cell), every lane adds its own window with shared atomics.
                               The FP64 form always uses PIC_ORDER_SLOT.                     */
    int32_t deterministic;  /* 0: the current is summed with floating-point atomics, so its
                               last bits depend on the order in which the GPU serves them.
                               1: every current contribution is added as a 64-bit fixed-point
                               integer (unit = s 2^-40 in the FP32 form; two words, units
                               s 2^-31 and s 2^-63, in the FP64 form; s = the largest
                               |q w dx_a / (V_c dt)| or |q w / V_c| of the loaded species, the
                               bound of one particle's contribution to one node), so the sums
                               are exact and order-independent and a run gives bit-identical
                               fields and particles every time; J is converted to FP64 after
                               the particle pass.  With the stable tile sort this makes pic_step
                               reproducible.  Costs integer atomics and, in the FP32 form, a
                               shared-memory current tile twice as large (default tile 32 x 8).
                               Batches (pic_batch_create) do not take deterministic runs.      */
} pic_options;

/* pic_create -- validate a run and build its host-side context (no device memory yet).
 *   grid[3]      cells per axis; grid[2] == 1 selects 2D (x3-independent fields, 2D3V).
 *   dx[3]        cell sizes (dx[2] ignored in 2D).
 *   dt           time step; requires sin^2(w dt/2) = (c dt)^2 sum_i A_i sin^2(k_i dx_i/2)/dx_i^2
 *                < 1 at every grid wavenumber (the Courant limit of App. C: for Yee, A_i = 1,
 *                c dt sqrt(sum 1/dx_i^2) < 1) and c dt / dx_i < 1 so a particle crosses at
 *                most one cell face per axis per step.
 *   spline_order l in 1..4: B-spline order of W_l (Sec. 2).
 *   scheme       PIC_SCHEME_WT: gather with Eq. interpolation-EB-real-mod (W along the
 *                component's half-offset axes, T_l along its integer-node axes), valid for any
 *                c dt / dx_i < 1 (the T_l definition of Eq. tau_l, not only the printed
 *                c dt <= dx/2 forms); PIC_SCHEME_MC: all-W gather, Eq. interpolation-EB-real-org.
 *   opt          may be NULL (defaults: FP64, 2 species, capacity 0 -> must be set).
 * On success *out owns the context; free it with pic_destroy.                              */
int pic_create(const int32_t grid[3], const double dx[3], double dt, int spline_order,
               int scheme, const pic_options *opt, pic_ctx **out);

/* Bytes of device memory the context needs (fields, particle stores x2, sort scratch, the
 * diagnostics' charge densities and, in the 3D FP32 form, the padded FP32 current). */
int pic_footprint(const pic_ctx *ctx, size_t *bytes);

/* Hand the context a device buffer of at least pic_footprint bytes (e.g. a torch tensor's
 * storage).  The caller keeps it alive until pic_destroy.  The fields are zeroed.            */
int pic_bind_memory(pic_ctx *ctx, void *dev_ptr, size_t bytes);

/* Alternative to pic_bind_memory: the library allocates (cudaMalloc) and frees the buffer. */
int pic_alloc(pic_ctx *ctx);

/* Load species `species` (0-based, < n_species): charge q, mass m, macro-particle weight w
 * (rho = q w W_l / V_c, Sec. 2 Eq. shape-real), n <= capacity particles.
 *   x: host, dim x n FP64 SoA, physical positions (wrapped into [0, n_i dx_i));
 *   u: host, 3 x n FP64 SoA, u = gamma v (units of c), the momentum at t^{n-1/2}.
 * Copies host -> device, packs into the context's precision form and tile-sorts. Syncs.
 * Page-locked host arrays that the device can address (cudaHostAlloc, cudaHostRegister) are
 * read in place by the packing kernel; pageable ones go through a staging buffer in chunks.
 * The arrays are not modified.                                                             */
int pic_load_particles(pic_ctx *ctx, int species, double q, double m, double w, int64_t n,
                       const double *x, const double *u);

/* Same as pic_load_particles with x, u already in device memory (not modified). */
int pic_load_particles_device(pic_ctx *ctx, int species, double q, double m, double w, int64_t n,
                              const double *x_dev, const double *u_dev);

/* Load species `species` as a drifting plasma generated on the device (App. D): per_cell
 * particles in every cell (n = ncell * per_cell <= capacity) at uniform in-cell offsets, and
 * momenta drawn in the co-moving frame, u' ~ N(0, u_th^2) per component (Box-Muller), the x1
 * component flipped to account for the volume transform (flip when an extra uniform X1 exceeds
 * (1 + beta u'_1 / E') / 2, E' = sqrt(1 + u'^2)), then boosted along x1 with gamma:
 * u_1 = gamma (u'_1 + beta E').  u_th = 0 gives the cold beam u = (sqrt(gamma^2 - 1), 0, 0).
 * Particle p sits in cell p / per_cell (x1 fastest).
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014), U[0,1) = 53 high bits of
 * mix(p * G + key), G = 0x9E3779B97F4A7C15, for stream keys
 *   key(ids) = mix(... mix(mix(seed + G) ^ ((id_0 + 1) G)) ^ ((id_1 + 1) G) ...)
 * with ids (run, pos_species, 10 + a) for the offset along axis a, (run, species, 20 + 2a) and
 * (run, species, 21 + 2a) for the two Box-Muller uniforms of u'_a (the first enters as
 * 1 - U), and (run, species, 30) for X1.  pos_species = species gives every species its own
 * positions; another species' index places this one on that species' positions.
 * gamma >= 1, u_th >= 0, per_cell >= 0.  Tile-sorts like pic_load_particles.  Syncs.
 * (The paper loads on the host; this is the same distribution generated in HBM.)            */
int pic_load_drifting_plasma(pic_ctx *ctx, int species, double q, double m, double w,
                             int64_t per_cell, double gamma, double u_th, uint64_t seed,
                             uint64_t run, int pos_species);

/* Same as pic_load_drifting_plasma with the co-moving momenta drawn from the Juttner-Synge
 * distribution of temperature theta = kT / (m c^2) (the App. D set-up for relativistically hot
 * plasmas), by Sobol's method: attempt a of particle p draws X1..X4 uniform on (0, 1] (1 - U
 * at counter p * 128 + a, stream ids (run, species, 40 + j) for X_{j+1}), sets
 * u = -theta ln(X1 X2 X3), eta = -theta ln(X1 X2 X3 X4), and accepts the first attempt with
 * eta^2 - u^2 > 1.  The direction is isotropic: cos = 2 X5 - 1, azimuth 2 pi X6, with X5, X6 at
 * counter p on ids (run, species, 44) and (run, species, 45).  The flip and boost along x1
 * follow as in pic_load_drifting_plasma; positions likewise.
 * theta >= PIC_JUTTNER_MIN_THETA (at 0.3 an attempt is accepted with probability 0.22, so
 * 128 attempts leave a particle unsampled with probability about 1e-14); else PIC_EINVAL.
 * A particle with no accepted attempt is loaded at rest in the co-moving frame, sets
 * PIC_ERR_TIMEOUT and the call returns PIC_ETIMEOUT.  Syncs.                                  */
#define PIC_JUTTNER_MIN_THETA 0.3
int pic_load_drifting_juttner(pic_ctx *ctx, int species, double q, double m, double w,
                              int64_t per_cell, double gamma, double theta, uint64_t seed,
                              uint64_t run, int pos_species);

/* Set field component comp (0..5 = E1 E2 E3 B1 B2 B3) from count = ncell FP64 host values. */
int pic_set_fields(pic_ctx *ctx, int comp, const double *host, size_t count);

/* Advance nsteps full PIC steps on the context's stream (asynchronous). */
int pic_step(pic_ctx *ctx, int nsteps);

/* Copy field comp (0..5 E, B; 6..8 J1 J2 J3 = J^{n-1/2} of the last step) to the host. Syncs. */
int pic_read_fields(pic_ctx *ctx, int comp, double *host, size_t count);

/* Copy species particles to the host in the current (tile-sorted) order: x dim x n physical
 * FP64, u 3 x n FP64, cell (may be NULL) the int64 linear cell index. Syncs.                */
int pic_read_particles(pic_ctx *ctx, int species, double *x, double *u, int64_t *cell, int64_t n);

/* Copy the tile offsets of the species' current order (ntiles + 1 int64 values). Syncs. */
int pic_read_tile_offsets(pic_ctx *ctx, int species, int64_t *offsets, int64_t count);

/* Tile extent, number of tiles and sort interval actually used, and the tile order:
 * *slot_major = 1 for (tile, slot, cell) -- one particle of every cell in turn, chosen for the
 * FP64 form and for sparse runs -- or 0 for (tile, cell, slot), chosen for dense FP32 runs.
 * Any out pointer may be NULL.                                                              */
int pic_tile_info(const pic_ctx *ctx, int32_t tile[3], int64_t *ntiles, int32_t *sort_interval,
                  int32_t *slot_major);

/* Dynamic shared memory per CTA of the 2D particle kernel of this context (*own_bytes) and of
 * this run's work items in the batched kernel (*batched_bytes; 0 for the FP64 form and in 3D),
 * and the largest per-CTA amount with which two CTAs still share an SM of the current device
 * (*two_per_sm_bytes; 0 when no device is present).  Host query: no device work.  A batch runs
 * at the largest *batched_bytes of its runs, so runs that stay within *two_per_sm_bytes keep two
 * CTAs per SM.  Any out pointer may be NULL.                                                  */
int pic_smem_info(const pic_ctx *ctx, size_t *own_bytes, size_t *batched_bytes,
                  size_t *two_per_sm_bytes);

/* Re-sort all species by tile now (also done automatically every sort_interval steps). */
int pic_sort(pic_ctx *ctx);

typedef struct {
    int64_t step;
    double field_energy;          /* 1/2 sum over nodes (E^2 + B^2) V_c, FP64               */
    double kinetic_energy;        /* sum w m (gamma - 1), FP64                              */
    double total_charge;          /* sum q w                                                */
    double max_gauss_residual;    /* max over nodes |D.E - rho| (App. B, Eq. gauss), with
                                     D the backward difference that takes E at its Yee
                                     position to the integer node of rho                     */
    double max_continuity_residual; /* max over nodes |(rho^{n+1} - rho^n)/dt + D.J^{n+1/2}|,
                                     the discrete continuity equation the Esirkepov deposit
                                     satisfies (Sec. 1; App. B): rho^{n+1} from the current
                                     particles, rho^n kept by the previous pic_diag, J the
                                     current of the last step.  Defined only when the previous
                                     pic_diag came exactly one step earlier with no load in
                                     between; NaN otherwise                                   */
    double max_gauss_residual_drift; /* max over nodes |G - G_0|, G = D.E - rho: the change of
                                     the Gauss residual (App. B: conserved by a
                                     charge-conserving deposit) since G_0, which the first
                                     pic_step (or batch) after the last load or field set
                                     records; 0 before that step                             */
    int32_t error_flags;          /* PIC_ERR_* bits latched since creation                  */
} pic_diag_t;

/* FP64 diagnostics of the current state (the particle deposit for rho, the reductions and the
 * residuals all on the device).  Syncs. */
int pic_diag(pic_ctx *ctx, pic_diag_t *out);

/* Wait for the context's stream; returns the latched error as a status. */
int pic_sync(pic_ctx *ctx);

/* ---- batched form ----
 * Many independent runs (2D, PIC_FP32_MIXED, spline order 2 or 3, not deterministic, same
 * species count, same stream; each created,
 * bound and loaded as usual) advanced together.  One batch step = device-side choice of the runs
 * due for a tile sort, the batched sort of those runs, ONE persistent gather-push-deposit
 * launch over the tiles of every run (heaviest tiles first, pulled from a device counter; when
 * the set holds few particles, tiles heavier than the average load of a CTA slot are split into
 * up to 8 work items that share their particles, so that small runs are not paced by one CTA), and
 * one launch per Yee half/full update covering all runs.  The step's launch sequence is captured
 * in a CUDA graph on the first pic_batch_step and replayed; its launches walk device-resident
 * tables, so the same graph serves any run set that fits the batch's capacities.  While a batch exists, its runs must
 * not be stepped on their own; pic_batch_sync writes the batch's device state back into them.
 * The physics of every run is exactly that of pic_step (same tile code).                    */
typedef struct pic_batch pic_batch;
int pic_batch_create(pic_ctx *const *runs, int n, pic_batch **out);

/* Room for other run sets than the initial one (see pic_batch_set_runs): totals over the runs
 * the batch may hold at once.  Call before binding memory; the capacities size the device
 * tables (pic_batch_footprint).  Never lowers a capacity below the initial set's.            */
typedef struct {
    int32_t runs;                  /* runs at once                                          */
    int64_t cells;                 /* cells, summed over the runs                           */
    int64_t tiles;                 /* work items of the particle kernel: the runs' tiles,
                                      summed; a set of few particles splits its heavier tiles
                                      into up to 8 items each, which count here too          */
    size_t stage_bytes;            /* largest dynamic shared memory per CTA a run's work
                                      items may need in the batched kernel (pic_smem_info's
                                      batched_bytes); fixes the persistent kernel's shared
                                      memory for the life of the batch                      */
    int32_t ctas_per_sm;           /* CTAs of the persistent particle kernel per SM (0: as
                                      many as fit, two).  The persistent CTAs hold their SM
                                      slots for the whole particle pass, so a batch that
                                      shares the GPU with a more urgent one (a server's batch
                                      of short requests on a higher-priority stream) can take
                                      one per SM and leave the other slot to it             */
} pic_batch_capacity;
int pic_batch_reserve(pic_batch *batch, const pic_batch_capacity *capacity);

int pic_batch_footprint(const pic_batch *batch, size_t *bytes);       /* device tables   */
int pic_batch_bind_memory(pic_batch *batch, void *dev_ptr, size_t bytes);
int pic_batch_alloc(pic_batch *batch);                                  /* cudaMalloc'd    */

/* Replace the runs of a bound batch between steps (n >= 0; the same conditions as
 * pic_batch_create).  The device state of the runs it held is written back into their
 * contexts first (as pic_batch_sync does), so they can be stepped, read or destroyed alone;
 * then the new set's descriptors and tables are uploaded.  Every batch launch reads its table
 * lengths from device memory on a fixed grid, so the captured graph of a step stays valid and
 * is not recaptured.  Returns PIC_ENOMEM when the set exceeds the batch's capacities (then
 * build a new batch).  Syncs.                                                                */
int pic_batch_set_runs(pic_batch *batch, pic_ctx *const *runs, int n);
int pic_batch_step(pic_batch *batch, int nsteps);                       /* asynchronous    */
/* one extra (uncaptured) batch step with CUDA events around the persistent particle kernel */
int pic_batch_time_gpp(pic_batch *batch, double *ms);
int pic_batch_info(const pic_batch *batch, int64_t *work_items, int64_t *launches_per_step);
int pic_batch_sync(pic_batch *batch);                                   /* syncs           */
void pic_batch_destroy(pic_batch *batch);

/* Time of the last pic_step's gather+push+deposit launches (ms, CUDA events on the context's
 * stream), summed over the steps of that call; syncs.  For measurement.                     */
int pic_last_gpp_ms(pic_ctx *ctx, double *ms, int64_t *launches);

/* Number of kernels this context has launched since creation (for measurement). */
int pic_kernel_launches(const pic_ctx *ctx, int64_t *count);

/* Measured arithmetic peak of this GPU for the roofline: kind 0 = FP64 FMA, kind 1 = FP32 FMA,
 * in TFLOP/s (2 flops per FMA), from a register-resident FMA loop over all SMs timed with CUDA
 * events on the legacy default stream.  Not part of the PIC path.                            */
int pic_probe_fma_peak(int kind, double *tflops);

/* Tile sort that allocates no device memory.  No counterpart in the paper: it exists for
 * callers that cannot allocate device memory when they need the sort (their device memory is
 * owned by another allocator, or they cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree).  Its scratch is a fixed file-scope device array of about 20.5 MB that
 * every GPU loading the library holds until the process exits.
 *   grid[3], tile[3]  grid extent and tile extent in cells (tile <= grid, cells per tile <= 1024)
 *   n                 particles, n <= 1,048,576
 *   cell_dev          device, n int32 linear cell indices (k*ny + j)*nx + i; cells outside the
 *                     grid (< 0 or >= nx*ny*nz) are left out of the order
 *   perm_dev          device, n int64 out: perm[p] = input index placed at position p of the
 *                     cell-major tile order, sorted by (tile, cell in tile, input index): the
 *                     same stable order as the context's sort.  Positions from
 *                     tile_start[ntiles] (the number of particles inside the grid) to n - 1
 *                     are set to -1.
 *   tile_start_dev    device, ntiles + 1 int64 out: first position of every tile
 *   stream            cudaStream_t (0 = legacy default stream); asynchronous on it
 * The current device must be the device that holds cell_dev, perm_dev and tile_start_dev: the
 * scratch array of that device is used.  Requires ntiles <= 65,536 and ntiles *
 * cells-per-tile <= 1,048,576; larger sizes return PIC_EINVAL.  The first call on a device
 * looks up the scratch array's device address (with that device current); make that first
 * call before any stream capture.  Every call on a device uses the same scratch array, so
 * calls that overlap on the GPU (other streams, other host threads) race: serialise them.    */
int pic_tile_sort_noalloc(const int32_t grid[3], const int32_t tile[3], int64_t n,
                          const int32_t *cell_dev, int64_t *perm_dev, int64_t *tile_start_dev,
                          uint64_t stream);

void pic_destroy(pic_ctx *ctx);
const char *pic_strerror(int status);

/* Host evaluation (no device work) of the integer-node interpolation weights the kernels use
 * along one axis: T_l(x; dtt) for PIC_SCHEME_WT (Sec. 2, Eq. tau_l: W_{l-1} averaged over
 * [x - dtt, x + dtt], any 0 < dtt < 1) or W_l for PIC_SCHEME_MC (Eq. shape-real), for a
 * particle at in-cell offset delta in [0,1), dtt = c dt / dx.  Writes the non-zero-range
 * weights w[0..*count-1] (count <= 6) of nodes *base .. *base + *count - 1 relative to the
 * particle's cell.                                                                         */
int pic_axis_weights(int spline_order, int scheme, double dtt, double delta, double *w,
                     int *base, int *count);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
