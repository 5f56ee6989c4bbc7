// Grid kernels: periodic Yee FDTD updates (FP64), FP32 field shadows, particle packing and
// unpacking, and the FP64 diagnostics.
#include "pic_grid_dev.cuh"
#include "pic_launch.h"

#include <cmath>

namespace pic {

namespace {

constexpr int kBlock = 256;

// B <- B - h curl E on the staggered grid (Sec. 1 Yee; App. C with A_i = 1).
__global__ void __launch_bounds__(kBlock) k_yee_b(const __grid_constant__ RunDev rd, double h,
                                                  int shadow)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < rd.ncell) yee_b_cell(rd, c, h, shadow);
}

// E <- E + dt curl B - dt J.
__global__ void __launch_bounds__(kBlock) k_yee_e(const __grid_constant__ RunDev rd, int shadow)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < rd.ncell) yee_e_cell(rd, c, shadow);
}

__global__ void __launch_bounds__(kBlock) k_shadow(const __grid_constant__ RunDev rd)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= rd.ncell) return;
#pragma unroll
    for (int f = 0; f < 6; ++f) rd.Fs[f][c] = (float)rd.F[f][c];
}

// FP64 physical (x, u) -> the context's particle form, for particles p0 .. p0 + m - 1.
// x[a * xs + i], u[a * us + i] hold particle p0 + i.  Positions are divided by dx (IEEE
// division, so the cell index floor(x/dx) matches a plain FP64 evaluation) and wrapped into
// [0, n).
__device__ __forceinline__ void pack_one(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                         const double *xp, const double *up)
{
    int cell[3] = {0, 0, 0};
    double off[3] = {0, 0, 0};
    for (int a = 0; a < rd.dim; ++a) {
        double xi = xp[a] / rd.dx[a];
        if (!isfinite(xi)) {  // a non-finite input position: flag it, keep the index in range
            set_err(rd.err, 2);  // PIC_ERR_NONFINITE
            xi = 0.0;
        }
        const double N = (double)rd.n[a];
        if (xi >= N) xi -= N;
        if (xi < 0.0) xi += N;
        if (xi >= N) xi = 0.0;  // -tiny + N rounded up to N
        const double f = floor(xi);
        cell[a] = (int)f;
        off[a] = xi - f;
    }
    if (rd.prec == 1) {
        int c[3] = {cell[0], cell[1], cell[2]};
        float o[3];
        for (int a = 0; a < rd.dim; ++a) {
            o[a] = (float)off[a];
            if (o[a] >= 1.0f) {  // offset rounded to 1: carry into the next cell
                o[a] = 0.0f;
                c[a] += 1;
                if (c[a] >= rd.n[a]) c[a] -= rd.n[a];
            }
            ((float *)sp.pos[a])[p] = o[a];
        }
        sp.cell[p] = (int32_t)gidx(rd, c[0], c[1], rd.dim == 3 ? c[2] : 0);
        for (int a = 0; a < 3; ++a) ((float *)sp.mom[a])[p] = (float)up[a];
    } else {
        for (int a = 0; a < rd.dim; ++a) ((double *)sp.pos[a])[p] = (double)cell[a] + off[a];
        for (int a = 0; a < 3; ++a) ((double *)sp.mom[a])[p] = up[a];
    }
}

__global__ void __launch_bounds__(kBlock) k_pack(const __grid_constant__ RunDev rd, int s,
                                                 const double *x, int64_t xs, const double *u,
                                                 int64_t us, int64_t m, int64_t p0)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double xp[3] = {0, 0, 0}, up[3];
    for (int a = 0; a < rd.dim; ++a) xp[a] = x[a * xs + i];
    for (int a = 0; a < 3; ++a) up[a] = u[a * us + i];
    pack_one(rd, rd.sp[s], p0 + i, xp, up);
}

// ---- drifting plasma generated on the device (App. D) ------------------------------------
// SplitMix64 finaliser (Steele, Lea, Flood 2014) and U[0,1) from its 53 high bits.
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int kJuttnerAttempts = 128;

__device__ __forceinline__ double sm64_uniform(uint64_t key, uint64_t ctr)
{
    return (double)(sm64_mix(ctr * 0x9E3779B97F4A7C15ull + key) >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void __launch_bounds__(kBlock) k_load_plasma(const __grid_constant__ RunDev rd, int s,
                                                        LoadKeys keys, int64_t per_cell,
                                                        double gamma, double u_th, double theta,
                                                        int64_t n)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t cell = p / per_cell;
    int64_t ci[3];
    ci[0] = cell % rd.n[0];
    ci[1] = (cell / rd.n[0]) % rd.n[1];
    ci[2] = cell / ((int64_t)rd.n[0] * rd.n[1]);
    double xp[3] = {0, 0, 0}, up[3] = {0, 0, 0};
    // every operation rounded on its own (no fused multiply-add), as a plain evaluation does
    for (int a = 0; a < rd.dim; ++a) {
        const double L = __dmul_rn((double)rd.n[a], rd.dx[a]);
        const double off = sm64_uniform(keys.pos[a], (uint64_t)p);
        double xa = __dmul_rn(__dadd_rn((double)ci[a], off), rd.dx[a]);
        if (xa >= L) xa = __dsub_rn(xa, L);
        xp[a] = xa;
    }
    const double beta = sqrt(__dsub_rn(1.0, __ddiv_rn(1.0, __dmul_rn(gamma, gamma))));
    if (theta > 0.0 || u_th > 0.0) {
        double v[3];
        if (theta > 0.0) {
            // Sobol's method: attempt a draws X1..X4 at counter p * kJuttnerAttempts + a;
            // u = -theta ln(X1 X2 X3), eta = -theta ln(X1 X2 X3 X4), accepted when
            // eta^2 - u^2 > 1.  The loop is bounded; a particle left without an accepted
            // attempt (about 1e-14 at theta = 0.3) is flagged and loaded at rest.
            double um = -1.0;
            for (int a = 0; a < kJuttnerAttempts && um < 0.0; ++a) {
                const uint64_t ctr = (uint64_t)p * kJuttnerAttempts + a;
                const double x1 = __dsub_rn(1.0, sm64_uniform(keys.jut[0], ctr));
                const double x2 = __dsub_rn(1.0, sm64_uniform(keys.jut[1], ctr));
                const double x3 = __dsub_rn(1.0, sm64_uniform(keys.jut[2], ctr));
                const double x4 = __dsub_rn(1.0, sm64_uniform(keys.jut[3], ctr));
                const double p3 = __dmul_rn(__dmul_rn(x1, x2), x3);
                const double u = __dmul_rn(-theta, log(p3));
                const double eta = __dmul_rn(-theta, log(__dmul_rn(p3, x4)));
                if (__dsub_rn(__dmul_rn(eta, eta), __dmul_rn(u, u)) > 1.0) um = u;
            }
            if (um < 0.0) {
                set_err(rd.err, 4);  // PIC_ERR_TIMEOUT: a bounded device loop gave up
                um = 0.0;
            }
            const double x5 = sm64_uniform(keys.dir[0], (uint64_t)p);
            const double x6 = sm64_uniform(keys.dir[1], (uint64_t)p);
            const double ct = __dsub_rn(__dmul_rn(2.0, x5), 1.0);
            const double st = __dmul_rn(2.0, sqrt(__dmul_rn(x5, __dsub_rn(1.0, x5))));
            const double ph = __dmul_rn(6.283185307179586, x6);
            v[0] = __dmul_rn(um, ct);
            v[1] = __dmul_rn(__dmul_rn(um, st), cos(ph));
            v[2] = __dmul_rn(__dmul_rn(um, st), sin(ph));
        } else
        for (int a = 0; a < 3; ++a) {
            const double u1 = __dsub_rn(1.0, sm64_uniform(keys.mom[2 * a], (uint64_t)p));  // (0, 1]
            const double u2 = sm64_uniform(keys.mom[2 * a + 1], (uint64_t)p);
            const double r = sqrt(__dmul_rn(-2.0, log(u1)));
            v[a] = __dmul_rn(u_th, __dmul_rn(r, cos(__dmul_rn(6.283185307179586, u2))));
        }
        const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])),
                                    __dmul_rn(v[2], v[2]));
        const double ep = sqrt(__dadd_rn(1.0, s2));
        const double x1 = sm64_uniform(keys.flip, (uint64_t)p);
        const double thr = __dmul_rn(0.5, __dadd_rn(1.0, __ddiv_rn(__dmul_rn(beta, v[0]), ep)));
        const double vx = (x1 > thr) ? -v[0] : v[0];
        up[0] = __dmul_rn(gamma, __dadd_rn(vx, __dmul_rn(beta, ep)));
        up[1] = v[1];
        up[2] = v[2];
    } else {
        up[0] = sqrt(__dsub_rn(__dmul_rn(gamma, gamma), 1.0));
    }
    pack_one(rd, rd.sp[s], p, xp, up);
}

// Particles p0 .. p0 + m - 1 -> FP64 physical x[a * m + i], u[a * m + i], cell[i].
__global__ void __launch_bounds__(kBlock) k_unpack(const __grid_constant__ RunDev rd, int s,
                                                   double *x, double *u, int64_t *cell,
                                                   int64_t m, int64_t p0)
{
    const SpeciesDev &sp = rd.sp[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t p = p0 + i;
    if (rd.prec == 1) {
        const int c = sp.cell[p];
        int ci[3];
        ci[0] = c % rd.n[0];
        ci[1] = (c / rd.n[0]) % rd.n[1];
        ci[2] = c / (rd.n[0] * rd.n[1]);
        for (int a = 0; a < rd.dim; ++a)
            x[a * m + i] = ((double)ci[a] + (double)((const float *)sp.pos[a])[p]) * rd.dx[a];
        for (int a = 0; a < 3; ++a) u[a * m + i] = (double)((const float *)sp.mom[a])[p];
        if (cell) cell[i] = c;
    } else {
        int ci[3] = {0, 0, 0};
        for (int a = 0; a < rd.dim; ++a) {
            const double xi = ((const double *)sp.pos[a])[p];
            ci[a] = (int)floor(xi);
            x[a * m + i] = xi * rd.dx[a];
        }
        for (int a = 0; a < 3; ++a) u[a * m + i] = ((const double *)sp.mom[a])[p];
        if (cell) cell[i] = gidx(rd, ci[0], ci[1], ci[2]);
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ double block_sum(double v)
{
    __shared__ double red[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

__device__ double block_max(double v)
{
    __shared__ double red[32];
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) v = warp_max(v);
    __syncthreads();
    return v;
}

__device__ __forceinline__ void atomic_max_nonneg(double *a, double v)
{
    atomicMax((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}

// sum over nodes of E^2 + B^2 (FP64); non-finite values raise the error bit.
__global__ void __launch_bounds__(kBlock) k_field_energy(const __grid_constant__ RunDev rd,
                                                         double *out)
{
    double acc = 0.0;
    bool bad = false;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < rd.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < 6; ++f) {
            const double v = rd.F[f][c];
            if (!isfinite(v)) bad = true;
            acc += v * v;
        }
    }
    if (bad) set_err(rd.err, 2);
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

// sum over particles of w m (gamma - 1)
__global__ void __launch_bounds__(kBlock) k_kinetic(const __grid_constant__ RunDev rd, int s,
                                                    double *out)
{
    const SpeciesDev &sp = rd.sp[s];
    double acc = 0.0;
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < sp.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double u0, u1, u2;
        if (rd.prec == 1) {
            u0 = ((const float *)sp.mom[0])[p];
            u1 = ((const float *)sp.mom[1])[p];
            u2 = ((const float *)sp.mom[2])[p];
        } else {
            u0 = ((const double *)sp.mom[0])[p];
            u1 = ((const double *)sp.mom[1])[p];
            u2 = ((const double *)sp.mom[2])[p];
        }
        const double u2s = u0 * u0 + u1 * u1 + u2 * u2;
        if (!isfinite(u2s)) bad = true;
        // gamma - 1 = u^2 / (sqrt(1 + u^2) + 1), free of cancellation for slow particles
        acc += u2s / (sqrt(1.0 + u2s) + 1.0);
    }
    if (bad) set_err(rd.err, 2);
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out, acc * sp.w * sp.m);
}

// rho = sum q w W_l / V_c at integer nodes (FP64 atomics): the l + 1 non-zero B-spline
// weights per axis from the basis polynomials, the same S0 the Esirkepov deposit starts from.
// A block covers kRhoPer * kBlock consecutive particles of the store, and the lanes of a warp
// take particles 32 apart: in the cell-major order 32 neighbours in the store usually share a
// cell, and their FP64 reductions to the same nodes would be serialised by L2, while particles
// 32 apart sit in different cells.
constexpr int kRhoPer = 4;
static_assert(kBlock / 32 * kRhoPer == 32, "a warp's lanes cover 32 particles 32 apart");

template <int L>
__device__ __forceinline__ void rho_particle(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                             double *rho);

template <int L>
__global__ void __launch_bounds__(kBlock) k_rho(const __grid_constant__ RunDev rd, int s,
                                                double *rho)
{
    const SpeciesDev &sp = rd.sp[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * (int64_t)kBlock * kRhoPer;
#pragma unroll 1
    for (int r = 0; r < kRhoPer; ++r) {
        const int64_t p = base + lane * 32 + warp + (kBlock / 32) * r;
        if (p < sp.n) rho_particle<L>(rd, sp, p, rho);
    }
}

template <int L>
__device__ __forceinline__ void rho_particle(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                             double *rho)
{
    int c[3] = {0, 0, 0};
    double d[3] = {0, 0, 0};
    if (rd.prec == 1) {
        const int cc = sp.cell[p];
        c[2] = fast_div(cc, rd.div_n01.m, rd.div_n01.s);
        const int r = cc - c[2] * rd.n[0] * rd.n[1];
        c[1] = fast_div(r, rd.div_n0.m, rd.div_n0.s);
        c[0] = r - c[1] * rd.n[0];
        for (int a = 0; a < rd.dim; ++a) d[a] = ((const float *)sp.pos[a])[p];
    } else {
        for (int a = 0; a < rd.dim; ++a) {
            const double xi = ((const double *)sp.pos[a])[p];
            const double f = floor(xi);
            c[a] = min(max((int)f, 0), rd.n[a] - 1);  // a non-finite position stays in range
            d[a] = xi - f;
        }
    }
    double w[3][L + 1];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double psi;
        b[a] = spline_base<L, double>(d[a], false, psi);
        bspline<L, double>(psi, w[a]);
    }
    const double vc = rd.dx[0] * rd.dx[1] * (rd.dim == 3 ? rd.dx[2] : 1.0);
    const double qw = sp.q * sp.w / vc;
    const int nk = rd.dim == 3 ? L + 1 : 1;
    for (int kk = 0; kk < nk; ++kk) {
        const int gk = rd.dim == 3 ? wrap_near(c[2] + b[2] + kk, rd.n[2]) : 0;
        const double wk = rd.dim == 3 ? qw * w[2][kk] : qw;
#pragma unroll
        for (int jj = 0; jj <= L; ++jj) {
            const int gj = wrap_near(c[1] + b[1] + jj, rd.n[1]);
            const double wjk = wk * w[1][jj];
#pragma unroll
            for (int ii = 0; ii <= L; ++ii) {
                const int gi = wrap_near(c[0] + b[0] + ii, rd.n[0]);
                atomicAdd(rho + gidx(rd, gi, gj, gk), wjk * w[0][ii]);
            }
        }
    }
}

// Backward-difference divergence at integer node c of a field whose component a sits half a
// cell up along a (E or J on the Yee grid): sum_a (F_a(c) - F_a(c - e_a)) / dx_a.
__device__ __forceinline__ double div_node(const RunDev &rd, const double *const *F, int64_t c)
{
    const int nx = rd.n[0], ny = rd.n[1], nz = rd.n[2];
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / ((int64_t)nx * ny));
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int jm = (j == 0) ? ny - 1 : j - 1;
    double dv = (F[0][c] - F[0][gidx(rd, im, j, k)]) * rd.idx[0]
                + (F[1][c] - F[1][gidx(rd, i, jm, k)]) * rd.idx[1];
    if (rd.dim == 3) {
        const int km = (k == 0) ? nz - 1 : k - 1;
        dv += (F[2][c] - F[2][gidx(rd, i, j, km)]) * rd.idx[2];
    }
    return dv;
}

// Charge-conservation residuals (App. B, Eq. gauss; Sec. 1 for the continuity equation of the
// Esirkepov deposit), with G = D.E - rho at every node:
//   out[0] = max |G|;
//   gref_out: G written per node (the reference the drift is measured from);
//   gref_in : out[1] = max |G - gref_in|;
//   rho_prev: out[2] = max |(rho - rho_prev) inv_dt + D.J|, J = F[6..8].
__global__ void __launch_bounds__(kBlock) k_gauss(const __grid_constant__ RunDev rd,
                                                  const double *rho, double *out,
                                                  const double *gref_in, double *gref_out,
                                                  const double *rho_prev, double inv_dt)
{
    double m = 0.0, md = 0.0, mc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < rd.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const double g = div_node(rd, rd.F, c) - rho[c];
        m = fmax(m, fabs(g));
        if (gref_out) gref_out[c] = g;
        if (gref_in) md = fmax(md, fabs(g - gref_in[c]));
        if (rho_prev) mc = fmax(mc, fabs((rho[c] - rho_prev[c]) * inv_dt + div_node(rd, rd.F + 6, c)));
    }
    m = block_max(m);
    if (threadIdx.x == 0) atomic_max_nonneg(out, m);
    if (gref_in) {
        md = block_max(md);
        if (threadIdx.x == 0) atomic_max_nonneg(out + 1, md);
    }
    if (rho_prev) {
        mc = block_max(mc);
        if (threadIdx.x == 0) atomic_max_nonneg(out + 2, mc);
    }
}

// Fixed-point current of a deterministic run (RunDev::det) -> FP64, in place.
__global__ void __launch_bounds__(kBlock) k_det_finish(const __grid_constant__ RunDev rd)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= rd.ncell) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long *w = (long long *)rd.F[6 + a];
        if (rd.prec == 1) {
            rd.F[6 + a][c] = (double)w[c] * (rd.det_scale * 0x1p-40);
        } else {
            const double v = (double)w[c] + (double)(long long)rd.Jlo[a][c] * 0x1p-32;
            rd.F[6 + a][c] = v * (rd.det_scale * 0x1p-31);
        }
    }
}

// The padded FP32 current (RunDev::J32) -> F[6..8]: every grid node gets the sum, in FP64, of
// its periodic images in the padded buffer (padded index i + jp_lo + m n along each axis).
__global__ void __launch_bounds__(kBlock) k_j32_finish(const __grid_constant__ RunDev rd)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= rd.ncell) return;
    const int i = (int)(c % rd.n[0]);
    const int64_t r = c / rd.n[0];
    const int j = (int)(r % rd.n[1]), k = (int)(r / rd.n[1]);
    double s[3] = {0.0, 0.0, 0.0};
    for (int kp = (k + rd.jp_lo) % rd.n[2]; kp < rd.jp[2]; kp += rd.n[2])
        for (int jq = (j + rd.jp_lo) % rd.n[1]; jq < rd.jp[1]; jq += rd.n[1])
            for (int ip = (i + rd.jp_lo) % rd.n[0]; ip < rd.jp[0]; ip += rd.n[0]) {
                const int64_t q = ((int64_t)kp * rd.jp[1] + jq) * rd.jp[0] + ip;
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] += (double)rd.J32[a][q];
            }
#pragma unroll
    for (int a = 0; a < 3; ++a) rd.F[6 + a][c] = s[a];
}

inline unsigned grid_for(int64_t n)
{
    return (unsigned)((n + kBlock - 1) / kBlock);
}

}  // namespace

cudaError_t launch_yee_b(const RunDev &rd, double h, bool shadow, cudaStream_t st)
{
    k_yee_b<<<grid_for(rd.ncell), kBlock, 0, st>>>(rd, h, shadow ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_yee_e(const RunDev &rd, bool shadow, cudaStream_t st)
{
    k_yee_e<<<grid_for(rd.ncell), kBlock, 0, st>>>(rd, shadow ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const RunDev &rd, cudaStream_t st)
{
    k_shadow<<<grid_for(rd.ncell), kBlock, 0, st>>>(rd);
    return cudaGetLastError();
}

cudaError_t launch_pack(const RunDev &rd, int s, const double *x, int64_t xs, const double *u,
                        int64_t us, int64_t m, int64_t p0, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    k_pack<<<grid_for(m), kBlock, 0, st>>>(rd, s, x, xs, u, us, m, p0);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const RunDev &rd, int s, double *x, double *u, int64_t *cell,
                          int64_t m, int64_t p0, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    k_unpack<<<grid_for(m), kBlock, 0, st>>>(rd, s, x, u, cell, m, p0);
    return cudaGetLastError();
}

// rho of all species at their current positions (FP64, into rho, cleared first)
static cudaError_t launch_rho(const RunDev &rd, double *rho, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(rho, 0, rd.ncell * sizeof(double), st);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < rd.nsp; ++s) {
        if (rd.sp[s].n == 0) continue;
        const unsigned g = grid_for((rd.sp[s].n + kRhoPer - 1) / kRhoPer);
        switch (rd.l) {
        case 1: k_rho<1><<<g, kBlock, 0, st>>>(rd, s, rho); break;
        case 2: k_rho<2><<<g, kBlock, 0, st>>>(rd, s, rho); break;
        case 3: k_rho<3><<<g, kBlock, 0, st>>>(rd, s, rho); break;
        default: k_rho<4><<<g, kBlock, 0, st>>>(rd, s, rho); break;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_diag(const RunDev &rd, double *out, double *rho, const double *gref,
                        const double *rho_prev, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 6 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const unsigned gr = 1024;
    k_field_energy<<<gr, kBlock, 0, st>>>(rd, out + 0);
    for (int s = 0; s < rd.nsp; ++s) k_kinetic<<<gr, kBlock, 0, st>>>(rd, s, out + 1);
    e = launch_rho(rd, rho, st);
    if (e != cudaSuccess) return e;
    k_gauss<<<gr, kBlock, 0, st>>>(rd, rho, out + 2, gref, nullptr, rho_prev, 1.0 / rd.dt);
    return cudaGetLastError();
}

cudaError_t launch_gauss_ref(const RunDev &rd, double *rho, double *gref, double *scratch,
                             cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = launch_rho(rd, rho, st);
    if (e != cudaSuccess) return e;
    k_gauss<<<1024, kBlock, 0, st>>>(rd, rho, scratch, nullptr, gref, nullptr, 0.0);
    return cudaGetLastError();
}

cudaError_t launch_det_finish(const RunDev &rd, cudaStream_t st)
{
    k_det_finish<<<grid_for(rd.ncell), kBlock, 0, st>>>(rd);
    return cudaGetLastError();
}

cudaError_t launch_j32_finish(const RunDev &rd, cudaStream_t st)
{
    k_j32_finish<<<grid_for(rd.ncell), kBlock, 0, st>>>(rd);
    return cudaGetLastError();
}

cudaError_t launch_load_plasma(const RunDev &rd, int s, const LoadKeys &keys, int64_t per_cell,
                               double gamma, double u_th, double theta, int64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_load_plasma<<<grid_for(n), kBlock, 0, st>>>(rd, s, keys, per_cell, gamma, u_th, theta, n);
    return cudaGetLastError();
}


}  // namespace pic
