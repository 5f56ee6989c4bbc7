// Fused gather -> Boris push -> move -> Esirkepov deposit for one particle tile: the WT (or MC)
// field interpolation of Sec. 2 (Eq. interpolation-EB-real-mod), the relativistic Boris push
// (Sec. 1, in the dimensionless equations of motion of App. E) and Esirkepov's charge-conserving
// current with the B-spline form factor W_l, which the WT scheme keeps (Sec. 1, end of Sec. 2).
//
// One CTA owns one tile of cells.  In 2D it stages the tile's E and B (plus a halo covering the
// interpolation stencils and the drift since the last sort) in shared memory, walks the tile's
// particles (contiguous in the sorted store), gathers, pushes and moves them.  The FP32 form sums
// its lanes' currents through shared memory into a J tile that is added to the global FP64
// current with one atomic per tile node and component, once per species; the FP64 form, bound
// by its FP64 pipe, adds every contribution to the global current as an L2 reduction.  In 3D
// the FP32 form stages its tile's fields in shared memory too (the FP64 form reads them through
// L1), and every current contribution goes straight to a global reduction (FP32 form: into an
// FP32 current converted to FP64 once per step).
#pragma once
#include "pic_common.cuh"

namespace pic {

template <typename R> struct Vec2;
template <> struct Vec2<float> { typedef float2 T; };
template <> struct Vec2<double> { typedef double2 T; };

// Particle state in registers, independent of the storage form.
template <typename R>
struct PState {
    int c[3];  // cell per axis
    R d[3];    // in-cell offset in [0,1)
    R u[3];
};

// ---- particle storage ---------------------------------------------------------------------

template <int DIM, typename R>
__device__ __forceinline__ void load_particle(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                              PState<R> &s)
{
    if constexpr (sizeof(R) == 4) {
        const int c = __ldg(sp.cell + p);
        if constexpr (DIM == 2) {
            s.c[1] = fast_div(c, rd.div_n0.m, rd.div_n0.s);
            s.c[0] = c - s.c[1] * rd.n[0];
            s.c[2] = 0;
        } else {
            const int nxy = rd.n[0] * rd.n[1];
            s.c[2] = fast_div(c, rd.div_n01.m, rd.div_n01.s);
            const int r = c - s.c[2] * nxy;
            s.c[1] = fast_div(r, rd.div_n0.m, rd.div_n0.s);
            s.c[0] = r - s.c[1] * rd.n[0];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) s.d[a] = __ldg((const float *)sp.pos[a] + p);
    } else {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double x = __ldg((const double *)sp.pos[a] + p);
            const double f = floor(x);
            s.c[a] = min(max((int)f, 0), rd.n[a] - 1);  // a non-finite position stays in range
            s.d[a] = x - f;
        }
        if (DIM == 2) s.c[2] = 0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) s.u[a] = __ldg((const R *)sp.mom[a] + p);
}

// ---- weights of one axis: W_l at half-integer nodes (Eq. shape-real), T_l of Eq. tau_l (WT) or
// W_l (MC) at integer nodes -------------------------------------------------------------------

template <int L, int KT, typename R>
struct AxisW {
    int bh;          // first half-integer node (relative to the cell)
    R wh[L + 1];     // W_l at half-integer nodes
    int bt;          // first integer node of the T (or MC W) stencil
    R wt[KT];
};

template <int L, int KT, typename R>
__device__ __forceinline__ void axis_weights(const TTable &tt, R d, AxisW<L, KT, R> &w)
{
    R psi;
    w.bh = spline_base<L, R>(d, true, psi);
    bspline<L, R>(psi, w.wh);
    w.bt = ttable_weights<L, KT, R>(tt, d, w.wt);
}

// Esirkepov window of one axis: S0 (old-position weights) and DS = S1 - S0 on l+2 nodes
// starting at node wb (relative to the old cell); the charge form factor is W_l (Sec. 1).
template <int L, typename R>
struct AxisS {
    int wb;
    bool wide;  // the window needs all l + 2 nodes (else node l + 1 carries S0 = DS = 0)
    R s0[L + 2];
    R ds[L + 2];
};

// FP64: S1 from the stored new position (cell shift sh, offset o_new), DS = S1 - S0.  The
// old-position weights are read from wsrc (l + 1 values wstride apart: what the previous step
// wrote for this position) when given, else evaluated; the new-position weights are written to
// wdst when given.
template <int L, typename R>
__device__ __forceinline__ void axis_shapes(R d_old, int sh, R o_new, AxisS<L, R> &s,
                                            const R *wsrc = nullptr, R *wdst = nullptr,
                                            int64_t wstride = 0)
{
    R p0, p1, w0[L + 1], w1[L + 1];
    const int b0 = spline_base<L, R>(d_old, false, p0);
    const int b1 = sh + spline_base<L, R>(o_new, false, p1);
    if (wsrc) {
#pragma unroll
        for (int k = 0; k <= L; ++k) w0[k] = __ldg(wsrc + (int64_t)k * wstride);
    } else {
        bspline<L, R>(p0, w0);
    }
    bspline<L, R>(p1, w1);
    if (wdst) {
#pragma unroll
        for (int k = 0; k <= L; ++k) wdst[(int64_t)k * wstride] = w1[k];
    }
    s.wb = min(b0, b1);
    s.wide = b0 != b1;
    const bool sh0 = b0 > s.wb, sh1 = b1 > s.wb;
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        const R a0 = (k <= L) ? w0[k] : R(0);
        const R a1 = (k >= 1) ? w0[k - 1] : R(0);
        const R c0 = (k <= L) ? w1[k] : R(0);
        const R c1 = (k >= 1) ? w1[k - 1] : R(0);
        s.s0[k] = sh0 ? a1 : a0;
        s.ds[k] = (sh1 ? c1 : c0) - s.s0[k];
    }
}

// Divided difference (P_k(b) - P_k(a)) / (b - a) of the B-spline basis polynomials of
// bspline<L> (monomial coefficients in psi), evaluated without cancellation for a, b in [0,1].
template <int L>
__device__ __forceinline__ void bspline_dd(float a, float b, float *D)
{
    const float h1 = a + b;
    if constexpr (L == 1) {
        D[0] = -1.0f;
        D[1] = 1.0f;
    } else if constexpr (L == 2) {
        D[0] = -1.0f + 0.5f * h1;
        D[1] = 1.0f - h1;
        D[2] = 0.5f * h1;
    } else if constexpr (L == 3) {
        const float h2 = a * a + a * b + b * b;
        const float s6 = 1.0f / 6.0f;
        D[0] = -0.5f + 0.5f * h1 - s6 * h2;
        D[1] = -h1 + 0.5f * h2;
        D[2] = 0.5f + 0.5f * h1 - 0.5f * h2;
        D[3] = s6 * h2;
    } else {
        const float h2 = a * a + a * b + b * b;
        const float h3 = (a * a + b * b) * h1;
        const float s24 = 1.0f / 24.0f;
        D[0] = s24 * (-4.0f + 6.0f * h1 - 4.0f * h2 + h3);
        D[1] = s24 * (-12.0f - 6.0f * h1 + 12.0f * h2 - 4.0f * h3);
        D[2] = s24 * (12.0f - 6.0f * h1 - 12.0f * h2 + 6.0f * h3);
        D[3] = s24 * (4.0f + 6.0f * h1 + 4.0f * h2 - 4.0f * h3);
        D[4] = s24 * h3;
    }
}

// FP32: DS from the displacement delta (cell units) by divided differences, so the current of
// a slowly moving particle is not lost to the cancellation of S1 - S0 in single precision.
// The particle moves from psi0 to psi0 + delta on the spline's local lattice; if that leaves
// [0,1) the stencil base moves by one node and the difference is split at the lattice point,
// where the basis polynomials of neighbouring nodes agree (P_{k-1}(0) = P_k(1)).  In every case
// DS[k] = al Da[k] + be Db[k - 1] with Da, Db divided differences over the two parts of the move:
//   same base: al = delta over [psi0, psi1], be = 0
//   up:        al = 1 - psi0 over [psi0, 1], be = delta - al over [0, be] (new psi)
//   down:      al = -e over [1 - e, 1], be = -psi0 over [0, psi0], with e = -delta - psi0 the
//              overshoot below the lattice point (new psi = 1 - e); the window starts one node
//              lower
// COLLECTIVE (all 32 lanes of the warp call together): a warp none of whose lanes changes base
// evaluates the one divided difference of the same-base case, any other warp evaluates the
// general form once, on every lane, instead of the cases one after the other.
template <int L, bool COLLECTIVE = false>
__device__ __forceinline__ void axis_shapes_dd(float d_old, float delta, AxisS<L, float> &s)
{
    float p0, w0[L + 1];
    const int b0 = spline_base<L, float>(d_old, false, p0);
    bspline<L, float>(p0, w0);
    const float p1 = p0 + delta;
    const bool up = p1 >= 1.0f, dn = p1 < 0.0f;
    if (COLLECTIVE ? !__any_sync(0xffffffffu, up || dn) : !(up || dn)) {
        s.wb = b0;
        s.wide = false;
        float D[L + 1];
        bspline_dd<L>(p0, p1, D);
#pragma unroll
        for (int k = 0; k < L + 2; ++k) {
            s.s0[k] = (k <= L) ? w0[k] : 0.0f;
            s.ds[k] = (k <= L) ? delta * D[k] : 0.0f;
        }
        return;
    }
    const float e = -delta - p0;
    const float al = up ? 1.0f - p0 : (dn ? -e : delta);
    const float alo = dn ? 1.0f - e : p0;
    const float ahi = (up || dn) ? 1.0f : p1;
    const float be = up ? delta - al : (dn ? -p0 : 0.0f);
    const float bhi = up ? be : (dn ? p0 : 0.0f);
    float Da[L + 1], Db[L + 1];
    bspline_dd<L>(alo, ahi, Da);
    bspline_dd<L>(0.0f, bhi, Db);
    s.wb = dn ? b0 - 1 : b0;
    s.wide = up || dn;
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        const float w_lo = (k <= L) ? w0[k] : 0.0f, w_hi = (k >= 1) ? w0[k - 1] : 0.0f;
        s.s0[k] = dn ? w_hi : w_lo;
        const float lo = (k <= L) ? al * Da[k] : 0.0f;
        const float hi = (k >= 1) ? be * Db[k - 1] : 0.0f;
        s.ds[k] = lo + hi;
    }
}

// ---- Boris push and move --------------------------------------------------------------------

__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_r(float x) { return __frcp_rn(x); }

// Relativistic Boris rotation u^{n-1/2} -> u^{n+1/2} (Sec. 1; units of App. E, u = gamma v,
// c = 1); h = q dt / (2 m).  Returns 1/gamma^{n+1/2}.
template <typename R>
__device__ __forceinline__ R boris(R h, const R *E, const R *B, R *u)
{
    R um[3], t[3], up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
    const R hg = h * rsqrt_r(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = hg * B[a];
    const R f = R(2) * rcp_r(R(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    // u+ = u- + u' x s with s = f t: the scale f applied once to u' x t (three products fewer)
    R q[3];
    q[0] = um[0] + f * (up[1] * t[2] - up[2] * t[1]);
    q[1] = um[1] + f * (up[2] * t[0] - up[0] * t[2]);
    q[2] = um[2] + f * (up[0] * t[1] - up[1] * t[0]);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = q[a] + h * E[a];
    return rsqrt_r(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Move one axis in cell units, x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2} (App. E): returns
// the cell shift sh in {-1,0,1} and the new offset o in [0,1).  In the FP64 form o is re-derived
// from the stored value cell + o so that the next step's old-position weights are bit-identical
// to this step's new-position weights; xs is that stored value (unused for FP32).
template <typename R>
__device__ __forceinline__ int move_axis(R d, R delta, int c, int n, R &o, int &cn, R &xs)
{
    const R xn = d + delta;
    int sh;
    R on;
    if constexpr (sizeof(R) == 8) {
        // xn - sh as xn plus a selected constant: the same rounding, without converting sh.
        // The compares are taken on the bit pattern (is_neg, ge_one): for finite values they
        // decide as the FP64 compares do (-0 aside, which moves to +0 here); a NaN position,
        // which only a non-finite momentum makes, leaves with a finite offset and a cell shift
        // of at most 1, while its current and kinetic energy carry the NaN that reports it.
        const bool lo = is_neg(xn), up = ge_one(xn);
        sh = lo ? -1 : (up ? 1 : 0);
        on = xn + (lo ? 1.0 : (up ? -1.0 : 0.0));
        if (ge_one(on)) { on = 0.0; sh = min(sh + 1, 1); }  // finite: only from sh = -1
        if (is_neg(on)) on = 0.0;
    } else {
        sh = (xn < R(0)) ? -1 : ((xn >= R(1)) ? 1 : 0);
        on = xn - R(sh);
        if (on >= R(1)) { on = R(0); sh += 1; }
        if (on < R(0)) on = R(0);
    }
    int cc = c + sh;
    if (cc < 0) cc += n;
    if (cc >= n) cc -= n;
    xs = R(0);
    if constexpr (sizeof(R) == 8) {
        const double stored = (double)cc + on;
        double o2 = stored - (double)cc;  // exact (Sterbenz)
        xs = stored;
        if (ge_one(o2)) {  // cc + on rounded up to the next integer, which is the stored value
            o2 = 0.0;
            sh += 1;
            cc += 1;
            if (cc >= n) { cc -= n; xs = 0.0; }
        }
        on = o2;
    }
    o = on;
    cn = cc;
    return sh;
}

}  // namespace pic
