// Fused gather -> Boris push -> move -> Esirkepov deposit for one particle tile.
//
// One CTA owns one tile of cells.  In 2D it stages the tile's E and B (plus a halo covering the
// interpolation stencils and the drift since the last sort) in shared memory, walks the tile's
// particles (contiguous in the sorted store), gathers with the WT (or MC) weights, pushes,
// moves, and accumulates the Esirkepov current of every particle in a shared-memory J tile,
// which is then added to the global FP64 current with one atomic per tile node and component,
// once per species.  In 3D the halo would not fit, so fields are read through the L1 cache and
// the current goes straight to global atomics.
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
            s.c[1] = c / rd.n[0];
            s.c[0] = c - s.c[1] * rd.n[0];
            s.c[2] = 0;
        } else {
            const int nxy = rd.n[0] * rd.n[1];
            s.c[2] = c / nxy;
            const int r = c - s.c[2] * nxy;
            s.c[1] = r / rd.n[0];
            s.c[0] = r - s.c[1] * rd.n[0];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) s.d[a] = __ldg((const float *)sp.pos[a] + p);
    } else {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double x = __ldg((const double *)sp.pos[a] + p);
            const double f = floor(x);
            s.c[a] = (int)f;
            s.d[a] = x - f;
        }
        if (DIM == 2) s.c[2] = 0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) s.u[a] = __ldg((const R *)sp.mom[a] + p);
}

// ---- weights of one axis ------------------------------------------------------------------

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

// Esirkepov window of one axis: S0 (old), S1 (new) on l+2 nodes starting at wb.
template <int L, typename R>
struct AxisS {
    int wb;
    R s0[L + 2];
    R s1[L + 2];
};

template <int L, typename R>
__device__ __forceinline__ void axis_shapes(R d_old, int sh, R o_new, AxisS<L, R> &s)
{
    R p0, p1, w0[L + 1], w1[L + 1];
    const int b0 = spline_base<L, R>(d_old, false, p0);
    const int b1 = sh + spline_base<L, R>(o_new, false, p1);
    bspline<L, R>(p0, w0);
    bspline<L, R>(p1, w1);
    s.wb = min(b0, b1);
    const bool sh0 = b0 > s.wb, sh1 = b1 > s.wb;
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        const R a0 = (k <= L) ? w0[k] : R(0);
        const R a1 = (k >= 1) ? w0[k - 1] : R(0);
        const R c0 = (k <= L) ? w1[k] : R(0);
        const R c1 = (k >= 1) ? w1[k - 1] : R(0);
        s.s0[k] = sh0 ? a1 : a0;
        s.s1[k] = sh1 ? c1 : c0;
    }
}

// ---- Boris push and move --------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ void boris(R h, const R *E, const R *B, R *u)
{
    R um[3], t[3], sv[3], up[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
    const R gm = sqrt(R(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    const R hg = h / gm;
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = hg * B[a];
    const R f = R(2) / (R(1) + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) sv[a] = f * t[a];
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    R q[3];
    q[0] = um[0] + (up[1] * sv[2] - up[2] * sv[1]);
    q[1] = um[1] + (up[2] * sv[0] - up[0] * sv[2]);
    q[2] = um[2] + (up[0] * sv[1] - up[1] * sv[0]);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = q[a] + h * E[a];
}

// Move one axis in cell units: returns the cell shift sh in {-1,0,1} and the new offset o in
// [0,1).  In the FP64 form o is re-derived from the stored value cell + o so that the next
// step's old-position weights are bit-identical to this step's new-position weights.
template <typename R>
__device__ __forceinline__ int move_axis(R d, R delta, int c, int n, R &o, int &cn)
{
    const R xn = d + delta;
    int sh = (xn < R(0)) ? -1 : ((xn >= R(1)) ? 1 : 0);
    R on = xn - R(sh);
    if (on >= R(1)) { on = R(0); sh += 1; }
    if (on < R(0)) on = R(0);
    int cc = c + sh;
    if (cc < 0) cc += n;
    if (cc >= n) cc -= n;
    if constexpr (sizeof(R) == 8) {
        const double stored = (double)cc + on;
        double o2 = stored - (double)cc;
        if (o2 >= 1.0) {  // cc + on rounded up to the next integer
            o2 = 0.0;
            sh += 1;
            cc += 1;
            if (cc >= n) cc -= n;
        }
        on = o2;
    }
    o = on;
    cn = cc;
    return sh;
}

}  // namespace pic
