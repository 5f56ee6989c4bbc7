// Shared device-side definitions of libpic: run descriptors, the 1-D interpolation weights of
// the WT scheme, and small helpers.  Everything here is written for sm_103a (GB300).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define PIC_NSP_MAX 4
#define PIC_TK_MAX 6  // max nodes of a T_l stencil: ceil(l + 2 c dt/dx) <= 6 for l <= 4

namespace pic {

// ------------------------------------------------------------------------------------------
// Per-axis table of the integer-node interpolation function of the WT scheme.
//
// T_l (Sec. 2, Eq. tau_l) is W_{l-1} averaged over a box of half-width dtt = c dt/dx: a
// piecewise polynomial of degree l with support radius R = l/2 + dtt.  For a particle at
// offset delta in [0,1) of its cell, let v = delta - R, phi = v - floor(v), first node
// b = floor(v) + 1 (relative to the cell).  The weight of node b + k (k = 0..K-1) is
// T_l(R - 1 + phi - k); as a function of phi it has breakpoints only at phi = 0 and at
// phi_b = frac(-2 dtt), so on each of the two sub-intervals it is one polynomial of degree l.
// coef[p][k][m] is its m-th Taylor coefficient about the sub-interval's left end a[p].
// For the MC scheme the same table holds W_l at integer nodes (R = (l+1)/2, one piece).
// ------------------------------------------------------------------------------------------
struct TTable {
    int K;            // nodes in the stencil window
    int Rint;         // floor(R)
    double Rfrac;     // R - floor(R)
    double phib;      // interior breakpoint (0 if none)
    double coef[2][PIC_TK_MAX][5];
    float Rfrac_f, phib_f;
    // coef in FP32, grouped for vector loads: cf4[p][m][g] = coefficient m of nodes 4g .. 4g + 3
    float4 cf4[2][5][2];
};

// Scratch of the tile sort (one set per run; the species are sorted one after the other).
struct SortScratch {
    int32_t *cnt;         // ntiles * TC
    int32_t *cell_first;  // ntiles * TC
    int32_t *slot;        // n_max: provisional place in the cell
    int32_t *key;         // n_max
    int32_t *idx;         // n_max: particle index at every cell-major position
    int32_t *pos;         // n_max (slot-major order only)
    int64_t *tile_count;  // ntiles + 1 (scan workspace)
};

struct SpeciesDev {
    double q, m, w;
    double qmdt_half;     // q dt / (2 m)
    double kx[3];         // -q w dx_a / (Vc dt): Esirkepov prefix scale per axis
    double kz;            // q w / Vc: out-of-plane current scale (2D)
    int64_t n;
    // particle store (current order).  FP64 form: xi[a] double (cell units), u[a] double.
    // FP32 form: cell int32, off[a] float, u[a] float.
    void *pos[3];
    void *mom[3];
    int32_t *cell;
    int64_t *tile_start;  // ntiles + 1
    // the other buffer of the ping-pong pair (target of the next sort)
    void *pos_alt[3];
    void *mom_alt[3];
    int32_t *cell_alt;
    // FP64 2D: the B-spline weights of each particle at its stored position, l + 1 per axis at
    // wc[(a (l + 1) + k) wc_stride + p], written by every step for the next one, whose
    // old-position deposit weights they are (bit-identical by construction of the move).
    // wc_mode: 0 no cache, 1 write only (the positions were loaded or re-ordered since the
    // last step), 2 read and write.
    double *wc;
    int64_t wc_stride;
    int wc_mode;
};

// Exact quotient n / d for 0 <= n < 2^31 and 1 <= d < 2^31 by one multiply and a shift:
// with s = ceil(log2 d) and m = ceil(2^(32+s) / d), floor(n m / 2^(32+s)) = floor(n / d).
// m d exceeds 2^(32+s) by e < d, so n m / 2^(32+s) exceeds n / d by n e / (d 2^(32+s)), which
// is below 2^-(s+1) <= 1/d and so never reaches the next integer; n m < 2^31 2^33 fits 64 bits.
struct FastDiv {
    uint64_t m;
    int s;
};

inline FastDiv make_fastdiv(int d)
{
    FastDiv f;
    f.s = 0;
    while (((int64_t)1 << f.s) < (int64_t)d) ++f.s;
    const uint64_t num = (uint64_t)1 << (32 + f.s);
    f.m = num / (uint64_t)d + (num % (uint64_t)d ? 1 : 0);
    return f;
}

__device__ __forceinline__ int fast_div(int n, uint64_t m, int s)
{
    return (int)(__umul64hi((uint64_t)(uint32_t)n << 32, m) >> s);
}

struct RunDev {
    int dim, l, scheme, prec;
    int n[3];
    int tile[3];
    int ntile[3];
    int64_t ntiles;
    int64_t ncell;
    double dx[3];
    double idx[3];  // 1 / dx
    double dt;
    double dtt[3];  // c dt / dx_a
    // staged region around a tile: node local index = cell - tile_origin + pre
    int pre[3], post[3], reg[3];
    int drift[3];      // max cells a particle can be away from its sorted tile (per axis)
    int slot_major;    // tile order: 1 = (tile, slot, cell), 0 = (tile, cell, slot)
    int m4;            // Faraday stencil: 0 = Yee, 1 = M4 (beta, delta below)
    double beta[3][3], delta[3];
    int64_t reg_nodes;
    FastDiv div_n0, div_n01;  // division by n[0] and by n[0] n[1] (cell index decode)
    // fields (FP64, index (k*ny + j)*nx + i) and FP32 shadows of E, B (precision form)
    double *F[9];
    float *Fs[6];
    // 3D FP32 form (not deterministic): the current summed by FP32 L2 reductions, converted
    // into F[6..8] after the particle pass; null otherwise.  It is padded: jp_lo ghost nodes
    // below and jp[a] - n[a] - jp_lo above the grid along every axis, so that every deposit
    // window lies inside it unwrapped (node (i, j, k) of the grid at ((k + jp_lo) jp[1] + j +
    // jp_lo) jp[0] + i + jp_lo); the conversion adds every node's periodic images.
    float *J32[3];
    int jp_lo;
    int jp[3];
    int64_t jp_nodes;
    TTable tt[3];
    int nsp;
    SpeciesDev sp[PIC_NSP_MAX];
    SortScratch sc;
    int32_t *err;
    // deterministic current (pic_options.deterministic): every contribution is added as a
    // 64-bit fixed-point integer, so the sums do not depend on the order of the atomics.
    // FP32 form: one word, unit s 2^-40 (det_inv32 = 2^40 / s).  FP64 form: two words, the
    // high one in units of s 2^-31 (det_inv64 = 2^31 / s) in F[6..8], the low one in units of
    // s 2^-63 in Jlo.  s (det_scale) bounds one particle's contribution to one node.
    int det;
    float det_inv32;
    double det_inv64;
    double det_scale;
    unsigned long long *Jlo[3];
};

// Fixed-point forms of a current contribution v (see RunDev::det).
__device__ __forceinline__ unsigned long long det_word32(float v, float inv)
{
    return (unsigned long long)__float2ll_rn(v * inv);
}

// High and low words of v in units of s 2^-31 and s 2^-63: t = v 2^31 / s = hi + lo 2^-32 with
// hi = floor(t) and lo = round((t - hi) 2^32) in [0, 2^32]; t - hi is exact.
__device__ __forceinline__ void det_words64(double v, double inv, unsigned long long &hi,
                                            unsigned long long &lo)
{
    const double t = v * inv;
    const double h = floor(t);
    hi = (unsigned long long)__double2ll_rn(h);
    lo = (unsigned long long)__double2ll_rn((t - h) * 4294967296.0);
}

// ------------------------------------------------------------------------------------------
// B-spline weights W_l at the l+1 nodes that carry a non-zero weight (Sec. 2, Eq. shape-real).
// psi in [0,1); node k (k = 0..L) sits at distance (L-1)/2 + psi - k from the particle.
// These are the uniform B-spline basis polynomials written in the local variable psi.
// ------------------------------------------------------------------------------------------
template <int L, typename R>
__device__ __forceinline__ void bspline(R p, R *w)
{
    const R one = R(1);
    const R q = one - p;
    if constexpr (L == 1) {
        w[0] = q;
        w[1] = p;
    } else if constexpr (L == 2) {
        w[0] = R(0.5) * q * q;
        w[1] = R(0.5) + p * q;
        w[2] = R(0.5) * p * p;
    } else if constexpr (L == 3 && sizeof(R) == 4) {
        // node k at psi is node L - k at 1 - psi: (w3, w0) and (w1, w2) are one polynomial
        // each, evaluated on the pair (psi, 1 - psi) with packed FP32 arithmetic
        const float2 pq = make_float2(p, q);
        const float2 s2 = __fmul2_rn(pq, pq);
        const float2 e = __fmul2_rn(s2, __fmul2_rn(pq, make_float2(1.0f / 6.0f, 1.0f / 6.0f)));
        const float2 h = __ffma2_rn(make_float2(0.5f, 0.5f), pq, make_float2(-1.0f, -1.0f));
        const float2 m = __ffma2_rn(h, s2, make_float2(2.0f / 3.0f, 2.0f / 3.0f));
        w[0] = e.y;
        w[1] = m.x;
        w[2] = m.y;
        w[3] = e.x;
    } else if constexpr (L == 3) {
        // Horner forms of w3 = psi^3/6 and w1 = 2/3 - psi^2 (1 - psi/2); w0 and w2 are the same
        // polynomials in 1 - psi (node k at psi is node 3 - k at 1 - psi): eleven FP64 operations
        const R p2 = p * p;
        const R q2 = q * q;
        w[0] = q2 * (q * R(1.0 / 6.0));
        w[1] = (R(0.5) * p - one) * p2 + R(2.0 / 3.0);
        w[2] = (R(0.5) * q - one) * q2 + R(2.0 / 3.0);
        w[3] = p2 * (p * R(1.0 / 6.0));
    } else if constexpr (sizeof(R) == 4) {
        // L = 4 on the pair (psi, 1 - psi): (w4, w0) = (psi^4, (1-psi)^4) / 24, and (w3, w1) one
        // Horner polynomial; the middle weight from the partition of unity (>= 11/24)
        const float2 pq = make_float2(p, q);
        const float2 s2 = __fmul2_rn(pq, pq);
        const float2 e = __fmul2_rn(s2, __fmul2_rn(s2, make_float2(1.0f / 24.0f, 1.0f / 24.0f)));
        float2 t = __ffma2_rn(make_float2(-1.0f / 6.0f, -1.0f / 6.0f), pq,
                              make_float2(1.0f / 6.0f, 1.0f / 6.0f));
        t = __ffma2_rn(t, pq, make_float2(0.25f, 0.25f));
        t = __ffma2_rn(t, pq, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
        t = __ffma2_rn(t, pq, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
        w[0] = e.y;
        w[1] = t.y;
        w[3] = t.x;
        w[4] = e.x;
        w[2] = 1.0f - (((w[0] + w[1]) + w[3]) + w[4]);
    } else {
        // Horner forms with the 1/24 folded into the coefficients; the middle weight from the
        // partition of unity (it is >= 11/24)
        const R p2 = p * p;
        const R q2 = q * q;
        w[0] = q2 * (q2 * R(1.0 / 24.0));
        w[1] = (((R(-1.0 / 6.0) * p + R(0.5)) * p - R(0.25)) * p - R(0.5)) * p + R(11.0 / 24.0);
        w[3] = (((R(-1.0 / 6.0) * p + R(1.0 / 6.0)) * p + R(0.25)) * p + R(1.0 / 6.0)) * p
               + R(1.0 / 24.0);
        w[4] = p2 * (p2 * R(1.0 / 24.0));
        w[2] = one - (((w[0] + w[1]) + w[3]) + w[4]);
    }
}

// Comparisons of non-negative FP64 values against non-negative constants, taken on the bit
// pattern: for x >= +0 and c >= +0, x >= c exactly when bits(x) >= bits(c) as integers, and for
// c = 1/2 or 1 (low word zero) the high words decide.  The FP64 pipe of this GPU completes two
// lanes per clock per SM, so an integer compare here frees one of its issue slots; R = float
// keeps the plain compare.  (A NaN offset only selects a branch whose indices stay in range.)
template <typename R>
__device__ __forceinline__ bool ge_half(R x)
{
    if constexpr (sizeof(R) == 8) return __double2hiint(x) >= 0x3FE00000;
    else return x >= R(0.5);
}

template <typename R>
__device__ __forceinline__ bool ge_one(R x)
{
    if constexpr (sizeof(R) == 8) return __double2hiint(x) >= 0x3FF00000;
    else return x >= R(1);
}

template <typename R>
__device__ __forceinline__ bool ge_pos(R x, R c)
{
    if constexpr (sizeof(R) == 8) return __double_as_longlong(x) >= __double_as_longlong(c);
    else return x >= c;
}

template <typename R>
__device__ __forceinline__ bool is_neg(R x)  // x < 0 for x != -0 (the callers never see -0)
{
    if constexpr (sizeof(R) == 8) return __double2hiint(x) < 0;
    else return x < R(0);
}

// Split an offset delta in [0,1) against a node lattice shifted by h = c + (L-1)/2 (c = 0 for
// integer nodes, 1/2 for half-integer nodes): returns the first node (relative to the cell)
// and the local coordinate psi in [0,1).
template <int L, typename R>
__device__ __forceinline__ int spline_base(R delta, bool half, R &psi)
{
    // h2 = 2h is an integer: 2c + L - 1
    const int h2 = (half ? 1 : 0) + L - 1;
    const int hi = h2 >> 1;            // integer part of h
    if (h2 & 1) {                      // h = hi + 1/2
        if (ge_half(delta)) { psi = delta - R(0.5); return -hi; }
        psi = delta + R(0.5);
        if (ge_one(psi)) { psi = R(0); return -hi; }  // delta + 1/2 rounded up to 1
        return -hi - 1;
    }
    psi = delta;
    return -hi;
}

// Weights of the integer-node factor from a TTable (WT: T_l, MC: W_l).  Returns the first
// node relative to the cell; w[0..KT-1] (entries beyond the table's K are zero).
template <int L, int KT, typename R>
__device__ __forceinline__ int ttable_weights(const TTable &t, R delta, R *w)
{
    R v;
    if constexpr (sizeof(R) == 8) v = delta - R(t.Rfrac);
    else v = delta - R(t.Rfrac_f);
    // v in (-1, 1)
    int fl = 0;
    R phi = v;
    if (is_neg(v)) {  // v = delta - Rfrac is never -0 (delta = Rfrac gives +0)
        phi = v + R(1);
        fl = -1;
        if (ge_one(phi)) { phi = R(0); fl = 0; }
    }
    const int base = fl - t.Rint + 1;
    R phib;
    if constexpr (sizeof(R) == 8) phib = R(t.phib);
    else phib = R(t.phib_f);
    const int p = ge_pos(phi, phib) ? 1 : 0;  // phi >= +0, phib >= +0
    const R tl = phi - (p ? phib : R(0));
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            R acc = R(t.coef[p][k][L]);
#pragma unroll
            for (int m = L - 1; m >= 0; --m) acc = acc * tl + R(t.coef[p][k][m]);
            w[k] = acc;
        }
    } else {
        // the same Horner steps for four nodes at a time: one 16-byte shared load per
        // coefficient and two packed FMAs (each rounded as the scalar FMA)
        const float2 t2 = make_float2(tl, tl);
#pragma unroll
        for (int g = 0; g < (KT + 3) / 4; ++g) {
            float4 c = t.cf4[p][L][g];
            float2 a01 = make_float2(c.x, c.y), a23 = make_float2(c.z, c.w);
#pragma unroll
            for (int m = L - 1; m >= 0; --m) {
                c = t.cf4[p][m][g];
                a01 = __ffma2_rn(a01, t2, make_float2(c.x, c.y));
                a23 = __ffma2_rn(a23, t2, make_float2(c.z, c.w));
            }
            const float v[4] = {a01.x, a01.y, a23.x, a23.y};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * g + j < KT) w[4 * g + j] = v[j];
        }
    }
    return base;
}

__device__ __forceinline__ int wrap_idx(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// wrap_idx for indices usually within one period of [0, n) (a compare and an add; the
// remainder only when that is not enough).
__device__ __forceinline__ int wrap_near(int i, int n)
{
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    return (i < 0 || i >= n) ? wrap_idx(i, n) : i;
}

__device__ __forceinline__ void set_err(int32_t *err, int bit)
{
    if (err) atomicOr(err, bit);
}

}  // namespace pic
