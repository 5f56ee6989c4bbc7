// Host-side construction of the per-axis interpolation tables (TTable) of the WT scheme.
//
// T_l (Sec. 2, Eq. tau_l and the real-space forms below it) is the inverse Fourier transform
// of tau_l = sinc^l(k dx/2) sinc(k c dt): the B-spline W_{l-1} averaged over a box of half
// width dtt = c dt/dx (cell units).  It is a piecewise polynomial of degree l.  The kernels
// evaluate it per particle from Taylor coefficients tabulated here once per run:
//   - W_{l-1} is written piece by piece in exact small-integer polynomial coefficients
//     (truncated-power form of the cardinal B-spline, expanded at each piece's left knot);
//   - T_l and its right derivatives at each sub-interval origin follow from
//     T^(m)(y) = [W_{l-1}^(m-1)(y + dtt) - W_{l-1}^(m-1)(y - dtt)] / (2 dtt)  (m >= 1)
//     and T(y) = integral of W_{l-1} over [y - dtt, y + dtt] / (2 dtt) piece by piece.
// This is valid for any dtt in (0, 1): the paper prints the forms for dtt <= 1/2 only
// (Sec. 2 restricts itself there); beyond that the support grows to l + 2 nodes.
#include "pic_common.cuh"

#include <cmath>
#include <cstring>

namespace pic {

typedef long double ld;

// Coefficients (in local t in [0,1)) of piece q of the centred B-spline of degree d
// (= W_d, support [-(d+1)/2, (d+1)/2], piece q on [-(d+1)/2 + q, -(d+1)/2 + q + 1)).
// W_d(y) = 1/d! sum_{j<=q} (-1)^j C(d+1, j) (q - j + t)^d.
static void bspline_piece(int d, int q, ld c[6])
{
    for (int m = 0; m < 6; ++m) c[m] = 0;
    ld fact = 1;
    for (int i = 2; i <= d; ++i) fact *= i;
    for (int j = 0; j <= q; ++j) {
        // C(d+1, j)
        ld binom = 1;
        for (int i = 0; i < j; ++i) binom = binom * (d + 1 - i) / (i + 1);
        const ld sgn = (j & 1) ? -1 : 1;
        const ld a = (ld)(q - j);
        // (a + t)^d = sum_m C(d, m) a^(d-m) t^m
        for (int m = 0; m <= d; ++m) {
            ld bm = 1;
            for (int i = 0; i < m; ++i) bm = bm * (d - i) / (i + 1);
            c[m] += sgn * binom * bm * std::pow(a, (ld)(d - m));
        }
    }
    for (int m = 0; m <= d; ++m) c[m] /= fact;
}

// m-th derivative at y of the polynomial piece of W_d that contains y_loc (so that a
// derivative taken exactly at a knot uses the piece of the interval it is meant for).
static ld bspline_deriv(int d, ld y, ld y_loc, int m)
{
    const ld left = -(ld)(d + 1) / 2;
    const ld s_loc = y_loc - left;
    if (s_loc < 0) return 0;
    const int q = (int)std::floor((double)s_loc);
    if (q > d) return 0;
    const ld t = (y - left) - q;
    ld c[6];
    bspline_piece(d, q, c);
    ld acc = 0;
    for (int k = d; k >= m; --k) {
        ld f = 1;
        for (int i = 0; i < m; ++i) f *= (k - i);
        acc = acc * t + c[k] * f;
    }
    return acc;
}

// integral of W_d over [a, b]
static ld bspline_integral(int d, ld a, ld b)
{
    const ld left = -(ld)(d + 1) / 2, right = -left;
    if (a < left) a = left;
    if (b > right) b = right;
    if (b <= a) return 0;
    ld sum = 0;
    for (int q = 0; q <= d; ++q) {
        const ld pl = left + q, pr = pl + 1;
        const ld lo = a > pl ? a : pl, hi = b < pr ? b : pr;
        if (hi <= lo) continue;
        ld c[6];
        bspline_piece(d, q, c);
        const ld ta = lo - pl, tb = hi - pl;
        ld s = 0;
        for (int k = d; k >= 0; --k) {
            // (tb^{k+1} - ta^{k+1})/(k+1) = (tb - ta) * sum_{r=0..k} tb^r ta^{k-r} / (k+1)
            ld h = 0;
            for (int r = 0; r <= k; ++r) h += std::pow(tb, (ld)r) * std::pow(ta, (ld)(k - r));
            s += c[k] * h / (k + 1);
        }
        sum += (tb - ta) * s;
    }
    return sum;
}

// T_l value and derivatives at y (m = 0..l), polynomial pieces chosen from y_loc.
static ld tfun_deriv(int l, ld dtt, ld y, ld y_loc, int m)
{
    if (m == 0) return bspline_integral(l - 1, y - dtt, y + dtt) / (2 * dtt);
    return (bspline_deriv(l - 1, y + dtt, y_loc + dtt, m - 1)
            - bspline_deriv(l - 1, y - dtt, y_loc - dtt, m - 1)) / (2 * dtt);
}

// Build the table of one axis.  scheme 1 = WT (T_l), 0 = MC (W_l at integer nodes).
bool build_ttable(int l, int scheme, double dtt_d, TTable *t)
{
    std::memset(t, 0, sizeof(*t));
    if (l < 1 || l > 4) return false;
    const ld dtt = dtt_d;
    ld R;
    if (scheme == 1) {
        if (!(dtt_d > 0.0 && dtt_d < 1.0)) return false;
        R = (ld)l / 2 + dtt;
    } else {
        R = (ld)(l + 1) / 2;
    }
    int K = (int)std::ceil((double)(2 * R) - 1e-12);
    if (K > PIC_TK_MAX) return false;
    t->K = K;
    t->Rint = (int)std::floor((double)R);
    t->Rfrac = (double)(R - t->Rint);
    ld phib = 0;
    if (scheme == 1) {
        ld f = -2 * dtt;
        f = f - std::floor((double)f);
        if (f > 1e-15 && f < 1 - 1e-15) phib = f;
    }
    t->phib = (double)phib;
    for (int p = 0; p < 2; ++p) {
        const ld a = p ? phib : 0;
        const ld b = (p == 0 && phib > 0) ? phib : 1;
        for (int k = 0; k < K; ++k) {
            const ld y0 = R - 1 + a - k;
            const ld ymid = R - 1 + (a + b) / 2 - k;
            ld fact = 1;
            for (int m = 0; m <= l; ++m) {
                if (m > 0) fact *= m;
                ld v;
                if (scheme == 1) v = tfun_deriv(l, dtt, y0, ymid, m);
                else v = bspline_deriv(l, y0, ymid, m);
                t->coef[p][k][m] = (double)(v / fact);
            }
        }
    }
    for (int p = 0; p < 2; ++p)
        for (int m = 0; m < 5; ++m)
            for (int g = 0; g < 2; ++g) {
                float v[4];
                for (int j = 0; j < 4; ++j) {
                    const int k = 4 * g + j;
                    v[j] = k < PIC_TK_MAX ? (float)t->coef[p][k][m] : 0.0f;
                }
                t->cf4[p][m][g] = make_float4(v[0], v[1], v[2], v[3]);
            }
    t->Rfrac_f = (float)t->Rfrac;
    t->phib_f = (float)t->phib;
    // the float split must reproduce the same breakpoint ordering
    if (t->Rfrac_f >= 1.0f) return false;
    return true;
}

// Host evaluation of a table (same arithmetic as the device code, in double).
int ttable_eval_host(const TTable *t, int l, double delta, double *w)
{
    double v = delta - t->Rfrac;
    int fl = 0;
    double phi = v;
    if (v < 0.0) {
        phi = v + 1.0;
        fl = -1;
        if (phi >= 1.0) { phi = 0.0; fl = 0; }
    }
    const int base = fl - t->Rint + 1;
    const int p = (phi >= t->phib) ? 1 : 0;
    const double tl = phi - (p ? t->phib : 0.0);
    for (int k = 0; k < t->K; ++k) {
        double acc = t->coef[p][k][l];
        for (int m = l - 1; m >= 0; --m) acc = acc * tl + t->coef[p][k][m];
        w[k] = acc;
    }
    return base;
}

}  // namespace pic
