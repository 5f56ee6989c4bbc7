/*
 * FP64 CPU oracle for the WT-scheme relativistic PIC step (Lu, Kilian, Guo, Li, Liang,
 * "Time-step dependent force interpolation scheme for suppressing numerical Cherenkov
 * instability in relativistic particle-in-cell simulations", arXiv:1909.09613).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
 * checked against.  It shares no code, header, table or constant with the CUDA library; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Everything is IEEE binary64, evaluated in the order the definitions are written (the file
 * is compiled with -ffp-contract=off so that no fused multiply-add changes the rounding).
 *
 * Code units (paper App. E, dimensionless system): c = 1, the 4*pi is absorbed, so
 *   du/dt = (q/m)(E + v x B),  dx/dt = v,  dE/dt = curl B - J,  dB/dt = -curl E,
 * with u = gamma*v the momentum per unit mass in units of c.
 *
 * Yee layout (standard reading of the half-grid offsets of Sec. 2, Eq. shapeEB-org):
 *   E1 (i+1/2, j, k)   E2 (i, j+1/2, k)   E3 (i, j, k+1/2)
 *   B1 (i, j+1/2, k+1/2)  B2 (i+1/2, j, k+1/2)  B3 (i+1/2, j+1/2, k)
 *   J co-located with E, rho at (i, j, k).
 * An array element [k][j][i] holds the value at the node whose integer parts are (i, j, k).
 * In 2D (nz = 1) every field is independent of x3 and the x3 interpolation factor is 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_SPECIES 4
#define ORC_MC 0
#define ORC_WT 1

/* ------------------------------------------------------------------------------------- */
/* 1-D interpolation functions                                                            */
/* ------------------------------------------------------------------------------------- */

/* Cardinal B-spline M_k on [0, k] by the textbook recurrence
 *   M_1 = indicator[0,1),  M_k(t) = ( t M_{k-1}(t) + (k - t) M_{k-1}(t - 1) ) / (k - 1).     */
static double cardinal_bspline(int k, double t)
{
    if (k == 1) return (t >= 0.0 && t < 1.0) ? 1.0 : 0.0;
    if (t <= 0.0 || t >= (double)k) return 0.0;
    return (t * cardinal_bspline(k - 1, t) + ((double)k - t) * cardinal_bspline(k - 1, t - 1.0))
           / (double)(k - 1);
}

/* W_l: the l-th order B-spline of width (l+1) cells, centred on 0 (Sec. 2, Eq. shape-real,
 * "W_l^(i) is the l-th order B-spline with width (l+1) dx_i").  Argument in cell units.     */
double orc_W(int l, double x)
{
    return cardinal_bspline(l + 1, x + 0.5 * (double)(l + 1));
}

/* T_l from its definition as the inverse Fourier transform of tau_l (Sec. 2, Eq. tau_l):
 * tau_l = sinc^l(k dx/2) * sinc(k c dt) is the product of the transform of W_{l-1} and of a
 * unit-area box of half-width c dt, so in cell units
 *   T_l(x; dtt) = 1/(2 dtt) * integral_{x-dtt}^{x+dtt} W_{l-1}(y) dy,  dtt = c dt / dx.
 * The integral is split at the knots of W_{l-1} (spacing 1, at -l/2 + j) and each polynomial
 * piece (degree l-1 <= 3) is integrated exactly by 4-point Gauss-Legendre.  This is valid for
 * any dtt > 0, including dtt > 1/2 where the paper's printed piecewise forms no longer apply. */
double orc_T(int l, double dtt, double x)
{
    static const double gx[4] = {-0.86113631159405257522, -0.33998104358485626480,
                                 0.33998104358485626480, 0.86113631159405257522};
    static const double gw[4] = {0.34785484513745385737, 0.65214515486254614263,
                                 0.65214515486254614263, 0.34785484513745385737};
    const double a = x - dtt, b = x + dtt;
    const double half = 0.5 * (double)l;       /* support of W_{l-1} is [-l/2, l/2] */
    double lo = a > -half ? a : -half;
    double hi = b < half ? b : half;
    if (hi <= lo) return 0.0;
    double sum = 0.0;
    double p = lo;
    while (p < hi) {
        /* next knot strictly above p */
        double q = ceil(p + half) - half;
        if (q <= p) q += 1.0;
        if (q > hi) q = hi;
        const double c = 0.5 * (p + q), h = 0.5 * (q - p);
        double s = 0.0;
        for (int g = 0; g < 4; ++g) s += gw[g] * orc_W(l - 1, c + h * gx[g]);
        sum += h * s;
        p = q;
    }
    return sum / (2.0 * dtt);
}

/* The paper's printed closed forms of T_1..T_4 (Sec. 2, the four piecewise equations below
 * Eq. tau_l), valid for 0 < dtt <= 1/2.  The outer piece of T_4 is read with 48*dtt in the
 * denominator (the printed "48 dt_i" lacks the tilde).  Kept as an independent routine so the
 * tests can pin orc_T against what the paper prints.                                       */
double orc_T_paper(int l, double d, double x)
{
    const double ax = fabs(x);
    switch (l) {
    case 1:
        if (ax <= 0.5 - d) return 1.0;
        if (ax <= 0.5 + d) return (1.0 + 2.0 * d - 2.0 * ax) / (4.0 * d);
        return 0.0;
    case 2:
        if (ax <= d) return (2.0 * d - d * d - x * x) / (2.0 * d);
        if (ax <= 1.0 - d) return 1.0 - ax;
        if (ax <= 1.0 + d) return (d + 1.0 - ax) * (d + 1.0 - ax) / (4.0 * d);
        return 0.0;
    case 3: {
        if (ax <= 0.5 - d) return (9.0 - 4.0 * d * d - 12.0 * x * x) / 12.0;
        if (ax <= 0.5 + d) {
            const double m = 1.0 - 2.0 * ax;
            return (-8.0 * d * d * d - 36.0 * d * d * m - 3.0 * m * m * m
                    + 6.0 * d * (15.0 - 12.0 * ax - 4.0 * x * x)) / (96.0 * d);
        }
        if (ax <= 1.5 - d) {
            const double m = 3.0 - 2.0 * ax;
            return (4.0 * d * d + 3.0 * m * m) / 24.0;
        }
        if (ax <= 1.5 + d) {
            const double m = 3.0 + 2.0 * d - 2.0 * ax;
            return m * m * m / (96.0 * d);
        }
        return 0.0;
    }
    case 4: {
        if (ax <= d)
            return (3.0 * x * x * x * x + d * (16.0 - 24.0 * x * x) + 18.0 * d * d * x * x
                    - 8.0 * d * d * d + 3.0 * d * d * d * d) / (24.0 * d);
        if (ax <= 1.0 - d)
            return (4.0 - 6.0 * x * x + 3.0 * ax * ax * ax - d * d * (2.0 - 3.0 * ax)) / 6.0;
        if (ax <= 1.0 + d) {
            const double m = 1.0 - ax;
            return (-m * m * m * m + 2.0 * d * (6.0 - 6.0 * ax + ax * ax * ax)
                    - 6.0 * d * d * m * m + 2.0 * d * d * d * ax - d * d * d * d) / (12.0 * d);
        }
        if (ax <= 2.0 - d) {
            const double m = 2.0 - ax;
            return m * (m * m + d * d) / 6.0;
        }
        if (ax <= 2.0 + d) {
            const double m = d + 2.0 - ax;
            return m * m * m * m / (48.0 * d);
        }
        return 0.0;
    }
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Simulation state                                                                       */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    double q, m, w;
    long n;
    double *x[3]; /* physical positions, [0, L_a) */
    double *u[3]; /* u = gamma v, units of c      */
} orc_species;

typedef struct {
    int dim;
    int n[3];
    double dx[3];
    double dt;
    int l;
    int scheme;
    long ncell;
    double *F[9]; /* E1 E2 E3 B1 B2 B3 J1 J2 J3 */
    int nsp;
    orc_species sp[ORC_MAX_SPECIES];
    long step;
    int m4;             /* 0: Yee Faraday stencil; 1: M4 (App. C) */
    double beta[3][3];  /* beta_ij of Eq. Maxwell-A */
    double delta[3];    /* delta_i of Eq. Maxwell-A */
} orc_sim;

static long wrapi(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

static long cidx(const orc_sim *s, long i, long j, long k)
{
    return (wrapi(k, s->n[2]) * s->n[1] + wrapi(j, s->n[1])) * s->n[0] + wrapi(i, s->n[0]);
}

orc_sim *orc_create(int nx, int ny, int nz, double dx, double dy, double dz, double dt, int l,
                    int scheme)
{
    if (nx < 1 || ny < 1 || nz < 1 || l < 1 || l > 4) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->dim = nz > 1 ? 3 : 2;
    s->n[0] = nx; s->n[1] = ny; s->n[2] = nz;
    s->dx[0] = dx; s->dx[1] = dy; s->dx[2] = (nz > 1) ? dz : 1.0;
    s->dt = dt;
    s->l = l;
    s->scheme = scheme;
    s->ncell = (long)nx * ny * nz;
    for (int c = 0; c < 9; ++c) s->F[c] = (double *)calloc((size_t)s->ncell, sizeof(double));
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    for (int c = 0; c < 9; ++c) free(s->F[c]);
    for (int p = 0; p < s->nsp; ++p)
        for (int a = 0; a < 3; ++a) { free(s->sp[p].x[a]); free(s->sp[p].u[a]); }
    free(s);
}

/* x: dim x n (SoA), u: 3 x n (SoA); physical units. Returns the species index or -1. */
int orc_add_species(orc_sim *s, double q, double m, double w, long n, const double *x,
                    const double *u)
{
    if (s->nsp >= ORC_MAX_SPECIES) return -1;
    orc_species *p = &s->sp[s->nsp];
    p->q = q; p->m = m; p->w = w; p->n = n;
    for (int a = 0; a < 3; ++a) {
        p->x[a] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        p->u[a] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (a < s->dim && n > 0) memcpy(p->x[a], x + (size_t)a * n, (size_t)n * sizeof(double));
        if (n > 0) memcpy(p->u[a], u + (size_t)a * n, (size_t)n * sizeof(double));
    }
    return s->nsp++;
}

void orc_set_field(orc_sim *s, int comp, const double *src)
{
    memcpy(s->F[comp], src, (size_t)s->ncell * sizeof(double));
}

void orc_get_field(const orc_sim *s, int comp, double *dst)
{
    memcpy(dst, s->F[comp], (size_t)s->ncell * sizeof(double));
}

void orc_get_particles(const orc_sim *s, int sp, double *x, double *u)
{
    const orc_species *p = &s->sp[sp];
    for (int a = 0; a < s->dim; ++a) memcpy(x + (size_t)a * p->n, p->x[a], (size_t)p->n * sizeof(double));
    for (int a = 0; a < 3; ++a) memcpy(u + (size_t)a * p->n, p->u[a], (size_t)p->n * sizeof(double));
}

void orc_set_particles(orc_sim *s, int sp, const double *x, const double *u)
{
    orc_species *p = &s->sp[sp];
    for (int a = 0; a < s->dim; ++a) memcpy(p->x[a], x + (size_t)a * p->n, (size_t)p->n * sizeof(double));
    for (int a = 0; a < 3; ++a) memcpy(p->u[a], u + (size_t)a * p->n, (size_t)p->n * sizeof(double));
}

long orc_step_count(const orc_sim *s) { return s->step; }

/* ------------------------------------------------------------------------------------- */
/* Field gather, Eq. interpolation-EB-real-org (MC) and Eq. interpolation-EB-real-mod (WT) */
/* ------------------------------------------------------------------------------------- */

/* Is field component comp (0..5 = E1,E2,E3,B1,B2,B3) offset by half a cell along axis a?
 * E_i is offset along i; B_i is offset along the two other axes.                          */
static int staggered(int comp, int a)
{
    return comp < 3 ? (a == comp) : (a != comp - 3);
}

/* 1-D factor of the interpolation function of component comp along axis a, for the node with
 * integer part n, at particle coordinate xt = x / dx_a.  Along an offset axis the node sits
 * at n + 1/2 and the factor is W_l; along a non-offset axis it is W_l (MC) or T_l (WT).      */
static double axis_factor(const orc_sim *s, int comp, int a, double xt, long n)
{
    if (staggered(comp, a)) return orc_W(s->l, xt - (double)n - 0.5);
    if (s->scheme == ORC_WT) return orc_T(s->l, s->dt / s->dx[a], xt - (double)n);
    return orc_W(s->l, xt - (double)n);
}

#define GWIN 12 /* nodes examined per axis: floor(xt)-5 .. floor(xt)+6 */

/* Windowed gather: sum over the nodes near the particle (weights vanish further away). */
void orc_gather(const orc_sim *s, const double *pos, double *eb)
{
    double xt[3] = {0, 0, 0};
    long base[3] = {0, 0, 0};
    for (int a = 0; a < s->dim; ++a) {
        xt[a] = pos[a] / s->dx[a];
        base[a] = (long)floor(xt[a]) - 5;
    }
    for (int comp = 0; comp < 6; ++comp) {
        double f[3][GWIN];
        for (int a = 0; a < 3; ++a)
            for (int t = 0; t < GWIN; ++t)
                f[a][t] = (a < s->dim) ? axis_factor(s, comp, a, xt[a], base[a] + t) : (t == 0 ? 1.0 : 0.0);
        const int n3 = (s->dim == 3) ? GWIN : 1;
        double acc = 0.0;
        for (int t3 = 0; t3 < n3; ++t3)
            for (int t2 = 0; t2 < GWIN; ++t2)
                for (int t1 = 0; t1 < GWIN; ++t1) {
                    const double wgt = f[0][t1] * f[1][t2] * f[2][t3];
                    if (wgt == 0.0) continue;
                    acc += wgt * s->F[comp][cidx(s, base[0] + t1, base[1] + t2, s->dim == 3 ? base[2] + t3 : 0)];
                }
        eb[comp] = acc;
    }
}

/* Brute-force gather: every grid node and its +-1 periodic images, no window.  Used only to
 * check the windowed gather on small grids.                                                */
void orc_gather_brute(const orc_sim *s, const double *pos, double *eb)
{
    double xt[3] = {0, 0, 0};
    for (int a = 0; a < s->dim; ++a) xt[a] = pos[a] / s->dx[a];
    for (int comp = 0; comp < 6; ++comp) {
        double acc = 0.0;
        const int nk = (s->dim == 3) ? s->n[2] : 1;
        for (long k = 0; k < nk; ++k)
            for (long j = 0; j < s->n[1]; ++j)
                for (long i = 0; i < s->n[0]; ++i) {
                    double f1 = 0, f2 = 0, f3 = 1.0;
                    for (int m = -1; m <= 1; ++m) f1 += axis_factor(s, comp, 0, xt[0], i + (long)m * s->n[0]);
                    for (int m = -1; m <= 1; ++m) f2 += axis_factor(s, comp, 1, xt[1], j + (long)m * s->n[1]);
                    if (s->dim == 3) {
                        f3 = 0.0;
                        for (int m = -1; m <= 1; ++m) f3 += axis_factor(s, comp, 2, xt[2], k + (long)m * s->n[2]);
                    }
                    acc += f1 * f2 * f3 * s->F[comp][(k * s->n[1] + j) * s->n[0] + i];
                }
        eb[comp] = acc;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Relativistic Boris push (Sec. 1 names the Boris algorithm; equations of motion App. E)  */
/* ------------------------------------------------------------------------------------- */

/* u in: u^{n-1/2}; out: u^{n+1/2}.  qmdt = q dt / m. */
void orc_boris(double qmdt, const double *E, const double *B, double *u)
{
    const double h = 0.5 * qmdt;
    double um[3], up[3], t[3], sv[3], uprime[3];
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) sv[a] = 2.0 * t[a] / (1.0 + t2);
    uprime[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    uprime[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    uprime[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
    up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
    up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
    for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];
}

/* ------------------------------------------------------------------------------------- */
/* Esirkepov charge-conserving deposit (Sec. 1 and Sec. 2: the unique combination of       */
/* form-factor differences consistent with discrete continuity; charge form factor W_l).   */
/* ------------------------------------------------------------------------------------- */

#define DWIN 8 /* window floor(x_old)-3 .. floor(x_old)+4 covers l <= 4 and |dx| < 1 cell */

/* Deposit the current of one particle moving from xo to xn (physical, xn NOT wrapped) with
 * velocity v (needed for the out-of-plane component in 2D).  Adds into J1, J2, J3.         */
void orc_deposit(orc_sim *s, double qw, const double *xo, const double *xn, const double *v)
{
    double S0[3][DWIN], S1[3][DWIN], DS[3][DWIN];
    long base[3] = {0, 0, 0};
    const double vc = s->dx[0] * s->dx[1] * (s->dim == 3 ? s->dx[2] : 1.0);
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < DWIN; ++t) { S0[a][t] = 0.0; S1[a][t] = 0.0; DS[a][t] = 0.0; }
    for (int a = 0; a < s->dim; ++a) {
        const double xo_t = xo[a] / s->dx[a], xn_t = xn[a] / s->dx[a];
        base[a] = (long)floor(xo_t) - 3;
        for (int t = 0; t < DWIN; ++t) {
            const double node = (double)(base[a] + t);
            S0[a][t] = orc_W(s->l, xo_t - node);
            S1[a][t] = orc_W(s->l, xn_t - node);
            DS[a][t] = S1[a][t] - S0[a][t];
        }
    }
    if (s->dim == 2) {
        const double cx = -qw * s->dx[0] / (vc * s->dt);
        const double cy = -qw * s->dx[1] / (vc * s->dt);
        const double cz = qw * v[2] / vc;
        for (int tj = 0; tj < DWIN; ++tj) {
            double acc = 0.0;
            for (int ti = 0; ti < DWIN; ++ti) {
                acc += DS[0][ti] * (S0[1][tj] + 0.5 * DS[1][tj]);       /* W_x */
                if (acc != 0.0) s->F[6][cidx(s, base[0] + ti, base[1] + tj, 0)] += cx * acc;
            }
        }
        for (int ti = 0; ti < DWIN; ++ti) {
            double acc = 0.0;
            for (int tj = 0; tj < DWIN; ++tj) {
                acc += DS[1][tj] * (S0[0][ti] + 0.5 * DS[0][ti]);       /* W_y */
                if (acc != 0.0) s->F[7][cidx(s, base[0] + ti, base[1] + tj, 0)] += cy * acc;
            }
        }
        for (int tj = 0; tj < DWIN; ++tj)
            for (int ti = 0; ti < DWIN; ++ti) {
                const double wz = S0[0][ti] * S0[1][tj] + 0.5 * DS[0][ti] * S0[1][tj]
                                  + 0.5 * S0[0][ti] * DS[1][tj] + DS[0][ti] * DS[1][tj] / 3.0;
                if (wz != 0.0) s->F[8][cidx(s, base[0] + ti, base[1] + tj, 0)] += cz * wz;
            }
        return;
    }
    /* 3D: W_x = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3) and cyclic. */
    const double cf[3] = {-qw * s->dx[0] / (vc * s->dt), -qw * s->dx[1] / (vc * s->dt),
                          -qw * s->dx[2] / (vc * s->dt)};
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int tb = 0; tb < DWIN; ++tb)
            for (int tc = 0; tc < DWIN; ++tc) {
                const double perp = S0[b][tb] * S0[c][tc] + 0.5 * DS[b][tb] * S0[c][tc]
                                    + 0.5 * S0[b][tb] * DS[c][tc] + DS[b][tb] * DS[c][tc] / 3.0;
                double acc = 0.0;
                for (int ta = 0; ta < DWIN; ++ta) {
                    acc += DS[a][ta] * perp;
                    if (acc == 0.0) continue;
                    long t[3];
                    t[a] = base[a] + ta; t[b] = base[b] + tb; t[c] = base[c] + tc;
                    s->F[6 + a][cidx(s, t[0], t[1], t[2])] += cf[a] * acc;
                }
            }
    }
}

/* Charge density of all particles at their current positions, rho = sum q w W_l / V_c
 * (Sec. 2, Eq. shape-real). */
void orc_rho(const orc_sim *s, double *rho)
{
    memset(rho, 0, (size_t)s->ncell * sizeof(double));
    const double vc = s->dx[0] * s->dx[1] * (s->dim == 3 ? s->dx[2] : 1.0);
    for (int sp = 0; sp < s->nsp; ++sp) {
        const orc_species *p = &s->sp[sp];
        for (long i = 0; i < p->n; ++i) {
            double S[3][DWIN];
            long base[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a)
                for (int t = 0; t < DWIN; ++t) S[a][t] = (t == 0) ? 1.0 : 0.0;
            for (int a = 0; a < s->dim; ++a) {
                const double xt = p->x[a][i] / s->dx[a];
                base[a] = (long)floor(xt) - 3;
                for (int t = 0; t < DWIN; ++t) S[a][t] = orc_W(s->l, xt - (double)(base[a] + t));
            }
            const int n3 = s->dim == 3 ? DWIN : 1;
            for (int t3 = 0; t3 < n3; ++t3)
                for (int t2 = 0; t2 < DWIN; ++t2)
                    for (int t1 = 0; t1 < DWIN; ++t1) {
                        const double wgt = S[0][t1] * S[1][t2] * S[2][t3];
                        if (wgt != 0.0)
                            rho[cidx(s, base[0] + t1, base[1] + t2, base[2] + t3)] += p->q * p->w * wgt / vc;
                    }
        }
    }
}

/* ------------------------------------------------------------------------------------- */
/* Yee FDTD (Sec. 1; "Yee solver", all beta = delta = 0 in Eq. Maxwell-A), periodic        */
/* ------------------------------------------------------------------------------------- */

/* Select the Faraday stencil: Yee (all beta = delta = 0) or M4, the fourth-order-dispersion
 * choice of App. C: beta_ij = (c dt/dx_j)^2 / 12, delta_i = ((c dt/dx_i)^2 - 1) / 12 (the last
 * equation of App. C).  Ampere's stencil is never modified. */
void orc_set_solver(orc_sim *s, int m4)
{
    s->m4 = m4;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            const double r = s->dt / s->dx[j];
            s->beta[i][j] = (m4 && i != j) ? r * r / 12.0 : 0.0;
        }
        const double r = s->dt / s->dx[i];
        s->delta[i] = m4 ? (r * r - 1.0) / 12.0 : 0.0;
    }
}

/* Forward difference of E component c along axis a at node (i, j, k):
 * (E_c(node + e_a) - E_c(node)) / dx_a. */
static double fdiff(const orc_sim *s, int c, int a, long i, long j, long k)
{
    long ii = i, jj = j, kk = k;
    if (a == 0) ii++;
    else if (a == 1) jj++;
    else kk++;
    return (s->F[c][cidx(s, ii, jj, kk)] - s->F[c][cidx(s, i, j, k)]) / s->dx[a];
}

/* Faraday's derivative of E component c along axis a at node (i, j, k).  Its Fourier symbol is
 * A_a times that of the Yee difference (Eq. Maxwell-A):
 *   A_a = 1 - 2 sum_{b != a} beta_ab [1 - cos(k_b dx_b)] - 2 delta_a [1 - cos(k_a dx_a)],
 * and -2 [1 - cos(k dx)] is the symbol of the second difference f(+1) - 2 f + f(-1), so the
 * derivative is the Yee difference plus beta_ab times its second difference along b and
 * delta_a times its second difference along a. */
static double fdiff_faraday(const orc_sim *s, int c, int a, long i, long j, long k)
{
    const double d0 = fdiff(s, c, a, i, j, k);
    if (!s->m4) return d0;
    double r = d0;
    for (int b = 0; b < 3; ++b) {
        const double coef = (b == a) ? s->delta[a] : s->beta[a][b];
        if (coef == 0.0) continue;
        const long di = (b == 0), dj = (b == 1), dk = (b == 2);
        const double dp = fdiff(s, c, a, i + di, j + dj, k + dk);
        const double dm = fdiff(s, c, a, i - di, j - dj, k - dk);
        r += coef * (dp - 2.0 * d0 + dm);
    }
    return r;
}

/* B <- B - h * curl E  (h = dt/2 for each half push), curl with Faraday's stencil. */
void orc_yee_b(orc_sim *s, double h)
{
    double *B1 = s->F[3], *B2 = s->F[4], *B3 = s->F[5];
    const long nc = s->ncell;
    double *c1 = (double *)malloc((size_t)nc * sizeof(double));
    double *c2 = (double *)malloc((size_t)nc * sizeof(double));
    double *c3 = (double *)malloc((size_t)nc * sizeof(double));
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i) {
                const long c = cidx(s, i, j, k);
                c1[c] = fdiff_faraday(s, 2, 1, i, j, k) - fdiff_faraday(s, 1, 2, i, j, k);
                c2[c] = fdiff_faraday(s, 0, 2, i, j, k) - fdiff_faraday(s, 2, 0, i, j, k);
                c3[c] = fdiff_faraday(s, 1, 0, i, j, k) - fdiff_faraday(s, 0, 1, i, j, k);
            }
    for (long c = 0; c < nc; ++c) {
        B1[c] -= h * c1[c];
        B2[c] -= h * c2[c];
        B3[c] -= h * c3[c];
    }
    free(c1); free(c2); free(c3);
}

/* E <- E + dt curl B - dt J. */
void orc_yee_e(orc_sim *s)
{
    double *E1 = s->F[0], *E2 = s->F[1], *E3 = s->F[2];
    double *B1 = s->F[3], *B2 = s->F[4], *B3 = s->F[5];
    double *J1 = s->F[6], *J2 = s->F[7], *J3 = s->F[8];
    const double dx = s->dx[0], dy = s->dx[1], dz = s->dx[2], dt = s->dt;
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i) {
                const long c = cidx(s, i, j, k);
                const double c1 = (B3[c] - B3[cidx(s, i, j - 1, k)]) / dy - (B2[c] - B2[cidx(s, i, j, k - 1)]) / dz;
                const double c2 = (B1[c] - B1[cidx(s, i, j, k - 1)]) / dz - (B3[c] - B3[cidx(s, i - 1, j, k)]) / dx;
                const double c3 = (B2[c] - B2[cidx(s, i - 1, j, k)]) / dx - (B1[c] - B1[cidx(s, i, j - 1, k)]) / dy;
                E1[c] += dt * c1 - dt * J1[c];
                E2[c] += dt * c2 - dt * J2[c];
                E3[c] += dt * c3 - dt * J3[c];
            }
}

/* ------------------------------------------------------------------------------------- */
/* One PIC step                                                                           */
/* ------------------------------------------------------------------------------------- */

/* Particle part of one step for one species: gather at x^n from E^n, B^n; Boris
 * u^{n-1/2} -> u^{n+1/2}; move x^{n+1} = x^n + dt u/gamma; Esirkepov deposit into J.   */
static void push_species(orc_sim *s, orc_species *p, long first, long count)
{
    const double qmdt = p->q * s->dt / p->m;
    const double qw = p->q * p->w;
    for (long i = first; i < first + count; ++i) {
        double xo[3] = {0, 0, 0}, xn[3] = {0, 0, 0}, eb[6], u[3], v[3];
        for (int a = 0; a < s->dim; ++a) xo[a] = p->x[a][i];
        orc_gather(s, xo, eb);
        for (int a = 0; a < 3; ++a) u[a] = p->u[a][i];
        orc_boris(qmdt, eb, eb + 3, u);
        const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) v[a] = u[a] / g;
        for (int a = 0; a < s->dim; ++a) xn[a] = xo[a] + s->dt * v[a];
        orc_deposit(s, qw, xo, xn, v);
        for (int a = 0; a < 3; ++a) p->u[a][i] = u[a];
        for (int a = 0; a < s->dim; ++a) {
            const double L = s->n[a] * s->dx[a];
            double x = xn[a];
            if (x >= L) x -= L;
            else if (x < 0.0) x += L;
            p->x[a][i] = x;
        }
    }
}

/* Gather at x^n, Boris u^{n-1/2} -> u^{n+1/2}, move x^{n+1} = x^n + dt u/gamma (wrapped) for
 * one particle of charge q and mass m, without depositing: the particle half of a step for a
 * sampled particle.  x: dim physical coordinates (updated), u: 3 (updated).               */
void orc_push_particle(const orc_sim *s, double q, double m, double *x, double *u)
{
    double xo[3] = {0, 0, 0}, eb[6];
    for (int a = 0; a < s->dim; ++a) xo[a] = x[a];
    orc_gather(s, xo, eb);
    orc_boris(q * s->dt / m, eb, eb + 3, u);
    const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < s->dim; ++a) {
        const double L = s->n[a] * s->dx[a];
        double xn = xo[a] + s->dt * (u[a] / g);
        if (xn >= L) xn -= L;
        else if (xn < 0.0) xn += L;
        x[a] = xn;
    }
}

/* Advance nsteps full PIC steps: particles, then B half, E full, B half. */
void orc_step(orc_sim *s, int nsteps)
{
    for (int it = 0; it < nsteps; ++it) {
        for (int c = 6; c < 9; ++c) memset(s->F[c], 0, (size_t)s->ncell * sizeof(double));
        for (int sp = 0; sp < s->nsp; ++sp) push_species(s, &s->sp[sp], 0, s->sp[sp].n);
        orc_yee_b(s, 0.5 * s->dt);
        orc_yee_e(s);
        orc_yee_b(s, 0.5 * s->dt);
        s->step++;
    }
}

/* Particle part of one step only (J zeroed first), on a contiguous sample of each species.
 * Used for the CPU-baseline timing, which measures the gather+push+deposit rate.          */
void orc_particle_pass(orc_sim *s, long first, long count)
{
    for (int c = 6; c < 9; ++c) memset(s->F[c], 0, (size_t)s->ncell * sizeof(double));
    for (int sp = 0; sp < s->nsp; ++sp) {
        long n = s->sp[sp].n - first;
        if (n > count) n = count;
        if (n > 0) push_species(s, &s->sp[sp], first, n);
    }
}

/* Particle pass of particles first .. first + count - 1 of every species over `threads` host
 * threads (the timing build, compiled with OpenMP; without it one thread does all): each
 * thread pushes a contiguous share of the particles and deposits into a private copy of J,
 * and the copies are then added into J in thread order.  The arithmetic of every particle is
 * that of push_species.  Returns the number of threads used.                              */
int orc_particle_pass_threads(orc_sim *s, long first, long count, int threads)
{
    for (int c = 6; c < 9; ++c) memset(s->F[c], 0, (size_t)s->ncell * sizeof(double));
#ifdef _OPENMP
    if (threads < 1) threads = omp_get_max_threads();
#else
    threads = 1;
#endif
    double *priv = (double *)calloc((size_t)threads * 3 * (size_t)s->ncell, sizeof(double));
    if (!priv) return 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#else
        const int t = 0, nt = 1;
#endif
        orc_sim local = *s;
        for (int c = 0; c < 3; ++c) local.F[6 + c] = priv + ((size_t)t * 3 + c) * (size_t)s->ncell;
        for (int sp = 0; sp < s->nsp; ++sp) {
            long n = s->sp[sp].n - first;
            if (n > count) n = count;
            if (n <= 0) continue;
            const long a = first + n * t / nt, b = first + n * (t + 1) / nt;
            if (b > a) push_species(&local, &local.sp[sp], a, b - a);
        }
    }
    for (int t = 0; t < threads; ++t)
        for (int c = 0; c < 3; ++c) {
            const double *src = priv + ((size_t)t * 3 + c) * (size_t)s->ncell;
            for (long i = 0; i < s->ncell; ++i) s->F[6 + c][i] += src[i];
        }
    free(priv);
    return threads;
}

/* ------------------------------------------------------------------------------------- */
/* Diagnostics                                                                            */
/* ------------------------------------------------------------------------------------- */

/* out[0] = field energy 1/2 sum (E^2 + B^2) V_c; out[1] = kinetic energy sum w m (gamma-1);
 * out[2] = total charge sum q w; out[3] = max |D.E - rho| over nodes (App. B, Eq. gauss).   */
void orc_diag(const orc_sim *s, double *out)
{
    const double vc = s->dx[0] * s->dx[1] * (s->dim == 3 ? s->dx[2] : 1.0);
    double ue = 0.0;
    for (int c = 0; c < 6; ++c)
        for (long i = 0; i < s->ncell; ++i) ue += s->F[c][i] * s->F[c][i];
    out[0] = 0.5 * ue * vc;
    double ke = 0.0, qt = 0.0;
    for (int sp = 0; sp < s->nsp; ++sp) {
        const orc_species *p = &s->sp[sp];
        for (long i = 0; i < p->n; ++i) {
            const double g = sqrt(1.0 + p->u[0][i] * p->u[0][i] + p->u[1][i] * p->u[1][i] + p->u[2][i] * p->u[2][i]);
            ke += p->w * p->m * (g - 1.0);
        }
        qt += p->q * p->w * (double)p->n;
    }
    out[1] = ke;
    out[2] = qt;
    double *rho = (double *)malloc((size_t)s->ncell * sizeof(double));
    orc_rho(s, rho);
    double mx = 0.0;
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i) {
                const long c = cidx(s, i, j, k);
                double dv = (s->F[0][c] - s->F[0][cidx(s, i - 1, j, k)]) / s->dx[0]
                            + (s->F[1][c] - s->F[1][cidx(s, i, j - 1, k)]) / s->dx[1];
                if (s->dim == 3) dv += (s->F[2][c] - s->F[2][cidx(s, i, j, k - 1)]) / s->dx[2];
                const double r = fabs(dv - rho[c]);
                if (r > mx) mx = r;
            }
    out[3] = mx;
    free(rho);
}

/* D.E - rho at every node (for the Gauss-law conservation pin). */
void orc_gauss_residual(const orc_sim *s, double *res)
{
    double *rho = (double *)malloc((size_t)s->ncell * sizeof(double));
    orc_rho(s, rho);
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i) {
                const long c = cidx(s, i, j, k);
                double dv = (s->F[0][c] - s->F[0][cidx(s, i - 1, j, k)]) / s->dx[0]
                            + (s->F[1][c] - s->F[1][cidx(s, i, j - 1, k)]) / s->dx[1];
                if (s->dim == 3) dv += (s->F[2][c] - s->F[2][cidx(s, i, j, k - 1)]) / s->dx[2];
                res[c] = dv - rho[c];
            }
    free(rho);
}

/* ------------------------------------------------------------------------------------- */
/* Particle tile sort (not in the paper; the layout the GPU path streams particles in)     */
/* ------------------------------------------------------------------------------------- */

/* Sort orders: cells are grouped into tiles of tile[0] x tile[1] (x tile[2]) cells (ragged at
 * the high edge); the tiles are numbered x-fastest, and so are the cells inside a tile.  Each
 * particle's slot is its rank among the particles of its cell in the input order.
 *   order 0 ("cell-major"): by (tile, cell-in-tile, slot);
 *   order 1 ("slot-major"): by (tile, slot, cell-in-tile), i.e. a tile runs through groups
 *   holding one particle of every cell that has more than `slot` particles.
 * In both, the cell at every output position is fixed by the cell counts alone.
 *
 * cell_of[i] = linear cell index (k*ny + j)*nx + i of particle i (input, computed by the
 * caller as floor(x/dx) per axis).  Outputs: perm[p] = input index placed at position p;
 * tile_start[t] = first position of tile t (ntiles + 1 entries).                           */
typedef struct { long tile, slot, cell, idx; } sort_rec;

static int sort_rec_cmp_cell(const void *pa, const void *pb)
{
    const sort_rec *a = (const sort_rec *)pa, *b = (const sort_rec *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

static int sort_rec_cmp_slot(const void *pa, const void *pb)
{
    const sort_rec *a = (const sort_rec *)pa, *b = (const sort_rec *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

long orc_tile_sort(const int *n, const int *tile, int order, long np, const long *cell_of,
                   long *perm, long *tile_start)
{
    const long nx = n[0], ny = n[1], nz = n[2];
    const long tx = tile[0], ty = tile[1], tz = tile[2];
    const long ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
    const long ntiles = ntx * nty * ntz;
    const long ncell = nx * ny * nz;
    long *cnt = (long *)calloc((size_t)ncell, sizeof(long));
    sort_rec *r = (sort_rec *)malloc((size_t)(np > 0 ? np : 1) * sizeof(sort_rec));
    for (long p = 0; p < np; ++p) {
        const long c = cell_of[p];
        const long i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        const long ti = i / tx, tj = j / ty, tk = k / tz;
        r[p].tile = (tk * nty + tj) * ntx + ti;
        /* cell-in-tile, x fastest, numbered with the full tile extent */
        r[p].cell = ((k - tk * tz) * ty + (j - tj * ty)) * tx + (i - ti * tx);
        r[p].slot = cnt[c]++;
        r[p].idx = p;
    }
    qsort(r, (size_t)np, sizeof(sort_rec), order == 1 ? sort_rec_cmp_slot : sort_rec_cmp_cell);
    for (long t = 0; t <= ntiles; ++t) tile_start[t] = 0;
    for (long p = 0; p < np; ++p) {
        perm[p] = r[p].idx;
        tile_start[r[p].tile + 1]++;
    }
    for (long t = 0; t < ntiles; ++t) tile_start[t + 1] += tile_start[t];
    free(cnt);
    free(r);
    return ntiles;
}

/* ------------------------------------------------------------------------------------- */
/* Particle loading: drifting plasma of App. D                                            */
/* ------------------------------------------------------------------------------------- */

/* Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the state advances by the odd constant
 * 0x9E3779B97F4A7C15 and each output is the state passed through the 64-bit finaliser below.
 * Value k of a stream with key K is mix(k * 0x9E3779B97F4A7C15 + K); a uniform deviate on
 * [0, 1) takes its 53 high bits.  Stream keys chain the finaliser over the stream's ids:
 * K = mix(... mix(mix(seed + G) ^ ((id_0 + 1) G)) ^ ((id_1 + 1) G) ...), G the constant above
 * (the schedule the library documents for its device loader).                              */
typedef unsigned long long u64;
static const u64 SM64_GAMMA = 0x9E3779B97F4A7C15ull;

static u64 sm64_finalise(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static u64 stream_key3(u64 seed, u64 a, u64 b, u64 c)
{
    u64 k = sm64_finalise(seed + SM64_GAMMA);
    k = sm64_finalise(k ^ ((a + 1) * SM64_GAMMA));
    k = sm64_finalise(k ^ ((b + 1) * SM64_GAMMA));
    k = sm64_finalise(k ^ ((c + 1) * SM64_GAMMA));
    return k;
}

static double uniform01(u64 key, u64 ctr)
{
    return (double)(sm64_finalise(ctr * SM64_GAMMA + key) >> 11) * (1.0 / 9007199254740992.0);
}

#define ORC_JUTTNER_ATTEMPTS 128

/* |u'| of the Juttner-Synge distribution of Eq. Maxwell-dist-relativistic (temperature
 * theta = k_B T / (m c^2), u' = p'/(m c)) by Sobol's rejection method: with X1..X4 uniform on
 * (0, 1], u = -theta ln(X1 X2 X3) and eta = -theta ln(X1 X2 X3 X4); the pair is accepted when
 * eta^2 - u^2 > 1, and u then has density proportional to u^2 exp(-sqrt(1 + u^2) / theta).
 * Attempt a (a < attempts <= ORC_JUTTNER_ATTEMPTS) of particle p uses counter
 * p * ORC_JUTTNER_ATTEMPTS + a.  Returns -1 when every attempt was rejected.              */
static double juttner_speed(double theta, const u64 *key, u64 p, int attempts)
{
    for (int a = 0; a < attempts; ++a) {
        const u64 ctr = p * ORC_JUTTNER_ATTEMPTS + (u64)a;
        double X[4];
        for (int j = 0; j < 4; ++j) X[j] = 1.0 - uniform01(key[j], ctr);
        const double prod3 = X[0] * X[1] * X[2];
        const double u = -theta * log(prod3);
        const double eta = -theta * log(prod3 * X[3]);
        if (eta * eta - u * u > 1.0) return u;
    }
    return -1.0;
}

/* Particles p0 .. p0 + m - 1 of one species of a plasma drifting along x1 (App. D, n = e_1):
 *   - particle p sits in cell p / per_cell (cells numbered x1 fastest) at uniform offsets
 *     U(key(seed, run, pos_species, 10 + a), p) per axis a;
 *   - co-moving momentum u' = p'/(m c): theta > 0 draws the Juttner-Synge speed above with an
 *     isotropic direction (cos = 2 X5 - 1, azimuth 2 pi X6, X5 and X6 at counter p of streams
 *     (run, species, 44) and (run, species, 45)); otherwise each component is u_th times a
 *     standard normal by Box-Muller, sqrt(-2 ln U1) cos(2 pi U2) with U1 = 1 - U(key(..,
 *     20 + 2a), p) in (0, 1] and U2 = U(key(.., 21 + 2a), p) (the Maxwell-Boltzmann limit,
 *     Eq. Maxwell-dist-non-relativistic); u_th = 0 and theta = 0 give u' = 0;
 *   - the volume transform of App. D by flipping instead of rejecting: with X1 = U(key(..,
 *     30), p) and E' = sqrt(1 + u'^2), u'_1 -> -u'_1 when X1 > (1 + beta u'_1 / E') / 2 (the
 *     reading of the flip rule under which the loaded density carries the weight
 *     1 + beta u'_1 / E' that App. D requires);
 *   - the Lorentz transform of App. D along n = e_1: u_1 = gamma (u'_1 + beta E'), the
 *     transverse components unchanged, beta = sqrt(1 - 1 / gamma^2).  For u' = 0 this is the
 *     cold beam u = (gamma beta, 0, 0), written as sqrt(gamma^2 - 1).
 * x: dim x m physical positions (SoA), u: 3 x m.  Returns the number of particles for which no
 * Sobol attempt was accepted (they are loaded at rest in the co-moving frame).              */
long orc_load_drifting(int dim, const int *n, const double *dx, long per_cell, long p0, long m,
                       double gamma, double u_th, double theta, u64 seed, u64 run, int species,
                       int pos_species, double *x, double *u)
{
    u64 kpos[3], kmom[6], kjut[4], kdir[2];
    for (int a = 0; a < 3; ++a) {
        kpos[a] = stream_key3(seed, run, (u64)pos_species, (u64)(10 + a));
        kmom[2 * a] = stream_key3(seed, run, (u64)species, (u64)(20 + 2 * a));
        kmom[2 * a + 1] = stream_key3(seed, run, (u64)species, (u64)(21 + 2 * a));
    }
    const u64 kflip = stream_key3(seed, run, (u64)species, 30);
    for (int j = 0; j < 4; ++j) kjut[j] = stream_key3(seed, run, (u64)species, (u64)(40 + j));
    kdir[0] = stream_key3(seed, run, (u64)species, 44);
    kdir[1] = stream_key3(seed, run, (u64)species, 45);
    const double beta = sqrt(1.0 - 1.0 / (gamma * gamma));
    const double two_pi = 6.28318530717958647692;  /* 2 pi */
    long failed = 0;
    for (long i = 0; i < m; ++i) {
        const long p = p0 + i;
        const long cell = p / per_cell;
        long ci[3];
        ci[0] = cell % n[0];
        ci[1] = (cell / n[0]) % n[1];
        ci[2] = cell / ((long)n[0] * n[1]);
        for (int a = 0; a < dim; ++a) {
            const double L = (double)n[a] * dx[a];
            double xa = ((double)ci[a] + uniform01(kpos[a], (u64)p)) * dx[a];
            if (xa >= L) xa -= L;
            x[(long)a * m + i] = xa;
        }
        if (theta > 0.0 || u_th > 0.0) {
            double v[3];
            if (theta > 0.0) {
                double um = juttner_speed(theta, kjut, (u64)p, ORC_JUTTNER_ATTEMPTS);
                if (um < 0.0) {
                    ++failed;
                    um = 0.0;
                }
                const double x5 = uniform01(kdir[0], (u64)p), x6 = uniform01(kdir[1], (u64)p);
                const double cos_t = 2.0 * x5 - 1.0;
                /* sin = sqrt(1 - cos^2) = 2 sqrt(X5 (1 - X5)), the form without cancellation */
                const double sin_t = 2.0 * sqrt(x5 * (1.0 - x5));
                const double phi = two_pi * x6;
                v[0] = um * cos_t;
                v[1] = um * sin_t * cos(phi);
                v[2] = um * sin_t * sin(phi);
            } else {
                for (int a = 0; a < 3; ++a) {
                    const double U1 = 1.0 - uniform01(kmom[2 * a], (u64)p);
                    const double U2 = uniform01(kmom[2 * a + 1], (u64)p);
                    v[a] = u_th * (sqrt(-2.0 * log(U1)) * cos(two_pi * U2));
                }
            }
            const double e_prime = sqrt(1.0 + (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            const double X1 = uniform01(kflip, (u64)p);
            const double v1 = (X1 > 0.5 * (1.0 + beta * v[0] / e_prime)) ? -v[0] : v[0];
            u[i] = gamma * (v1 + beta * e_prime);
            u[m + i] = v[1];
            u[2 * m + i] = v[2];
        } else {
            u[i] = sqrt(gamma * gamma - 1.0);
            u[m + i] = 0.0;
            u[2 * m + i] = 0.0;
        }
    }
    return failed;
}

/* The Juttner-Synge speeds alone (the co-moving |u'| of particles p0 .. p0 + m - 1 of one
 * species' streams) with at most `attempts` Sobol attempts each; -1 where none was accepted. */
void orc_juttner_speeds(double theta, int attempts, u64 seed, u64 run, int species, long p0,
                        long m, double *out)
{
    u64 kjut[4];
    for (int j = 0; j < 4; ++j) kjut[j] = stream_key3(seed, run, (u64)species, (u64)(40 + j));
    if (attempts > ORC_JUTTNER_ATTEMPTS) attempts = ORC_JUTTNER_ATTEMPTS;
    for (long i = 0; i < m; ++i) out[i] = juttner_speed(theta, kjut, (u64)(p0 + i), attempts);
}
