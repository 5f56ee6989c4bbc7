// Device bodies of the periodic Yee update (Sec. 1 Yee grid; App. C with A_i = 1), shared
// by the single-run launches (pic_grid.cu) and the batched launches (pic_batch.cu).
#pragma once
#include "pic_common.cuh"

namespace pic {

__device__ __forceinline__ int64_t gidx(const RunDev &rd, int i, int j, int k)
{
    return ((int64_t)k * rd.n[1] + j) * rd.n[0] + i;
}

// Forward difference of E component ec along axis a at node (i, j, k), periodic.
__device__ __forceinline__ double fdiff_e(const RunDev &rd, int ec, int a, int i, int j, int k)
{
    int ip = i, jp = j, kp = k;
    if (a == 0) ip = (i + 1 == rd.n[0]) ? 0 : i + 1;
    else if (a == 1) jp = (j + 1 == rd.n[1]) ? 0 : j + 1;
    else kp = (k + 1 == rd.n[2]) ? 0 : k + 1;
    return (rd.F[ec][gidx(rd, ip, jp, kp)] - rd.F[ec][gidx(rd, i, j, k)]) * rd.idx[a];
}

// Cell (i, j, k) of linear cell index c (c < 2^30).
__device__ __forceinline__ void cell_ijk(const RunDev &rd, int64_t c, int &i, int &j, int &k)
{
    const int ci = (int)c;
    k = fast_div(ci, rd.div_n01.m, rd.div_n01.s);
    const int r = ci - k * rd.n[0] * rd.n[1];
    j = fast_div(r, rd.div_n0.m, rd.div_n0.s);
    i = r - j * rd.n[0];
}

// Faraday's derivative of E component ec along axis a at node (i, j, k).  Yee: the forward
// difference.  M4 (App. C): its Fourier symbol is A_a times the Yee one (Eq. Maxwell-A), i.e. the
// Yee difference plus beta_ab times its second difference along each other axis b and delta_a
// times its second difference along a.
__device__ __forceinline__ double faraday_d(const RunDev &rd, int ec, int a, int i, int j, int k)
{
    const double d0 = fdiff_e(rd, ec, a, i, j, k);
    if (!rd.m4) return d0;
    double r = d0;
    for (int b = 0; b < 3; ++b) {
        const double coef = (b == a) ? rd.delta[a] : rd.beta[a][b];
        if (coef == 0.0 || rd.n[b] == 1) continue;
        int ip = i, jp = j, kp = k, im = i, jm = j, km = k;
        if (b == 0) { ip = (i + 1 == rd.n[0]) ? 0 : i + 1; im = (i == 0) ? rd.n[0] - 1 : i - 1; }
        else if (b == 1) { jp = (j + 1 == rd.n[1]) ? 0 : j + 1; jm = (j == 0) ? rd.n[1] - 1 : j - 1; }
        else { kp = (k + 1 == rd.n[2]) ? 0 : k + 1; km = (k == 0) ? rd.n[2] - 1 : k - 1; }
        r += coef * (fdiff_e(rd, ec, a, ip, jp, kp) - 2.0 * d0 + fdiff_e(rd, ec, a, im, jm, km));
    }
    return r;
}

// B <- B - h curl E at cell c (FP32 shadow of B written when `shadow`).
__device__ __forceinline__ void yee_b_cell(const RunDev &rd, int64_t c, double h, int shadow)
{
    int i, j, k;
    cell_ijk(rd, c, i, j, k);
    double c1, c2, c3;
    if (rd.m4) {
        c1 = faraday_d(rd, 2, 1, i, j, k) - faraday_d(rd, 1, 2, i, j, k);
        c2 = faraday_d(rd, 0, 2, i, j, k) - faraday_d(rd, 2, 0, i, j, k);
        c3 = faraday_d(rd, 1, 0, i, j, k) - faraday_d(rd, 0, 1, i, j, k);
    } else {
        const int ip = (i + 1 == rd.n[0]) ? 0 : i + 1;
        const int jp = (j + 1 == rd.n[1]) ? 0 : j + 1;
        const int kp = (k + 1 == rd.n[2]) ? 0 : k + 1;
        const double *E1 = rd.F[0], *E2 = rd.F[1], *E3 = rd.F[2];
        const double e1 = E1[c], e2 = E2[c], e3 = E3[c];
        const double idx = rd.idx[0], idy = rd.idx[1], idz = rd.idx[2];
        if (rd.dim == 2) {  // the z differences are exact zeros: the same values, fewer FP64 ops
            c1 = (E3[gidx(rd, i, jp, k)] - e3) * idy;
            c2 = -((E3[gidx(rd, ip, j, k)] - e3) * idx);
            c3 = (E2[gidx(rd, ip, j, k)] - e2) * idx - (E1[gidx(rd, i, jp, k)] - e1) * idy;
        } else {
            c1 = (E3[gidx(rd, i, jp, k)] - e3) * idy - (E2[gidx(rd, i, j, kp)] - e2) * idz;
            c2 = (E1[gidx(rd, i, j, kp)] - e1) * idz - (E3[gidx(rd, ip, j, k)] - e3) * idx;
            c3 = (E2[gidx(rd, ip, j, k)] - e2) * idx - (E1[gidx(rd, i, jp, k)] - e1) * idy;
        }
    }
    const double b1 = rd.F[3][c] - h * c1;
    const double b2 = rd.F[4][c] - h * c2;
    const double b3 = rd.F[5][c] - h * c3;
    rd.F[3][c] = b1;
    rd.F[4][c] = b2;
    rd.F[5][c] = b3;
    if (shadow) {
        rd.Fs[3][c] = (float)b1;
        rd.Fs[4][c] = (float)b2;
        rd.Fs[5][c] = (float)b3;
    }
}

// E <- E + dt curl B - dt J at cell c.
__device__ __forceinline__ void yee_e_cell(const RunDev &rd, int64_t c, int shadow)
{
    const int nx = rd.n[0], ny = rd.n[1], nz = rd.n[2];
    int i, j, k;
    cell_ijk(rd, c, i, j, k);
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int jm = (j == 0) ? ny - 1 : j - 1;
    const int km = (k == 0) ? nz - 1 : k - 1;
    const double *B1 = rd.F[3], *B2 = rd.F[4], *B3 = rd.F[5];
    const double b1 = B1[c], b2 = B2[c], b3 = B3[c];
    const double idx = rd.idx[0], idy = rd.idx[1], idz = rd.idx[2];
    const double dt = rd.dt;
    const double dB3dy = (b3 - B3[gidx(rd, i, jm, k)]) * idy;
    const double dB3dx = (b3 - B3[gidx(rd, im, j, k)]) * idx;
    const double dB2dx = (b2 - B2[gidx(rd, im, j, k)]) * idx;
    const double dB1dy = (b1 - B1[gidx(rd, i, jm, k)]) * idy;
    double e1, e2;
    if (rd.dim == 2) {  // the z differences are exact zeros: the same values, fewer FP64 ops
        e1 = rd.F[0][c] + dt * dB3dy - dt * rd.F[6][c];
        e2 = rd.F[1][c] + dt * (-dB3dx) - dt * rd.F[7][c];
    } else {
        const double dB2dz = (b2 - B2[gidx(rd, i, j, km)]) * idz;
        const double dB1dz = (b1 - B1[gidx(rd, i, j, km)]) * idz;
        e1 = rd.F[0][c] + dt * (dB3dy - dB2dz) - dt * rd.F[6][c];
        e2 = rd.F[1][c] + dt * (dB1dz - dB3dx) - dt * rd.F[7][c];
    }
    const double e3 = rd.F[2][c] + dt * (dB2dx - dB1dy) - dt * rd.F[8][c];
    rd.F[0][c] = e1;
    rd.F[1][c] = e2;
    rd.F[2][c] = e3;
    if (shadow) {
        rd.Fs[0][c] = (float)e1;
        rd.Fs[1][c] = (float)e2;
        rd.Fs[2][c] = (float)e3;
    }
}

}  // namespace pic
