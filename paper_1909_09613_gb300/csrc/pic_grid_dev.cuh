// Device bodies of the periodic Yee update (Sec. 1 Yee grid; App. C with A_i = 1), shared
// by the single-run launches (pic_grid.cu) and the batched launches (pic_batch.cu).
#pragma once
#include "pic_common.cuh"

namespace pic {

__device__ __forceinline__ int64_t gidx(const RunDev &rd, int i, int j, int k)
{
    return ((int64_t)k * rd.n[1] + j) * rd.n[0] + i;
}

// B <- B - h curl E at cell c (FP32 shadow of B written when `shadow`).
__device__ __forceinline__ void yee_b_cell(const RunDev &rd, int64_t c, double h, int shadow)
{
    const int nx = rd.n[0], ny = rd.n[1], nz = rd.n[2];
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / ((int64_t)nx * ny));
    const int ip = (i + 1 == nx) ? 0 : i + 1;
    const int jp = (j + 1 == ny) ? 0 : j + 1;
    const int kp = (k + 1 == nz) ? 0 : k + 1;
    const double *E1 = rd.F[0], *E2 = rd.F[1], *E3 = rd.F[2];
    const double e1 = E1[c], e2 = E2[c], e3 = E3[c];
    const double idx = 1.0 / rd.dx[0], idy = 1.0 / rd.dx[1], idz = 1.0 / rd.dx[2];
    const double dE3dy = (E3[gidx(rd, i, jp, k)] - e3) * idy;
    const double dE2dz = (E2[gidx(rd, i, j, kp)] - e2) * idz;
    const double dE1dz = (E1[gidx(rd, i, j, kp)] - e1) * idz;
    const double dE3dx = (E3[gidx(rd, ip, j, k)] - e3) * idx;
    const double dE2dx = (E2[gidx(rd, ip, j, k)] - e2) * idx;
    const double dE1dy = (E1[gidx(rd, i, jp, k)] - e1) * idy;
    const double b1 = rd.F[3][c] - h * (dE3dy - dE2dz);
    const double b2 = rd.F[4][c] - h * (dE1dz - dE3dx);
    const double b3 = rd.F[5][c] - h * (dE2dx - dE1dy);
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
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / ((int64_t)nx * ny));
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int jm = (j == 0) ? ny - 1 : j - 1;
    const int km = (k == 0) ? nz - 1 : k - 1;
    const double *B1 = rd.F[3], *B2 = rd.F[4], *B3 = rd.F[5];
    const double b1 = B1[c], b2 = B2[c], b3 = B3[c];
    const double idx = 1.0 / rd.dx[0], idy = 1.0 / rd.dx[1], idz = 1.0 / rd.dx[2];
    const double dt = rd.dt;
    const double dB3dy = (b3 - B3[gidx(rd, i, jm, k)]) * idy;
    const double dB2dz = (b2 - B2[gidx(rd, i, j, km)]) * idz;
    const double dB1dz = (b1 - B1[gidx(rd, i, j, km)]) * idz;
    const double dB3dx = (b3 - B3[gidx(rd, im, j, k)]) * idx;
    const double dB2dx = (b2 - B2[gidx(rd, im, j, k)]) * idx;
    const double dB1dy = (b1 - B1[gidx(rd, i, jm, k)]) * idy;
    const double e1 = rd.F[0][c] + dt * (dB3dy - dB2dz) - dt * rd.F[6][c];
    const double e2 = rd.F[1][c] + dt * (dB1dz - dB3dx) - dt * rd.F[7][c];
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
