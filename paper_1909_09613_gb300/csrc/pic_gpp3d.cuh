// Tile kernel of the fused particle pass in 3D: the FP32 form stages the tile's fields in
// shared memory, the FP64 form reads them through L1; both add the current by global
// reductions.
#pragma once
#include "pic_gpp_kernels.cuh"

namespace pic {

// Stage the FP32 fields of 3D tile (x0, y0, z0) and its halo in shared memory: six arrays of
// reg_nodes floats (E1, E2, E3, B1, B2, B3), x fastest.  The loads bypass L1 (ld.global.cg),
// which keeps the particle stream requested ahead of its iteration there.
__device__ inline void stage3d_load(const RunDev &rd, float *sf, int x0, int y0, int z0)
{
    const int RX = rd.reg[0], RY = rd.reg[1];
    const int nodes = (int)rd.reg_nodes;
    for (int n = threadIdx.x; n < nodes; n += blockDim.x) {
        const int rx = n % RX, r2 = n / RX;
        const int ry = r2 % RY, rz = r2 / RY;
        const int gx = wrap_idx(x0 - rd.pre[0] + rx, rd.n[0]);
        const int gy = wrap_idx(y0 - rd.pre[1] + ry, rd.n[1]);
        const int gz = wrap_idx(z0 - rd.pre[2] + rz, rd.n[2]);
        const int64_t g = ((int64_t)gz * rd.n[1] + gy) * rd.n[0] + gx;
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = __ldcg(rd.Fs[c] + g);
#pragma unroll
        for (int c = 0; c < 6; ++c) sf[c * nodes + n] = v[c];
    }
}

// The stored state of one particle as loaded (FP32 form: cell index, offsets, momenta; FP64
// form: positions in cell units, momenta).
template <typename R>
struct Raw3 {
    int cell;
    R x[3];
    R u[3];
};

template <typename R>
__device__ __forceinline__ void load_raw3(const SpeciesDev &sp, int64_t p, Raw3<R> &r)
{
    if constexpr (sizeof(R) == 4) r.cell = __ldg(sp.cell + p);
    else r.cell = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.x[a] = __ldg((const R *)sp.pos[a] + p);
        r.u[a] = __ldg((const R *)sp.mom[a] + p);
    }
}

template <typename R>
__device__ __forceinline__ void decode_raw3(const RunDev &rd, const Raw3<R> &r, PState<R> &s)
{
    if constexpr (sizeof(R) == 4) {
        const int nxy = rd.n[0] * rd.n[1];
        s.c[2] = fast_div(r.cell, rd.div_n01.m, rd.div_n01.s);
        const int q = r.cell - s.c[2] * nxy;
        s.c[1] = fast_div(q, rd.div_n0.m, rd.div_n0.s);
        s.c[0] = q - s.c[1] * rd.n[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) s.d[a] = r.x[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double f = floor(r.x[a]);
            s.c[a] = min(max((int)f, 0), rd.n[a] - 1);  // a non-finite position stays in range
            s.d[a] = r.x[a] - f;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) s.u[a] = r.u[a];
}

// One staggered field component at a particle from the staged tile: sum over the stencil
// nodes of wz[c] wy[b] wx[a] F(zs + c, ys + b, xs + a), the nodes of each axis consecutive in
// the stage (row stride RX, plane stride RXY; 32-bit shared-memory offsets).
template <int NA, int NB, int NC, typename R>
__device__ __forceinline__ R gather3_staged(const float *f, int RX, int RXY, int xs, int ys,
                                            int zs, const R *wx, const R *wy, const R *wz)
{
    const float *base = f + (zs * RXY + ys * RX + xs);
    R acc = R(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        R r2 = R(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float *row = base + (c * RXY + b * RX);
            R r1 = R(0);
#pragma unroll
            for (int a = 0; a < NA; ++a) r1 += wx[a] * row[a];
            r2 += wy[b] * r1;
        }
        acc += wz[c] * r2;
    }
    return acc;
}

// The same through L1 from the global field (wrapped node indices per axis).
template <int NA, int NB, int NC, typename R, typename F>
__device__ __forceinline__ R gather3_global(const F *f, int64_t nx, int64_t ny, const int *xi,
                                            const int *yi, const int *zi, const R *wx,
                                            const R *wy, const R *wz)
{
    R acc = R(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        R r2 = R(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int64_t row = ((int64_t)zi[c] * ny + yi[b]) * nx;
            R r1 = R(0);
#pragma unroll
            for (int a = 0; a < NA; ++a) r1 += wx[a] * (R)__ldg(f + row + xi[a]);
            r2 += wy[b] * r1;
        }
        acc += wz[c] * r2;
    }
    return acc;
}

// One particle, 3D: fields from the tile's shared-memory stage (STAGED, FP32 form: sf, tile
// origin x0, y0, z0) or through L1 (FP64 form), current by global reductions (FP32 form: into
// the padded FP32 current RunDev::J32, whose windows need no wrapping, so each row of a window
// is one pointer and its x nodes go in as aligned pairs, red.global.add.v2.f32 -- fewer
// reduction requests for the L2, which bounds this kernel; FP64 form and deterministic runs:
// into F[6..8]).  Called by all 32 lanes of a warp together (the window-row skips of the
// deposit are decided per warp); lanes with act == false carry no particle.  raw: the
// particle's stored state, loaded by the caller.
template <int L, int KT, typename R, bool STAGED = false>
__device__ __forceinline__ void particle_3d(const RunDev &rd, const SpeciesDev &sp, int64_t p,
                                            bool act, const Raw3<R> &raw,
                                            const float *sf = nullptr, int x0 = 0, int y0 = 0,
                                            int z0 = 0)
{
    PState<R> s;
    decode_raw3<R>(rd, raw, s);
    const int nx = rd.n[0], ny = rd.n[1];
    int lc[3] = {0, 0, 0};
    if constexpr (STAGED) {
        const int org[3] = {x0, y0, z0};
        bool ok = act;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (ok) ok = local_coord(s.c[a], org[a], rd.tile[a], rd.drift[a], rd.n[a], lc[a]);
        if (act && !ok) {
            set_err(rd.err, 1);  // outside the staged halo: the sort interval was exceeded
            act = false;
        }
    }
    if (!act) {
        // a harmless stand-in particle at the tile origin; it deposits and stores nothing
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s.c[a] = a == 0 ? x0 : (a == 1 ? y0 : z0);
            s.d[a] = R(0.5);
            s.u[a] = R(0);
            lc[a] = 0;
        }
    }
    AxisW<L, KT, R> w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) axis_weights<L, KT, R>(rd.tt[a], s.d[a], w[a]);

    // ---- gather (Eq. interpolation-EB-real-mod in 3D):
    // E1: W T T ; E2: T W T ; E3: T T W ; B1: T W W ; B2: W T W ; B3: W W T (x, y, z)
    R E[3], B[3];
    if constexpr (STAGED) {
        const int RX = rd.reg[0], RXY = rd.reg[0] * rd.reg[1], nodes = (int)rd.reg_nodes;
        int h[3], t[3];  // first staged node of the half-integer and integer stencils
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[a] = lc[a] + rd.pre[a] + w[a].bh;
            t[a] = lc[a] + rd.pre[a] + w[a].bt;
        }
        E[0] = gather3_staged<L + 1, KT, KT, R>(sf, RX, RXY, h[0], t[1], t[2], w[0].wh, w[1].wt, w[2].wt);
        E[1] = gather3_staged<KT, L + 1, KT, R>(sf + nodes, RX, RXY, t[0], h[1], t[2], w[0].wt, w[1].wh, w[2].wt);
        E[2] = gather3_staged<KT, KT, L + 1, R>(sf + 2 * nodes, RX, RXY, t[0], t[1], h[2], w[0].wt, w[1].wt, w[2].wh);
        B[0] = gather3_staged<KT, L + 1, L + 1, R>(sf + 3 * nodes, RX, RXY, t[0], h[1], h[2], w[0].wt, w[1].wh, w[2].wh);
        B[1] = gather3_staged<L + 1, KT, L + 1, R>(sf + 4 * nodes, RX, RXY, h[0], t[1], h[2], w[0].wh, w[1].wt, w[2].wh);
        B[2] = gather3_staged<L + 1, L + 1, KT, R>(sf + 5 * nodes, RX, RXY, h[0], h[1], t[2], w[0].wh, w[1].wh, w[2].wt);
    } else {
        int ih[3][L + 1], it[3][KT];  // wrapped global node indices
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int k = 0; k <= L; ++k) ih[a][k] = wrap_idx(s.c[a] + w[a].bh + k, rd.n[a]);
#pragma unroll
            for (int k = 0; k < KT; ++k) it[a][k] = wrap_idx(s.c[a] + w[a].bt + k, rd.n[a]);
        }
        if constexpr (sizeof(R) == 4) {
            E[0] = gather3_global<L + 1, KT, KT, R>(rd.Fs[0], nx, ny, ih[0], it[1], it[2], w[0].wh, w[1].wt, w[2].wt);
            E[1] = gather3_global<KT, L + 1, KT, R>(rd.Fs[1], nx, ny, it[0], ih[1], it[2], w[0].wt, w[1].wh, w[2].wt);
            E[2] = gather3_global<KT, KT, L + 1, R>(rd.Fs[2], nx, ny, it[0], it[1], ih[2], w[0].wt, w[1].wt, w[2].wh);
            B[0] = gather3_global<KT, L + 1, L + 1, R>(rd.Fs[3], nx, ny, it[0], ih[1], ih[2], w[0].wt, w[1].wh, w[2].wh);
            B[1] = gather3_global<L + 1, KT, L + 1, R>(rd.Fs[4], nx, ny, ih[0], it[1], ih[2], w[0].wh, w[1].wt, w[2].wh);
            B[2] = gather3_global<L + 1, L + 1, KT, R>(rd.Fs[5], nx, ny, ih[0], ih[1], it[2], w[0].wh, w[1].wh, w[2].wt);
        } else {
            E[0] = gather3_global<L + 1, KT, KT, R>(rd.F[0], nx, ny, ih[0], it[1], it[2], w[0].wh, w[1].wt, w[2].wt);
            E[1] = gather3_global<KT, L + 1, KT, R>(rd.F[1], nx, ny, it[0], ih[1], it[2], w[0].wt, w[1].wh, w[2].wt);
            E[2] = gather3_global<KT, KT, L + 1, R>(rd.F[2], nx, ny, it[0], it[1], ih[2], w[0].wt, w[1].wt, w[2].wh);
            B[0] = gather3_global<KT, L + 1, L + 1, R>(rd.F[3], nx, ny, it[0], ih[1], ih[2], w[0].wt, w[1].wh, w[2].wh);
            B[1] = gather3_global<L + 1, KT, L + 1, R>(rd.F[4], nx, ny, ih[0], it[1], ih[2], w[0].wh, w[1].wt, w[2].wh);
            B[2] = gather3_global<L + 1, L + 1, KT, R>(rd.F[5], nx, ny, ih[0], ih[1], it[2], w[0].wh, w[1].wh, w[2].wt);
        }
    }

    // ---- Boris push and move ----
    const R ig = boris<R>(R(sp.qmdt_half), E, B, s.u);
    R o[3], dl[3], xs[3];
    int cn[3], shv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dl[a] = R(rd.dtt[a]) * s.u[a] * ig;
        shv[a] = move_axis<R>(s.d[a], dl[a], s.c[a], rd.n[a], o[a], cn[a], xs[a]);
    }

    // ---- Esirkepov deposit ----
    AxisS<L, R> S[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(R) == 4) axis_shapes_dd<L, true>(s.d[a], dl[a], S[a]);
        else axis_shapes<L, R>(s.d[a], shv[a], o[a], S[a]);
    }
    R DS[3][L + 2], P[3][L + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < L + 2; ++k) {
            DS[a][k] = S[a].ds[k];
            acc += DS[a][k];
            P[a][k] = acc;
        }
    }
    // Along an axis on which no lane of the warp moved its window base, every lane's window
    // has S0 = DS = 0 on its last node (l + 1), and the prefix sum P[l] = sum of DS over the
    // window is zero (in exact arithmetic; its computed value is round-off): those rows of the
    // current are zero and the warp skips them together (branches uniform across the warp).
    // With a drift along x1 the y and z windows rarely move: 75 of the 144 products for l = 2.
    bool mv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mv[a] = __any_sync(0xffffffffu, act && S[a].wide);
    const R third = R(1) / R(3);
    // W_a = DS_a (S0_b S0_c + DS_b S0_c / 2 + S0_b DS_c / 2 + DS_b DS_c / 3), prefix along a:
    // J_a(ka, kb, kc) = kx_a P_a[ka] (S0_b[kb] fc0_c[kc] + DS_b[kb] fc1_c[kc]) with
    // fc0 = S0 + DS / 2, fc1 = S0 / 2 + DS / 3 of axis c
    R fc0[3][L + 2], fc1[3][L + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int k = 0; k < L + 2; ++k) {
            fc0[a][k] = S[a].s0[k] + R(0.5) * DS[a][k];
            fc1[a][k] = R(0.5) * S[a].s0[k] + third * DS[a][k];
        }
    }
    if (sizeof(R) == 4 && !rd.det) {
        // padded FP32 current: the window of axis a starts at c_a + wb_a + jp_lo, unwrapped
        const int PX = rd.jp[0], PXY = rd.jp[0] * rd.jp[1];
        const int w0 = ((s.c[2] + S[2].wb + rd.jp_lo) * rd.jp[1] + (s.c[1] + S[1].wb + rd.jp_lo)) * PX
                       + (s.c[0] + S[0].wb + rd.jp_lo);
        const int xodd = (s.c[0] + S[0].wb + rd.jp_lo) & 1;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int bx = (ax + 1) % 3, cx = (ax + 2) % 3;
            const R kk = R(sp.kx[ax]);
            R kP[L + 1];
#pragma unroll
            for (int ka = 0; ka <= L; ++ka) kP[ka] = kk * P[ax][ka];
            // nodes per axis of this component's rows (x, y, z): the prefix axis has l + 1
            // (l when no lane moved along it), the others l + 2 (l + 1 likewise)
            int nk[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) nk[a] = (a == ax ? L : L + 1) + (mv[a] ? 1 : 0);
            // the row's x nodes as aligned pairs from the even node at or below its first node
            // (x rows have even length, so every pair is 8-byte aligned): npair pairs cover
            // the nk[0] nodes shifted by the lane's parity
            float *J = (float *)rd.J32[ax] + (w0 - xodd);
            const int npair = (nk[0] + 2) / 2;
#pragma unroll
            for (int kz = 0; kz < L + 2; ++kz) {
                if (kz >= nk[2]) break;
#pragma unroll
                for (int ky = 0; ky < L + 2; ++ky) {
                    if (ky >= nk[1]) break;
                    float *row = J + (kz * PXY + ky * PX);
                    float v[L + 2];
#pragma unroll
                    for (int kx = 0; kx < L + 2; ++kx) {
                        const int k3[3] = {kx, ky, kz};
                        const int ka = k3[ax], kb = k3[bx], kc = k3[cx];
                        if (ka > L || kx >= nk[0]) { v[kx] = 0.0f; continue; }
                        const R perp = S[bx].s0[kb] * fc0[cx][kc] + DS[bx][kb] * fc1[cx][kc];
                        v[kx] = (float)(kP[ka] * perp);
                    }
#pragma unroll
                    for (int j = 0; j < (L + 3) / 2 + 1; ++j) {
                        if (j >= npair) break;
                        const float lo = xodd ? (2 * j >= 1 && 2 * j - 1 < L + 2 ? v[2 * j - 1] : 0.0f)
                                              : (2 * j < L + 2 ? v[2 * j] : 0.0f);
                        const float hi = xodd ? (2 * j < L + 2 ? v[2 * j] : 0.0f)
                                              : (2 * j + 1 < L + 2 ? v[2 * j + 1] : 0.0f);
                        if (act && (lo != 0.0f || hi != 0.0f))
                            asm volatile("red.global.add.v2.f32 [%0], {%1, %2};"
                                         ::"l"(row + 2 * j), "f"(lo), "f"(hi) : "memory");
                    }
                }
            }
        }
    } else {
        // node offsets of the window along each axis (the grid has at most 2^30 cells)
        int off[3][L + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int stride = a == 0 ? 1 : (a == 1 ? nx : nx * ny);
#pragma unroll
            for (int k = 0; k < L + 2; ++k) off[a][k] = wrap_near(s.c[a] + S[a].wb + k, rd.n[a]) * stride;
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int bx = (ax + 1) % 3, cx = (ax + 2) % 3;
            const R kk = R(sp.kx[ax]);
            R kP[L + 1];
#pragma unroll
            for (int ka = 0; ka <= L; ++ka) kP[ka] = kk * P[ax][ka];
#pragma unroll
            for (int kb = 0; kb < L + 2; ++kb) {
                if (kb == L + 1 && !mv[bx]) break;
#pragma unroll
                for (int kc = 0; kc < L + 2; ++kc) {
                    if (kc == L + 1 && !mv[cx]) break;
                    const R perp = S[bx].s0[kb] * fc0[cx][kc] + DS[bx][kb] * fc1[cx][kc];
                    const int base = off[bx][kb] + off[cx][kc];
#pragma unroll
                    for (int ka = 0; ka <= L; ++ka) {
                        if (ka == L && !mv[ax]) break;
                        const int g = base + off[ax][ka];
                        const R v = kP[ka] * perp;
                        if (!act || v == R(0)) continue;
                        if (rd.det) {
                            if constexpr (sizeof(R) == 4) {
                                atomicAdd((unsigned long long *)(rd.F[6 + ax] + g),
                                          det_word32(v, rd.det_inv32));
                            } else {
                                unsigned long long hi, lo;
                                det_words64(v, rd.det_inv64, hi, lo);
                                atomicAdd((unsigned long long *)(rd.F[6 + ax] + g), hi);
                                atomicAdd(rd.Jlo[ax] + g, lo);
                            }
                        } else {
                            atomicAdd(rd.F[6 + ax] + g, (double)v);
                        }
                    }
                }
            }
        }
    }
    if (!act) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) ((R *)sp.mom[a])[p] = s.u[a];
    if constexpr (sizeof(R) == 4) {
        sp.cell[p] = (cn[2] * ny + cn[1]) * nx + cn[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) ((float *)sp.pos[a])[p] = o[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) ((double *)sp.pos[a])[p] = xs[a];  // = cn + o
    }
}

// Ask the memory system for the particle stream of a later iteration, 3D (see
// prefetch_particle): three positions, three momenta and (FP32 form) the cell index.
template <typename R>
__device__ __forceinline__ void prefetch_particle_3d(const SpeciesDev &sp, int64_t p)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"((const char *)sp.pos[a] + p * (int64_t)sizeof(R)));
        asm volatile("prefetch.global.L1 [%0];" ::"l"((const char *)sp.mom[a] + p * (int64_t)sizeof(R)));
    }
    if constexpr (sizeof(R) == 4)
        asm volatile("prefetch.global.L1 [%0];" ::"l"((const char *)sp.cell + p * 4));
}

// All particles of one 3D tile.  FP32 form: the tile's fields and halo are staged in shared
// memory first (sf, 6 x reg_nodes floats; the FP32 3D sort interval keeps every particle
// within one cell of its sorted tile); FP64 form: fields through L1.  A warp's lanes take 32
// consecutive particles (warp-uniform trip count) and ask for the stream of their next
// iteration ahead (into L1); the first particles of every species are requested before the
// stage load.
template <int L, int KT, typename R>
__device__ void tile_3d(const RunDev &rd, int64_t tile, float *sf = nullptr)
{
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < rd.nsp; ++s) {
        const int64_t p = rd.sp[s].tile_start[tile] + threadIdx.x;
        if (p < rd.sp[s].tile_start[tile + 1]) prefetch_particle_3d<R>(rd.sp[s], p);
    }
    int x0 = 0, y0 = 0, z0 = 0;
    if constexpr (sizeof(R) == 4) {
        const int tx = (int)(tile % rd.ntile[0]);
        const int ty = (int)((tile / rd.ntile[0]) % rd.ntile[1]);
        const int tz = (int)(tile / ((int64_t)rd.ntile[0] * rd.ntile[1]));
        x0 = tx * rd.tile[0];
        y0 = ty * rd.tile[1];
        z0 = tz * rd.tile[2];
        stage3d_load(rd, sf, x0, y0, z0);
        __syncthreads();
    }
    for (int s = 0; s < rd.nsp; ++s) {
        const SpeciesDev &sp = rd.sp[s];
        const int64_t a = sp.tile_start[tile], b = sp.tile_start[tile + 1];
        for (int64_t q = a + (threadIdx.x & ~31); q < b; q += blockDim.x) {
            const int64_t p = q + lane;
            const bool act = p < b;
            if (p + blockDim.x < b) prefetch_particle_3d<R>(sp, p + blockDim.x);
            Raw3<R> cur = {};
            if (act) load_raw3<R>(sp, p, cur);
            if constexpr (sizeof(R) == 4)
                particle_3d<L, KT, R, true>(rd, sp, p, act, cur, sf, x0, y0, z0);
            else
                particle_3d<L, KT, R>(rd, sp, p, act, cur);
        }
    }
}

// Dynamic shared memory of a 3D tile block (FP32 form: the staged fields).
__host__ __device__ inline size_t stage3d_bytes(const RunDev &rd)
{
    return (size_t)6 * rd.reg_nodes * sizeof(float);
}

}  // namespace pic
