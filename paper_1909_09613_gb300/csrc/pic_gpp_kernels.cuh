// Tile kernels of the fused particle pass in 2D (shared-memory staged) and the per-tile
// driver shared by the single-run and the batched launches (3D: pic_gpp3d.cuh).
#pragma once
#include "pic_gpp.cuh"

namespace pic {

// Accumulation type of the shared-memory current tile: FP32 in the precision form, FP64 in
// the plain form.
template <typename R> struct AccT { typedef R T; };

// Shared-memory layout of a staged 2D tile (all arrays reg_nodes long, x fastest):
//   pa = (E1, B2) pairs  [both sit at (i+1/2, j): W along x, T along y]
//   pb = (E2, B1) pairs  [both sit at (i, j+1/2): T along x, W along y]
//   e3 = E3 [(i, j): T T],  b3 = B3 [(i+1/2, j+1/2): W W],  j1, j2, j3 (R), or, for a
//   deterministic run, q1, q2, q3 (64-bit fixed point, RunDev::det) in their place.
//   rec = per-warp factor records of the FP32 deposit (see DepFrame), FP32 form only.
template <typename R>
struct Stage2D {
    typename Vec2<R>::T *pa, *pb;
    R *e3, *b3;
    R *j1, *j2, *j3;
    unsigned long long *q1, *q2, *q3;
    TTable *tt;
    float *rec;
};

// Warps of a 2D tile block (the kernels launch 256 threads).
constexpr int kTileWarps = 8;

// Frame of the FP32 warp deposit.  The Esirkepov current of a group of lanes whose windows
// start at most SXM nodes apart along x and SYM along y is a sum over lanes of outer products
// (J1 = sum px (x) Ay, J2 = sum Ax (x) py, J3 = sum Ax (x) S0y + Bx (x) DSy, in the notation of
// particle_2d) on a common NX x NY block of nodes.  Every lane writes its factor vectors,
// shifted into the block, as a record (x part: px, Ax, Bx over NX nodes; y part: Ay, py, S0y,
// DSy over NY nodes); then the lanes sum the 32 records, each lane one term (J1, J2, or one of
// the two products of J3) on a block of nodes with packed FMAs, every load a shared-memory
// broadcast within its record: on a HALF frame (NY = 2 or 4) the two half warps take the even
// and the odd records, each lane a 2 x NY block from one 64-bit and one 64- or 128-bit load per
// record; otherwise each lane takes a 2 x BY block (BY = NY / 2) over all 32 records, from one
// 64-bit and BY 32-bit loads.  The sums are bound by shared-memory wavefronts and issue, not by
// arithmetic (a 128-bit load takes a wavefront per quarter warp, a 64-bit one per half warp).
// RS (floats per record) is a multiple of 4 with RS / 4 odd, so that the float4 stores of 8
// consecutive lanes fall in distinct banks.  NARROW: no lane of the group moved its y window
// base, so every window's last row (node l + 1) is zero and the frame has l + 1 + SYM rows
// (rounded up to even) instead of l + 2 + SYM.
template <int L, bool NARROW = false>
struct DepFrame {
    // Along y the windows of a group start at most SYM rows apart: for odd l a particle's
    // integer-node window starts at a fixed offset from its cell, so the lanes of one cell row
    // share it (SYM = 0; a warp straddling the end of a tile row takes a second pass); for even
    // l the start moves by one with the in-cell offset (SYM = 1).  Along x, up to SXM nodes.
    static constexpr int SYM = (L % 2 == 0) ? 1 : 0;
    static constexpr int WYN = NARROW ? L + 1 : L + 2;  // y nodes of one lane's window
    static constexpr int PX = (L + 2 + 2 + 1) / 2, PY = (WYN + SYM + 1) / 2;
    static constexpr int NX = 2 * PX, NY = 2 * PY;
    static constexpr int SXM = NX - (L + 2);
    static constexpr int BY = NY / 2;            // y nodes of a lane's sub-block
    static constexpr int NBT = (NX / 2) * 2;     // sub-blocks of one term
    // x part padded to a multiple of 4 floats, so that every term's y factors start 16-byte
    // aligned within the record
    static constexpr int XS = (3 * NX + 3) / 4 * 4, YS = 4 * NY;
    // HALF: the two half warps sum the even and the odd records, each lane one term on a
    // 2 x NY block (one 64-bit and one 64- or 128-bit load and NY packed FMAs per record)
    static constexpr bool HALF = (NY == 2 || NY == 4) && 4 * (NX / 2) <= 16;
    static constexpr int RS0 = XS + YS;
    static constexpr int RS1 = (RS0 + 3) / 4 * 4;
    static constexpr int RS = ((RS1 / 4) % 2 == 0) ? RS1 + 4 : RS1;
    static_assert(4 * NBT <= 32, "one lane per sub-block and term");
};

// Floats of one warp's deposit records for spline order l (host-side sizing).
__host__ __device__ inline int dep_record_floats(int l)
{
    switch (l) {
    case 1: return 32 * DepFrame<1>::RS;
    case 2: return 32 * DepFrame<2>::RS;
    case 3: return 32 * DepFrame<3>::RS;
    default: return 32 * DepFrame<4>::RS;
    }
}

// Bytes per node of the shared current tile: R per component, or (FP32 form of a
// deterministic run) a 64-bit fixed-point word per component.
template <typename R>
__host__ __device__ inline size_t stage2d_j_bytes(bool det)
{
    return (sizeof(R) == 4 && det) ? 8 : sizeof(R);
}

// own_tt: the stage holds its own copy of the two T tables (false when the caller already
// keeps the run descriptor, tables included, in shared memory).
template <typename R>
__host__ __device__ inline size_t stage2d_fields_bytes(int64_t nodes, bool own_tt = true,
                                                       bool det = false)
{
    size_t b = own_tt ? 2 * sizeof(TTable) : 0;
    b += (size_t)nodes * (2 * sizeof(typename Vec2<R>::T) + 2 * sizeof(R)
                          + 3 * stage2d_j_bytes<R>(det));
    return (b + 15) / 16 * 16;
}

// Dynamic shared memory of a 2D tile block: staged fields and current, plus (FP32 form) the
// deposit records of its warps.
template <typename R>
__host__ __device__ inline size_t stage2d_bytes(int64_t nodes, int l, bool own_tt = true,
                                                bool det = false)
{
    size_t b = stage2d_fields_bytes<R>(nodes, own_tt, det);
    if (sizeof(R) == 4) b += (size_t)kTileWarps * dep_record_floats(l) * sizeof(float);
    return b;
}

// tt_shared: T tables already in shared memory (else the stage carries a copy)
template <typename R>
__device__ __forceinline__ Stage2D<R> stage2d_carve(char *smem, int64_t nodes,
                                                    const TTable *tt_shared = nullptr,
                                                    bool det = false)
{
    Stage2D<R> s;
    s.tt = tt_shared ? (TTable *)tt_shared : (TTable *)smem;
    char *p = smem + (tt_shared ? 0 : 2 * sizeof(TTable));
    s.pa = (typename Vec2<R>::T *)p; p += nodes * sizeof(typename Vec2<R>::T);
    s.pb = (typename Vec2<R>::T *)p; p += nodes * sizeof(typename Vec2<R>::T);
    s.e3 = (R *)p; p += nodes * sizeof(R);
    s.b3 = (R *)p; p += nodes * sizeof(R);
    s.j1 = s.j2 = s.j3 = nullptr;
    s.q1 = s.q2 = s.q3 = nullptr;
    if (sizeof(R) == 4 && det) {
        s.q1 = (unsigned long long *)p; p += nodes * 8;
        s.q2 = (unsigned long long *)p; p += nodes * 8;
        s.q3 = (unsigned long long *)p;
    } else {
        s.j1 = (R *)p; p += nodes * sizeof(R);
        s.j2 = (R *)p; p += nodes * sizeof(R);
        s.j3 = (R *)p;
    }
    s.rec = (float *)(smem + stage2d_fields_bytes<R>(nodes, tt_shared == nullptr, det));
    return s;
}

// Stage fields of tile (tx, ty) and zero the current tile.
template <typename R>
__device__ void stage2d_load(const RunDev &rd, const Stage2D<R> &st, int x0, int y0)
{
    const int RX = rd.reg[0];
    const int64_t nodes = rd.reg_nodes;
    if (st.tt != rd.tt)
        for (int i = threadIdx.x; i < (int)(2 * sizeof(TTable) / sizeof(int)); i += blockDim.x)
            ((int *)st.tt)[i] = ((const int *)rd.tt)[i];
    for (int64_t n = threadIdx.x; n < nodes; n += blockDim.x) {
        const int rx = (int)(n % RX), ry = (int)(n / RX);
        const int gx = wrap_idx(x0 - rd.pre[0] + rx, rd.n[0]);
        const int gy = wrap_idx(y0 - rd.pre[1] + ry, rd.n[1]);
        const int64_t g = (int64_t)gy * rd.n[0] + gx;
        typename Vec2<R>::T a, b;
        if constexpr (sizeof(R) == 4) {
            a.x = __ldg(rd.Fs[0] + g); a.y = __ldg(rd.Fs[4] + g);
            b.x = __ldg(rd.Fs[1] + g); b.y = __ldg(rd.Fs[3] + g);
            st.e3[n] = __ldg(rd.Fs[2] + g);
            st.b3[n] = __ldg(rd.Fs[5] + g);
        } else {
            a.x = __ldg(rd.F[0] + g); a.y = __ldg(rd.F[4] + g);
            b.x = __ldg(rd.F[1] + g); b.y = __ldg(rd.F[3] + g);
            st.e3[n] = __ldg(rd.F[2] + g);
            st.b3[n] = __ldg(rd.F[5] + g);
        }
        st.pa[n] = a;
        st.pb[n] = b;
        if (st.q1) {
            st.q1[n] = 0ull;
            st.q2[n] = 0ull;
            st.q3[n] = 0ull;
        } else {
            st.j1[n] = R(0);
            st.j2[n] = R(0);
            st.j3[n] = R(0);
        }
    }
}

// Add the current tile to the global FP64 current and clear it.
template <typename R>
__device__ void stage2d_flush(const RunDev &rd, const Stage2D<R> &st, int x0, int y0)
{
    const int RX = rd.reg[0];
    const int64_t nodes = rd.reg_nodes;
    if (st.q1) {  // deterministic run: integer sums, exact in any order
        for (int64_t n = threadIdx.x; n < nodes; n += blockDim.x) {
            const unsigned long long a = st.q1[n], b = st.q2[n], c = st.q3[n];
            if ((a | b | c) == 0ull) continue;
            const int rx = (int)(n % RX), ry = (int)(n / RX);
            const int gx = wrap_idx(x0 - rd.pre[0] + rx, rd.n[0]);
            const int gy = wrap_idx(y0 - rd.pre[1] + ry, rd.n[1]);
            const int64_t g = (int64_t)gy * rd.n[0] + gx;
            if (a) atomicAdd((unsigned long long *)(rd.F[6] + g), a);
            if (b) atomicAdd((unsigned long long *)(rd.F[7] + g), b);
            if (c) atomicAdd((unsigned long long *)(rd.F[8] + g), c);
            st.q1[n] = 0ull;
            st.q2[n] = 0ull;
            st.q3[n] = 0ull;
        }
        return;
    }
    for (int64_t n = threadIdx.x; n < nodes; n += blockDim.x) {
        const R a = st.j1[n], b = st.j2[n], c = st.j3[n];
        if (a == R(0) && b == R(0) && c == R(0)) continue;
        const int rx = (int)(n % RX), ry = (int)(n / RX);
        const int gx = wrap_idx(x0 - rd.pre[0] + rx, rd.n[0]);
        const int gy = wrap_idx(y0 - rd.pre[1] + ry, rd.n[1]);
        const int64_t g = (int64_t)gy * rd.n[0] + gx;
        if (a != R(0)) atomicAdd(rd.F[6] + g, (double)a);
        if (b != R(0)) atomicAdd(rd.F[7] + g, (double)b);
        if (c != R(0)) atomicAdd(rd.F[8] + g, (double)c);
        st.j1[n] = R(0);
        st.j2[n] = R(0);
        st.j3[n] = R(0);
    }
}

// Local coordinate of a cell index along one axis, relative to the tile origin, taking the
// periodic image that lies within [-D, tile + D).  Returns false if none does.
__device__ __forceinline__ bool local_coord(int c, int origin, int tile, int drift, int n, int &lc)
{
    int l = c - origin;
    if (l < -drift) l += n;
    if (l >= tile + drift) l -= n;
    lc = l;
    return l >= -drift && l < tile + drift;
}

// Add (a, b) to the two FP32 values at p (8-byte aligned: two neighbouring x nodes of a staged
// row that starts at an even node) with one 64-bit compare-and-swap loop and a packed add, each
// half rounded as the scalar add.  Shared-memory FP32 additions are compare-and-swap loops
// either way; this one serves two nodes.
__device__ __forceinline__ void atomic_add_pair(float *p, float a, float b)
{
    unsigned long long *q = (unsigned long long *)p;
    unsigned long long old = *q, got;
    do {
        float2 f = make_float2(__uint_as_float((unsigned)old),
                               __uint_as_float((unsigned)(old >> 32)));
        f = __fadd2_rn(f, make_float2(a, b));
        const unsigned long long nw = (unsigned long long)__float_as_uint(f.x)
                                      | ((unsigned long long)__float_as_uint(f.y) << 32);
        got = atomicCAS(q, old, nw);
        if (got == old) break;
        old = got;
    } while (true);
}

// One lane's Esirkepov window (Sec. 1: W_x = DSx (S0y + DSy/2) summed along x, W_y likewise,
// W_z = S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3) added to the shared current tile with
// atomics (WY as in deposit_lane_global below); DET: as fixed-point words (RunDev::det).
template <int L, typename R, bool WY = true, bool DET = false>
__device__ __forceinline__ void deposit_lane(const Stage2D<R> &st, int RX, int jx0, int jy0, R kx,
                                             R ky, R kz, const R *px, const R *py, const R *Ax,
                                             const R *Ay, const R *Bx, const AxisS<L, R> &Sy,
                                             float dinv = 0.0f)
{
#pragma unroll
    for (int b = 0; b < (WY ? L + 2 : L + 1); ++b) {
        const int row = (jy0 + b) * RX + jx0;
        const R ayk = kx * Ay[b];
        const R pyk = (b <= L) ? ky * py[b] : R(0);
        const R zs = kz * Sy.s0[b], zd = kz * Sy.ds[b];
#pragma unroll
        for (int a = 0; a < L + 2; ++a) {
            if constexpr (DET) {
                if (a <= L) atomicAdd(st.q1 + row + a, det_word32(ayk * px[a], dinv));
                if (b <= L) atomicAdd(st.q2 + row + a, det_word32(pyk * Ax[a], dinv));
                atomicAdd(st.q3 + row + a, det_word32(zs * Ax[a] + zd * Bx[a], dinv));
            } else {
                if (a <= L) atomicAdd(st.j1 + row + a, ayk * px[a]);
                if (b <= L) atomicAdd(st.j2 + row + a, pyk * Ax[a]);
                atomicAdd(st.j3 + row + a, zs * Ax[a] + zd * Bx[a]);
            }
        }
    }
}

// One lane's Esirkepov window added straight to the global FP64 current (FP64 form).  The
// reductions (red.global.add.f64) are performed by L2, so unlike shared-memory FP64 atomics
// (compare-and-swap loops around a DADD) they take no issue slots of the SM's FP64 pipe, which
// bounds this form.  gx0, gy0: global node of the window's first column and row (unwrapped).
// WY = false when no lane of the warp changed its y window base: row l + 1 then carries exact
// zeros (S0y = DSy = 0) and is skipped.
template <int L, typename R, typename Hot, bool WY = true, bool DET = false>
__device__ __forceinline__ void deposit_lane_global(const Hot &h, int gx0, int gy0, R kx, R ky,
                                                    R kz, const R *px, const R *py, const R *Ax,
                                                    const R *Ay, const R *Bx,
                                                    const AxisS<L, R> &Sy)
{
    int gx[L + 2];
    int64_t gy[L + 2];
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        gx[k] = wrap_near(gx0 + k, h.n0);
        gy[k] = (int64_t)wrap_near(gy0 + k, h.n1) * h.n0;
    }
#pragma unroll
    for (int b = 0; b < (WY ? L + 2 : L + 1); ++b) {
        const R ayk = kx * Ay[b];
        const R pyk = (b <= L) ? ky * py[b] : R(0);
        const R zs = kz * Sy.s0[b], zd = kz * Sy.ds[b];
#pragma unroll
        for (int a = 0; a < L + 2; ++a) {
            const int64_t g = gy[b] + gx[a];
            if constexpr (DET) {
                unsigned long long hi, lo;
                if (a <= L) {
                    det_words64((double)(ayk * px[a]), h.dinv64, hi, lo);
                    atomicAdd((unsigned long long *)(h.J0 + g), hi);
                    atomicAdd(h.Jlo0 + g, lo);
                }
                if (b <= L) {
                    det_words64((double)(pyk * Ax[a]), h.dinv64, hi, lo);
                    atomicAdd((unsigned long long *)(h.J1 + g), hi);
                    atomicAdd(h.Jlo1 + g, lo);
                }
                det_words64((double)(zs * Ax[a] + zd * Bx[a]), h.dinv64, hi, lo);
                atomicAdd((unsigned long long *)(h.J2 + g), hi);
                atomicAdd(h.Jlo2 + g, lo);
            } else {
                if (a <= L) atomicAdd(h.J0 + g, (double)(ayk * px[a]));
                if (b <= L) atomicAdd(h.J1 + g, (double)(pyk * Ax[a]));
                atomicAdd(h.J2 + g, (double)(zs * Ax[a] + zd * Bx[a]));
            }
        }
    }
}

// Scalars the particle loop uses, held in registers for the whole tile (a run descriptor in
// shared or global memory would be re-read for every particle).
struct Hot2D {
    int n0, n1, tile0, tile1, drift0, drift1, pre0, pre1, RX, RY, slot_major;
    double *J0, *J1, *J2;  // global FP64 current (high fixed-point words of a deterministic run)
    double dtt0, dtt1;
    uint64_t dm;  // division by n0 (FastDiv)
    int ds;
    int32_t *err;
    int det;  // RunDev::det and its fixed-point scales and low words
    float dinv32;
    double dinv64;
    unsigned long long *Jlo0, *Jlo1, *Jlo2;
};

template <typename R>
struct HotSp {
    void *pos0, *pos1, *mom0, *mom1, *mom2;
    int32_t *cell;
    double qmdt_half, kx0, kx1, kz;
    double *wc;  // FP64 weight cache (SpeciesDev::wc)
    int64_t wc_stride;
    int wc_mode;
};

__device__ __forceinline__ Hot2D make_hot2d(const RunDev &rd)
{
    Hot2D h;
    h.n0 = rd.n[0]; h.n1 = rd.n[1];
    h.tile0 = rd.tile[0]; h.tile1 = rd.tile[1];
    h.drift0 = rd.drift[0]; h.drift1 = rd.drift[1];
    h.pre0 = rd.pre[0]; h.pre1 = rd.pre[1];
    h.RX = rd.reg[0];
    h.RY = rd.reg[1];
    h.J0 = rd.F[6]; h.J1 = rd.F[7]; h.J2 = rd.F[8];
    h.slot_major = rd.slot_major;
    h.dtt0 = rd.dtt[0]; h.dtt1 = rd.dtt[1];
    h.dm = rd.div_n0.m; h.ds = rd.div_n0.s;
    h.err = rd.err;
    h.det = rd.det;
    h.dinv32 = rd.det_inv32;
    h.dinv64 = rd.det_inv64;
    h.Jlo0 = rd.Jlo[0]; h.Jlo1 = rd.Jlo[1]; h.Jlo2 = rd.Jlo[2];
    return h;
}

template <typename R>
__device__ __forceinline__ HotSp<R> make_hotsp(const SpeciesDev &sp)
{
    HotSp<R> h;
    h.pos0 = sp.pos[0]; h.pos1 = sp.pos[1];
    h.mom0 = sp.mom[0]; h.mom1 = sp.mom[1]; h.mom2 = sp.mom[2];
    h.cell = sp.cell;
    h.qmdt_half = sp.qmdt_half;
    h.kx0 = sp.kx[0]; h.kx1 = sp.kx[1]; h.kz = sp.kz;
    h.wc = sp.wc; h.wc_stride = sp.wc_stride; h.wc_mode = sp.wc_mode;
    return h;
}

// Ask the memory system for the particle stream of a later iteration (lines land in L1 while
// the current particle is processed; the particle loop is otherwise stalled on these loads).
template <typename R>
__device__ __forceinline__ void prefetch_particle(const HotSp<R> &hs, int64_t p)
{
    const void *ptrs[6] = {hs.pos0, hs.pos1, hs.mom0, hs.mom1, hs.mom2, hs.cell};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (i == 5 && sizeof(R) == 8) break;  // the FP64 form has no cell array
        const char *a = (const char *)ptrs[i] + p * (i == 5 ? 4 : (int64_t)sizeof(R));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
}

// The cached old-position weights of a later iteration (FP64 form, 2 (l + 1) arrays).
template <int L>
__device__ __forceinline__ void prefetch_weights(const HotSp<double> &hs, int64_t p)
{
#pragma unroll
    for (int i = 0; i < 2 * (L + 1); ++i) {
        const double *a = hs.wc + (int64_t)i * hs.wc_stride + p;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
}

// FP32 gather on packed pairs: __ffma2_rn performs two FP32 fused multiply-adds in one
// instruction (sm_100 and later), each rounded exactly as the scalar FMA, so the result is the
// scalar loop's bit for bit.  (E1, B2) and (E2, B1) are staged as pairs that share their
// weights; E3 (T x T) and B3 (W x W) pair up when the two stencils have the same size.
template <int L, int KT>
__device__ __forceinline__ void gather_2d_x2(const Stage2D<float> &st, const AxisW<L, KT, float> &wx,
                                             const AxisW<L, KT, float> &wy, int sx, int sy,
                                             int RX, float *E, float *B)
{
    const float2 z2 = make_float2(0.0f, 0.0f);
    float2 e1b2 = z2, e2b1 = z2;
#pragma unroll
    for (int b = 0; b < KT; ++b) {  // (E1, B2): W along x (half nodes), T along y
        const int row = (sy + wy.bt + b) * RX + sx + wx.bh;
        float2 r = z2;
#pragma unroll
        for (int a = 0; a <= L; ++a) r = __ffma2_rn(make_float2(wx.wh[a], wx.wh[a]), st.pa[row + a], r);
        e1b2 = __ffma2_rn(make_float2(wy.wt[b], wy.wt[b]), r, e1b2);
    }
#pragma unroll
    for (int b = 0; b <= L; ++b) {  // (E2, B1): T along x, W along y
        const int row = (sy + wy.bh + b) * RX + sx + wx.bt;
        float2 r = z2;
#pragma unroll
        for (int a = 0; a < KT; ++a) r = __ffma2_rn(make_float2(wx.wt[a], wx.wt[a]), st.pb[row + a], r);
        e2b1 = __ffma2_rn(make_float2(wy.wh[b], wy.wh[b]), r, e2b1);
    }
    E[0] = e1b2.x; B[1] = e1b2.y;
    E[1] = e2b1.x; B[0] = e2b1.y;
    if constexpr (KT == L + 1) {
        float2 e3b3 = z2;
#pragma unroll
        for (int b = 0; b < KT; ++b) {  // E3: T T, B3: W W
            const int rt = (sy + wy.bt + b) * RX + sx + wx.bt;
            const int rw = (sy + wy.bh + b) * RX + sx + wx.bh;
            float2 r = z2;
#pragma unroll
            for (int a = 0; a < KT; ++a)
                r = __ffma2_rn(make_float2(wx.wt[a], wx.wh[a]), make_float2(st.e3[rt + a], st.b3[rw + a]), r);
            e3b3 = __ffma2_rn(make_float2(wy.wt[b], wy.wh[b]), r, e3b3);
        }
        E[2] = e3b3.x; B[2] = e3b3.y;
    } else {
        float e3 = 0.0f, b3 = 0.0f;
#pragma unroll
        for (int b = 0; b < KT; ++b) {
            const int row = (sy + wy.bt + b) * RX + sx + wx.bt;
            float r = 0.0f;
#pragma unroll
            for (int a = 0; a < KT; ++a) r += wx.wt[a] * st.e3[row + a];
            e3 += wy.wt[b] * r;
        }
#pragma unroll
        for (int b = 0; b <= L; ++b) {
            const int row = (sy + wy.bh + b) * RX + sx + wx.bh;
            float r = 0.0f;
#pragma unroll
            for (int a = 0; a <= L; ++a) r += wx.wh[a] * st.b3[row + a];
            b3 += wy.wh[b] * r;
        }
        E[2] = e3; B[2] = b3;
    }
}

// One pass of the FP32 warp deposit on frame FR (DepFrame): every lane writes its factor
// record, shifted by (ox, oy) into the frame and scaled by gin (1 for the lanes of this pass's
// group, 0 for the others), then each lane sums its term on its sub-block over the 32 records and
// adds it to the shared current.  The two products of J3 (terms 2 and 3, lanes NBT apart) are
// added together first, so that no two lanes of one atomic instruction address the same node.
// mnx, mny: frame origin (tile-local node); kx, ky, kz: the species' current scales.
template <class FR, int L, bool DET>
__device__ __forceinline__ void warp_frame_pass(const Hot2D &h, const Stage2D<float> &st,
                                                float gin, int ox, int oy, int mnx, int mny,
                                                float kx, float ky, float kz, const float *px,
                                                const float *py, const float *Ax, const float *Ay,
                                                const float *Bx, const AxisS<L, float> &Sy)
{
    const int lane = threadIdx.x & 31;
    // the warp's record area is sized for the widest frame of order l
    float *rec = st.rec + (threadIdx.x >> 5) * (32 * DepFrame<L>::RS);
    float4 *mine = (float4 *)(rec + lane * FR::RS);
    // the record: block node A holds this lane's window node A - ox (zero outside it); the x
    // factors are scaled first, then shifted by ox = 0..SXM in two steps (ox & 1, ox & 2); the
    // y factors are shifted by oy (0 when SYM = 0)
    float r[FR::RS1];
    float sp[L + 2], sa[L + 2], sb2[L + 2];
    const float gkx = gin * kx;
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        sp[k] = (k <= L) ? gkx * px[k] : 0.0f;
        sa[k] = gin * Ax[k];
        sb2[k] = gin * Bx[k];
    }
    const bool sh1 = (ox & 1) != 0, sh2 = (ox & 2) != 0;
    float tp[L + 3], ta[L + 3], tb[L + 3];
#pragma unroll
    for (int k = 0; k < L + 3; ++k) {
        const float p0 = (k < L + 2) ? sp[k] : 0.0f, p1 = (k >= 1) ? sp[k - 1] : 0.0f;
        const float a0 = (k < L + 2) ? sa[k] : 0.0f, a1 = (k >= 1) ? sa[k - 1] : 0.0f;
        const float b0 = (k < L + 2) ? sb2[k] : 0.0f, b1 = (k >= 1) ? sb2[k - 1] : 0.0f;
        tp[k] = sh1 ? p1 : p0;
        ta[k] = sh1 ? a1 : a0;
        tb[k] = sh1 ? b1 : b0;
    }
#pragma unroll
    for (int A = 0; A < FR::NX; ++A) {
        const float p0 = (A < L + 3) ? tp[A] : 0.0f;
        const float p2 = (A >= 2 && A - 2 < L + 3) ? tp[A - 2] : 0.0f;
        const float a0 = (A < L + 3) ? ta[A] : 0.0f;
        const float a2 = (A >= 2 && A - 2 < L + 3) ? ta[A - 2] : 0.0f;
        const float b0 = (A < L + 3) ? tb[A] : 0.0f;
        const float b2 = (A >= 2 && A - 2 < L + 3) ? tb[A - 2] : 0.0f;
        r[A] = sh2 ? p2 : p0;
        r[FR::NX + A] = sh2 ? a2 : a0;
        r[2 * FR::NX + A] = sh2 ? b2 : b0;
    }
    float ty[4][L + 2];  // Ay, ky py, kz S0y, kz DSy
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        ty[0][k] = Ay[k];
        ty[1][k] = (k <= L) ? ky * py[k] : 0.0f;
        ty[2][k] = kz * Sy.s0[k];
        ty[3][k] = kz * Sy.ds[k];
    }
#pragma unroll
    for (int Bn = 0; Bn < FR::NY; ++Bn) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float v0 = (Bn <= L + 1) ? ty[f][Bn] : 0.0f;
            if constexpr (FR::SYM == 0) {
                r[FR::XS + f * FR::NY + Bn] = v0;
            } else {
                const float v1 = (Bn >= 1 && Bn - 1 <= L + 1) ? ty[f][Bn - 1] : 0.0f;
                r[FR::XS + f * FR::NY + Bn] = (oy == 1) ? v1 : v0;
            }
        }
    }
#pragma unroll
    for (int k = 3 * FR::NX; k < FR::XS; ++k) r[k] = 0.0f;
#pragma unroll
    for (int k = FR::RS0; k < FR::RS1; ++k) r[k] = 0.0f;
#pragma unroll
    for (int v = 0; v < FR::RS1 / 4; ++v)
        mine[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    __syncwarp();
    if constexpr (FR::HALF) {
        // lane (half, term, bx): term t (0: J1 = px Ay, 1: J2 = Ax py, 2: J3 from Ax S0y, 3: J3
        // from Bx DSy; lanes past the four terms idle) on the frame columns 2 bx, 2 bx + 1 and
        // all NY rows, summed over the records of parity `half`, as packed pairs (each lane
        // rounded as the scalar FMA)
        constexpr int NBX = FR::NX / 2;
        const int half = lane >> 4, hl = lane & 15;
        const int term = hl / NBX, bx = hl % NBX;
        const bool sums = term < 4;
        const int xo = sums ? (term == 0 ? 0 : (term == 3 ? 2 * FR::NX : FR::NX)) + 2 * bx : 0;
        const int yo = sums ? FR::XS + term * FR::NY : FR::XS;
        float2 o[FR::NY];
#pragma unroll
        for (int j = 0; j < FR::NY; ++j) o[j] = make_float2(0.0f, 0.0f);
#pragma unroll 8
        for (int q = 0; q < 16; ++q) {
            const float *rq = rec + (2 * q + half) * FR::RS;
            const float2 xv = *(const float2 *)(rq + xo);
            float yv[FR::NY];
            if constexpr (FR::NY == 4) {
                const float4 t = *(const float4 *)(rq + yo);
                yv[0] = t.x; yv[1] = t.y; yv[2] = t.z; yv[3] = t.w;
            } else {
                const float2 t = *(const float2 *)(rq + yo);
                yv[0] = t.x; yv[1] = t.y;
            }
#pragma unroll
            for (int j = 0; j < FR::NY; ++j) o[j] = __ffma2_rn(xv, make_float2(yv[j], yv[j]), o[j]);
        }
        // both halves' sums (a + b = b + a: the halves hold the same value), then J3's two
        // products (terms 2 and 3, NBX lanes apart within the half)
#pragma unroll
        for (int j = 0; j < FR::NY; ++j) {
            o[j].x += __shfl_xor_sync(0xffffffffu, o[j].x, 16);
            o[j].y += __shfl_xor_sync(0xffffffffu, o[j].y, 16);
        }
#pragma unroll
        for (int j = 0; j < FR::NY; ++j) {
            const float ox3 = __shfl_down_sync(0xffffffffu, o[j].x, NBX);
            const float oy3 = __shfl_down_sync(0xffffffffu, o[j].y, NBX);
            if (term == 2) {
                o[j].x += ox3;
                o[j].y += oy3;
            }
        }
        // the halves add the lower and the upper NY / 2 rows; with an even frame origin each
        // lane's two x nodes are one aligned pair (the row stride is even)
        if (!DET && (mnx & 1) == 0) {
            if (term < 3) {
                float *t = term == 0 ? st.j1 : (term == 1 ? st.j2 : st.j3);
#pragma unroll
                for (int jj = 0; jj < FR::NY / 2; ++jj) {
                    const float2 v = half ? o[FR::NY / 2 + jj] : o[jj];
                    const int gx = mnx + 2 * bx, gy = mny + (half ? FR::NY / 2 + jj : jj);
                    if (gx >= h.RX || gy >= h.RY || (v.x == 0.0f && v.y == 0.0f)) continue;
                    atomic_add_pair(t + gy * h.RX + gx, v.x, v.y);
                }
            }
        } else if (term < 3) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
#pragma unroll
                for (int jj = 0; jj < FR::NY / 2; ++jj) {
                    const int j = half ? FR::NY / 2 + jj : jj;
                    const float vlo = i == 0 ? o[jj].x : o[jj].y;
                    const float vhi = i == 0 ? o[FR::NY / 2 + jj].x : o[FR::NY / 2 + jj].y;
                    const float v = half ? vhi : vlo;
                    const int gx = mnx + 2 * bx + i, gy = mny + j;
                    if (gx >= h.RX || gy >= h.RY || v == 0.0f) continue;
                    const int node = gy * h.RX + gx;
                    if (DET) {  // fixed-point words: the warps' sums commute exactly
                        unsigned long long *t = term == 0 ? st.q1 : (term == 1 ? st.q2 : st.q3);
                        atomicAdd(t + node, det_word32(v, h.dinv32));
                    } else {
                        float *t = term == 0 ? st.j1 : (term == 1 ? st.j2 : st.j3);
                        atomicAdd(t + node, v);
                    }
                }
            }
        }
    } else {
        // this lane's sum: term t (0: J1 = px Ay, 1: J2 = Ax py, 2: J3 from Ax S0y, 3: J3 from
        // Bx DSy; lanes past the four terms idle) on the sub-block (bx, by) of the frame, as packed
        // pairs (the sub-block's two x nodes; each lane rounded as the scalar FMA)
        const int term = lane / FR::NBT, sb = lane % FR::NBT;
        const int bx = sb % (FR::NX / 2), by = sb / (FR::NX / 2);
        const bool sums = term < 4;
        const int xo = sums ? (term == 0 ? 0 : (term == 3 ? 2 * FR::NX : FR::NX)) + 2 * bx : 0;
        const int yo = sums ? FR::XS + term * FR::NY + FR::BY * by : FR::XS;
        float2 o[FR::BY];
#pragma unroll
        for (int k = 0; k < FR::BY; ++k) o[k] = make_float2(0.0f, 0.0f);
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            const float *rq = rec + q * FR::RS;
            const float2 xv = *(const float2 *)(rq + xo);
#pragma unroll
            for (int k = 0; k < FR::BY; ++k) {
                const float yv = rq[yo + k];
                o[k] = __ffma2_rn(xv, make_float2(yv, yv), o[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < FR::BY; ++k) {
            const float ox3 = __shfl_down_sync(0xffffffffu, o[k].x, FR::NBT);
            const float oy3 = __shfl_down_sync(0xffffffffu, o[k].y, FR::NBT);
            if (term == 2) {
                o[k].x += ox3;
                o[k].y += oy3;
            }
        }
        if (!DET && (mnx & 1) == 0) {
            if (term < 3) {
                float *t = term == 0 ? st.j1 : (term == 1 ? st.j2 : st.j3);
#pragma unroll
                for (int k = 0; k < FR::BY; ++k) {
                    const int gx = mnx + 2 * bx, gy = mny + FR::BY * by + k;
                    if (gx >= h.RX || gy >= h.RY || (o[k].x == 0.0f && o[k].y == 0.0f)) continue;
                    atomic_add_pair(t + gy * h.RX + gx, o[k].x, o[k].y);
                }
            }
        } else if (term < 3) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
#pragma unroll
                for (int k = 0; k < FR::BY; ++k) {
                    const int gx = mnx + 2 * bx + i, gy = mny + FR::BY * by + k;
                    const float v = i == 0 ? o[k].x : o[k].y;
                    if (gx >= h.RX || gy >= h.RY || v == 0.0f) continue;
                    const int node = gy * h.RX + gx;
                    if (DET) {  // fixed-point words: the warps' sums commute exactly
                        unsigned long long *t = term == 0 ? st.q1 : (term == 1 ? st.q2 : st.q3);
                        atomicAdd(t + node, det_word32(v, h.dinv32));
                    } else {
                        float *t = term == 0 ? st.j1 : (term == 1 ? st.j2 : st.j3);
                        atomicAdd(t + node, v);
                    }
                }
            }
        }
    }
}

// One particle per lane, 2D, staged tile.  Called by all 32 lanes of a warp together (the
// deposit is warp-collective); lanes with act == false carry no particle.  DET: a
// deterministic run (RunDev::det), whose current goes in as fixed-point words; a template
// parameter so that the default instances carry none of its code.
template <int L, int KT, typename R, bool DET = false>
__device__ __forceinline__ void particle_2d(const Hot2D h, const HotSp<R> hs,
                                            const Stage2D<R> &st, int64_t p, bool act, int x0,
                                            int y0)
{
    const int lane = threadIdx.x & 31;
    PState<R> s;
    int lx = 0, ly = 0;
    if (act) {
        if constexpr (sizeof(R) == 4) {
            const int c = __ldg(hs.cell + p);
            s.c[1] = fast_div(c, h.dm, h.ds);
            s.c[0] = c - s.c[1] * h.n0;
            s.d[0] = __ldg((const float *)hs.pos0 + p);
            s.d[1] = __ldg((const float *)hs.pos1 + p);
        } else {
            const double x0v = __ldg((const double *)hs.pos0 + p);
            const double x1v = __ldg((const double *)hs.pos1 + p);
            const double f0 = floor(x0v), f1 = floor(x1v);
            // in [0, n) by construction; the clamp keeps a non-finite position's index valid
            s.c[0] = min(max((int)f0, 0), h.n0 - 1);
            s.c[1] = min(max((int)f1, 0), h.n1 - 1);
            s.d[0] = x0v - f0;
            s.d[1] = x1v - f1;
        }
        s.c[2] = 0;
        s.u[0] = __ldg((const R *)hs.mom0 + p);
        s.u[1] = __ldg((const R *)hs.mom1 + p);
        s.u[2] = __ldg((const R *)hs.mom2 + p);
        const bool okx = local_coord(s.c[0], x0, h.tile0, h.drift0, h.n0, lx);
        const bool oky = local_coord(s.c[1], y0, h.tile1, h.drift1, h.n1, ly);
        if (!(okx && oky)) {
            set_err(h.err, 1);
            act = false;
        }
    }
    if (!act) {
        // a harmless stand-in particle at the tile origin; its current is weighted by zero
        s.c[0] = x0; s.c[1] = y0; s.c[2] = 0;
        s.d[0] = R(0.5); s.d[1] = R(0.5); s.d[2] = R(0);
        s.u[0] = s.u[1] = s.u[2] = R(0);
        lx = 0; ly = 0;
    }
    const int RX = h.RX;
    const int sx = lx + h.pre0, sy = ly + h.pre1;

    AxisW<L, KT, R> wx, wy;
    axis_weights<L, KT, R>(st.tt[0], s.d[0], wx);
    axis_weights<L, KT, R>(st.tt[1], s.d[1], wy);

    // ---- gather (Eq. interpolation-EB-real-mod; MC when the tables hold W_l) ----
    R E[3], B[3];
    if constexpr (sizeof(R) == 4) {
        gather_2d_x2<L, KT>(st, wx, wy, sx, sy, RX, E, B);
    } else {
        // (E1, B2): W along x (half nodes), T along y (integer nodes)
        R e1 = R(0), b2 = R(0);
#pragma unroll
        for (int b = 0; b < KT; ++b) {
            const int row = (sy + wy.bt + b) * RX + sx + wx.bh;
            R re = R(0), rb = R(0);
#pragma unroll
            for (int a = 0; a <= L; ++a) {
                const typename Vec2<R>::T v = st.pa[row + a];
                re += wx.wh[a] * v.x;
                rb += wx.wh[a] * v.y;
            }
            e1 += wy.wt[b] * re;
            b2 += wy.wt[b] * rb;
        }
        // (E2, B1): T along x, W along y
        R e2 = R(0), b1 = R(0);
#pragma unroll
        for (int b = 0; b <= L; ++b) {
            const int row = (sy + wy.bh + b) * RX + sx + wx.bt;
            R re = R(0), rb = R(0);
#pragma unroll
            for (int a = 0; a < KT; ++a) {
                const typename Vec2<R>::T v = st.pb[row + a];
                re += wx.wt[a] * v.x;
                rb += wx.wt[a] * v.y;
            }
            e2 += wy.wh[b] * re;
            b1 += wy.wh[b] * rb;
        }
        // E3: T T
        R e3 = R(0);
#pragma unroll
        for (int b = 0; b < KT; ++b) {
            const int row = (sy + wy.bt + b) * RX + sx + wx.bt;
            R r = R(0);
#pragma unroll
            for (int a = 0; a < KT; ++a) r += wx.wt[a] * st.e3[row + a];
            e3 += wy.wt[b] * r;
        }
        // B3: W W
        R b3 = R(0);
#pragma unroll
        for (int b = 0; b <= L; ++b) {
            const int row = (sy + wy.bh + b) * RX + sx + wx.bh;
            R r = R(0);
#pragma unroll
            for (int a = 0; a <= L; ++a) r += wx.wh[a] * st.b3[row + a];
            b3 += wy.wh[b] * r;
        }
        E[0] = e1; E[1] = e2; E[2] = e3;
        B[0] = b1; B[1] = b2; B[2] = b3;
    }

    // ---- Boris push ----
    const R ig = boris<R>(R(hs.qmdt_half), E, B, s.u);

    // ---- move ----
    R o[2], dl[2], xs[2];
    int cn[2], shv[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        dl[a] = R(a == 0 ? h.dtt0 : h.dtt1) * s.u[a] * ig;
        shv[a] = move_axis<R>(s.d[a], dl[a], s.c[a], a == 0 ? h.n0 : h.n1, o[a], cn[a], xs[a]);
    }

    // ---- Esirkepov deposit ----
    AxisS<L, R> Sx, Sy;
    if constexpr (sizeof(R) == 4) {
        axis_shapes_dd<L, true>(s.d[0], dl[0], Sx);  // all 32 lanes take part
        axis_shapes_dd<L, true>(s.d[1], dl[1], Sy);
    } else {
        // old-position weights: from the cache the previous step wrote at this particle's
        // stored position (bit-identical to evaluating them), else evaluated.  (l = 4 keeps
        // evaluating: its cache would not fit the register budget of two CTAs per SM.)
        double *wc = (L <= 3 && act && hs.wc_mode != 0) ? hs.wc + p : nullptr;
        const double *wr = hs.wc_mode == 2 ? wc : nullptr;
        const int64_t ws = hs.wc_stride;
        axis_shapes<L, R>(s.d[0], shv[0], o[0], Sx, wr, wc, ws);
        axis_shapes<L, R>(s.d[1], shv[1], o[1], Sy, wr ? wr + (L + 1) * ws : nullptr,
                          wc ? wc + (L + 1) * ws : nullptr, ws);
    }
    // the FP32 warp-collective deposit carries idle lanes with zero weight; the FP64 form
    // deposits active lanes only, and saves the three products
    const R wgt = (sizeof(R) == 8 || act) ? R(1) : R(0);
    const R kx = (sizeof(R) == 8) ? R(hs.kx0) : wgt * R(hs.kx0);
    const R ky = (sizeof(R) == 8) ? R(hs.kx1) : wgt * R(hs.kx1);
    const R kz = ((sizeof(R) == 8) ? R(hs.kz) : wgt * R(hs.kz)) * s.u[2] * ig;
    const R third = R(1) / R(3);
    // W_x = DSx (S0y + DSy/2), prefix along x; W_y = DSy (S0x + DSx/2), prefix along y;
    // W_z = S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3 = S0y Ax + DSy Bx.
    R Ax[L + 2], Ay[L + 2], Bx[L + 2], px[L + 2], py[L + 2];
    R acc_x = R(0), acc_y = R(0);
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        Ax[k] = Sx.s0[k] + R(0.5) * Sx.ds[k];
        Ay[k] = Sy.s0[k] + R(0.5) * Sy.ds[k];
        Bx[k] = R(0.5) * Sx.s0[k] + third * Sx.ds[k];
        acc_x += Sx.ds[k];
        acc_y += Sy.ds[k];
        px[k] = acc_x;
        py[k] = acc_y;
    }
    const int jx0 = sx + Sx.wb, jy0 = sy + Sy.wb;

    if constexpr (sizeof(R) == 4) {
        // Warp-collective path (cell-major order): lanes whose windows start at most SXM nodes
        // apart in x and SYM in y (up to three or four neighbouring cells along a row) form a
        // group; the group's current is a sum of per-lane outer products on a common block
        // (DepFrame), which the warp sums through shared memory and adds node by node.
        // Otherwise every lane adds its own window with shared atomics (the slot-major order,
        // lanes in different cells).
        using FR = DepFrame<L>;
        if (h.slot_major) {  // lanes in different cells: per-lane atomics do not collide
            // (shared-memory CAS atomics: measured faster here than global FP64 reductions,
            // which would need an FP32 -> FP64 conversion per node)
            const bool wide = __any_sync(0xffffffffu, act && Sy.wide);
            if (!act) {
            } else if (DET) {
                if (wide)
                    deposit_lane<L, R, true, true>(st, RX, jx0, jy0, kx, ky, kz, px, py, Ax, Ay,
                                                   Bx, Sy, h.dinv32);
                else
                    deposit_lane<L, R, false, true>(st, RX, jx0, jy0, kx, ky, kz, px, py, Ax, Ay,
                                                    Bx, Sy, h.dinv32);
            } else if (wide) {
                deposit_lane<L, R, true>(st, RX, jx0, jy0, kx, ky, kz, px, py, Ax, Ay, Bx, Sy);
            } else {
                deposit_lane<L, R, false>(st, RX, jx0, jy0, kx, ky, kz, px, py, Ax, Ay, Bx, Sy);
            }
        } else {
        // passes over groups of lanes that fit one common block (usually one pass; a warp that
        // straddles the end of a tile row takes two)
        bool todo = act;
        while (__any_sync(0xffffffffu, todo)) {
            const int mny = __reduce_min_sync(0xffffffffu, todo ? jy0 : 0x7fffffff);
            const bool rowok = todo && jy0 <= mny + FR::SYM;
            const int mnx = __reduce_min_sync(0xffffffffu, rowok ? jx0 : 0x7fffffff);
            const bool in = rowok && jx0 <= mnx + FR::SXM;
            todo = todo && !in;
            const int ox = in ? jx0 - mnx : 0, oy = in ? jy0 - mny : 0;
            const R gin = in ? R(1) : R(0);
            __syncwarp();  // the previous pass has read every record
            // a group none of whose lanes moved its y window base leaves row l + 1 of every
            // window at exact zeros (S0y = DSy = 0): its frame is two rows lower
            if (__any_sync(0xffffffffu, in && Sy.wide))
                warp_frame_pass<DepFrame<L, false>, L, DET>(h, st, gin, ox, oy, mnx, mny, kx, ky,
                                                            kz, px, py, Ax, Ay, Bx, Sy);
            else
                warp_frame_pass<DepFrame<L, true>, L, DET>(h, st, gin, ox, oy, mnx, mny, kx, ky,
                                                           kz, px, py, Ax, Ay, Bx, Sy);
        }
        }
    } else {
        // a drift along x1 rarely moves the y window: skip its empty last row warp-uniformly
        const bool wide = __any_sync(0xffffffffu, act && Sy.wide);
        const int gx0 = x0 - h.pre0 + jx0, gy0 = y0 - h.pre1 + jy0;
        if (!act) {
        } else if (DET) {
            if (wide)
                deposit_lane_global<L, R, Hot2D, true, true>(h, gx0, gy0, kx, ky, kz, px, py, Ax,
                                                             Ay, Bx, Sy);
            else
                deposit_lane_global<L, R, Hot2D, false, true>(h, gx0, gy0, kx, ky, kz, px, py,
                                                              Ax, Ay, Bx, Sy);
        } else if (wide) {
            deposit_lane_global<L, R, Hot2D, true>(h, gx0, gy0, kx, ky, kz, px, py, Ax, Ay, Bx, Sy);
        } else {
            deposit_lane_global<L, R, Hot2D, false>(h, gx0, gy0, kx, ky, kz, px, py, Ax, Ay, Bx,
                                                    Sy);
        }
    }
    if (!act) return;

    // ---- store ----
    ((R *)hs.mom0)[p] = s.u[0];
    ((R *)hs.mom1)[p] = s.u[1];
    ((R *)hs.mom2)[p] = s.u[2];
    if constexpr (sizeof(R) == 4) {
        hs.cell[p] = cn[1] * h.n0 + cn[0];
        ((float *)hs.pos0)[p] = o[0];
        ((float *)hs.pos1)[p] = o[1];
    } else {
        ((double *)hs.pos0)[p] = xs[0];  // = cn + o
        ((double *)hs.pos1)[p] = xs[1];
    }
}

// All particles of one tile (both species), 2D.  tt_shared as in stage2d_carve.  split (in
// shared memory: part, parts), when given with parts > 1: only that part of every species'
// particles of the tile (a contiguous share of its range) -- the batched kernel splits the
// heavy tiles of a small run set over several CTAs, each staging the tile and adding its own
// share of the current.  (Read where used, so that it holds no registers across the tile.)
template <int L, int KT, typename R, bool DET = false>
__device__ void tile_2d(const RunDev &rd, char *smem, int64_t tile,
                        const TTable *tt_shared = nullptr, const int *split = nullptr)
{
    Stage2D<R> st = stage2d_carve<R>(smem, rd.reg_nodes, tt_shared, DET);
    const int tx = (int)(tile % rd.ntile[0]);
    const int ty = (int)(tile / rd.ntile[0]);
    const int x0 = tx * rd.tile[0], y0 = ty * rd.tile[1];
    stage2d_load<R>(rd, st, x0, y0);
    const Hot2D h = make_hot2d(rd);
    __syncthreads();
    for (int s = 0; s < rd.nsp; ++s) {
        const SpeciesDev &sp = rd.sp[s];
        const HotSp<R> hs = make_hotsp<R>(sp);
        int64_t a = sp.tile_start[tile], b = sp.tile_start[tile + 1];
        if (split != nullptr && split[1] > 1) {  // (fewer than 2^27 particles per tile)
            const int len = (int)(b - a), part = split[0], parts = split[1];
            b = a + (len * (part + 1)) / parts;
            a += (len * part) / parts;
        }
        if constexpr (sizeof(R) == 4) {
            // every warp takes a contiguous chunk of the tile's particles of this species (for a
            // uniform plasma in the cell-major order, one row of cells), so that the warps'
            // frames, a row apart, rarely race for the same nodes of the tile: 5.53 -> 5.38 ms
            // on the 134M-particle FP32 step (slot-major runs, whose lanes deposit one by one,
            // lose about 5%; a runtime choice between the two loops cost the dense kernel more)
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int64_t groups = (b - a + 31) / 32;
            const int64_t gw = (groups + kTileWarps - 1) / kTileWarps;
            const int64_t ca = a + 32 * min(groups, (int64_t)w * gw);
            const int64_t cb = min(b, a + 32 * min(groups, (int64_t)(w + 1) * gw));
            for (int64_t q = ca; q < cb; q += 32) {  // warp-uniform trip count
                const int64_t p = q + lane;
                if (p + 32 < cb) prefetch_particle<R>(hs, p + 32);
                particle_2d<L, KT, R, DET>(h, hs, st, p, p < cb, x0, y0);
            }
        } else {
            // warp-uniform trip count: a warp's lanes take 32 consecutive particles
            const int64_t wbase = a + (threadIdx.x & ~31);
            for (int64_t q = wbase; q < b; q += blockDim.x) {
                const int64_t p = q + (threadIdx.x & 31);
                if (p + blockDim.x < b) {
                    prefetch_particle<R>(hs, p + blockDim.x);
                    if constexpr (sizeof(R) == 8 && L <= 3)
                        if (hs.wc_mode == 2) prefetch_weights<L>(hs, p + blockDim.x);
                }
                particle_2d<L, KT, R, DET>(h, hs, st, p, p < b, x0, y0);
            }
        }
        if constexpr (sizeof(R) == 4) {  // the FP64 form deposits to global memory directly
            __syncthreads();
            stage2d_flush<R>(rd, st, x0, y0);
            __syncthreads();
        }
    }
}

}  // namespace pic
