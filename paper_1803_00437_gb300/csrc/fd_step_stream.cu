// fd_step_stream.cu -- FD-LBM step (Sec. 2, Eq. 2) for periodic lattices,
// streaming each warp down a strip of rows.
//
// Work decomposition.  A warp owns an output strip of 120 columns and a
// segment of rows.  Lane L holds 4 consecutive columns starting at
// strip0 - 4 + 4 L, so lanes 0 and 31 are halo lanes: they reconstruct the
// populations one column outside the strip (where the gradients they need
// are still exact) and store nothing.  Warps never synchronise with each
// other.
//
// Data path per warp.  Rows of (rho - 1, ux, uy) for the strip plus 8 halo
// columns are copied by 1-D bulk (TMA) copies into a private ring of
// shared-memory slots, each slot completed by an mbarrier, several rows
// ahead of use.  Each lane reads its 4 columns (one 16-byte load per field
// for FP32).  Derivatives along y use a register window over rows (for five
// points, d1(c) = f(c+1) - f(c-1) and 8 d/dy = 6 d1(c) - d1(c-1) - d1(c+1),
// so four rows are held); derivatives along x use warp shuffles of the two
// neighbouring columns on each side.  After the reconstruction the
// populations that cross a lane boundary are exchanged by shuffles, summed
// per destination row and closed when the row below has contributed.
// Outputs are written with 16-byte (FP32) stores.
#include <algorithm>

#include "fd_common.cuh"
#include "tma_ring.cuh"

namespace fdlbm {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kStrip = 120;     // output columns per warp
constexpr int kLoadCols = 136;  // columns staged per row: strip0 - 8 .. strip0 + 128
constexpr int kSlots = 6;       // ring depth (rows)
// Resident CTAs per SM requested from the register allocator (168
// registers for three): measured on GB300, three is fastest for both
// stencils (five points: 137.5 vs 133.8 GLUPS at two).
#ifndef FDLBM_STREAM_MIN_BLOCKS5
#define FDLBM_STREAM_MIN_BLOCKS5 3
#endif
template <int R>
constexpr int min_blocks() { return R == 1 ? 3 : FDLBM_STREAM_MIN_BLOCKS5; }
constexpr unsigned kFull = 0xffffffffu;

// Paired FP32 arithmetic (two lattice columns per instruction).
__device__ __forceinline__ float2 sp(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b (b * -1 is exact, so this rounds once like a subtraction)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, sp(-1.f), a); }

// Hardware reciprocal (relative error ~2^-23).  Used only where it scales a
// small correction term, so its error is far below FP32 resolution.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec4<__half> {
    static __device__ __forceinline__ void load(const __half* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(__half* p, const float v[4]) {
        __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t*>(&a);
        q.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};
template <>
struct Vec4<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, const float v[4]) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t*>(&a);
        q.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};

// Fields kept in the y window: rho - 1, Jx, Jy, Jx Jy / rho, Jy Jy / rho.
enum { W_R = 0, W_JX, W_JY, W_PXY, W_PYY, W_N };

// v[f][0] holds columns (0, 1), v[f][1] columns (2, 3) of this lane.
struct Win {
    float2 v[W_N][2];
};

struct StreamArgs {
    const void* src;   // 3 planes (rho - 1, ux, uy), [ny][pitch]
    void* dst;
    size_t plane;      // elements per plane
    size_t pitch;      // elements per row
    int nx, ny;
    int nstrips, seg_rows, nsegs, nitems;
    FdCoeffs c;
    int* status;       // device status word (FDLBM_ERR_TIMEOUT on a lost copy)
};

template <typename T>
struct Ring {
    T* slot_base;       // kSlots x 3 x kLoadCols elements
    uint64_t* bars;     // kSlots barriers
};

template <typename T>
__device__ __forceinline__ T* slot_field(const Ring<T>& ring, int slot, int field) {
    return ring.slot_base + ((size_t)slot * 3 + field) * kLoadCols;
}

// Column pieces of a strip's staged row: kLoadCols columns starting at x0
// (wrapping once at nx).  Fixed for a work item.
struct Cols {
    int x0, first;
};

__device__ __forceinline__ Cols strip_cols(const StreamArgs& a, int strip0) {
    Cols c;
    c.x0 = wrap_index(strip0 - 8, a.nx);
    c.first = min(kLoadCols, a.nx - c.x0);
    return c;
}

// Issue the copies of one row (3 fields) into a slot; row already in
// [0, ny).  Called by the whole warp: lane 0 arms the barrier with the
// row's byte count, then lanes 0..2 each copy one field (one or two pieces).
template <typename T>
__device__ __forceinline__ void issue_row(const StreamArgs& a, const Ring<T>& ring, int slot,
                                          int r, const Cols& cols, int lane) {
    uint64_t* bar = &ring.bars[slot];
    if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, 3u * kLoadCols * sizeof(T));
    }
    __syncwarp();
    if (lane < 3) {
        fence_proxy_async_smem();
        const T* rowp = static_cast<const T*>(a.src) + lane * a.plane + (size_t)r * a.pitch;
        T* dst = slot_field(ring, slot, lane);
        tma_load_1d(dst, rowp + cols.x0, cols.first * sizeof(T), bar);
        if (cols.first < kLoadCols)
            tma_load_1d(dst + cols.first, rowp, (kLoadCols - cols.first) * sizeof(T), bar);
    }
}

__device__ __forceinline__ int next_row(int r, int ny) { return r + 1 == ny ? 0 : r + 1; }

// x-derivative (scaled by 2 or 8) at the 4 columns of this lane of one
// field given as two column pairs.
template <int R>
__device__ __forceinline__ void deriv_x(const float2 v[2], float2 d[2]) {
    const float f0 = v[0].x, f1 = v[0].y, f2 = v[1].x, f3 = v[1].y;
    const float l1 = __shfl_up_sync(kFull, f3, 1);
    const float r0 = __shfl_down_sync(kFull, f0, 1);
    if (R == 1) {
        // 2 d/dx = f(+1) - f(-1)
        d[0] = make_float2(f1 - l1, f2 - f0);
        d[1] = make_float2(f3 - f1, r0 - f2);
    } else {
        // 8 d/dx = 6 (f(+1) - f(-1)) - (f(+2) - f(-2))
        const float l2 = __shfl_up_sync(kFull, f2, 1);
        const float r1 = __shfl_down_sync(kFull, f1, 1);
        d[0] = fma2(sp(6.f), make_float2(f1 - l1, f2 - f0), make_float2(l2 - f2, l1 - f3));
        d[1] = fma2(sp(6.f), make_float2(f3 - f1, r0 - f2), make_float2(f0 - r0, f1 - r1));
    }
}

// g = M^-1 m' in deviation form for two columns at once; same arithmetic
// as moments_to_populations (conserved moments reproduced with unbiased
// roundings: sx = (jx - 2 tx)/4, g0 = dr - 4 (axis + diag)), with q = -J.
__device__ __forceinline__ void populations2(float2 dr, float2 jx, float2 jy, float2 Jx, float2 Jy,
                                             float2 e, float2 xx, float2 xy, float2 ep,
                                             float2 g[9]) {
    const float2 r9 = mul2(dr, sp(1.f / 9.f));
    const float2 axis = fma2(e, sp(-1.f / 36.f), fma2(ep, sp(-1.f / 18.f), r9));
    const float2 diag = fma2(e, sp(1.f / 18.f), fma2(ep, sp(1.f / 36.f), r9));
    g[0] = fma2(sp(-4.f), add2(axis, diag), dr);
    const float2 tx = mul2(add2(jx, Jx), sp(1.f / 6.f));  // (jx - qx) / 6
    const float2 ty = mul2(add2(jy, Jy), sp(1.f / 6.f));
    const float2 sx = mul2(fma2(sp(-2.f), tx, jx), sp(0.25f));
    const float2 sy = mul2(fma2(sp(-2.f), ty, jy), sp(0.25f));
    const float2 ax = fma2(xx, sp(0.25f), axis), ay = fma2(xx, sp(-0.25f), axis);
    const float2 dp = fma2(xy, sp(0.25f), diag), dm = fma2(xy, sp(-0.25f), diag);
    const float2 spp = add2(sx, sy), smm = sub2(sy, sx);
    g[1] = add2(ax, tx);
    g[3] = sub2(ax, tx);
    g[2] = add2(ay, ty);
    g[4] = sub2(ay, ty);
    g[5] = add2(dp, spp);
    g[7] = sub2(dp, spp);
    g[6] = add2(dm, smm);
    g[8] = sub2(dm, smm);
}

// Reconstruction (Sec. 2) of two columns from scaled derivatives; the
// derivative scale is folded into the relaxation factors a_e, a_xx.
__device__ __forceinline__ void reconstruct2(float2 dr, float2 ux, float2 uy, float2 Jx, float2 Jy,
                                             float2 dxr,
                                             float2 dyr, float2 dxjx, float2 dyjx, float2 dxjy,
                                             float2 dyjy, float2 dxpxx, float2 dxpxy,
                                             float2 dypxy, float2 dypyy, float2 a_e, float2 a_xx,
                                             float2 hf_x, float2 hf_y, float2 g[9]) {
    const float2 nuy = mul2(uy, sp(-1.f));
    const float2 uxx = mul2(ux, ux), uyy = mul2(uy, uy), uxy = mul2(ux, uy);
    const float2 u2 = add2(uxx, uyy);
    const float2 mx = add2(dxpxx, dypxy);
    const float2 my = add2(dxpxy, dypyy);
    // theta_E = (2 + 6 u^2)(d.J) - 2 (u . grad rho)
    const float2 udr = fma2(uy, dyr, mul2(ux, dxr));
    const float2 th_e = fma2(sp(-2.f), udr, mul2(fma2(sp(6.f), u2, sp(2.f)), add2(dxjx, dyjy)));
    // theta_XX = 2/3 ((dxJx - dyJy) - (ux dxr - uy dyr)) - 2 (ux mx - uy my)
    const float2 b = sub2(sub2(dxjx, dyjy), fma2(ux, dxr, mul2(nuy, dyr)));
    const float2 th_xx = fma2(sp(2.f / 3.f), b, mul2(sp(-2.f), fma2(ux, mx, mul2(nuy, my))));
    // theta_XY = 1/3 ((dxJy + dyJx) - (ux dyr + uy dxr)) - (ux my + uy mx)
    const float2 c = sub2(add2(dxjy, dyjx), fma2(ux, dyr, mul2(uy, dxr)));
    const float2 th_xy = sub2(mul2(sp(1.f / 3.f), c), fma2(ux, my, mul2(uy, mx)));
    const float2 ru2 = fma2(dr, u2, u2);
    const float2 dxx = sub2(uxx, uyy);
    const float2 e = fma2(sp(-2.f), dr, fma2(sp(3.f), ru2, mul2(a_e, th_e)));
    const float2 xx = fma2(a_xx, th_xx, fma2(dr, dxx, dxx));
    const float2 xy = fma2(a_xx, th_xy, fma2(dr, uxy, uxy));
    const float2 ep = fma2(sp(-3.f), ru2, dr);
    populations2(dr, add2(Jx, hf_x), add2(Jy, hf_y), Jx, Jy, e, xx, xy, ep, g);
}

// Per-lane gather state, in column pairs: destination row c (partial, "A")
// and c + 1 (contribution of row c's upward populations, "U").
struct Acc {
    float2 ar[2], ax[2], ay[2];  // row c: rho - 1, Jx, Jy (missing row c + 1)
    float2 us[2], ud[2];         // row c + 1: sum and x-difference of g2, g5, g6
};

template <typename T>
__device__ __forceinline__ void load4(const T* p, float2 v[2]) {
    float f[4];
    Vec4<T>::load(p, f);
    v[0] = make_float2(f[0], f[1]);
    v[1] = make_float2(f[2], f[3]);
}

template <typename T>
__device__ __forceinline__ void store4(T* p, const float2 v[2]) {
    const float f[4] = {v[0].x, v[0].y, v[1].x, v[1].y};
    Vec4<T>::store(p, f);
}

// Per-item constants of a warp.
struct Item {
    int strip0, yb, ye, row_first, nrows;
    Cols cols;
};

template <int R, typename T>
struct RowStep {
    // Field row k of the item: wait for it, read it, update the y window and
    // reconstruct the centre row c = row k - R; close and store row c - 1.
    static __device__ __forceinline__ void run(const StreamArgs& a, const Ring<T>& ring,
                                               const Item& it, int lane, int k, uint32_t load_no,
                                               Win& fm2, Win& fm1, Win& dm3, Win& dm2, Acc& acc,
                                               bool& ok, uint32_t& issued, int& next_load_row) {
        const int slot = load_no % kSlots;
        const uint32_t phase = (load_no / kSlots) & 1u;
        const bool landed = __all_sync(kFull, mbar_wait_bounded(&ring.bars[slot], phase));
        if (!landed) {
            ok = false;
            return;
        }
        const int col = 4 + 4 * lane;  // slot column of this lane's first column
        float2 nr[2], nux[2], nuy[2];
        load4<T>(slot_field(ring, slot, 0) + col, nr);
        load4<T>(slot_field(ring, slot, 1) + col, nux);
        load4<T>(slot_field(ring, slot, 2) + col, nuy);
        Win nw;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 jx = fma2(nr[h], nux[h], nux[h]), jy = fma2(nr[h], nuy[h], nuy[h]);
            nw.v[W_R][h] = nr[h];
            nw.v[W_JX][h] = jx;
            nw.v[W_JY][h] = jy;
            nw.v[W_PXY][h] = mul2(jx, nuy[h]);
            nw.v[W_PYY][h] = mul2(jy, nuy[h]);
        }
        // centre row c = r - R from its ring slot (still resident); before
        // the window is full the centre row does not exist yet
        const int cslot = (load_no + kSlots - R) % kSlots;
        float2 cdr[2] = {sp(0.f), sp(0.f)}, cux[2] = {sp(0.f), sp(0.f)};
        float2 cuy[2] = {sp(0.f), sp(0.f)};
        if (k >= R) {
            if (R == 2) load4<T>(slot_field(ring, cslot, 0) + col, cdr);
            load4<T>(slot_field(ring, cslot, 1) + col, cux);
            load4<T>(slot_field(ring, cslot, 2) + col, cuy);
        }
        // Five points: the centre row's fields are rebuilt from the ring
        // (only the differences d1 are held in registers).  Three points:
        // the centre row is held (fm1).
        Win rebuilt;
        if (R == 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 jx = fma2(cdr[h], cux[h], cux[h]), jy = fma2(cdr[h], cuy[h], cuy[h]);
                rebuilt.v[W_R][h] = cdr[h];
                rebuilt.v[W_JX][h] = jx;
                rebuilt.v[W_JY][h] = jy;
                rebuilt.v[W_PXY][h] = mul2(jx, cuy[h]);
                rebuilt.v[W_PYY][h] = mul2(jy, cuy[h]);
            }
        }
        const Win& cen = (R == 1) ? fm1 : rebuilt;
        // y derivatives at the centre row (scaled by 2 or 8):
        //   three points: 2 d/dy = f(c+1) - f(c-1)
        //   five points:  8 d/dy = 6 d1(c) - d1(c-1) - d1(c+1), d1(c+1) = f(r) - f(c);
        //   the window holds n1 = -d1, so 8 d/dy = -6 n1(c) + n1(c-1) + n1(c+1)
        Win dy, d1new;
#pragma unroll
        for (int f = 0; f < W_N; ++f)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (R == 1) {
                    dy.v[f][h] = sub2(nw.v[f][h], fm2.v[f][h]);
                } else {
                    d1new.v[f][h] = sub2(cen.v[f][h], nw.v[f][h]);
                    dy.v[f][h] = fma2(sp(-6.f), dm2.v[f][h], add2(dm3.v[f][h], d1new.v[f][h]));
                }
            }
        // x derivatives at the centre row
        float2 pxx[2], dxr[2], dxjx[2], dxjy[2], dxpxx[2], dxpxy[2];
        pxx[0] = mul2(cen.v[W_JX][0], cux[0]);
        pxx[1] = mul2(cen.v[W_JX][1], cux[1]);
        deriv_x<R>(cen.v[W_R], dxr);
        deriv_x<R>(cen.v[W_JX], dxjx);
        deriv_x<R>(cen.v[W_JY], dxjy);
        deriv_x<R>(pxx, dxpxx);
        deriv_x<R>(cen.v[W_PXY], dxpxy);

        const float sc = (R == 1) ? 0.5f : 0.125f;
        const float2 a_e = sp(a.c.a_e * sc), a_xx = sp(a.c.a_xx * sc);
        const float2 hf_x = sp(0.5f * a.c.fx), hf_y = sp(0.5f * a.c.fy);
        float2 g[2][9];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            reconstruct2(cen.v[W_R][h], cux[h], cuy[h], cen.v[W_JX][h], cen.v[W_JY][h], dxr[h],
                         dy.v[W_R][h], dxjx[h],
                         dy.v[W_JX][h], dxjy[h], dy.v[W_JY][h], dxpxx[h], dxpxy[h],
                         dy.v[W_PXY][h], dy.v[W_PYY][h], a_e, a_xx, hf_x, hf_y, g[h]);

        // populations crossing lane boundaries: right-going (1, 5, 8) of
        // column 3 to the next lane, left-going (3, 6, 7) of column 0 back
        const float in1 = __shfl_up_sync(kFull, g[1][1].y, 1);
        const float in5 = __shfl_up_sync(kFull, g[1][5].y, 1);
        const float in8 = __shfl_up_sync(kFull, g[1][8].y, 1);
        const float in3 = __shfl_down_sync(kFull, g[0][3].x, 1);
        const float in6 = __shfl_down_sync(kFull, g[0][6].x, 1);
        const float in7 = __shfl_down_sync(kFull, g[0][7].x, 1);
        // per destination column j: from j - 1 (1, 5, 8) and from j + 1 (3, 6, 7)
        const float2 p1[2] = {make_float2(in1, g[0][1].x), make_float2(g[0][1].y, g[1][1].x)};
        const float2 p5[2] = {make_float2(in5, g[0][5].x), make_float2(g[0][5].y, g[1][5].x)};
        const float2 p8[2] = {make_float2(in8, g[0][8].x), make_float2(g[0][8].y, g[1][8].x)};
        const float2 p3[2] = {make_float2(g[0][3].y, g[1][3].x), make_float2(g[1][3].y, in3)};
        const float2 p6[2] = {make_float2(g[0][6].y, g[1][6].x), make_float2(g[1][6].y, in6)};
        const float2 p7[2] = {make_float2(g[0][7].y, g[1][7].x), make_float2(g[1][7].y, in7)};

        // destination row c - 1 is complete once row c's downward
        // populations arrive; c is the centre row
        const int c_row = it.row_first + k - R;
        const bool store = (c_row - 1 >= it.yb) && (c_row - 1 < it.ye) && lane >= 1 &&
                           lane <= 30 && (it.strip0 - 4 + 4 * lane) < a.nx;
        float2 odr[2], oux[2], ouy[2];
        const float2 hfx = sp(0.5f * a.c.fx), hfy = sp(0.5f * a.c.fy);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 ss = add2(g[h][0], add2(p1[h], p3[h])), ds = sub2(p1[h], p3[h]);
            const float2 su = add2(g[h][2], add2(p5[h], p6[h])), du = sub2(p5[h], p6[h]);
            const float2 sd = add2(g[h][4], add2(p7[h], p8[h])), dd = sub2(p8[h], p7[h]);
            // close row c - 1: u = J - J dr / (1 + dr)
            const float2 drn = add2(acc.ar[h], sd);
            const float2 px = add2(add2(acc.ax[h], dd), hfx);
            const float2 py = add2(sub2(acc.ay[h], sd), hfy);
            const float2 nrho = fma2(drn, sp(-1.f), sp(-1.f));  // -(1 + dr)
            const float2 ninv = make_float2(rcp_approx(nrho.x), rcp_approx(nrho.y));
            odr[h] = drn;
            oux[h] = fma2(mul2(px, drn), ninv, px);
            ouy[h] = fma2(mul2(py, drn), ninv, py);
            // row c: upward part of row c - 1 plus the same-row part
            acc.ar[h] = add2(acc.us[h], ss);
            acc.ax[h] = add2(acc.ud[h], ds);
            acc.ay[h] = acc.us[h];
            acc.us[h] = su;
            acc.ud[h] = du;
        }
        if (store) {
            T* dst = static_cast<T*>(a.dst);
            const size_t o = (size_t)(c_row - 1) * a.pitch + (it.strip0 - 4 + 4 * lane);
            store4<T>(dst + o, odr);
            store4<T>(dst + a.plane + o, oux);
            store4<T>(dst + 2 * a.plane + o, ouy);
        }

        // rotate the window: the oldest row/difference take the new ones
        if (R == 1) fm2 = nw;
        if (R == 2) dm3 = d1new;

        // the centre row's slot is no longer needed: refill it with the row
        // kSlots ahead
        __syncwarp();
        if (k >= R && k - R + kSlots < it.nrows) {
            issue_row<T>(a, ring, cslot, next_load_row, it.cols, lane);
            next_load_row = next_row(next_load_row, a.ny);
            ++issued;
        }
    }
};

template <int R, typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, min_blocks<R>())
    fd_step_stream_kernel(StreamArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t slot_bytes = (size_t)3 * kLoadCols * sizeof(T);
    const size_t warp_bytes = kSlots * slot_bytes;
    Ring<T> ring;
    ring.slot_base = reinterpret_cast<T*>(smem + warp * warp_bytes);
    ring.bars = reinterpret_cast<uint64_t*>(smem + kWarpsPerBlock * warp_bytes) + warp * kSlots;
    if (lane == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(&ring.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    uint32_t loads = 0;   // rows consumed by this warp in finished items (ring position)
    uint32_t issued = 0;  // row copies issued by this warp
    uint32_t consumed = 0;
    bool ok = true;
    for (int item = blockIdx.x * kWarpsPerBlock + warp; item < a.nitems && ok;
         item += gridDim.x * kWarpsPerBlock) {
        Item it;
        const int strip = item % a.nstrips, seg = item / a.nstrips;
        it.strip0 = strip * kStrip;
        it.yb = seg * a.seg_rows;
        it.ye = min(a.ny, it.yb + a.seg_rows);
        it.row_first = it.yb - 1 - R;
        it.nrows = it.ye - it.yb + 2 + 2 * R;
        it.cols = strip_cols(a, it.strip0);
        int next_load_row = wrap_index(it.row_first, a.ny);
        const int prologue = min(kSlots, it.nrows);
        for (int k = 0; k < prologue; ++k) {
            issue_row<T>(a, ring, (loads + k) % kSlots, next_load_row, it.cols, lane);
            next_load_row = next_row(next_load_row, a.ny);
        }
        issued += prologue;
        __syncwarp();
        Win w0 = {}, w1 = {}, w2 = {}, w3 = {};
        Acc acc = {};
        int k = 0;
        for (; k + 1 < it.nrows; k += 2) {
            RowStep<R, T>::run(a, ring, it, lane, k, loads + k, w0, w1, w2, w3, acc, ok, issued,
                               next_load_row);
            if (!ok) {
                consumed = loads + k;
                break;
            }
            RowStep<R, T>::run(a, ring, it, lane, k + 1, loads + k + 1, w1, w0, w3, w2, acc, ok,
                               issued, next_load_row);
            if (!ok) {
                consumed = loads + k + 1;
                break;
            }
        }
        if (ok && k < it.nrows) {
            RowStep<R, T>::run(a, ring, it, lane, k, loads + k, w0, w1, w2, w3, acc, ok, issued,
                               next_load_row);
            if (!ok) consumed = loads + k;
        }
        loads += it.nrows;
    }
    if (!ok) {
        // A copy did not complete in time: record it, then give every copy
        // still in flight a bounded chance to land before the CTA exits.
        if (lane == 0) atomicExch(a.status, FDLBM_ERR_TIMEOUT);
        for (uint32_t n = consumed; n < issued; ++n)
            mbar_wait_bounded(&ring.bars[n % kSlots], (n / kSlots) & 1u);
    }
}

struct Plan {
    int seg_rows, nsegs, nitems, blocks;
};

// Segment length that balances the waves: the critical path is
// ceil(items / resident warps) * (segment + halo rows).
Plan make_plan(int nx, int ny, int R, int resident_warps) {
    const int nstrips = (nx + kStrip - 1) / kStrip;
    Plan best{ny, 1, nstrips, 0};
    long long best_cost = -1;
    for (int s = 16; s <= ny; s += (s < 128 ? 8 : 16)) {
        const int nsegs = (ny + s - 1) / s;
        const int items = nstrips * nsegs;
        const long long waves = (items + resident_warps - 1) / resident_warps;
        const long long cost = waves * (long long)(s + 2 + 2 * R);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best.seg_rows = s;
            best.nsegs = nsegs;
            best.nitems = items;
        }
    }
    if (ny < 16) {
        best.seg_rows = ny;
        best.nsegs = 1;
        best.nitems = nstrips;
    }
    best.blocks = (best.nitems + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return best;
}

template <int R, typename T>
cudaError_t launch_stream_typed(fdlbm_s* h, const void* src, void* dst) {
    const size_t smem = kWarpsPerBlock * (kSlots * 3 * kLoadCols * sizeof(T) + kSlots * 8);
    static bool attr_set = false;  // per template instance; set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fd_step_stream_kernel<R, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (h->stream_plan_warps == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fd_step_stream_kernel<R, T>,
                                                      kWarpsPerBlock * 32, smem);
        h->stream_plan_warps = std::max(1, sms * per_sm * kWarpsPerBlock);
    }
    const Plan plan = make_plan(h->p.nx, h->p.ny, R, h->stream_plan_warps);
    StreamArgs a;
    a.src = src;
    a.dst = dst;
    a.plane = h->L.plane;
    a.pitch = h->L.pitch;
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.nstrips = (h->p.nx + kStrip - 1) / kStrip;
    a.seg_rows = plan.seg_rows;
    a.nsegs = plan.nsegs;
    a.nitems = plan.nitems;
    a.c.a_e = (float)(1.0 - 1.0 / h->p.s_e);
    a.c.a_xx = (float)(1.0 - 1.0 / h->p.s_xx);
    a.c.fx = (float)h->p.force_x;
    a.c.fy = (float)h->p.force_y;
    a.c.xi = (float)h->p.wall_xi;
    a.status = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    fd_step_stream_kernel<R, T><<<plan.blocks, kWarpsPerBlock * 32, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stream_stencil(fdlbm_s* h, const void* src, void* dst) {
    if (h->p.scheme == FDLBM_SCHEME_FD3) return launch_stream_typed<1, T>(h, src, dst);
    return launch_stream_typed<2, T>(h, src, dst);
}

}  // namespace

bool fd_stream_supported(const fdlbm_params& p) {
    return p.boundary == FDLBM_BOUNDARY_PERIODIC && p.nx % 8 == 0 && p.nx >= 256 && p.ny >= 16;
}

cudaError_t launch_fd_step_stream(fdlbm_s* h, const void* src, void* dst) {
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return launch_stream_stencil<__half>(h, src, dst);
        case FDLBM_STORAGE_BF16: return launch_stream_stencil<__nv_bfloat16>(h, src, dst);
        default: return launch_stream_stencil<float>(h, src, dst);
    }
}

}  // namespace fdlbm
