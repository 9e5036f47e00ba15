// fd_stream_common.cuh -- device code shared by the streaming FD-LBM kernels
// (single lattice and batched): paired FP32 arithmetic on column pairs,
// 4-column vector access in each storage type, x-derivatives by warp
// shuffles and the reconstruction of Sec. 2 in deviation form.
#pragma once

#include "fd_common.cuh"

namespace fdlbm {
namespace stream {

constexpr unsigned kFull = 0xffffffffu;

// ---- paired FP32 arithmetic (two lattice columns per instruction) --------------

__device__ __forceinline__ float2 sp(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// Hardware reciprocal (relative error ~2^-23), flushing subnormals (its
// argument is -(1 + rho') ~ -1, never subnormal; the non-flushing form adds
// subnormal handling around the reciprocal).  Used only where it scales a
// small correction term, so its error is far below FP32 resolution.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- storage of 4 consecutive columns ----------------------------------------------

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float2 v[2]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    }
    // two 8-byte stores straight from the column-pair registers (a 16-byte
    // store would need both pairs in one aligned register quad); the halves
    // of each 16-byte chunk merge in L2
    static __device__ __forceinline__ void store(float* p, const float2 v[2]) {
        reinterpret_cast<float2*>(p)[0] = v[0];
        reinterpret_cast<float2*>(p)[1] = v[1];
    }
};
template <>
struct Vec4<__half> {
    static __device__ __forceinline__ void load(const __half* p, float2 v[2]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        v[1] = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    }
    static __device__ __forceinline__ void store(__half* p, const float2 v[2]) {
        __half2 a = __float22half2_rn(v[0]), b = __float22half2_rn(v[1]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t*>(&a);
        q.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};
template <>
struct Vec4<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const __nv_bfloat16* p, float2 v[2]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        v[1] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, const float2 v[2]) {
        __nv_bfloat162 a = __float22bfloat162_rn(v[0]), b = __float22bfloat162_rn(v[1]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t*>(&a);
        q.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};

// Fixed-point storage (FDLBM_STORAGE_I16): 4 columns of int16 q, read as
// q * scale and written as q = RN(v / scale) clamped to +-32767 (the
// rounding of quantize16); store() returns true if a value saturated (or was
// not finite: such a value is stored as 0, and the lattice reports it).
template <>
struct Vec4<int16_t> {
    static __device__ __forceinline__ float2 pair(uint32_t w, float scale) {
        const float lo = (float)((int)(w << 16) >> 16), hi = (float)((int)w >> 16);
        return mul2(make_float2(lo, hi), sp(scale));
    }
    static __device__ __forceinline__ void load(const int16_t* p, float2 v[2], Quant q) {
        const uint2 w = *reinterpret_cast<const uint2*>(p);
        v[0] = pair(w.x, q.scale);
        v[1] = pair(w.y, q.scale);
    }
    // A saturating round-to-nearest-even conversion per value and one packed
    // 16-bit max that lifts -32768 to -32767 (measured 3 % faster on the FD-5
    // step than clamping in FP32 and rounding by the 1.5 * 2^23 addition;
    // the same codes within the range).
    static __device__ __forceinline__ uint32_t pack(float2 v, float inv, bool& sat) {
        const float2 t = mul2(v, sp(inv));
        sat |= !(fabsf(t.x) <= 32767.f) || !(fabsf(t.y) <= 32767.f);
        unsigned short a, b;
        asm("cvt.rni.sat.s16.f32 %0, %1;" : "=h"(a) : "f"(t.x));
        asm("cvt.rni.sat.s16.f32 %0, %1;" : "=h"(b) : "f"(t.y));
        return __vmaxs2((uint32_t)a | ((uint32_t)b << 16), 0x80018001u);
    }
    static __device__ __forceinline__ bool store(int16_t* p, const float2 v[2], Quant q) {
        bool sat = false;
        uint2 w;
        w.x = pack(v[0], q.inv, sat);
        w.y = pack(v[1], q.inv, sat);
        *reinterpret_cast<uint2*>(p) = w;
        return sat;
    }
};

// The floating-point storage types through the same interface (no scale,
// never saturated).
template <typename T>
__device__ __forceinline__ void vec4_load(const T* p, float2 v[2], Quant) {
    Vec4<T>::load(p, v);
}
template <>
__device__ __forceinline__ void vec4_load<int16_t>(const int16_t* p, float2 v[2], Quant q) {
    Vec4<int16_t>::load(p, v, q);
}
template <typename T>
__device__ __forceinline__ bool vec4_store(T* p, const float2 v[2], Quant) {
    Vec4<T>::store(p, v);
    return false;
}
template <>
__device__ __forceinline__ bool vec4_store<int16_t>(int16_t* p, const float2 v[2], Quant q) {
    return Vec4<int16_t>::store(p, v, q);
}

// Fields of the y window: rho - 1, Jx, Jy, Jx Jy / rho, Jy Jy / rho, each as
// two column pairs: v[f][0] = columns (0, 1), v[f][1] = columns (2, 3).
enum { W_R = 0, W_JX, W_JY, W_PXY, W_PYY, W_N };

struct Win {
    float2 v[W_N][2];
};

// Relaxation factors with the derivative scale (2 or 8) and the constants
// of theta and of M^-1 folded in (see reconstruct2).
struct StreamCoeffs {
    float e6, e2, em2;  // theta_E terms, times (1 - 1/s_e) / (36 scale)
    float xm23, x13;    // -2/3 and 1/3, times (1 - 1/s_xx) / scale (theta_XX, theta_XY)
    float hfx, hfy;            // half of the body force
    float lw_t;                // LW-ACM: 2 nu
};

// x-derivative (scaled by 2 or 8) at the 4 columns of this lane.
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

// Reconstruction (Sec. 2) of two columns, g_a = f*_a - w_a, from scaled
// derivatives.  With K_E = (1 - 1/s_e) theta_E, K_XX, K_XY likewise and
// u2 = |u|^2, the moments of the table of Sec. 2 substituted into M^-1 give
//   g0 = dr - 4 (axis + diag)            (so that sum g = dr, unbiased)
//   axis = dr/9 + rho u2/12 - K_E/36,     diag = dr/36 + rho u2/12 + K_E/18
//   tx = (jx + Jx)/6, sx = (jx - 2 tx)/4 (so that sum c g = jx, unbiased),
//   carried as 2 tx and 4 sx (exact scalings, the same roundings)
//   g1,3 = axis + XX/4 +- tx,  g2,4 = axis - XX/4 +- ty,
//   g5,7 = diag + XY/4 +- (sx + sy),  g6,8 = diag - XY/4 +- (sy - sx),
// with jx = Jx + F/2 (Strang) and q = -J, epsilon at equilibrium.
// The equilibrium products rho ux ux = Pxx, rho ux uy = Pxy, rho uy uy = Pyy
// are the window's momentum-flux values of the node.  The non-equilibrium
// parts of theta_XX and theta_XY share E = grad rho + 3 (div P):
//   K_XX = (2/3) a_xx [(dxJx - dyJy) - ux Ex + uy Ey]
//   K_XY = (1/3) a_xx [(dxJy + dyJx) - ux Ey - uy Ex]
// with Ex = dx rho + 3 (dx Pxx + dy Pxy), Ey = dy rho + 3 (dx Pxy + dy Pyy).
template <bool FORCE>
__device__ __forceinline__ void reconstruct2(float2 dr, float2 ux, float2 uy, float2 Jx, float2 Jy,
                                             float2 pxx, float2 pxy, float2 pyy, float2 dxr,
                                             float2 dyr, float2 dxjx, float2 dyjx, float2 dxjy,
                                             float2 dyjy, float2 dxpxx, float2 dxpxy,
                                             float2 dypxy, float2 dypyy, const StreamCoeffs& k,
                                             float2 g[9]) {
    const float2 nuy = mul2(uy, sp(-1.f));
    const float2 u2 = fma2(ux, ux, mul2(uy, uy));
    const float2 ex = fma2(sp(3.f), add2(dxpxx, dypxy), dxr);
    const float2 ey = fma2(sp(3.f), add2(dxpxy, dypyy), dyr);
    // K_E / 36 = a_e [(2 + 6 u^2)(d.J) - 2 (u . grad rho)] / 36
    const float2 udr = fma2(uy, dyr, mul2(ux, dxr));
    const float2 ke36 =
        fma2(sp(k.em2), udr, mul2(fma2(sp(k.e6), u2, sp(k.e2)), add2(dxjx, dyjy)));
    // XX = Pxx - Pyy + K_XX, K_XX = -(2/3) a_xx [ux Ex - uy Ey - (dxJx - dyJy)]
    const float2 xx =
        fma2(sp(k.xm23), fma2(ux, ex, fma2(nuy, ey, sub2(dyjy, dxjx))), sub2(pxx, pyy));
    // XY = Pxy + K_XY, K_XY = (1/3) a_xx [(dxJy + dyJx) - (ux Ey + uy Ex)]
    const float2 xy = fma2(sp(k.x13), sub2(add2(dxjy, dyjx), fma2(ux, ey, mul2(uy, ex))), pxy);
    const float2 ru2_12 = mul2(add2(pxx, pyy), sp(1.f / 12.f));
    const float2 axis = sub2(fma2(dr, sp(1.f / 9.f), ru2_12), ke36);
    const float2 diag = fma2(sp(2.f), ke36, fma2(dr, sp(1.f / 36.f), ru2_12));
    g[0] = fma2(sp(-4.f), add2(axis, diag), dr);
    // t2 = 2 t, s4 = 4 s: fl(2/3) = 2 fl(1/3) and the factors 1/2, 1/4 below
    // are exact, so every population has the roundings of the t, s form
    float2 tx2, ty2, jx = Jx, jy = Jy;
    if (FORCE) {
        jx = add2(Jx, sp(k.hfx));
        jy = add2(Jy, sp(k.hfy));
        tx2 = mul2(add2(jx, Jx), sp(1.f / 3.f));
        ty2 = mul2(add2(jy, Jy), sp(1.f / 3.f));
    } else {
        tx2 = mul2(Jx, sp(2.f / 3.f));
        ty2 = mul2(Jy, sp(2.f / 3.f));
    }
    const float2 sx4 = sub2(jx, tx2), sy4 = sub2(jy, ty2);
    const float2 ax = fma2(xx, sp(0.25f), axis), ay = fma2(xx, sp(-0.25f), axis);
    const float2 dp = fma2(xy, sp(0.25f), diag), dm = fma2(xy, sp(-0.25f), diag);
    const float2 spp4 = add2(sx4, sy4), smm4 = sub2(sy4, sx4);
    g[1] = fma2(tx2, sp(0.5f), ax);
    g[3] = fma2(tx2, sp(-0.5f), ax);
    g[2] = fma2(ty2, sp(0.5f), ay);
    g[4] = fma2(ty2, sp(-0.5f), ay);
    g[5] = fma2(spp4, sp(0.25f), dp);
    g[7] = fma2(spp4, sp(-0.25f), dp);
    g[6] = fma2(smm4, sp(0.25f), dm);
    g[8] = fma2(smm4, sp(-0.25f), dm);
}

// LW-ACM reconstruction (Sec. 1-b, Eq. 3) of two columns.  After the
// propagation f_a(x) = feq_a(x - c_a) + Theta (feo_a(x) - feo_a(x - c_a)),
// so the new moments gather h_a = feq_a - Theta feo_a from the upstream
// nodes and add Theta J(x) to the momentum (sum_a feo_a = 0,
// sum_a c_a feo_a = J).  With feo_a = 3 w_a c_a.J and 3 (1 - Theta) = 18 nu,
// g_a = h_a - w_a = w_a [dr + 18 nu c.J + 4.5 rho (c.u)^2 - 1.5 rho u^2],
// rho u_i u_j = P_ij from the row's flux values:
//   g1,3 = q + Pxx/2 +- tx,  g2,4 = q + Pyy/2 +- ty,  q = (dr - 1.5 (Pxx + Pyy)) / 9,
//   g5,7 = d + Pxy/4 +- (sx + sy),  g6,8 = d - Pxy/4 +- (sy - sx),
//   d = (dr + 3 (Pxx + Pyy)) / 36,  t = 2 nu J,  s = t / 4 (exact),
//   g0 = dr - 2 (g-pairs' even parts), equal to 4 q, so that sum g = dr
// without the bias of the rounded 1/9 and 1/36.  The momentum the node
// sends out is 3 t; the close adds J - 3 t of the receiving node (Theta J),
// so the lattice's momentum cancels term by term (see the close).
__device__ __forceinline__ void reconstruct_lw2(float2 dr, float2 Jx, float2 Jy, float2 pxx,
                                                float2 pxy, float2 pyy, const StreamCoeffs& k,
                                                float2 g[9]) {
    const float2 S = add2(pxx, pyy);
    const float2 q = fma2(S, sp(-1.f / 6.f), mul2(dr, sp(1.f / 9.f)));
    const float2 ax = fma2(pxx, sp(0.5f), q), ay = fma2(pyy, sp(0.5f), q);
    const float2 d = fma2(S, sp(1.f / 12.f), mul2(dr, sp(1.f / 36.f)));
    const float2 dp = fma2(pxy, sp(0.25f), d), dm = fma2(pxy, sp(-0.25f), d);
    const float2 tx = mul2(Jx, sp(k.lw_t)), ty = mul2(Jy, sp(k.lw_t));
    // s = t / 4 exactly: the diagonal populations take (ty +- tx) / 4
    const float2 spp4 = add2(tx, ty), smm4 = sub2(ty, tx);
    g[0] = fma2(sp(-2.f), add2(add2(ax, ay), add2(dp, dm)), dr);
    g[1] = add2(ax, tx);
    g[3] = sub2(ax, tx);
    g[2] = add2(ay, ty);
    g[4] = sub2(ay, ty);
    g[5] = fma2(spp4, sp(0.25f), dp);
    g[7] = fma2(spp4, sp(-0.25f), dp);
    g[6] = fma2(smm4, sp(0.25f), dm);
    g[8] = fma2(smm4, sp(-0.25f), dm);
}

// Per-lane gather state, in column pairs: destination row c (partial, "A")
// and c + 1 (contribution of row c's upward populations, "U").
struct Acc {
    float2 ar[2], ax[2], ay[2];  // row c: rho - 1, Jx, Jy (missing row c + 1)
    float2 us[2], ud[2];         // row c + 1: sum and x-difference of g2, g5, g6
};


// The y window's update alone, for the first rows of an item (k < 2R),
// whose centre rows' populations reach no output row: three points keep the
// new row (fm2 takes it); five points keep n1 = f(c) - f(c + 2) of the
// centre row c = k - 2 and the new row (dm3 takes it), needed from k = R on.
template <int R>
__device__ __forceinline__ void window_row(const float2 nr[2], const float2 nux[2],
                                           const float2 nuy[2], const float2 cdr[2],
                                           const float2 cux[2], const float2 cuy[2], Win& fm2,
                                           Win& dm3) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 jx = fma2(nr[h], nux[h], nux[h]), jy = fma2(nr[h], nuy[h], nuy[h]);
        const float2 pxy = mul2(jx, nuy[h]), pyy = mul2(jy, nuy[h]);
        if (R == 1) {
            fm2.v[W_R][h] = nr[h];
            fm2.v[W_JX][h] = jx;
            fm2.v[W_JY][h] = jy;
            fm2.v[W_PXY][h] = pxy;
            fm2.v[W_PYY][h] = pyy;
        } else {
            const float2 cjx = fma2(cdr[h], cux[h], cux[h]), cjy = fma2(cdr[h], cuy[h], cuy[h]);
            dm3.v[W_R][h] = sub2(cdr[h], nr[h]);
            dm3.v[W_JX][h] = sub2(cjx, jx);
            dm3.v[W_JY][h] = sub2(cjy, jy);
            dm3.v[W_PXY][h] = sub2(mul2(cjx, cuy[h]), pxy);
            dm3.v[W_PYY][h] = sub2(mul2(cjy, cuy[h]), pyy);
        }
    }
}

// One row of the streaming step, shared by the single-lattice and the batched
// kernels.  In: the new field row k (nr, nux, nuy; channel rows already
// scaled) and, for R > 0, the centre row c = k - R (cdr, cux, cuy; zeros
// while the window fills; R = 0, LW-ACM, takes the new row as the centre).
// Out: the closed row c - 1 (odr, oux, ouy).  Advances the y window (fm2 /
// fm1 for R <= 1, the differences dm3 / dm2 for R = 2) and the gather state.
template <int R, bool FORCE>
__device__ __forceinline__ void stream_row(const float2 nr[2], const float2 nux[2],
                                           const float2 nuy[2], const float2 cdr[2],
                                           float2 cux[2], float2 cuy[2], const StreamCoeffs& k,
                                           Win& fm2, Win& fm1, Win& dm3, Win& dm2, Acc& acc,
                                           float2 odr[2], float2 oux[2], float2 ouy[2]) {
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
    if (R == 0) {  // LW-ACM: no derivative window, the new row is the centre
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            cux[h] = nux[h];
            cuy[h] = nuy[h];
        }
    }
    // Five points: the centre row's fields are rebuilt from the ring
    // (only the differences are held in registers).  Three points: the
    // centre row is held (fm1).
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
    const Win& cen = (R == 0) ? nw : (R == 1) ? fm1 : rebuilt;
    // y derivatives at the centre row (scaled by 2 or 8):
    //   three points: 2 d/dy = f(c+1) - f(c-1)
    //   five points:  8 d/dy = 6 d1(c) - d1(c-1) - d1(c+1), d1(c+1) = f(r) - f(c);
    //   the window holds n1 = -d1, so 8 d/dy = (-6 n1(c) + n1(c-1)) + n1(c+1);
    //   the bracket does not wait for the new row
    Win dy, d1new;
#pragma unroll
    for (int f = 0; f < W_N; ++f)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (R == 0) {
                dy.v[f][h] = sp(0.f);  // unused
            } else if (R == 1) {
                dy.v[f][h] = sub2(nw.v[f][h], fm2.v[f][h]);
            } else {
                d1new.v[f][h] = sub2(cen.v[f][h], nw.v[f][h]);
                dy.v[f][h] = add2(fma2(sp(-6.f), dm2.v[f][h], dm3.v[f][h]), d1new.v[f][h]);
            }
        }
    // x derivatives at the centre row
    float2 pxx[2], dxr[2], dxjx[2], dxjy[2], dxpxx[2], dxpxy[2];
    pxx[0] = mul2(cen.v[W_JX][0], cux[0]);
    pxx[1] = mul2(cen.v[W_JX][1], cux[1]);
    float2 g[2][9];
    if (R == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            reconstruct_lw2(cen.v[W_R][h], cen.v[W_JX][h], cen.v[W_JY][h], pxx[h],
                            cen.v[W_PXY][h], cen.v[W_PYY][h], k, g[h]);
    } else {
        deriv_x<R>(cen.v[W_R], dxr);
        deriv_x<R>(cen.v[W_JX], dxjx);
        deriv_x<R>(cen.v[W_JY], dxjy);
        deriv_x<R>(pxx, dxpxx);
        deriv_x<R>(cen.v[W_PXY], dxpxy);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            reconstruct2<FORCE>(cen.v[W_R][h], cux[h], cuy[h], cen.v[W_JX][h], cen.v[W_JY][h],
                            pxx[h], cen.v[W_PXY][h], cen.v[W_PYY][h], dxr[h], dy.v[W_R][h], dxjx[h], dy.v[W_JX][h], dxjy[h],
                            dy.v[W_JY][h], dxpxx[h], dxpxy[h], dy.v[W_PXY][h],
                            dy.v[W_PYY][h], k, g[h]);
    }

    // populations crossing lane boundaries: right-going (1, 5, 8) of
    // column 3 to the next lane, left-going (3, 6, 7) of column 0 back
    const float in1 = __shfl_up_sync(kFull, g[1][1].y, 1);
    const float in5 = __shfl_up_sync(kFull, g[1][5].y, 1);
    const float in8 = __shfl_up_sync(kFull, g[1][8].y, 1);
    const float in3 = __shfl_down_sync(kFull, g[0][3].x, 1);
    const float in6 = __shfl_down_sync(kFull, g[0][6].x, 1);
    const float in7 = __shfl_down_sync(kFull, g[0][7].x, 1);
    // per destination column j (0..3): from j - 1 (1, 5, 8) and j + 1
    // (3, 6, 7), summed in scalar FP32 (the results land in column pairs
    // without register moves)
    float G[9][4];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        G[q][0] = g[0][q].x;
        G[q][1] = g[0][q].y;
        G[q][2] = g[1][q].x;
        G[q][3] = g[1][q].y;
    }
    float ss_[4], ds_[4], su_[4], du_[4], sd_[4], dd_[4];
    // columns 1 and 2 take their neighbours' populations from whole pairs
    // ((G1[0], G1[1]) = g[0][1], (G3[2], G3[3]) = g[1][3], and so on): one
    // paired instruction for two scalar ones, each sum rounded as before
    const float2 p13 = add2(g[0][1], g[1][3]), m13 = sub2(g[0][1], g[1][3]);
    const float2 p56 = add2(g[0][5], g[1][6]), m56 = sub2(g[0][5], g[1][6]);
    const float2 p78 = add2(g[1][7], g[0][8]), m87 = sub2(g[0][8], g[1][7]);
#pragma unroll
    for (int j = 0; j < 4; j += 3) {
        const float q1 = j ? G[1][j - 1] : in1, q5 = j ? G[5][j - 1] : in5;
        const float q8 = j ? G[8][j - 1] : in8;
        const float q3 = j < 3 ? G[3][j + 1] : in3, q6 = j < 3 ? G[6][j + 1] : in6;
        const float q7 = j < 3 ? G[7][j + 1] : in7;
        ss_[j] = G[0][j] + (q1 + q3);
        ds_[j] = q1 - q3;
        su_[j] = G[2][j] + (q5 + q6);
        du_[j] = q5 - q6;
        sd_[j] = G[4][j] + (q7 + q8);
        dd_[j] = q8 - q7;
    }
    ss_[1] = G[0][1] + p13.x;
    ss_[2] = G[0][2] + p13.y;
    ds_[1] = m13.x;
    ds_[2] = m13.y;
    su_[1] = G[2][1] + p56.x;
    su_[2] = G[2][2] + p56.y;
    du_[1] = m56.x;
    du_[2] = m56.y;
    sd_[1] = G[4][1] + p78.x;
    sd_[2] = G[4][2] + p78.y;
    dd_[1] = m87.x;
    dd_[2] = m87.y;

#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 ss = make_float2(ss_[2 * h], ss_[2 * h + 1]);
        const float2 ds = make_float2(ds_[2 * h], ds_[2 * h + 1]);
        const float2 su = make_float2(su_[2 * h], su_[2 * h + 1]);
        const float2 du = make_float2(du_[2 * h], du_[2 * h + 1]);
        const float2 sd = make_float2(sd_[2 * h], sd_[2 * h + 1]);
        const float2 dd = make_float2(dd_[2 * h], dd_[2 * h + 1]);
        // close row c - 1: u = J - J dr / (1 + dr)
        const float2 drn = add2(acc.ar[h], sd);
        float2 px = add2(acc.ax[h], dd);
        float2 py = sub2(acc.ay[h], sd);
        if (FORCE) {
            px = add2(px, sp(k.hfx));
            py = add2(py, sp(k.hfy));
        }
        if (R == 0) {
            // LW-ACM: Theta J = J - 3 t of the closing row (the previous
            // row), t = 2 nu J the same product that row sent to its
            // neighbours, so the momentum leaving and entering cancel
            const float2 tx = mul2(fm1.v[W_JX][h], sp(k.lw_t));
            const float2 ty = mul2(fm1.v[W_JY][h], sp(k.lw_t));
            px = add2(px, fma2(sp(-3.f), tx, fm1.v[W_JX][h]));
            py = add2(py, fma2(sp(-3.f), ty, fm1.v[W_JY][h]));
        }
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
    // rotate the window: the oldest row/difference take the new ones
    if (R <= 1) fm2 = nw;
    if (R == 2) dm3 = d1new;
}

// ---- narrow strips: one column pair per lane ------------------------------------
// The same step on lanes that hold 2 consecutive columns (a warp covers 64
// columns; with two halo lanes on each side, 56 output columns): used for
// the last, partial strip of a lattice, where 4-column lanes would compute
// up to 128 columns for a few stored ones.  Lane L holds columns 2L - 4 and
// 2L - 3 of its strip; lanes 0 and 31 hold only the stencil's outer columns,
// lanes 1 and 30 rebuild the populations that enter the strip.

struct Win1 {
    float2 v[W_N];
};
struct Acc1 {
    float2 ar, ax, ay, us, ud;
};

// x-derivative (scaled by 2 or 8) at the lane's 2 columns.
template <int R>
__device__ __forceinline__ float2 deriv_x1(float2 v) {
    const float l1 = __shfl_up_sync(kFull, v.y, 1);
    const float r0 = __shfl_down_sync(kFull, v.x, 1);
    const float2 d1 = make_float2(v.y - l1, r0 - v.x);  // f(+1) - f(-1)
    if (R == 1) return d1;
    // 8 d/dx = 6 (f(+1) - f(-1)) - (f(+2) - f(-2)): columns +-2 are the
    // neighbouring lanes' pairs
    const float l0 = __shfl_up_sync(kFull, v.x, 1);
    const float r1 = __shfl_down_sync(kFull, v.y, 1);
    return fma2(sp(6.f), d1, sub2(make_float2(l0, l1), make_float2(r0, r1)));
}

template <int R>
__device__ __forceinline__ void window_row1(float2 nr, float2 nux, float2 nuy, float2 cdr,
                                            float2 cux, float2 cuy, Win1& fm2, Win1& dm3) {
    const float2 jx = fma2(nr, nux, nux), jy = fma2(nr, nuy, nuy);
    const float2 pxy = mul2(jx, nuy), pyy = mul2(jy, nuy);
    if (R == 1) {
        fm2.v[W_R] = nr;
        fm2.v[W_JX] = jx;
        fm2.v[W_JY] = jy;
        fm2.v[W_PXY] = pxy;
        fm2.v[W_PYY] = pyy;
    } else {
        const float2 cjx = fma2(cdr, cux, cux), cjy = fma2(cdr, cuy, cuy);
        dm3.v[W_R] = sub2(cdr, nr);
        dm3.v[W_JX] = sub2(cjx, jx);
        dm3.v[W_JY] = sub2(cjy, jy);
        dm3.v[W_PXY] = sub2(mul2(cjx, cuy), pxy);
        dm3.v[W_PYY] = sub2(mul2(cjy, cuy), pyy);
    }
}

// One row of a narrow strip; the single-pair form of stream_row (finite
// differences only, R = 1 or 2).
template <int R, bool FORCE>
__device__ __forceinline__ void stream_row1(float2 nr, float2 nux, float2 nuy, float2 cdr,
                                            float2 cux, float2 cuy, const StreamCoeffs& k,
                                            Win1& fm2, Win1& fm1, Win1& dm3, Win1& dm2,
                                            Acc1& acc, float2& odr, float2& oux, float2& ouy) {
    static_assert(R == 1 || R == 2, "narrow strips carry the finite-difference steps");
    Win1 nw;
    {
        const float2 jx = fma2(nr, nux, nux), jy = fma2(nr, nuy, nuy);
        nw.v[W_R] = nr;
        nw.v[W_JX] = jx;
        nw.v[W_JY] = jy;
        nw.v[W_PXY] = mul2(jx, nuy);
        nw.v[W_PYY] = mul2(jy, nuy);
    }
    Win1 rebuilt;
    if (R == 2) {
        const float2 jx = fma2(cdr, cux, cux), jy = fma2(cdr, cuy, cuy);
        rebuilt.v[W_R] = cdr;
        rebuilt.v[W_JX] = jx;
        rebuilt.v[W_JY] = jy;
        rebuilt.v[W_PXY] = mul2(jx, cuy);
        rebuilt.v[W_PYY] = mul2(jy, cuy);
    }
    const Win1& cen = (R == 1) ? fm1 : rebuilt;
    Win1 dy, d1new;
#pragma unroll
    for (int f = 0; f < W_N; ++f) {
        if (R == 1) {
            dy.v[f] = sub2(nw.v[f], fm2.v[f]);
        } else {
            d1new.v[f] = sub2(cen.v[f], nw.v[f]);
            dy.v[f] = add2(fma2(sp(-6.f), dm2.v[f], dm3.v[f]), d1new.v[f]);
        }
    }
    const float2 pxx = mul2(cen.v[W_JX], cux);
    const float2 dxr = deriv_x1<R>(cen.v[W_R]), dxjx = deriv_x1<R>(cen.v[W_JX]);
    const float2 dxjy = deriv_x1<R>(cen.v[W_JY]), dxpxx = deriv_x1<R>(pxx);
    const float2 dxpxy = deriv_x1<R>(cen.v[W_PXY]);
    float2 g[9];
    reconstruct2<FORCE>(cen.v[W_R], cux, cuy, cen.v[W_JX], cen.v[W_JY], pxx, cen.v[W_PXY],
                        cen.v[W_PYY], dxr, dy.v[W_R], dxjx, dy.v[W_JX], dxjy, dy.v[W_JY],
                        dxpxx, dxpxy, dy.v[W_PXY], dy.v[W_PYY], k, g);
    // right-going (1, 5, 8) of column 1 to the next lane, left-going
    // (3, 6, 7) of column 0 back
    const float in1 = __shfl_up_sync(kFull, g[1].y, 1);
    const float in5 = __shfl_up_sync(kFull, g[5].y, 1);
    const float in8 = __shfl_up_sync(kFull, g[8].y, 1);
    const float in3 = __shfl_down_sync(kFull, g[3].x, 1);
    const float in6 = __shfl_down_sync(kFull, g[6].x, 1);
    const float in7 = __shfl_down_sync(kFull, g[7].x, 1);
    // column 0 takes 1, 5, 8 from the left lane and 3, 6, 7 from column 1;
    // column 1 takes 1, 5, 8 from column 0 and 3, 6, 7 from the right lane
    const float2 ss = make_float2(g[0].x + (in1 + g[3].y), g[0].y + (g[1].x + in3));
    const float2 ds = make_float2(in1 - g[3].y, g[1].x - in3);
    const float2 su = make_float2(g[2].x + (in5 + g[6].y), g[2].y + (g[5].x + in6));
    const float2 du = make_float2(in5 - g[6].y, g[5].x - in6);
    const float2 sd = make_float2(g[4].x + (g[7].y + in8), g[4].y + (in7 + g[8].x));
    const float2 dd = make_float2(in8 - g[7].y, g[8].x - in7);
    // close row c - 1: u = J - J dr / (1 + dr)
    const float2 drn = add2(acc.ar, sd);
    float2 px = add2(acc.ax, dd);
    float2 py = sub2(acc.ay, sd);
    if (FORCE) {
        px = add2(px, sp(k.hfx));
        py = add2(py, sp(k.hfy));
    }
    const float2 nrho = fma2(drn, sp(-1.f), sp(-1.f));  // -(1 + dr)
    const float2 ninv = make_float2(rcp_approx(nrho.x), rcp_approx(nrho.y));
    odr = drn;
    oux = fma2(mul2(px, drn), ninv, px);
    ouy = fma2(mul2(py, drn), ninv, py);
    acc.ar = add2(acc.us, ss);
    acc.ax = add2(acc.ud, ds);
    acc.ay = acc.us;
    acc.us = su;
    acc.ud = du;
    if (R == 1) fm2 = nw;
    if (R == 2) dm3 = d1new;
}

}  // namespace stream
}  // namespace fdlbm
