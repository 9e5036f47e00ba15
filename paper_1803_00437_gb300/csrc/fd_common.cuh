// fd_common.cuh -- per-node arithmetic of the FD-LBM step (Sec. 2), shared
// by the FD-LBM kernels of this library.
#pragma once

#include "fdlbm_internal.cuh"

namespace fdlbm {

// Derivative estimate at p[0] from neighbours p[+-stride] (Sec. 2):
//   three points  d = (f(+1) - f(-1)) / 2
//   five points   d = 3/4 (f(+1) - f(-1)) - 1/8 (f(+2) - f(-2))
template <int R>
__device__ __forceinline__ float fd_deriv(const float* p, int stride);

template <>
__device__ __forceinline__ float fd_deriv<1>(const float* p, int s) {
    return 0.5f * (p[s] - p[-s]);
}

template <>
__device__ __forceinline__ float fd_deriv<2>(const float* p, int s) {
    return 0.75f * (p[s] - p[-s]) - 0.125f * (p[2 * s] - p[-2 * s]);
}

// The ten finite-difference derivatives one node needs.  Following the
// definition of theta (Eq. theta) they act on the density, on the momentum
// J = rho u and on the momentum flux P = J J / rho.
struct NodeDerivs {
    float drx, dry;         // d_x rho, d_y rho
    float dJx_x, dJx_y;     // d_x Jx, d_y Jx
    float dJy_x, dJy_y;     // d_x Jy, d_y Jy
    float dPxx_x;           // d_x (Jx Jx / rho)
    float dPxy_x, dPxy_y;   // d_x, d_y (Jx Jy / rho)
    float dPyy_y;           // d_y (Jy Jy / rho)
};

// g = M^-1 m' for the 9 moments in deviation form (moments of the fluid at
// rest subtracted: E + 2, epsilon - 1).  M^-1 = M^T diag(1/9, 1/6, 1/6,
// 1/36, 1/4, 1/4, 1/12, 1/12, 1/36), M the table of Sec. 1.
//
// FP32 note: 1/6, 1/9, ... are not representable, and 6 fl(1/6) = 1 + 3e-8.
// Written naively, the momentum carried by the populations would be
// (1 + 3e-8) J every step (2.5e-5 after 1000 steps).  The diagonal terms sx,
// sy and the rest population g0 are therefore formed from the others so that
// sum g = rho - 1 and sum c g = J hold up to unbiased roundings:
//   sx = (jx - 2 tx)/4 (= jx/6 + qx/12),  g0 = dr - 4 (axis + diag).
__device__ __forceinline__ void moments_to_populations(float dr, float jx, float jy, float e,
                                                       float xx, float xy, float qx, float qy,
                                                       float ep, float g[9]) {
    const float r9 = dr * (1.f / 9.f);
    const float axis = r9 - e * (1.f / 36.f) - ep * (1.f / 18.f);
    const float diag = r9 + e * (1.f / 18.f) + ep * (1.f / 36.f);
    g[0] = dr - 4.f * (axis + diag);
    const float tx = (jx - qx) * (1.f / 6.f);
    const float ty = (jy - qy) * (1.f / 6.f);
    const float sx = 0.25f * (jx - 2.f * tx);
    const float sy = 0.25f * (jy - 2.f * ty);
    const float ax = axis + 0.25f * xx, ay = axis - 0.25f * xx;
    const float dp = diag + 0.25f * xy, dm = diag - 0.25f * xy;
    g[1] = ax + tx;
    g[3] = ax - tx;
    g[2] = ay + ty;
    g[4] = ay - ty;
    g[5] = dp + (sx + sy);
    g[7] = dp - (sx + sy);
    g[6] = dm + (sy - sx);
    g[8] = dm - (sy - sx);
}

// Reconstructed post-collision populations, as deviations g_a = f*_a - w_a,
// at one node of state (rho - 1, ux, uy) (Sec. 2):
//   E  = -2 rho + 3 |J|^2/rho + (1 - 1/s_e)  theta_E
//   XX = (Jx^2 - Jy^2)/rho    + (1 - 1/s_xx) theta_XX
//   XY = Jx Jy / rho          + (1 - 1/s_xx) theta_XY
//   q = -J, epsilon = rho - 3 |J|^2/rho, momentum J + F/2 (Strang).
__device__ __forceinline__ void fd_reconstruct(float dr, float ux, float uy, const NodeDerivs& d,
                                               const FdCoeffs& c, float g[9]) {
    const float uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const float u2 = uxx + uyy;
    const float mx = d.dPxx_x + d.dPxy_y;
    const float my = d.dPxy_x + d.dPyy_y;
    const float th_e = (2.f + 6.f * u2) * (d.dJx_x + d.dJy_y) - 2.f * (ux * d.drx + uy * d.dry);
    const float th_xx = (2.f / 3.f) * ((d.dJx_x - d.dJy_y) - (ux * d.drx - uy * d.dry)) -
                        2.f * (ux * mx - uy * my);
    const float th_xy = (1.f / 3.f) * ((d.dJy_x + d.dJx_y) - (ux * d.dry + uy * d.drx)) -
                        ux * my - uy * mx;
    // rho v = v + (rho - 1) v: avoids rounding 1 + dr
    const float Jx = fmaf(dr, ux, ux), Jy = fmaf(dr, uy, uy);
    const float ru2 = fmaf(dr, u2, u2);
    const float dxx = uxx - uyy;
    const float e = -2.f * dr + 3.f * ru2 + c.a_e * th_e;
    const float xx = fmaf(dr, dxx, dxx) + c.a_xx * th_xx;
    const float xy = fmaf(dr, uxy, uxy) + c.a_xx * th_xy;
    const float ep = dr - 3.f * ru2;
    moments_to_populations(dr, Jx + 0.5f * c.fx, Jy + 0.5f * c.fy, e, xx, xy, -Jx, -Jy, ep, g);
}

// Moments of the 9 arriving populations p_a = g_a(x - c_a) (Eq. 2) and the
// new primitive state: rho - 1 = sum p, J = sum c p, u = (J + F/2) / rho.
__device__ __forceinline__ void fd_close(const float p[9], const FdCoeffs& c, float* dr,
                                         float* ux, float* uy) {
    const float drn = p[0] + (p[1] + p[3]) + (p[2] + p[4]) + (p[5] + p[7]) + (p[6] + p[8]);
    const float d57 = p[5] - p[7], d86 = p[8] - p[6];
    const float jx = (p[1] - p[3]) + d57 + d86;
    const float jy = (p[2] - p[4]) + d57 - d86;
    // u = J / rho = J - J dr / (1 + dr): the rounding of 1 + dr only touches
    // the small correction
    const float inv = __frcp_rn(1.f + drn);
    const float px = jx + 0.5f * c.fx, py = jy + 0.5f * c.fy;
    *dr = drn;
    *ux = fmaf(-px * drn, inv, px);
    *uy = fmaf(-py * drn, inv, py);
}

// Primitive state at lattice node (x, y), x already inside [0, nx).  With
// walls, rows outside [0, ny) are virtual nodes: u extrapolated linearly to
// zero at the wall (from the first fluid row if xi >= 1/2, else from the
// second), rho - 1 copied from the first fluid row (Sec. 3-b, 3-c).
template <bool WALLS, typename T>
__device__ __forceinline__ void fd_load_node(const FdState<T>& s, int x, int y, int ny,
                                             size_t pitch, float xi, Quant q, float* dr,
                                             float* ux, float* uy) {
    if (!WALLS) {
        const size_t o = (size_t)wrap_index(y, ny) * pitch + x;
        *dr = Storage<T>::load(s.drho + o, q);
        *ux = Storage<T>::load(s.ux + o, q);
        *uy = Storage<T>::load(s.uy + o, q);
        return;
    }
    if (y >= 0 && y < ny) {
        const size_t o = (size_t)y * pitch + x;
        *dr = Storage<T>::load(s.drho + o, q);
        *ux = Storage<T>::load(s.ux + o, q);
        *uy = Storage<T>::load(s.uy + o, q);
        return;
    }
    const bool below = y < 0;
    const int edge = below ? 0 : ny - 1;
    const int jref = xi >= 0.5f ? edge : (below ? 1 : ny - 2);
    const float ywall = below ? -xi : (float)(ny - 1) + xi;
    const float factor = ((float)y - ywall) / ((float)jref - ywall);
    const size_t oe = (size_t)edge * pitch + x, orf = (size_t)jref * pitch + x;
    *dr = Storage<T>::load(s.drho + oe, q);
    *ux = Storage<T>::load(s.ux + orf, q) * factor;
    *uy = Storage<T>::load(s.uy + orf, q) * factor;
}

}  // namespace fdlbm
