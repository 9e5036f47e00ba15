// mrt_common.cuh -- per-node arithmetic of the MRT D2Q9 scheme (Sec. 1,
// Sec. 1-a) in deviation form, shared by the MRT kernels of this library.
#pragma once

#include "fd_common.cuh"

namespace fdlbm {

// Moments (deviation form: E + 2, epsilon - 1) of 9 populations h_a.
__device__ __forceinline__ void populations_to_moments(const float f[9], float m[9]) {
    const float s_axis = (f[1] + f[2]) + (f[3] + f[4]);
    const float s_diag = (f[5] + f[6]) + (f[7] + f[8]);
    const float d57 = f[5] - f[7], d68 = f[6] - f[8];
    m[0] = f[0] + s_axis + s_diag;                       // rho - 1
    m[1] = (f[1] - f[3]) + d57 - d68;                    // Jx
    m[2] = (f[2] - f[4]) + d57 + d68;                    // Jy
    m[3] = -4.f * f[0] - s_axis + 2.f * s_diag;          // E + 2
    m[4] = (f[1] + f[3]) - (f[2] + f[4]);                // XX
    m[5] = (f[5] + f[7]) - (f[6] + f[8]);                // XY
    m[6] = 2.f * (f[3] - f[1]) + d57 - d68;              // qx
    m[7] = 2.f * (f[4] - f[2]) + d57 + d68;              // qy
    m[8] = 4.f * f[0] - 2.f * s_axis + s_diag;           // epsilon - 1
}

// Equilibria of Sec. 1-a in deviation form at (rho - 1, J').
__device__ __forceinline__ void mrt_equilibrium(float dr, float jx, float jy, float* e,
                                                float* xx, float* xy, float* ep) {
    const float inv = __frcp_rn(1.f + dr);
    const float j2 = (jx * jx + jy * jy) * inv;
    *e = -2.f * dr + 3.f * j2;
    *xx = (jx * jx - jy * jy) * inv;
    *xy = jx * jy * inv;
    *ep = dr - 3.f * j2;
}

// Populations arriving at (x, y) (Eq. 2) from the post-collision planes h:
// f_a(x) = h_a(x - c_a), or h_opp(a)(x) when x - c_a lies in a wall
// (half-way bounce-back).
template <bool WALLS>
__device__ __forceinline__ void mrt_pull(const float* __restrict__ h, int x, int y, int nx,
                                         int ny, size_t pitch, size_t plane, float f[9]) {
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    int ym = y - 1, yp = y + 1;
    bool wall_lo = false, wall_hi = false;
    if (WALLS) {
        wall_lo = ym < 0;
        wall_hi = yp >= ny;
    } else {
        ym = ym < 0 ? ny - 1 : ym;
        yp = yp >= ny ? 0 : yp;
    }
    const size_t r0 = (size_t)y * pitch, rm = (size_t)ym * pitch, rp = (size_t)yp * pitch;
    f[0] = h[r0 + x];
    f[1] = h[plane + r0 + xm];
    f[3] = h[3 * plane + r0 + xp];
    if (WALLS && wall_lo) {
        f[2] = h[4 * plane + r0 + x];
        f[5] = h[7 * plane + r0 + x];
        f[6] = h[8 * plane + r0 + x];
    } else {
        f[2] = h[2 * plane + rm + x];
        f[5] = h[5 * plane + rm + xm];
        f[6] = h[6 * plane + rm + xp];
    }
    if (WALLS && wall_hi) {
        f[4] = h[2 * plane + r0 + x];
        f[7] = h[5 * plane + r0 + x];
        f[8] = h[6 * plane + r0 + x];
    } else {
        f[4] = h[4 * plane + rp + x];
        f[7] = h[7 * plane + rp + xp];
        f[8] = h[8 * plane + rp + xm];
    }
}

}  // namespace fdlbm
