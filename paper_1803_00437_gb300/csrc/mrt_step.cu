// mrt_step.cu -- MRT D2Q9 step (Sec. 1 and 1-a; Eq. 1 and Eq. 2).
//
// Storage: 9 planes of h_a = f*_a - w_a, the post-collision populations of
// the previous step ("pull" layout).  One step at node x:
//   1. pull f_a(x) = h_a(x - c_a) (Eq. 2); if x - c_a lies in a wall the
//      link is bounced back half-way: f_a(x) = h_opp(a)(x);
//   2. moments m = M f (deviation form), J' = J + F/2 (first half force);
//   3. relax E, XX, XY, qx, qy, epsilon towards the equilibria of Sec. 1-a
//      computed with J' (Eq. 1); momentum J' + F/2 (second half);
//   4. h* = M^-1 m*, stored at x.
#include "mrt_common.cuh"

namespace fdlbm {

namespace {

constexpr int kThreads = 256;

template <bool WALLS>
__global__ void __launch_bounds__(kThreads)
    mrt_step_kernel(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny,
                    size_t pitch, size_t plane, MrtCoeffs c) {
    const int x = blockIdx.x * kThreads + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    float f[9];
    mrt_pull<WALLS>(src, x, y, nx, ny, pitch, plane, f);
    const size_t r0 = (size_t)y * pitch;
    float m[9];
    populations_to_moments(f, m);
    const float jx = m[1] + 0.5f * c.fx, jy = m[2] + 0.5f * c.fy;
    float e_eq, xx_eq, xy_eq, ep_eq;
    mrt_equilibrium(m[0], jx, jy, &e_eq, &xx_eq, &xy_eq, &ep_eq);
    const float e = m[3] + c.s_e * (e_eq - m[3]);
    const float xx = m[4] + c.s_xx * (xx_eq - m[4]);
    const float xy = m[5] + c.s_xx * (xy_eq - m[5]);
    const float qx = m[6] + c.s_q * (-jx - m[6]);
    const float qy = m[7] + c.s_q * (-jy - m[7]);
    const float ep = m[8] + c.s_eps * (ep_eq - m[8]);
    float g[9];
    moments_to_populations(m[0], jx + 0.5f * c.fx, jy + 0.5f * c.fy, e, xx, xy, qx, qy, ep, g);
#pragma unroll
    for (int a = 0; a < 9; ++a) dst[a * plane + r0 + x] = g[a];
}

}  // namespace

MrtCoeffs mrt_coeffs(const fdlbm_params& p) {
    MrtCoeffs c;
    c.s_e = (float)p.s_e;
    c.s_xx = (float)p.s_xx;
    c.s_q = (float)p.s_q;
    c.s_eps = (float)p.s_eps;
    c.fx = (float)p.force_x;
    c.fy = (float)p.force_y;
    return c;
}

cudaError_t launch_mrt_step(fdlbm_s* h, const void* src, void* dst) {
    dim3 grid((h->p.nx + kThreads - 1) / kThreads, h->p.ny);
    const MrtCoeffs c = mrt_coeffs(h->p);
    if (h->p.boundary == FDLBM_BOUNDARY_WALLS_Y)
        mrt_step_kernel<true><<<grid, kThreads, 0, h->stream>>>(
            static_cast<const float*>(src), static_cast<float*>(dst), h->p.nx, h->p.ny,
            h->L.pitch, h->L.plane, c);
    else
        mrt_step_kernel<false><<<grid, kThreads, 0, h->stream>>>(
            static_cast<const float*>(src), static_cast<float*>(dst), h->p.nx, h->p.ny,
            h->L.pitch, h->L.plane, c);
    return cudaGetLastError();
}

}  // namespace fdlbm
