// fd_step_tiled.cu -- general FD-LBM step kernel (Sec. 2, Eq. 2): 2-D tiles
// staged in shared memory with a halo of r + 1 nodes.  Handles periodic and
// channel (walls in y) lattices of any size and every storage type.
// Stencil radius r = 0 is LW-ACM (Sec. 1-b, Eq. 3): no finite differences,
// a one-node halo for the gather.  The nine-point stencil of Sec. 2 has
// radius 1 and also reads the diagonal neighbours, which the 2-D tile holds.
//
// Per CTA (TX x TY outputs):
//   1. load (rho-1, u) of the tile plus a halo of H = r + 1 nodes (gradients
//      are needed at the upstream nodes, one link away), and form J = rho u
//      and the momentum flux J J / rho;
//   2. at every node of the tile plus a one-node ring, estimate the ten
//      derivatives, form theta, the reconstructed moments and the 9
//      populations g_a = f*_a - w_a (kept in shared memory);
//   3. every output node gathers g_a(x - c_a) (propagation, Eq. 2), closes
//      rho and u and stores them.
#include "fd_common.cuh"

namespace fdlbm {
namespace {

constexpr int kTX = 32, kTY = 16, kThreads = 256;

// LW-ACM populations g_a = h_a - w_a, h_a = feq_a - Theta feo_a, of one node
// (Sec. 1-b, Eq. 3), with 3 (1 - Theta) = 18 nu and t = 2 nu J:
//   g1,3 = q + Pxx/2 +- tx, g2,4 = q + Pyy/2 +- ty, q = (dr - 1.5 (Pxx + Pyy)) / 9,
//   g5,7 = d + Pxy/4 +- (tx + ty)/4, g6,8 = d - Pxy/4 +- (ty - tx)/4,
//   d = (dr + 3 (Pxx + Pyy)) / 36, g0 = dr - 2 (even parts)  (sum g = dr).
__device__ __forceinline__ void lw_reconstruct(float dr, float Jx, float Jy, float pxx,
                                               float pxy, float pyy, float lw_t, float g[9]) {
    const float S = pxx + pyy;
    const float q = fmaf(S, -1.f / 6.f, dr * (1.f / 9.f));
    const float ax = fmaf(pxx, 0.5f, q), ay = fmaf(pyy, 0.5f, q);
    const float d = fmaf(S, 1.f / 12.f, dr * (1.f / 36.f));
    const float dp = fmaf(pxy, 0.25f, d), dm = fmaf(pxy, -0.25f, d);
    const float tx = Jx * lw_t, ty = Jy * lw_t;
    const float spp = 0.25f * tx + 0.25f * ty, smm = 0.25f * ty - 0.25f * tx;
    g[0] = fmaf(-2.f, (ax + ay) + (dp + dm), dr);
    g[1] = ax + tx;
    g[3] = ax - tx;
    g[2] = ay + ty;
    g[4] = ay - ty;
    g[5] = dp + spp;
    g[7] = dp - spp;
    g[6] = dm + smm;
    g[8] = dm - smm;
}

// Nine-point difference (Sec. 2, D2Q9 footprint) along the axis of stride s,
// the other axis having stride t:
//   d = f(+s) - f(-s) - [(f(+s+t) - f(-s+t)) + (f(+s-t) - f(-s-t))] / 4
__device__ __forceinline__ float fd_deriv9(const float* p, int s, int t) {
    return (p[s] - p[-s]) - 0.25f * ((p[s + t] - p[-s + t]) + (p[s - t] - p[-s - t]));
}

template <int R, bool NINE, bool WALLS, typename T>
__global__ void __launch_bounds__(kThreads)
    fd_step_tiled_kernel(FdState<T> src, FdState<T> dst, int nx, int ny, size_t pitch,
                         FdCoeffs c, float lw_t, int* status) {
    constexpr int H = R + 1;
    constexpr int LX = kTX + 2 * H, LY = kTY + 2 * H, LN = LX * LY;
    constexpr int GX = kTX + 2, GY = kTY + 2, GN = GX * GY;
    // rho-1, ux, uy, Jx, Jy, Jx Jx/rho, Jx Jy/rho, Jy Jy/rho
    __shared__ float sf[8][LN];
    __shared__ float sg[9][GN];

    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;

    for (int t = threadIdx.x; t < LN; t += kThreads) {
        const int lx = t % LX, ly = t / LX;
        const int x = wrap_index(x0 - H + lx, nx);
        const int y = y0 - H + ly;
        float dr, ux, uy;
        fd_load_node<WALLS>(src, x, y, ny, pitch, c.xi, c.q, &dr, &ux, &uy);
        const float Jx = fmaf(dr, ux, ux), Jy = fmaf(dr, uy, uy);
        sf[0][t] = dr;
        sf[1][t] = ux;
        sf[2][t] = uy;
        sf[3][t] = Jx;
        sf[4][t] = Jy;
        sf[5][t] = Jx * ux;
        sf[6][t] = Jx * uy;
        sf[7][t] = Jy * uy;
    }
    __syncthreads();

    for (int t = threadIdx.x; t < GN; t += kThreads) {
        const int gx = t % GX, gy = t / GX;
        const int l = (gy + H - 1) * LX + (gx + H - 1);
        float g[9];
        if (R == 0) {
            lw_reconstruct(sf[0][l], sf[3][l], sf[4][l], sf[5][l], sf[6][l], sf[7][l], lw_t, g);
#pragma unroll
            for (int a = 0; a < 9; ++a) sg[a][t] = g[a];
            continue;
        }
        NodeDerivs d;
        if (NINE) {
            d.drx = fd_deriv9(&sf[0][l], 1, LX);
            d.dry = fd_deriv9(&sf[0][l], LX, 1);
            d.dJx_x = fd_deriv9(&sf[3][l], 1, LX);
            d.dJx_y = fd_deriv9(&sf[3][l], LX, 1);
            d.dJy_x = fd_deriv9(&sf[4][l], 1, LX);
            d.dJy_y = fd_deriv9(&sf[4][l], LX, 1);
            d.dPxx_x = fd_deriv9(&sf[5][l], 1, LX);
            d.dPxy_x = fd_deriv9(&sf[6][l], 1, LX);
            d.dPxy_y = fd_deriv9(&sf[6][l], LX, 1);
            d.dPyy_y = fd_deriv9(&sf[7][l], LX, 1);
        } else {
            d.drx = fd_deriv<R>(&sf[0][l], 1);
            d.dry = fd_deriv<R>(&sf[0][l], LX);
            d.dJx_x = fd_deriv<R>(&sf[3][l], 1);
            d.dJx_y = fd_deriv<R>(&sf[3][l], LX);
            d.dJy_x = fd_deriv<R>(&sf[4][l], 1);
            d.dJy_y = fd_deriv<R>(&sf[4][l], LX);
            d.dPxx_x = fd_deriv<R>(&sf[5][l], 1);
            d.dPxy_x = fd_deriv<R>(&sf[6][l], 1);
            d.dPxy_y = fd_deriv<R>(&sf[6][l], LX);
            d.dPyy_y = fd_deriv<R>(&sf[7][l], LX);
        }
        fd_reconstruct(sf[0][l], sf[1][l], sf[2][l], d, c, g);
#pragma unroll
        for (int a = 0; a < 9; ++a) sg[a][t] = g[a];
    }
    __syncthreads();

    bool sat = false;
    for (int t = threadIdx.x; t < kTX * kTY; t += kThreads) {
        const int ox = t % kTX, oy = t / kTX;
        const int x = x0 + ox, y = y0 + oy;
        if (x >= nx || y >= ny) continue;
        const int b = (oy + 1) * GX + (ox + 1);
        float p[9];
        p[0] = sg[0][b];
        p[1] = sg[1][b - 1];        // from (x-1, y)
        p[2] = sg[2][b - GX];       // from (x, y-1)
        p[3] = sg[3][b + 1];        // from (x+1, y)
        p[4] = sg[4][b + GX];       // from (x, y+1)
        p[5] = sg[5][b - GX - 1];   // from (x-1, y-1)
        p[6] = sg[6][b - GX + 1];   // from (x+1, y-1)
        p[7] = sg[7][b + GX + 1];   // from (x+1, y+1)
        p[8] = sg[8][b + GX - 1];   // from (x-1, y+1)
        float dr, ux, uy;
        if (R == 0) {
            // LW-ACM: Theta J of the node added as J - 3 t, t = 2 nu J the
            // product this node sent to its neighbours (no bias in the totals)
            const int l = (oy + H) * LX + (ox + H);
            const float Jx = sf[3][l], Jy = sf[4][l];
            const float drn =
                p[0] + (p[1] + p[3]) + (p[2] + p[4]) + (p[5] + p[7]) + (p[6] + p[8]);
            const float d57 = p[5] - p[7], d86 = p[8] - p[6];
            const float px = ((p[1] - p[3]) + d57 + d86) + fmaf(-3.f, Jx * lw_t, Jx);
            const float py = ((p[2] - p[4]) + d57 - d86) + fmaf(-3.f, Jy * lw_t, Jy);
            const float inv = __frcp_rn(1.f + drn);
            dr = drn;
            ux = fmaf(-px * drn, inv, px);
            uy = fmaf(-py * drn, inv, py);
        } else {
            fd_close(p, c, &dr, &ux, &uy);
        }
        const size_t o = (size_t)y * pitch + x;
        sat |= Storage<T>::store(dst.drho + o, dr, c.q);
        sat |= Storage<T>::store(dst.ux + o, ux, c.q);
        sat |= Storage<T>::store(dst.uy + o, uy, c.q);
    }
    if (sat) report_saturation(status);
}

template <int R, bool NINE, bool WALLS, typename T>
cudaError_t launch_typed(fdlbm_s* h, const void* src, void* dst) {
    const size_t plane = h->L.plane;
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    FdState<T> S{const_cast<T*>(s), const_cast<T*>(s + plane), const_cast<T*>(s + 2 * plane)};
    FdState<T> D{d, d + plane, d + 2 * plane};
    FdCoeffs c;
    c.a_e = (float)(1.0 - 1.0 / h->p.s_e);
    c.a_xx = (float)(1.0 - 1.0 / h->p.s_xx);
    c.fx = (float)h->p.force_x;
    c.fy = (float)h->p.force_y;
    c.xi = (float)h->p.wall_xi;
    c.q = quant_of(h->p);
    const float lw_t = (float)(2.0 * (1.0 / h->p.s_xx - 0.5) / 3.0);  // LW-ACM: 2 nu
    dim3 grid((h->p.nx + kTX - 1) / kTX, (h->p.ny + kTY - 1) / kTY);
    fd_step_tiled_kernel<R, NINE, WALLS, T>
        <<<grid, kThreads, 0, h->stream>>>(S, D, h->p.nx, h->p.ny, h->L.pitch, c, lw_t,
                                           reinterpret_cast<int*>(h->ws + h->L.off_flag));
    return cudaGetLastError();
}

template <int R, bool NINE, typename T>
cudaError_t launch_boundary(fdlbm_s* h, const void* src, void* dst) {
    if (h->p.boundary == FDLBM_BOUNDARY_WALLS_Y)
        return launch_typed<R, NINE, true, T>(h, src, dst);
    return launch_typed<R, NINE, false, T>(h, src, dst);
}

template <typename T>
cudaError_t launch_stencil(fdlbm_s* h, const void* src, void* dst) {
    if (h->p.scheme == FDLBM_SCHEME_LWACM) return launch_typed<0, false, false, T>(h, src, dst);
    if (h->p.scheme == FDLBM_SCHEME_FD3) return launch_boundary<1, false, T>(h, src, dst);
    if (h->p.scheme == FDLBM_SCHEME_FD9) return launch_boundary<1, true, T>(h, src, dst);
    return launch_boundary<2, false, T>(h, src, dst);
}

}  // namespace

cudaError_t launch_fd_step_tiled(fdlbm_s* h, const void* src, void* dst) {
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return launch_stencil<__half>(h, src, dst);
        case FDLBM_STORAGE_BF16: return launch_stencil<__nv_bfloat16>(h, src, dst);
        case FDLBM_STORAGE_I16: return launch_stencil<int16_t>(h, src, dst);
        default: return launch_stencil<float>(h, src, dst);
    }
}

}  // namespace fdlbm
