// aux_kernels.cu -- initialisation, moment extraction and FP64 reductions.
#include <algorithm>

#include "mrt_common.cuh"

namespace fdlbm {
namespace {

constexpr int kThreads = 256;

// ---- FD-LBM: contiguous FP32 (rho-1, ux, uy) -> stored state ---------------

template <typename T>
__global__ void fd_init_kernel(const float* __restrict__ drho, const float* __restrict__ ux,
                               const float* __restrict__ uy, T* __restrict__ dst, int nx, int ny,
                               size_t pitch, size_t plane, Quant q, int* status) {
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const size_t i = (size_t)y * nx + x, o = (size_t)y * pitch + x;
    bool sat = Storage<T>::store(dst + o, drho[i], q);
    sat |= Storage<T>::store(dst + plane + o, ux[i], q);
    sat |= Storage<T>::store(dst + 2 * plane + o, uy[i], q);
    if (sat) report_saturation(status);
}

// Four consecutive columns per thread (nx % 4 == 0, sources 16-byte
// aligned): 16-byte loads, which is what keeps the host link busy when the
// sources are page-locked host memory read in place.
template <typename T>
__device__ __forceinline__ bool store4(T* p, float4 v, Quant q) {
    bool sat = Storage<T>::store(p, v.x, q);
    sat |= Storage<T>::store(p + 1, v.y, q);
    sat |= Storage<T>::store(p + 2, v.z, q);
    sat |= Storage<T>::store(p + 3, v.w, q);
    return sat;
}
template <>
__device__ __forceinline__ bool store4<float>(float* p, float4 v, Quant) {
    *reinterpret_cast<float4*>(p) = v;  // rows start 256-byte aligned
    return false;
}

template <typename T>
__global__ void fd_init_vec4_kernel(const float4* __restrict__ drho, const float4* __restrict__ ux,
                                    const float4* __restrict__ uy, T* __restrict__ dst, int nx4,
                                    int ny, size_t pitch, size_t plane, Quant q, int* status) {
    const int x4 = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x4 >= nx4) return;
    const size_t i = (size_t)y * nx4 + x4, o = (size_t)y * pitch + 4 * (size_t)x4;
    const float4 a = drho[i], b = ux[i], c = uy[i];
    bool sat = store4(dst + o, a, q);
    sat |= store4(dst + plane + o, b, q);
    sat |= store4(dst + 2 * plane + o, c, q);
    if (sat) report_saturation(status);
}

// ---- MRT: equilibrium start --------------------------------------------------

// Deviation populations h^eq_a at node n for (rho-1, u): the equilibria of
// Sec. 1-a at J = rho u - F/2 (so that the reported velocity is u).
__device__ __forceinline__ void mrt_eq_node(const float* drho, const float* ux, const float* uy,
                                            size_t n, const MrtCoeffs& c, float g[9]) {
    const float dr = drho[n];
    const float jx = fmaf(dr, ux[n], ux[n]) - 0.5f * c.fx;
    const float jy = fmaf(dr, uy[n], uy[n]) - 0.5f * c.fy;
    float e, xx, xy, ep;
    mrt_equilibrium(dr, jx, jy, &e, &xx, &xy, &ep);
    moments_to_populations(dr, jx, jy, e, xx, xy, -jx, -jy, ep, g);
}

// Pull layout: stored h_b(y) must be what the next step pulls, so that the
// first step sees f^0 = f^eq everywhere: h_b(y) = h^eq_b(y + c_b) when
// y + c_b is fluid, otherwise (bounce-back link) h^eq_opp(b)(y).
template <bool WALLS>
__global__ void mrt_init_kernel(const float* __restrict__ drho, const float* __restrict__ ux,
                                const float* __restrict__ uy, float* __restrict__ dst, int nx,
                                int ny, size_t pitch, size_t plane, MrtCoeffs c) {
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    float own[9];
    mrt_eq_node(drho, ux, uy, (size_t)y * nx + x, c, own);
    for (int b = 0; b < 9; ++b) {
        const int xd = wrap_index(x + cx[b], nx);
        int yd = y + cy[b];
        float v;
        if (WALLS && (yd < 0 || yd >= ny)) {
            v = own[opp[b]];
        } else {
            yd = wrap_index(yd, ny);
            float g[9];
            mrt_eq_node(drho, ux, uy, (size_t)yd * nx + xd, c, g);
            v = g[b];
        }
        dst[b * plane + (size_t)y * pitch + x] = v;
    }
}

// ---- transverse plane waves (shear waves / Stokes modes) ---------------------

struct ModeList {
    int n;
    double mean_ux, mean_uy;
    double rec[kMaxModes][4];  // m, n, amplitude, phase
};

// Rows per block.  A cos(kx x + ky y + phase) = cos(kx x) C(y) - sin(kx x) S(y)
// with C, S = A (cos, sin)(ky y + phase): the row factors of the block's rows
// are tabulated once per block in shared memory (FP64 sincos of each row),
// the column factor once per thread and mode, so each node costs four FP64
// multiply-adds per mode instead of a sincos.
constexpr int kModeRows = 16;

__global__ void __launch_bounds__(kThreads)
    modes_kernel(ModeList ml, int nx, int ny, float* __restrict__ drho, float* __restrict__ ux,
                 float* __restrict__ uy) {
    __shared__ double2 rowf[kMaxModes][kModeRows];
    const int x = blockIdx.x * kThreads + threadIdx.x;
    const int y0 = blockIdx.y * kModeRows;
    const int nrows = min(kModeRows, ny - y0);
    for (int t = threadIdx.x; t < ml.n * kModeRows; t += kThreads) {
        const int k = t / kModeRows, r = t % kModeRows;
        const double ky = 2.0 * M_PI * ml.rec[k][1] / ny;
        double sn, cs;
        sincos(ky * (double)(y0 + r) + ml.rec[k][3], &sn, &cs);
        rowf[k][r] = make_double2(ml.rec[k][2] * cs, ml.rec[k][2] * sn);
    }
    __syncthreads();
    if (x >= nx) return;
    double vx[kModeRows], vy[kModeRows];
#pragma unroll
    for (int r = 0; r < kModeRows; ++r) {
        vx[r] = ml.mean_ux;
        vy[r] = ml.mean_uy;
    }
    for (int k = 0; k < ml.n; ++k) {
        const double kx = 2.0 * M_PI * ml.rec[k][0] / nx, ky = 2.0 * M_PI * ml.rec[k][1] / ny;
        const double kk = sqrt(kx * kx + ky * ky);
        const double tx = -ky / kk, ty = kx / kk;  // unit vector across k
        double sx, cx;
        sincos(kx * (double)x, &sx, &cx);
#pragma unroll
        for (int r = 0; r < kModeRows; ++r) {
            const double2 f = rowf[k][r];
            const double w = fma(cx, f.x, -sx * f.y);
            vx[r] = fma(w, tx, vx[r]);
            vy[r] = fma(w, ty, vy[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < kModeRows; ++r) {
        if (r < nrows) {
            const size_t i = (size_t)(y0 + r) * nx + x;
            drho[i] = 0.f;
            ux[i] = (float)vx[r];
            uy[i] = (float)vy[r];
        }
    }
}

// ---- moments ---------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void fd_node(const T* s, size_t plane, size_t o, Quant q, float* dr,
                                        float* ux, float* uy) {
    *dr = Storage<T>::load(s + o, q);
    *ux = Storage<T>::load(s + plane + o, q);
    *uy = Storage<T>::load(s + 2 * plane + o, q);
}

template <bool WALLS>
__device__ __forceinline__ void mrt_node(const float* s, int x, int y, int nx, int ny,
                                         size_t pitch, size_t plane, float fx, float fy,
                                         float* dr, float* ux, float* uy) {
    float f[9], m[9];
    mrt_pull<WALLS>(s, x, y, nx, ny, pitch, plane, f);
    populations_to_moments(f, m);
    const float inv = __frcp_rn(1.f + m[0]);
    const float px = m[1] + 0.5f * fx, py = m[2] + 0.5f * fy;
    *dr = m[0];
    *ux = fmaf(-px * m[0], inv, px);
    *uy = fmaf(-py * m[0], inv, py);
}

template <typename T, int KIND>  // KIND 0: FD-LBM, 1: MRT periodic, 2: MRT walls
__device__ __forceinline__ void node_state(const void* s, int x, int y, int nx, int ny,
                                           size_t pitch, size_t plane, float fx, float fy,
                                           Quant q, float* dr, float* ux, float* uy) {
    if (KIND == 0)
        fd_node(static_cast<const T*>(s), plane, (size_t)y * pitch + x, q, dr, ux, uy);
    else
        mrt_node<KIND == 2>(static_cast<const float*>(s), x, y, nx, ny, pitch, plane, fx, fy,
                            dr, ux, uy);
}

template <typename T, int KIND>
__global__ void moments_kernel(const void* s, int nx, int ny, size_t pitch, size_t plane,
                               float fx, float fy, Quant q, float* __restrict__ drho,
                               float* __restrict__ ux, float* __restrict__ uy) {
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    float dr, vx, vy;
    node_state<T, KIND>(s, x, y, nx, ny, pitch, plane, fx, fy, q, &dr, &vx, &vy);
    const size_t i = (size_t)y * nx + x;
    drho[i] = dr;
    ux[i] = vx;
    uy[i] = vy;
}

// ---- FP64 reductions ----------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Compensated FP32 sum (Knuth's TwoSum; no products, so nothing to contract
// into FMAs): s + c carries ~48 significant bits.  The FP32 pipes of this GPU
// are ~60x faster than its FP64 pipe, so the per-node work of the mass and
// momentum sums stays in FP32 and only each thread's chunk total (<= 64
// terms) is added in FP64.
struct Sum2f {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        const float bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double flush() {
        const double r = (double)s + (double)c;
        s = c = 0.f;
        return r;
    }
};

// rho u = u + dr u, with dr u split exactly into p + e (FMA product error).
__device__ __forceinline__ void add_rho_u(Sum2f& acc, float dr, float u) {
    const float p = dr * u;
    const float e = fmaf(dr, u, -p);
    acc.add(u);
    acc.add(p);
    acc.add(e);
}

// Rows per block iteration; for the mode projection their phases
// e^{i ky y} are tabulated in shared memory once per block.
constexpr int kRowChunk = 64;

// One column per thread (x = column chunk of the block + thread), rows in
// chunks strided over gridDim.y; slot 3 counts non-finite nodes in every
// reduction.  The mode projection uses the separable phase
// e^{i(kx x + ky y)} = e^{i kx x} e^{i ky y}: the column factor once per
// thread and row chunk, the row factors from the shared table (FP64 sincos
// of exact integer multiples, no accumulated rotation).
template <typename T, int KIND, int WHAT>
__global__ void __launch_bounds__(kThreads)
    reduce_kernel(const void* s, int nx, int ny, size_t pitch, size_t plane, float fx, float fy,
                  Quant q, double a0, double a1, double* __restrict__ partial) {
    double acc[kReduceSlots] = {0.0, 0.0, 0.0, 0.0};
    __shared__ double2 rowph[kRowChunk];
    double kx = 0.0, ky = 0.0, tx = 0.0, ty = 0.0;
    if (WHAT == FDLBM_REDUCE_MODE) {
        kx = 2.0 * M_PI * a0 / nx;
        ky = 2.0 * M_PI * a1 / ny;
        const double kk = sqrt(kx * kx + ky * ky);
        tx = kk > 0.0 ? -ky / kk : 0.0;
        ty = kk > 0.0 ? kx / kk : 0.0;
    }
    for (int y0 = blockIdx.y * kRowChunk; y0 < ny; y0 += gridDim.y * kRowChunk) {
        const int nrows = min(kRowChunk, ny - y0);
        if (WHAT == FDLBM_REDUCE_MODE) {
            __syncthreads();
            if (threadIdx.x < nrows) {
                double sn, cs;
                sincos(ky * (double)(y0 + (int)threadIdx.x), &sn, &cs);
                rowph[threadIdx.x] = make_double2(cs, sn);
            }
            __syncthreads();
        }
        for (int x = blockIdx.x * kThreads + threadIdx.x; x < nx; x += gridDim.x * kThreads) {
            double cxc = 1.0, cxs = 0.0;
            if (WHAT == FDLBM_REDUCE_MODE) sincos(kx * (double)x, &cxs, &cxc);
            Sum2f f0, f1;
            int bad = 0;
            // max |u|: FP32 |u|^2 (relative error < 2.4e-7) screens the nodes and
            // only those within 1e-4 of the running FP32 maximum are squared in
            // FP64, so the node holding the true maximum is always among them
            float m32 = 0.f, dmax = 0.f;
            double m64 = 0.0;
            // rows in batches of kBatch: all loads of a batch are issued before
            // any is used (several rows in flight per warp); a non-finite node
            // is counted and contributes zero
            constexpr int kBatch = 8;
            for (int r0 = 0; r0 < nrows; r0 += kBatch) {
                float bdr[kBatch], bux[kBatch], buy[kBatch];
#pragma unroll
                for (int i = 0; i < kBatch; ++i) {
                    bdr[i] = bux[i] = buy[i] = 0.f;
                    if (r0 + i < nrows)
                        node_state<T, KIND>(s, x, y0 + r0 + i, nx, ny, pitch, plane, fx, fy,
                                            q, &bdr[i], &bux[i], &buy[i]);
                }
#pragma unroll
                for (int i = 0; i < kBatch; ++i) {
                    const bool ok = isfinite(bdr[i]) && isfinite(bux[i]) && isfinite(buy[i]);
                    bad += ok ? 0 : 1;
                    const float dr = ok ? bdr[i] : 0.f;
                    const float ux = ok ? bux[i] : 0.f;
                    const float uy = ok ? buy[i] : 0.f;
                    const double rho = 1.0 + (double)dr;
                    if (WHAT == FDLBM_REDUCE_MASS) {
                        f0.add(dr);
                    } else if (WHAT == FDLBM_REDUCE_MOMENTUM) {
                        add_rho_u(f0, dr, ux);
                        add_rho_u(f1, dr, uy);
                    } else if (WHAT == FDLBM_REDUCE_ENERGY) {
                        acc[0] += 0.5 * rho * ((double)ux * ux + (double)uy * uy);
                    } else if (WHAT == FDLBM_REDUCE_MODE) {
                        const double ut = tx * ux + ty * uy;
                        const double2 ry = rowph[r0 + i];
                        const double cs = cxc * ry.x - cxs * ry.y;  // cos(kx x + ky y)
                        const double sn = cxs * ry.x + cxc * ry.y;  // sin(kx x + ky y)
                        acc[0] += ut * cs;
                        acc[1] -= ut * sn;
                    } else {
                        const float s32 = fmaf(ux, ux, uy * uy);
                        if (s32 >= 0.9999f * m32) {
                            m64 = fmax(m64, (double)ux * ux + (double)uy * uy);
                            m32 = fmaxf(m32, s32);
                        }
                        dmax = fmaxf(dmax, fabsf(dr));
                    }
                }
            }
            acc[3] += (double)bad;
            if (WHAT == FDLBM_REDUCE_MAXABS) {
                acc[0] = fmax(acc[0], sqrt(m64));
                acc[1] = fmax(acc[1], (double)dmax);
            }
            if (WHAT == FDLBM_REDUCE_MASS || WHAT == FDLBM_REDUCE_MOMENTUM) {
                acc[0] += f0.flush();
                acc[1] += f1.flush();
            }
        }
    }
    __shared__ double sh[kThreads / 32][kReduceSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool maxw = WHAT == FDLBM_REDUCE_MAXABS;
    for (int k = 0; k < kReduceSlots; ++k) {
        const double v = (maxw && k < 2) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kReduceSlots) {
        const int k = threadIdx.x;
        const bool is_max = maxw && k < 2;
        double v = sh[0][k];
        for (int w = 1; w < kThreads / 32; ++w) v = is_max ? fmax(v, sh[w][k]) : v + sh[w][k];
        partial[(blockIdx.y * gridDim.x + blockIdx.x) * kReduceSlots + k] = v;
    }
}

constexpr int kFinalThreads = 128;

// Combine the block partials: per slot, each thread folds a fixed strided
// subset, then a fixed tree over the threads (deterministic order).
__global__ void __launch_bounds__(kFinalThreads)
    reduce_final_kernel(const double* __restrict__ partial, int nblocks, int what,
                        double* __restrict__ result) {
    __shared__ double sh[kFinalThreads / 32][kReduceSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kReduceSlots; ++k) {
        const bool is_max = what == FDLBM_REDUCE_MAXABS && k < 2;
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kFinalThreads) {
            const double p = partial[b * kReduceSlots + k];
            v = is_max ? fmax(v, p) : v + p;
        }
        v = is_max ? warp_max(v) : warp_sum(v);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kReduceSlots) {
        const int k = threadIdx.x;
        const bool is_max = what == FDLBM_REDUCE_MAXABS && k < 2;
        double v = sh[0][k];
        for (int w = 1; w < kFinalThreads / 32; ++w) v = is_max ? fmax(v, sh[w][k]) : v + sh[w][k];
        result[k] = v;
    }
}

template <typename F>
cudaError_t dispatch_kind(fdlbm_s* h, F&& f) {
    if (h->p.scheme == FDLBM_SCHEME_MRT) {
        if (h->p.boundary == FDLBM_BOUNDARY_WALLS_Y) return f.template run<float, 2>();
        return f.template run<float, 1>();
    }
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return f.template run<__half, 0>();
        case FDLBM_STORAGE_BF16: return f.template run<__nv_bfloat16, 0>();
        case FDLBM_STORAGE_I16: return f.template run<int16_t, 0>();
        default: return f.template run<float, 0>();
    }
}

template <typename T>
cudaError_t launch_fd_init_typed(fdlbm_s* h, const float* drho, const float* ux,
                                 const float* uy, void* dst) {
    const Quant q = quant_of(h->p);
    int* status = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    const bool vec4 = h->p.nx % 4 == 0 &&
                      ((reinterpret_cast<uintptr_t>(drho) | reinterpret_cast<uintptr_t>(ux) |
                        reinterpret_cast<uintptr_t>(uy)) & 15) == 0;
    if (vec4) {
        const int nx4 = h->p.nx / 4;
        dim3 grid4((nx4 + kThreads - 1) / kThreads, h->p.ny);
        fd_init_vec4_kernel<T><<<grid4, kThreads, 0, h->stream>>>(
            reinterpret_cast<const float4*>(drho), reinterpret_cast<const float4*>(ux),
            reinterpret_cast<const float4*>(uy), static_cast<T*>(dst), nx4, h->p.ny,
            h->L.pitch, h->L.plane, q, status);
        return cudaGetLastError();
    }
    dim3 grid((h->p.nx + kThreads - 1) / kThreads, h->p.ny);
    fd_init_kernel<T><<<grid, kThreads, 0, h->stream>>>(drho, ux, uy, static_cast<T*>(dst),
                                                        h->p.nx, h->p.ny, h->L.pitch,
                                                        h->L.plane, q, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fd_init(fdlbm_s* h, const float* drho, const float* ux, const float* uy,
                           void* dst) {
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return launch_fd_init_typed<__half>(h, drho, ux, uy, dst);
        case FDLBM_STORAGE_BF16: return launch_fd_init_typed<__nv_bfloat16>(h, drho, ux, uy, dst);
        case FDLBM_STORAGE_I16: return launch_fd_init_typed<int16_t>(h, drho, ux, uy, dst);
        default: return launch_fd_init_typed<float>(h, drho, ux, uy, dst);
    }
}

cudaError_t launch_mrt_init(fdlbm_s* h, const float* drho, const float* ux, const float* uy,
                            void* dst) {
    dim3 grid((h->p.nx + kThreads - 1) / kThreads, h->p.ny);
    const MrtCoeffs c = mrt_coeffs(h->p);
    if (h->p.boundary == FDLBM_BOUNDARY_WALLS_Y)
        mrt_init_kernel<true><<<grid, kThreads, 0, h->stream>>>(
            drho, ux, uy, static_cast<float*>(dst), h->p.nx, h->p.ny, h->L.pitch, h->L.plane, c);
    else
        mrt_init_kernel<false><<<grid, kThreads, 0, h->stream>>>(
            drho, ux, uy, static_cast<float*>(dst), h->p.nx, h->p.ny, h->L.pitch, h->L.plane, c);
    return cudaGetLastError();
}

cudaError_t launch_modes_eval(fdlbm_s* h, int n_modes, const double* modes_host, double mean_ux,
                              double mean_uy, float* drho, float* ux, float* uy) {
    ModeList ml;
    ml.n = n_modes;
    ml.mean_ux = mean_ux;
    ml.mean_uy = mean_uy;
    for (int k = 0; k < n_modes; ++k)
        for (int j = 0; j < 4; ++j) ml.rec[k][j] = modes_host[4 * k + j];
    dim3 grid((h->p.nx + kThreads - 1) / kThreads, (h->p.ny + kModeRows - 1) / kModeRows);
    modes_kernel<<<grid, kThreads, 0, h->stream>>>(ml, h->p.nx, h->p.ny, drho, ux, uy);
    return cudaGetLastError();
}

namespace {
struct MomentsLaunch {
    fdlbm_s* h;
    const void* s;
    float *dr, *ux, *uy;
    template <typename T, int KIND>
    cudaError_t run() {
        dim3 grid((h->p.nx + kThreads - 1) / kThreads, h->p.ny);
        moments_kernel<T, KIND><<<grid, kThreads, 0, h->stream>>>(
            s, h->p.nx, h->p.ny, h->L.pitch, h->L.plane, (float)h->p.force_x,
            (float)h->p.force_y, quant_of(h->p), dr, ux, uy);
        return cudaGetLastError();
    }
};

// Grid of the reduction: column chunks x row chunks, at most kReduceBlocks
// blocks (the size of the partial-sum area).
dim3 reduce_grid(int nx, int ny) {
    const int gx = std::min((nx + kThreads - 1) / kThreads, kReduceBlocks);
    const int gy = std::max(1, std::min((ny + kRowChunk - 1) / kRowChunk, kReduceBlocks / gx));
    return dim3(gx, gy);
}

struct ReduceLaunch {
    fdlbm_s* h;
    const void* s;
    int what;
    double a0, a1;
    double* partial;
    template <typename T, int KIND, int WHAT>
    cudaError_t go() {
        reduce_kernel<T, KIND, WHAT><<<reduce_grid(h->p.nx, h->p.ny), kThreads, 0, h->stream>>>(
            s, h->p.nx, h->p.ny, h->L.pitch, h->L.plane, (float)h->p.force_x,
            (float)h->p.force_y, quant_of(h->p), a0, a1, partial);
        return cudaGetLastError();
    }
    template <typename T, int KIND>
    cudaError_t run() {
        switch (what) {
            case FDLBM_REDUCE_MASS: return go<T, KIND, FDLBM_REDUCE_MASS>();
            case FDLBM_REDUCE_MOMENTUM: return go<T, KIND, FDLBM_REDUCE_MOMENTUM>();
            case FDLBM_REDUCE_ENERGY: return go<T, KIND, FDLBM_REDUCE_ENERGY>();
            case FDLBM_REDUCE_MODE: return go<T, KIND, FDLBM_REDUCE_MODE>();
            default: return go<T, KIND, FDLBM_REDUCE_MAXABS>();
        }
    }
};
}  // namespace

cudaError_t launch_moments(fdlbm_s* h, const void* state, float* drho, float* ux, float* uy) {
    MomentsLaunch ml{h, state, drho, ux, uy};
    return dispatch_kind(h, ml);
}

cudaError_t launch_reduce(fdlbm_s* h, const void* state, int what, double a0, double a1,
                          double* partial, double* result) {
    ReduceLaunch rl{h, state, what, a0, a1, partial};
    cudaError_t e = dispatch_kind(h, rl);
    if (e != cudaSuccess) return e;
    const dim3 g = reduce_grid(h->p.nx, h->p.ny);
    reduce_final_kernel<<<1, kFinalThreads, 0, h->stream>>>(partial, (int)(g.x * g.y), what,
                                                           result);
    return cudaGetLastError();
}

}  // namespace fdlbm
