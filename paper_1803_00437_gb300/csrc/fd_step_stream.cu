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
constexpr unsigned kFull = 0xffffffffu;

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

struct Win {
    float v[W_N][4];
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

// Issue the copies of one row (3 fields, kLoadCols columns starting at
// column xl, wrapping periodically) into a slot.  Called by one lane.
template <typename T>
__device__ __forceinline__ void issue_row(const StreamArgs& a, const Ring<T>& ring, int slot,
                                          int row, int xl) {
    const int r = wrap_index(row, a.ny);
    const int x0 = wrap_index(xl, a.nx);
    const int first = min(kLoadCols, a.nx - x0);
    uint64_t* bar = &ring.bars[slot];
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, 3u * kLoadCols * sizeof(T));
    const T* src = static_cast<const T*>(a.src);
    for (int f = 0; f < 3; ++f) {
        const T* rowp = src + f * a.plane + (size_t)r * a.pitch;
        T* dst = slot_field(ring, slot, f);
        tma_load_1d(dst, rowp + x0, first * sizeof(T), bar);
        if (first < kLoadCols) tma_load_1d(dst + first, rowp, (kLoadCols - first) * sizeof(T), bar);
    }
}

// x-derivative (scaled) at the 4 columns of this lane of one field.
template <int R>
__device__ __forceinline__ void deriv_x(const float v[4], float d[4]) {
    const float l1 = __shfl_up_sync(kFull, v[3], 1);
    const float r0 = __shfl_down_sync(kFull, v[0], 1);
    if (R == 1) {
        // 2 d/dx = f(+1) - f(-1)
        d[0] = v[1] - l1;
        d[1] = v[2] - v[0];
        d[2] = v[3] - v[1];
        d[3] = r0 - v[2];
    } else {
        // 8 d/dx = 6 (f(+1) - f(-1)) - (f(+2) - f(-2))
        const float l2 = __shfl_up_sync(kFull, v[2], 1);
        const float r1 = __shfl_down_sync(kFull, v[1], 1);
        d[0] = fmaf(6.f, v[1] - l1, -(v[2] - l2));
        d[1] = fmaf(6.f, v[2] - v[0], -(v[3] - l1));
        d[2] = fmaf(6.f, v[3] - v[1], -(r0 - v[0]));
        d[3] = fmaf(6.f, r0 - v[2], -(r1 - v[1]));
    }
}

// Reconstruction of one node from scaled derivatives (see fd_reconstruct;
// the derivative scale is folded into the relaxation factors).
__device__ __forceinline__ void reconstruct_scaled(float dr, float ux, float uy, float dxr,
                                                   float dyr, float dxjx, float dyjx, float dxjy,
                                                   float dyjy, float dxpxx, float dxpxy,
                                                   float dypxy, float dypyy, float a_e,
                                                   float a_xx, float fx, float fy, float g[9]) {
    const float uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const float u2 = uxx + uyy;
    const float mx = dxpxx + dypxy;
    const float my = dxpxy + dypyy;
    const float th_e = (2.f + 6.f * u2) * (dxjx + dyjy) - 2.f * (ux * dxr + uy * dyr);
    const float th_xx =
        (2.f / 3.f) * ((dxjx - dyjy) - (ux * dxr - uy * dyr)) - 2.f * (ux * mx - uy * my);
    const float th_xy =
        (1.f / 3.f) * ((dxjy + dyjx) - (ux * dyr + uy * dxr)) - ux * my - uy * mx;
    const float Jx = fmaf(dr, ux, ux), Jy = fmaf(dr, uy, uy);
    const float ru2 = fmaf(dr, u2, u2);
    const float dxx = uxx - uyy;
    const float e = -2.f * dr + 3.f * ru2 + a_e * th_e;
    const float xx = fmaf(dr, dxx, dxx) + a_xx * th_xx;
    const float xy = fmaf(dr, uxy, uxy) + a_xx * th_xy;
    const float ep = dr - 3.f * ru2;
    moments_to_populations(dr, Jx + 0.5f * fx, Jy + 0.5f * fy, e, xx, xy, -Jx, -Jy, ep, g);
}

// Per-lane gather state: for destination row c (partial, "A") and c + 1
// (contribution of row c's upward populations, "U").
struct Acc {
    float ar[4], ax[4], ay[4];  // row c: rho - 1, Jx, Jy (still missing row c + 1)
    float us[4], ud[4];         // row c + 1: sum and x-difference of g2, g5, g6
};

template <int R, typename T>
struct RowStep {
    // One field row: read it, update the y window, and (when the centre row
    // is inside the computed range) reconstruct the centre row, gather and
    // store the row above the centre... i.e. the destination row c - 1.
    static __device__ __forceinline__ void run(const StreamArgs& a, const Ring<T>& ring,
                                               int lane, int k, int nrows, uint32_t load_no,
                                               int row_first, int yb, int ye, int strip0,
                                               Win& fm2, Win& fm1, Win& dm3, Win& dm2, Acc& acc,
                                               bool& ok, uint32_t& issued) {
        const int slot = load_no % kSlots;
        const uint32_t phase = (load_no / kSlots) & 1u;
        const bool landed = __all_sync(kFull, mbar_wait_bounded(&ring.bars[slot], phase));
        if (!landed) {
            ok = false;
            return;
        }
        // new row r = row_first + k
        float nr[4], nux[4], nuy[4];
        const int col = 4 + 4 * lane;  // slot column of this lane's first column
        Vec4<T>::load(slot_field(ring, slot, 0) + col, nr);
        Vec4<T>::load(slot_field(ring, slot, 1) + col, nux);
        Vec4<T>::load(slot_field(ring, slot, 2) + col, nuy);
        Win nw;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float jx = fmaf(nr[j], nux[j], nux[j]), jy = fmaf(nr[j], nuy[j], nuy[j]);
            nw.v[W_R][j] = nr[j];
            nw.v[W_JX][j] = jx;
            nw.v[W_JY][j] = jy;
            nw.v[W_PXY][j] = jx * nuy[j];
            nw.v[W_PYY][j] = jy * nuy[j];
        }
        // y derivatives at the centre row c = r - R (scaled by 2 or 8)
        Win dy, d1new;
        const Win& cen = (R == 1) ? fm1 : fm2;
#pragma unroll
        for (int f = 0; f < W_N; ++f)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (R == 1) {
                    dy.v[f][j] = nw.v[f][j] - fm2.v[f][j];
                } else {
                    d1new.v[f][j] = nw.v[f][j] - fm2.v[f][j];
                    dy.v[f][j] = fmaf(6.f, dm2.v[f][j], -(dm3.v[f][j] + d1new.v[f][j]));
                }
            }
        // centre row velocities from its ring slot (still resident); before
        // the window is full the centre row does not exist yet
        const int cslot = (load_no + kSlots - R) % kSlots;
        float cux[4] = {0.f, 0.f, 0.f, 0.f}, cuy[4] = {0.f, 0.f, 0.f, 0.f};
        if (k >= R) {
            Vec4<T>::load(slot_field(ring, cslot, 1) + col, cux);
            Vec4<T>::load(slot_field(ring, cslot, 2) + col, cuy);
        }

        // x derivatives at the centre row
        float pxx[4], dxr[4], dxjx[4], dxjy[4], dxpxx[4], dxpxy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) pxx[j] = cen.v[W_JX][j] * cux[j];
        deriv_x<R>(cen.v[W_R], dxr);
        deriv_x<R>(cen.v[W_JX], dxjx);
        deriv_x<R>(cen.v[W_JY], dxjy);
        deriv_x<R>(pxx, dxpxx);
        deriv_x<R>(cen.v[W_PXY], dxpxy);

        const float sc = (R == 1) ? 0.5f : 0.125f;
        const float a_e = a.c.a_e * sc, a_xx = a.c.a_xx * sc;
        float g[4][9];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            reconstruct_scaled(cen.v[W_R][j], cux[j], cuy[j], dxr[j], dy.v[W_R][j], dxjx[j],
                               dy.v[W_JX][j], dxjy[j], dy.v[W_JY][j], dxpxx[j], dxpxy[j],
                               dy.v[W_PXY][j], dy.v[W_PYY][j], a_e, a_xx, a.c.fx, a.c.fy, g[j]);

        // populations crossing lane boundaries
        const float in1 = __shfl_up_sync(kFull, g[3][1], 1);
        const float in5 = __shfl_up_sync(kFull, g[3][5], 1);
        const float in8 = __shfl_up_sync(kFull, g[3][8], 1);
        const float in3 = __shfl_down_sync(kFull, g[0][3], 1);
        const float in6 = __shfl_down_sync(kFull, g[0][6], 1);
        const float in7 = __shfl_down_sync(kFull, g[0][7], 1);

        // destination row c - 1 is complete once row c's downward populations
        // arrive; c is the centre row
        const int c_row = row_first + k - R;
        const bool store = (c_row - 1 >= yb) && (c_row - 1 < ye) && lane >= 1 && lane <= 30 &&
                           (strip0 - 4 + 4 * lane) < a.nx;
        float odr[4], oux[4], ouy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float p1 = j > 0 ? g[j - 1][1] : in1;
            const float p5 = j > 0 ? g[j - 1][5] : in5;
            const float p8 = j > 0 ? g[j - 1][8] : in8;
            const float p3 = j < 3 ? g[j + 1][3] : in3;
            const float p6 = j < 3 ? g[j + 1][6] : in6;
            const float p7 = j < 3 ? g[j + 1][7] : in7;
            const float ss = g[j][0] + (p1 + p3), ds = p1 - p3;
            const float su = g[j][2] + (p5 + p6), du = p5 - p6;
            const float sd = g[j][4] + (p7 + p8), dd = p8 - p7;
            // close row c - 1
            const float drn = acc.ar[j] + sd;
            const float jxn = acc.ax[j] + dd;
            const float jyn = acc.ay[j] - sd;
            const float inv = __frcp_rn(1.f + drn);
            const float px = jxn + 0.5f * a.c.fx, py = jyn + 0.5f * a.c.fy;
            odr[j] = drn;
            oux[j] = fmaf(-px * drn, inv, px);
            ouy[j] = fmaf(-py * drn, inv, py);
            // row c: upward part of row c - 1 plus the same-row part
            acc.ar[j] = acc.us[j] + ss;
            acc.ax[j] = acc.ud[j] + ds;
            acc.ay[j] = acc.us[j];
            acc.us[j] = su;
            acc.ud[j] = du;
        }
        if (store) {
            T* dst = static_cast<T*>(a.dst);
            const size_t o = (size_t)(c_row - 1) * a.pitch + (strip0 - 4 + 4 * lane);
            Vec4<T>::store(dst + o, odr);
            Vec4<T>::store(dst + a.plane + o, oux);
            Vec4<T>::store(dst + 2 * a.plane + o, ouy);
        }

        // rotate the window: the oldest row/difference slots take the new ones
        fm2 = nw;
        if (R == 2) dm3 = d1new;

        // the centre row's slot is no longer needed: refill it with the row
        // kSlots ahead
        __syncwarp();
        const int knext = k - R + kSlots;
        if (k >= R && knext < nrows) {
            if (lane == 0) issue_row<T>(a, ring, cslot, row_first + knext, strip0 - 8);
            ++issued;
        }
    }
};

template <int R, typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
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
        const int strip = item % a.nstrips, seg = item / a.nstrips;
        const int strip0 = strip * kStrip;
        const int yb = seg * a.seg_rows, ye = min(a.ny, yb + a.seg_rows);
        const int row_first = yb - 1 - R;
        const int nrows = ye - yb + 2 + 2 * R;
        if (lane == 0)
            for (int k = 0; k < kSlots && k < nrows; ++k)
                issue_row<T>(a, ring, (loads + k) % kSlots, row_first + k, strip0 - 8);
        issued += min(kSlots, nrows);
        __syncwarp();
        Win w0 = {}, w1 = {}, w2 = {}, w3 = {};
        Acc acc = {};
        int k = 0;
        for (; k + 1 < nrows && ok; k += 2) {
            RowStep<R, T>::run(a, ring, lane, k, nrows, loads + k, row_first, yb, ye, strip0, w0,
                               w1, w2, w3, acc, ok, issued);
            if (!ok) {
                consumed = loads + k;
                break;
            }
            RowStep<R, T>::run(a, ring, lane, k + 1, nrows, loads + k + 1, row_first, yb, ye,
                               strip0, w1, w0, w3, w2, acc, ok, issued);
            if (!ok) consumed = loads + k + 1;
        }
        if (ok && k < nrows) {
            RowStep<R, T>::run(a, ring, lane, k, nrows, loads + k, row_first, yb, ye, strip0, w0,
                               w1, w2, w3, acc, ok, issued);
            if (!ok) consumed = loads + k;
        }
        loads += nrows;
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
