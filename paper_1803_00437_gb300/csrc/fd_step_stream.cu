// fd_step_stream.cu -- FD-LBM step (Sec. 2, Eq. 2) for lattices periodic in
// x (periodic or walled in y), streaming each warp down a strip of rows.
//
// Work decomposition.  A warp owns an output strip of 120 columns and a
// segment of rows.  Lane L holds 4 consecutive columns starting at
// strip0 - 4 + 4 L, so lanes 0 and 31 are halo lanes: they reconstruct the
// populations one column outside the strip (where the gradients they need
// are still exact) and store nothing.  Warps never synchronise with each
// other.
//
// Data path per warp.  Rows of (rho - 1, ux, uy) for the strip plus 8 halo
// columns are copied by 1-D bulk (TMA) copies into a private ring of 8
// shared-memory slots, each completed by an mbarrier, several rows ahead of
// use (two rows per issue, six lanes issuing one copy each).  Each lane
// reads its 4 columns (one 16-byte load per field for FP32).  Derivatives
// along y: three points hold the two previous rows in registers; five points
// hold only the (negated) differences d1(c) = f(c+1) - f(c-1) and use
// 8 d/dy = 6 d1(c) - d1(c-1) - d1(c+1), the centre row being re-read from the
// ring.  Derivatives along x use warp shuffles of the two neighbouring
// columns on each side.  Arithmetic on column pairs uses the paired FP32
// instructions of sm_100-family GPUs.  After the reconstruction the
// populations that cross a lane boundary are exchanged by shuffles, summed
// per destination row and closed when the row below has contributed.
#include <algorithm>

#include "fd_stream_common.cuh"
#include "tma_ring.cuh"

namespace fdlbm {
namespace {

using namespace stream;

constexpr int kWarpsPerBlock = 1;
constexpr int kStrip = 120;     // output columns per warp
constexpr int kLoadCols = 136;  // columns staged per row: strip0 - 8 .. strip0 + 128
constexpr int kSlots = 8;       // ring depth (rows); a power of two
constexpr int kSlotMask = kSlots - 1;

// One warp per CTA (warps never synchronise), 16 resident per SM: the
// register allocator then fits the step in 128 registers without spills and
// occupancy is set by registers and shared memory (16 x 13 KB rings), not by
// CTA granularity.  Measured on GB300: 16 one-warp CTAs beat 3 four-warp CTAs
// (168 registers) by 6 %.
#ifndef FDLBM_STREAM_MIN_BLOCKS
#define FDLBM_STREAM_MIN_BLOCKS 16
#endif
template <int R>
constexpr int min_blocks() {
    return FDLBM_STREAM_MIN_BLOCKS;
}

struct StreamArgs {
    const void* src;  // 3 planes (rho - 1, ux, uy), [ny][pitch]
    void* dst;
    size_t plane;     // elements per plane
    size_t pitch;     // elements per row
    int nx, ny;
    float xi;         // wall offset (channels)
    int nstrips, seg_rows, nsegs, nitems;
    StreamCoeffs k;
    int* status;      // device status word (FDLBM_ERR_TIMEOUT on a lost copy)
};

template <typename T>
struct Ring {
    T* slot_base;    // kSlots x 3 x kLoadCols elements
    uint64_t* bars;  // kSlots barriers
};

template <typename T>
__device__ __forceinline__ T* slot_field(const Ring<T>& ring, int slot, int field) {
    return ring.slot_base + (slot * 3 + field) * kLoadCols;
}

// Per-item constants of a warp.
struct Item {
    int strip0, yb, ye, row_first, nrows;
    int x0, first;     // staged columns: kLoadCols from x0, wrapping once at nx
    bool lane_stores;  // this lane's 4 columns are output columns
    uint32_t base;     // ring position of the item's row 0
    size_t out;        // element offset of this lane's columns in output row yb
};

// Issue rows k0 .. k0 + count - 1 (count 1 or 2) of the item into their ring
// slots: lanes 0..count-1 first arm the rows' barriers with the byte count,
// then lanes 0..3 count - 1 each copy one field of one row.
// Channel (walls in y): a row outside [0, ny) is virtual (Sec. 3-b, 3-c
// closure): its rho - 1 is the first fluid row's and its u the reference
// row's (the first fluid row if xi >= 1/2, else the second) times the linear
// extrapolation factor to u = 0 at the wall, applied when the row is read.
__device__ __forceinline__ int wall_edge(int r, int ny) { return r < 0 ? 0 : ny - 1; }
__device__ __forceinline__ int wall_ref(int r, int ny, float xi) {
    return xi >= 0.5f ? wall_edge(r, ny) : (r < 0 ? 1 : ny - 2);
}
__device__ __forceinline__ float wall_factor(int r, int ny, float xi) {
    if (r >= 0 && r < ny) return 1.f;
    const float ywall = r < 0 ? -xi : (float)(ny - 1) + xi;
    return ((float)r - ywall) / ((float)wall_ref(r, ny, xi) - ywall);
}

template <bool WALLS, typename T>
__device__ __forceinline__ void issue_rows(const StreamArgs& a, const Ring<T>& ring,
                                           const Item& it, int k0, int count, int lane) {
    if (lane < count) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&ring.bars[(it.base + k0 + lane) & kSlotMask],
                              3u * kLoadCols * sizeof(T));
    }
    __syncwarp();
    if (lane < 3 * count) {
        const int j = lane >= 3 ? 1 : 0;  // which row this lane copies
        const int f = lane - 3 * j;       // which field
        const int slot = (it.base + k0 + j) & kSlotMask;
        int r = it.row_first + k0 + j;
        if (!WALLS) {
            if (r < 0) r += a.ny;
            if (r >= a.ny) r -= a.ny;
        } else if (r < 0 || r >= a.ny) {
            r = f == 0 ? wall_edge(r, a.ny) : wall_ref(r, a.ny, a.xi);
        }
        fence_proxy_async_smem();
        const T* rowp = static_cast<const T*>(a.src) + f * a.plane + (size_t)r * a.pitch;
        T* dst = slot_field(ring, slot, f);
        uint64_t* bar = &ring.bars[slot];
        tma_load_1d(dst, rowp + it.x0, it.first * sizeof(T), bar);
        if (it.first < kLoadCols)
            tma_load_1d(dst + it.first, rowp, (kLoadCols - it.first) * sizeof(T), bar);
    }
}

// Rows before this one are the window's warm-up: the centre row does not
// exist yet (k < R) or the closed row is above the segment (k < 2R + 2).
template <int R>
__host__ __device__ constexpr int warm_rows() {
    return 2 * R + 2;
}

// Wait (bounded) for field row k of the item to land in its slot.
template <typename T>
__device__ __forceinline__ bool row_landed(const Ring<T>& ring, const Item& it, int k) {
    const uint32_t pos = it.base + k;
    return mbar_wait_bounded(&ring.bars[pos & kSlotMask], (pos / kSlots) & 1u);
}

template <int R, bool FORCE, bool WALLS, typename T>
struct RowStep {
    // Field row k of the item (already landed): read it, update the y window
    // and reconstruct the centre row c = row k - R; close and store row c - 1.
    // WARM: k may be below warm_rows<R>(), so the centre-row read and the
    // store are guarded; otherwise both are unconditional.
    template <bool WARM>
    static __device__ __forceinline__ void run(const StreamArgs& a, const Ring<T>& ring,
                                               const Item& it, int lane, int k, Win& fm2,
                                               Win& fm1, Win& dm3, Win& dm2, Acc& acc) {
        const uint32_t pos = it.base + k;
        const int slot = pos & kSlotMask;
        const int col = 4 + 4 * lane;  // slot column of this lane's first column
        float2 nr[2], nux[2], nuy[2];
        Vec4<T>::load(slot_field(ring, slot, 0) + col, nr);
        Vec4<T>::load(slot_field(ring, slot, 1) + col, nux);
        Vec4<T>::load(slot_field(ring, slot, 2) + col, nuy);
        if (WALLS) {
            const int r = it.row_first + k;
            if (r < 0 || r >= a.ny) {  // uniform across the warp
                const float2 fac = sp(wall_factor(r, a.ny, a.xi));
                nux[0] = mul2(nux[0], fac);
                nux[1] = mul2(nux[1], fac);
                nuy[0] = mul2(nuy[0], fac);
                nuy[1] = mul2(nuy[1], fac);
            }
        }
        // centre row c = r - R from its ring slot (still resident); before
        // the window is full the centre row does not exist yet
        const int cslot = (pos - R) & kSlotMask;
        float2 cdr[2] = {sp(0.f), sp(0.f)}, cux[2] = {sp(0.f), sp(0.f)};
        float2 cuy[2] = {sp(0.f), sp(0.f)};
        if (R > 0 && (!WARM || k >= R)) {
            if (R == 2) Vec4<T>::load(slot_field(ring, cslot, 0) + col, cdr);
            Vec4<T>::load(slot_field(ring, cslot, 1) + col, cux);
            Vec4<T>::load(slot_field(ring, cslot, 2) + col, cuy);
            if (WALLS) {
                const int r = it.row_first + k - R;
                if (r < 0 || r >= a.ny) {
                    const float2 fac = sp(wall_factor(r, a.ny, a.xi));
                    cux[0] = mul2(cux[0], fac);
                    cux[1] = mul2(cux[1], fac);
                    cuy[0] = mul2(cuy[0], fac);
                    cuy[1] = mul2(cuy[1], fac);
                }
            }
        }
        float2 odr[2], oux[2], ouy[2];
        stream_row<R, FORCE>(nr, nux, nuy, cdr, cux, cuy, a.k, fm2, fm1, dm3, dm2, acc, odr, oux,
                             ouy);
        // destination row c - 1 = yb + k - 2R - 2 is an output row from k = 2R + 2
        if ((!WARM || k >= warm_rows<R>()) && it.lane_stores) {
            T* dst = static_cast<T*>(a.dst) + it.out + (size_t)(k - 2 * R - 2) * a.pitch;
            Vec4<T>::store(dst, odr);
            Vec4<T>::store(dst + a.plane, oux);
            Vec4<T>::store(dst + 2 * a.plane, ouy);
        }
    }
};

template <int R, bool FORCE, bool WALLS, typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, min_blocks<R>())
    fd_step_stream_kernel(StreamArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp_bytes = kSlots * 3 * kLoadCols * (int)sizeof(T);
    Ring<T> ring;
    ring.slot_base = reinterpret_cast<T*>(smem + warp * warp_bytes);
    ring.bars = reinterpret_cast<uint64_t*>(smem + kWarpsPerBlock * warp_bytes) + warp * kSlots;
    if (lane == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(&ring.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    uint32_t base = 0;      // ring position of the current item's row 0
    uint32_t issued = 0;    // ring positions issued so far
    uint32_t consumed = 0;  // ring positions waited for so far
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
        it.x0 = wrap_index(it.strip0 - 8, a.nx);
        it.first = min(kLoadCols, a.nx - it.x0);
        it.lane_stores = lane >= 1 && lane <= 30 && (it.strip0 - 4 + 4 * lane) < a.nx;
        it.base = base;
        it.out = (size_t)it.yb * a.pitch + (it.strip0 - 4 + 4 * lane);
        // every lane is done with the slots of the previous item
        __syncwarp();
        // prologue: the first kSlots rows, two per issue
        for (int k0 = 0; k0 < kSlots && k0 < it.nrows; k0 += 2)
            issue_rows<WALLS, T>(a, ring, it, k0, min(2, it.nrows - k0), lane);
        issued = base + min(kSlots, it.nrows);
        Win w0 = {}, w1 = {}, w2 = {}, w3 = {};
        Acc acc = {};
        int k = 0;
        using Step = RowStep<R, FORCE, WALLS, T>;
        for (; k + 1 < it.nrows; k += 2) {
            // one vote for both rows keeps their arithmetic in one block,
            // free to interleave
            const bool l0 = row_landed(ring, it, k), l1 = row_landed(ring, it, k + 1);
            if (!__all_sync(kFull, l0 && l1)) {
                ok = false;
                break;
            }
            if (k >= warm_rows<R>()) {
                Step::template run<false>(a, ring, it, lane, k, w0, w1, w2, w3, acc);
                Step::template run<false>(a, ring, it, lane, k + 1, w1, w0, w3, w2, acc);
            } else {
                Step::template run<true>(a, ring, it, lane, k, w0, w1, w2, w3, acc);
                Step::template run<true>(a, ring, it, lane, k + 1, w1, w0, w3, w2, acc);
            }
            // the centre rows of these two steps (k - R, k + 1 - R) are no
            // longer needed: refill their slots with the rows kSlots ahead
            __syncwarp();
            const int m1 = k + 1 - R;
            const int n0 = (int)(issued - base);
            const int cnt = min(m1 + kSlots + 1, it.nrows) - n0;
            if (m1 >= 0 && cnt > 0) {
                issue_rows<WALLS, T>(a, ring, it, n0, cnt, lane);
                issued += cnt;
            }
        }
        if (ok && k < it.nrows) {
            if (__all_sync(kFull, row_landed(ring, it, k))) {
                Step::template run<true>(a, ring, it, lane, k, w0, w1, w2, w3, acc);
                ++k;
            } else {
                ok = false;
            }
        }
        consumed = base + k;
        base += it.nrows;
    }
    if (!ok) {
        // A copy did not complete in time: record it, then give every copy
        // still in flight a bounded chance to land before the CTA exits.
        if (lane == 0) atomicExch(a.status, FDLBM_ERR_TIMEOUT);
        for (uint32_t n = consumed; n < issued; ++n)
            mbar_wait_bounded(&ring.bars[n & kSlotMask], (n / kSlots) & 1u);
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

template <int R, bool FORCE, bool WALLS, typename T>
cudaError_t launch_stream_typed(fdlbm_s* h, const void* src, void* dst) {
    auto kernel = fd_step_stream_kernel<R, FORCE, WALLS, T>;
    const size_t smem = kWarpsPerBlock * (kSlots * 3 * kLoadCols * sizeof(T) + kSlots * 8);
    if (h->stream_plan_warps == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarpsPerBlock * 32, smem);
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
    a.xi = (float)h->p.wall_xi;
    a.nstrips = (h->p.nx + kStrip - 1) / kStrip;
    a.seg_rows = plan.seg_rows;
    a.nsegs = plan.nsegs;
    a.nitems = plan.nitems;
    const double sc = (R == 1) ? 0.5 : 0.125;  // derivatives are computed times 2 or 8
    const double ae = (1.0 - 1.0 / h->p.s_e) * sc / 36.0;
    const double axx = (1.0 - 1.0 / h->p.s_xx) * sc;
    a.k.e6 = (float)(6.0 * ae);
    a.k.e2 = (float)(2.0 * ae);
    a.k.em2 = (float)(-2.0 * ae);
    a.k.xm23 = (float)(-2.0 / 3.0 * axx);
    a.k.x13 = (float)(axx / 3.0);
    a.k.hfx = (float)(0.5 * h->p.force_x);
    a.k.hfy = (float)(0.5 * h->p.force_y);
    const double nu = (1.0 / h->p.s_xx - 0.5) / 3.0;  // LW-ACM (Sec. 1-b)
    a.k.lw_t = (float)(2.0 * nu);
    a.k.lw_s = a.k.lw_t * 0.25f;
    a.status = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    kernel<<<plan.blocks, kWarpsPerBlock * 32, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <bool WALLS, typename T>
cudaError_t launch_stream_stencil(fdlbm_s* h, const void* src, void* dst) {
    const bool force = h->p.force_x != 0.0 || h->p.force_y != 0.0;
    // LW-ACM: no finite differences (radius 0), periodic, no force
    if (h->p.scheme == FDLBM_SCHEME_LWACM) return launch_stream_typed<0, false, false, T>(h, src, dst);
    if (h->p.scheme == FDLBM_SCHEME_FD3)
        return force ? launch_stream_typed<1, true, WALLS, T>(h, src, dst)
                     : launch_stream_typed<1, false, WALLS, T>(h, src, dst);
    return force ? launch_stream_typed<2, true, WALLS, T>(h, src, dst)
                 : launch_stream_typed<2, false, WALLS, T>(h, src, dst);
}

template <typename T>
cudaError_t launch_stream_boundary(fdlbm_s* h, const void* src, void* dst) {
    return h->p.boundary == FDLBM_BOUNDARY_WALLS_Y ? launch_stream_stencil<true, T>(h, src, dst)
                                                   : launch_stream_stencil<false, T>(h, src, dst);
}

}  // namespace

bool fd_stream_supported(const fdlbm_params& p) {
    return (p.boundary == FDLBM_BOUNDARY_PERIODIC || p.boundary == FDLBM_BOUNDARY_WALLS_Y) &&
           p.nx % 8 == 0 && p.nx >= 256 && p.ny >= 16;
}

cudaError_t launch_fd_step_stream(fdlbm_s* h, const void* src, void* dst) {
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return launch_stream_boundary<__half>(h, src, dst);
        case FDLBM_STORAGE_BF16: return launch_stream_boundary<__nv_bfloat16>(h, src, dst);
        default: return launch_stream_boundary<float>(h, src, dst);
    }
}

}  // namespace fdlbm
