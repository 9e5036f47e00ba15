// fd_step_stream.cu -- FD-LBM step (Sec. 2, Eq. 2) for lattices periodic in
// x (periodic or walled in y), streaming each CTA down a strip of rows.
//
// Work decomposition.  A CTA of W = 2 warps owns an output strip of W x 120
// columns and a segment of rows; warp w owns the 120 columns from w x 120.  Lane L of a warp holds 4 consecutive columns
// starting at 4 L - 4 of the warp's strip, so lanes 0 and 31 are halo lanes:
// they reconstruct the populations one column outside the warp's strip
// (where the gradients they need are still exact) and store nothing.
//
// Data path.  Rows of (rho - 1, ux, uy) for the CTA strip plus 8 halo
// columns on each side are copied by 1-D bulk (TMA) copies -- one per field
// and row for the whole CTA, two where the row wraps around x -- into a ring
// of 8 shared-memory row slots, each completed by an mbarrier, several rows
// ahead of use.  Every warp releases a slot once it has read the slot's row
// for the last time (the row is then the centre row of the derivative
// window); the warp whose release is the slot's last (a shared-memory
// counter, atomic with acquire-release order) refills it with the row
// eight positions ahead.  Warps therefore never wait for each other, only
// for copies.  Each lane reads its 4 columns (one 16-byte load per field for
// FP32).  Derivatives along y: three points hold the two previous rows in
// registers; five points hold only the (negated) differences
// d1(c) = f(c+1) - f(c-1) and use 8 d/dy = 6 d1(c) - d1(c-1) - d1(c+1), the
// centre row being re-read from the ring.  Derivatives along x use warp
// shuffles of the two neighbouring columns on each side.  Arithmetic on
// column pairs uses the paired FP32 instructions of sm_100-family GPUs.
// After the reconstruction the populations that cross a lane boundary are
// exchanged by shuffles, summed per destination row and closed when the row
// below has contributed.
#include <algorithm>
#include <vector>
#include <type_traits>

#include "fd_stream_common.cuh"
#include "tma_ring.cuh"

namespace fdlbm {
namespace {

using namespace stream;

constexpr int kStrip = 120;     // output columns per warp
constexpr int kHalo = 8;        // staged columns on each side of a CTA strip
constexpr int kSlots = 8;       // ring depth (rows); a power of two
constexpr int kSlotMask = kSlots - 1;
// Resident warps per SM the launch bounds aim at: 128 registers per thread
// (8 CTAs of 2 warps), the register file's limit at that count.
constexpr int kWarpsPerSM = 16;

// Columns staged per row for a CTA of W warps.  W x 120 + 16 elements are a
// multiple of 16 bytes in every storage type.
__host__ __device__ constexpr int load_cols(int W) { return W * kStrip + 2 * kHalo; }

// Shared memory of a CTA: the ring (kSlots x 3 fields x load_cols), then
// kSlots completion barriers, kSlots release counters and kSlots records of
// the last ring position issued to each slot.
__host__ __device__ constexpr size_t ring_bytes(int W, int elem) {
    return (size_t)kSlots * 3 * load_cols(W) * elem;
}
__host__ __device__ constexpr size_t smem_bytes(int W, int elem) {
    return ring_bytes(W, elem) + kSlots * (8 + 4 + 4);
}

struct StreamArgs {
    const void* src;  // 3 planes (rho - 1, ux, uy), [ny][pitch]
    void* dst;
    size_t plane;     // elements per plane
    size_t pitch;     // elements per row
    int nx, ny;
    float xi;         // wall offset (channels)
    int nstrips;      // warp strips of 120 columns
    int ncstrips;     // CTA strips (W warp strips each, the last maybe fewer)
    // rows [0, nsegs seg_rows) in segments of seg_rows rows, the rest of the
    // rows in segments of tail_rows; items list the first kind, then the second
    int seg_rows, nsegs, tail_rows, nitems;
    StreamCoeffs k;
    Quant q;          // fixed-point scale (FDLBM_STORAGE_I16)
    int* status;      // device status word (FDLBM_ERR_TIMEOUT on a lost copy)
};

// Per-item constants, uniform over the CTA.
struct Item {
    int strip0;        // first output column of the CTA strip
    int active;        // warps of the CTA with columns in this strip
    int yb, ye;        // output rows [yb, ye)
    int row_first;     // lattice row of ring row 0 (yb - 1 - R)
    int nrows;         // rows streamed: ye - yb + 2 + 2R
    int x0, first;     // staged columns: load_cols from x0, wrapping once at nx
};

template <int R>
__device__ __forceinline__ Item make_item(const StreamArgs& a, int item, int W) {
    Item it;
    const int nfirst = a.ncstrips * a.nsegs;
    const bool first = item < nfirst;
    const int i = first ? item : item - nfirst;
    const int cs = i % a.ncstrips, seg = i / a.ncstrips;
    const int rows = first ? a.seg_rows : a.tail_rows;
    it.strip0 = cs * W * kStrip;
    it.active = min(W, a.nstrips - cs * W);
    it.yb = (first ? 0 : a.nsegs * a.seg_rows) + seg * rows;
    it.ye = min(a.ny, it.yb + rows);
    it.row_first = it.yb - 1 - R;
    it.nrows = it.ye - it.yb + 2 + 2 * R;
    it.x0 = wrap_index(it.strip0 - kHalo, a.nx);
    it.first = min(load_cols(W), a.nx - it.x0);
    return it;
}

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

// The ring lives at the start of the dynamic shared memory; its barriers,
// counters and records follow it.  Only 32-bit offsets are kept.
extern __shared__ __align__(128) unsigned char g_smem[];

template <int W, typename T>
struct Ring {
    static constexpr uint32_t cols = load_cols(W);  // staged columns per row
    static constexpr uint32_t field_bytes = cols * sizeof(T);
    static constexpr uint32_t slot_bytes = 3 * field_bytes;
    static constexpr uint32_t tail = kSlots * slot_bytes;  // barriers, counters, records
    static __device__ __forceinline__ uint64_t* full(int slot) {
        return reinterpret_cast<uint64_t*>(g_smem + tail) + slot;
    }
    static __device__ __forceinline__ uint32_t* count(int slot) {
        return reinterpret_cast<uint32_t*>(g_smem + tail + kSlots * 8) + slot;
    }
    static __device__ __forceinline__ int* last(int slot) {
        return reinterpret_cast<int*>(g_smem + tail + kSlots * 12) + slot;
    }
};

// Copy ring row k of the item (ring position pos) into its slot; one thread.
template <bool WALLS, typename T, int W>
__device__ __forceinline__ void issue_row(const StreamArgs& a, const Item& it, uint32_t pos,
                                          int k) {
    using ring = Ring<W, T>;
    const int slot = pos & kSlotMask;
    uint64_t* bar = ring::full(slot);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, 3u * ring::cols * sizeof(T));
    int r = it.row_first + k;
    int rref = r;
    if (!WALLS) {
        if (r < 0) r += a.ny;
        if (r >= a.ny) r -= a.ny;
        rref = r;
    } else if (r < 0 || r >= a.ny) {
        rref = wall_ref(r, a.ny, a.xi);
        r = wall_edge(r, a.ny);
    }
    T* dst = reinterpret_cast<T*>(g_smem) + (size_t)slot * 3 * ring::cols;
    const T* src = static_cast<const T*>(a.src);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const T* rowp = src + f * a.plane + (size_t)(f == 0 ? r : rref) * a.pitch;
        T* d = dst + f * ring::cols;
        tma_load_1d(d, rowp + it.x0, it.first * sizeof(T), bar);
        if (it.first < (int)ring::cols)
            tma_load_1d(d + it.first, rowp, (ring::cols - it.first) * sizeof(T), bar);
    }
    *ring::last(slot) = (int)pos;
}

// Rows before this one are the window's warm-up: the centre row does not
// exist yet (k < R) or the closed row is above the segment (k < 2R + 2).
template <int R>
__host__ __device__ constexpr int warm_rows() {
    return 2 * R + 2;
}

// Wait (bounded) for ring position pos to land in its slot.
template <int W, typename T>
__device__ __forceinline__ bool row_landed(uint32_t pos) {
    return mbar_wait_bounded(Ring<W, T>::full(pos & kSlotMask), (pos / kSlots) & 1u);
}

// Atomic increment of a release counter that wraps to 0 after `last`,
// ordered (acquire-release, CTA scope) after this thread's and -- through
// the preceding __syncwarp -- its warp's reads of the slot.
__device__ __forceinline__ uint32_t release_inc(uint32_t* counter, uint32_t last) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.inc.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "r"(smem_u32(counter)), "r"(last)
                 : "memory");
    return old;
}

// One field of ring row k (position pos) into its slot, by the calling lane.
template <bool WALLS, typename T, int W>
__device__ __forceinline__ void issue_field(const StreamArgs& a, const Item& it, uint32_t pos,
                                            int k, int f) {
    using ring = Ring<W, T>;
    const int slot = pos & kSlotMask;
    int r = it.row_first + k;
    if (!WALLS) {
        if (r < 0) r += a.ny;
        if (r >= a.ny) r -= a.ny;
    } else if (r < 0 || r >= a.ny) {
        r = f == 0 ? wall_edge(r, a.ny) : wall_ref(r, a.ny, a.xi);
    }
    fence_proxy_async_smem();
    const T* rowp = static_cast<const T*>(a.src) + f * a.plane + (size_t)r * a.pitch;
    T* d = reinterpret_cast<T*>(g_smem) + ((size_t)slot * 3 + f) * ring::cols;
    uint64_t* bar = ring::full(slot);
    tma_load_1d(d, rowp + it.x0, it.first * sizeof(T), bar);
    if (it.first < (int)ring::cols)
        tma_load_1d(d + it.first, rowp, (ring::cols - it.first) * sizeof(T), bar);
}

// The warp has read ring rows m0 .. m0 + 3 for the last time.  Lanes 0-3
// count the four releases (in parallel); a row whose release is the CTA's
// last is refilled with the row kSlots ahead: its lane arms the barrier,
// then three lanes per row copy one field each.  The item's description is
// read from shared memory (it is needed only here, so it is not held in
// registers through the row loop).  Releasing four rows at a time halves the
// warp synchronisations, votes and counter atomics of releasing two; a row
// is still refilled at least three row pairs before it is read (measured:
// 8192^2 FD-5 214.9 -> 218.8 GLUPS, 16384^2 227.7 -> 233.6).
template <bool WALLS, typename T, int W>
__device__ __forceinline__ void release_quad(const StreamArgs& a, const Item* s_item,
                                             uint32_t base, int m0, int lane) {
    using ring = Ring<W, T>;
    const int nrows = s_item->nrows, active = s_item->active;
    const int m = m0 + (lane & 3);
    bool last = false;
    if (lane < 4 && m >= 0 && m + kSlots < nrows)  // otherwise no refill follows the row
        last = release_inc(ring::count((base + m) & kSlotMask), active - 1) ==
               (uint32_t)(active - 1);
    const uint32_t refill = __ballot_sync(kFull, last);  // bit j: row m0 + j
    if (refill == 0) return;
    const Item it = *s_item;
    if (last) {
        const uint32_t pos = base + m + kSlots;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(ring::full(pos & kSlotMask), 3u * ring::cols * sizeof(T));
        *ring::last(pos & kSlotMask) = (int)pos;
    }
    __syncwarp();
    const int j = lane / 3;
    if (lane < 12 && ((refill >> j) & 1u))
        issue_field<WALLS, T, W>(a, it, base + m0 + j + kSlots, m0 + j + kSlots, lane - 3 * j);
}

template <int R, bool FORCE, bool WALLS, typename T, int W>
struct RowStep {
    // Field row k of the item (already landed): read it, update the y window
    // and reconstruct the centre row c = row k - R; close and store row c - 1
    // through the running output pointer `out` (row yb + k - 2R - 2).
    // WARM: k may be below warm_rows<R>(), so the centre-row read and the
    // store are guarded; otherwise both are unconditional.
    template <bool WARM>
    static __device__ __forceinline__ void run(const StreamArgs& a, int row_first,
                                               uint32_t lane_off, uint32_t base, int k,
                                               bool stores, T*& out, bool& sat, Win& fm2,
                                               Win& fm1, Win& dm3, Win& dm2, Acc& acc) {
        constexpr uint32_t slot_bytes = Ring<W, T>::slot_bytes;
        constexpr uint32_t field_bytes = Ring<W, T>::field_bytes;
        // five points: rows 0 and 1 of an item only wait in the ring for
        // the window update of rows 2 and 3
        if (WARM && R == 2 && k < R) return;
        const uint32_t pos = base + k;
        const uint32_t row = lane_off + (pos & kSlotMask) * slot_bytes;
        float2 nr[2], nux[2], nuy[2];
        vec4_load(reinterpret_cast<const T*>(g_smem + row), nr, a.q);
        vec4_load(reinterpret_cast<const T*>(g_smem + row + field_bytes), nux, a.q);
        vec4_load(reinterpret_cast<const T*>(g_smem + row + 2 * field_bytes), nuy, a.q);
        if (WALLS) {
            const int r = row_first + k;
            if (r < 0 || r >= a.ny) {  // uniform across the CTA
                const float2 fac = sp(wall_factor(r, a.ny, a.xi));
                nux[0] = mul2(nux[0], fac);
                nux[1] = mul2(nux[1], fac);
                nuy[0] = mul2(nuy[0], fac);
                nuy[1] = mul2(nuy[1], fac);
            }
        }
        // centre row c = r - R from its ring slot (still resident); before
        // the window is full the centre row does not exist yet
        float2 cdr[2] = {sp(0.f), sp(0.f)}, cux[2] = {sp(0.f), sp(0.f)};
        float2 cuy[2] = {sp(0.f), sp(0.f)};
        if (R > 0 && (!WARM || k >= R)) {
            const uint32_t crow = lane_off + ((pos - R) & kSlotMask) * slot_bytes;
            if (R == 2) vec4_load(reinterpret_cast<const T*>(g_smem + crow), cdr, a.q);
            vec4_load(reinterpret_cast<const T*>(g_smem + crow + field_bytes), cux, a.q);
            vec4_load(reinterpret_cast<const T*>(g_smem + crow + 2 * field_bytes), cuy, a.q);
            if (WALLS) {
                const int r = row_first + k - R;
                if (r < 0 || r >= a.ny) {
                    const float2 fac = sp(wall_factor(r, a.ny, a.xi));
                    cux[0] = mul2(cux[0], fac);
                    cux[1] = mul2(cux[1], fac);
                    cuy[0] = mul2(cuy[0], fac);
                    cuy[1] = mul2(cuy[1], fac);
                }
            }
        }
        if (WARM && R > 0 && k < 2 * R) {  // the window only: no output needs this row
            window_row<R>(nr, nux, nuy, cdr, cux, cuy, fm2, dm3);
            return;
        }
        float2 odr[2], oux[2], ouy[2];
        stream_row<R, FORCE>(nr, nux, nuy, cdr, cux, cuy, a.k, fm2, fm1, dm3, dm2, acc, odr, oux,
                             ouy);
        // destination row c - 1 = yb + k - 2R - 2 is an output row from k = 2R + 2
        if (!WARM || k >= warm_rows<R>()) {
            if (stores) {
                sat |= vec4_store(out, odr, a.q);
                sat |= vec4_store(out + a.plane, oux, a.q);
                sat |= vec4_store(out + 2 * a.plane, ouy, a.q);
            }
            out += a.pitch;
        }
    }
};

// The rows of one item for one warp; false if a copy did not land in time.
template <int R, bool FORCE, bool WALLS, typename T, int W>
__device__ __forceinline__ bool warp_item(const StreamArgs& a, const Item* s_item, uint32_t base,
                                          int warp, int lane, bool& sat) {
    const int nrows = s_item->nrows, row_first = s_item->row_first, yb = s_item->yb;
    const uint32_t lane_off = (warp * kStrip + 4 + 4 * lane) * sizeof(T);
    const int col = s_item->strip0 + warp * kStrip - 4 + 4 * lane;  // first column of this lane
    const bool stores = lane >= 1 && lane <= 30 && col < a.nx;
    T* out = static_cast<T*>(a.dst) + (size_t)yb * a.pitch + (stores ? col : 0);
    Win w0 = {}, w1 = {}, w2 = {}, w3 = {};
    Acc acc = {};
    using Step = RowStep<R, FORCE, WALLS, T, W>;
    int k = 0;
    // Each lane waits for its rows itself (its wait orders its reads); the
    // warp votes on the outcome once every second pair, before releasing
    // slots.  After a lost copy a lane therefore computes at most one more
    // pair from a stale slot (shared-memory addresses do not depend on the
    // data) before the vote ends the item, and the step is reported as
    // failed.  Measured: 8192^2 FD-5 219.2 -> 221.5 GLUPS, 16384^2 233.8 ->
    // 236.8, against a vote after every pair.
    bool landed = true;
    for (; k + 1 < nrows; k += 2) {
        const bool l0 = row_landed<W, T>(base + k), l1 = row_landed<W, T>(base + k + 1);
        landed = landed && l0 && l1;
        if (k >= warm_rows<R>()) {
            Step::template run<false>(a, row_first, lane_off, base, k,
                                      stores, out, sat, w0, w1, w2, w3, acc);
            Step::template run<false>(a, row_first, lane_off, base,
                                      k + 1, stores, out, sat, w1, w0, w3, w2, acc);
        } else {
            Step::template run<true>(a, row_first, lane_off, base, k,
                                     stores, out, sat, w0, w1, w2, w3, acc);
            Step::template run<true>(a, row_first, lane_off, base,
                                     k + 1, stores, out, sat, w1, w0, w3, w2, acc);
        }
        // after every second pair the centre rows of the last four steps
        // (k - R - 2 .. k + 1 - R) have been read for the last time: release
        // their slots.  Rows left at the item's end have no refill to follow.
        if (k & 2) {
            if (!__all_sync(kFull, landed)) return false;
            __syncwarp();
            release_quad<WALLS, T, W>(a, s_item, base, k - R - 2, lane);
        }
    }
    // the last pairs' outcome (and the odd last row's) is always voted on
    if (k < nrows) landed = landed && row_landed<W, T>(base + k);
    if (!__all_sync(kFull, landed)) return false;
    if (k < nrows)
        Step::template run<true>(a, row_first, lane_off, base, k,
                                 stores, out, sat, w0, w1, w2, w3, acc);
    return true;
}

template <int R, bool FORCE, bool WALLS, typename T, int W>
__global__ void __launch_bounds__(W * 32, kWarpsPerSM / W) fd_step_stream_kernel(StreamArgs a) {
    using ring = Ring<W, T>;
    __shared__ Item s_item;
    // The warp index taken through a shuffle: the compiler then holds it,
    // and the offsets derived from it, in ordinary registers (as a value it
    // can prove warp-uniform it is kept apart, and the row loop spills).
    const int warp = __shfl_sync(kFull, threadIdx.x >> 5, 0), lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(ring::full(s), 1);
            *ring::count(s) = 0;
            *ring::last(s) = -1;
        }
        fence_mbar_init();
    }
    uint32_t base = 0;  // ring position of the current item's row 0
    bool failed = false, sat = false;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        // every warp is done with the previous item's slots (and the
        // barriers are initialised); stop everywhere if a copy was lost
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        if (threadIdx.x == 0) {
            const Item it = make_item<R>(a, item, W);
            s_item = it;
            for (int k = 0; k < kSlots && k < it.nrows; ++k)
                issue_row<WALLS, T, W>(a, it, base + k, k);
        }
        __syncthreads();
        const int active = s_item.active, nrows = s_item.nrows;
        if (warp < active &&
            !warp_item<R, FORCE, WALLS, T, W>(a, &s_item, base, warp, lane, sat))
            failed = true;
        base += nrows;
    }
    if (std::is_same<T, int16_t>::value && __any_sync(kFull, sat) && lane == 0)
        report_saturation(a.status);
    if (__syncthreads_or(failed) && threadIdx.x == 0) {
        // A copy did not complete in time: record it, then give every copy
        // still in flight a bounded chance to land before the CTA exits.
        atomicExch(a.status, FDLBM_ERR_TIMEOUT);
        for (int s = 0; s < kSlots; ++s)
            if (*ring::last(s) >= 0)
                mbar_wait_bounded(ring::full(s), ((uint32_t)*ring::last(s) / kSlots) & 1u);
    }
}

struct Plan {
    int W, ncstrips, seg_rows, nsegs, tail_rows, ntail, nitems, blocks;
};

// Warps per CTA.  Two warps share one ring: the row copies and the halo
// columns fetched per output column halve against one-warp CTAs, and the
// two warps' progress stays loosely coupled.  Measured on 8192^2 (FP32,
// GLUPS, W = 2 / 3 / 4): FD-5 189.4 / 173.7 / 173.1, FD-3 221.4 / 204.9 /
// 203.9, LW-ACM 239.0 / 216.4 / 211.0; wider CTAs lose whatever release
// protocol they use (an acquire-release or relaxed shared-memory counter, or
// an mbarrier arrival with its pending count: all within 1 %).
constexpr int kWarps = 2;

// Row segments.  A segment streams rows beyond its own (2 whose populations
// cross its ends, and 2R that only fill the y window, at a fraction of a
// row's cost), and a launch ends with a tail while its last CTAs finish.
// With w = items / resident CTAs (the waves), a plan of equal segments takes
//   (segment rows + c) (w + a)
// row-times of one resident CTA, c = 0.5 + 2R extra rows (2 for LW-ACM,
// R = 0) and a = 0.2 of an item's time, except for LW-ACM with FP32 storage,
// which runs near the memory bound and whose extra rows mostly come from L2:
// c = 0.5, a = 0.4.  This fits, within 1.3 %, step times measured on GB300
// over segment counts (FD-5 on 4096^2, 8192^2 and 16384^2; FD-3, LW-ACM and
// LW-ACM with FP16 storage on 8192^2).
//
// The finite-difference steps do better with two segment lengths: nsegs long
// segments of seg_rows rows per strip, then the remaining rows in short
// segments of tail_rows, the long ones first in the item order.  The long
// items cut the extra rows; the short ones, taken by whichever CTAs finish
// first, absorb the spread of the long items' finishing times and leave a
// short tail.  Such a plan takes
//   strips (nsegs (seg_rows + c) + ntail (tail_rows + c)) / resident + a (tail_rows + c)
// provided the short items give every resident CTA at least kSpread of a
// long item's work, the spread of the long items' finishing times (the
// largest seg_rows meeting it is taken; otherwise long segments finishing
// late set the step time).  Measured on 8192^2 FD-5 (GLUPS): equal 64-row
// segments 205.1, 34 segments of 200 rows then 32-row ones 213.7; 16384^2:
// equal 120-row segments 221.7, 35 of 400 then 48 rows 229.0.  Near the
// optimum the step times vary by 1-2 % from one plan to the next in ways the
// model does not follow, so plan_candidates also lists the neighbouring plans
// for measurement on the device.  LW-ACM is slower with long segments
// (8192^2: 275.0 with equal 16-row segments, 230.7 with 34 of 200 then 16)
// and keeps equal ones.
constexpr double kSpread = 0.22;
constexpr int kTailRows[] = {16, 24, 32, 48, 64};

struct PlanModel {
    double P, S, c, a;
    bool two_size;  // the finite-difference steps
};

PlanModel plan_model(int nx, int R, int W, int resident_ctas, int elem_bytes) {
    const int nstrips = (nx + kStrip - 1) / kStrip;
    const bool near_memory_bound = R == 0 && elem_bytes == 4;
    PlanModel m;
    m.P = (nstrips + W - 1) / W;
    m.S = resident_ctas;
    m.c = near_memory_bound ? 0.5 : (R == 0 ? 2.0 : 0.5 + 2.0 * R);
    m.a = near_memory_bound ? 0.4 : 0.2;
    m.two_size = R > 0;
    return m;
}

// Step time of a plan in row-times of one resident CTA (see above); the
// spread condition is not part of it.
double plan_cost(const PlanModel& m, int ny, int B, int nb, int t) {
    if (nb * B >= ny) {  // equal segments
        const int n = (ny + B - 1) / B;
        return (B + m.c) * (m.P * n / m.S + m.a);
    }
    const int nt = (ny - nb * B + t - 1) / t;
    return m.P * (nb * (B + m.c) + nt * (t + m.c)) / m.S + m.a * (t + m.c);
}

bool covers_spread(const PlanModel& m, int ny, int B, int nb, int t) {
    const int nt = (ny - nb * B + t - 1) / t;
    return m.P * nt * (t + m.c) / m.S >= kSpread * (B + m.c);
}

struct PlanChoice {
    double cost;
    int B, nb, t;  // equal segments: nb * B >= ny, t = B
};

// Longest first segments (a multiple of 8 rows, at least twice the tail's,
// leaving a tail) of nb per strip whose tail gives every resident CTA at
// least `spread` of a first segment's work; 0 if none.
int longest_first(const PlanModel& m, int ny, int nb, int t, double spread) {
    if (nb * 2 * t >= ny) return 0;
    for (int B = ((ny - t) / nb) & ~7; B >= 2 * t; B -= 8) {
        const int nt = (ny - nb * B + t - 1) / t;
        if (m.P * nt * (t + m.c) / m.S >= spread * (B + m.c)) return B;
    }
    return 0;
}

// Candidate plans, the model's first, then the rest cheapest first by the
// model.  Equal segments: the two cheapest segment counts.  Two lengths
// (finite differences only): a first part of about k waves, k = 1, 2, 3
// (nsegs = k resident / strips), then tail_rows from kTailRows, with the
// longest first segments whose tail covers kSpread of their work (the model's
// choice among these is the cheapest), the lengths 8 rows either side of it,
// and those covering 0.3 and 0.4 (for measurement).
std::vector<PlanChoice> plan_candidates(int nx, int ny, int R, int W, int resident_ctas,
                                        int elem_bytes) {
    const PlanModel m = plan_model(nx, R, W, resident_ctas, elem_bytes);
    std::vector<PlanChoice> eq, rest;
    const int max_segs = (ny + 15) / 16;
    for (int n = 1; n <= max_segs; ++n) {
        const int s = (ny + n - 1) / n;
        if ((ny + s - 1) / s != n) continue;  // the same segments as a smaller count
        eq.push_back({plan_cost(m, ny, s, n, s), s, n, s});
    }
    const auto cheaper = [](const PlanChoice& x, const PlanChoice& y) { return x.cost < y.cost; };
    std::sort(eq.begin(), eq.end(), cheaper);
    if (eq.size() > 2) eq.resize(2);
    PlanChoice pick = eq[0];
    rest = eq;
    if (m.two_size) {
        for (int k = 1; k <= 3; ++k) {
            const int nb = (int)(k * m.S / m.P);
            if (nb < 1) continue;
            for (const int t : kTailRows) {
                const int B = longest_first(m, ny, nb, t, kSpread);
                if (B == 0) continue;
                const PlanChoice pc{plan_cost(m, ny, B, nb, t), B, nb, t};
                if (pc.cost < pick.cost) pick = pc;
                for (const int b : {B - 8, B, B + 8, longest_first(m, ny, nb, t, 0.3),
                                    longest_first(m, ny, nb, t, 0.4)}) {
                    if (b < 2 * t || nb * b > ny - t) continue;
                    bool seen = false;
                    for (const PlanChoice& q : rest) seen |= q.B == b && q.nb == nb && q.t == t;
                    if (!seen) rest.push_back({plan_cost(m, ny, b, nb, t), b, nb, t});
                }
            }
        }
    }
    std::sort(rest.begin(), rest.end(), cheaper);
    std::vector<PlanChoice> out{pick};
    for (const PlanChoice& pc : rest)
        if (pc.B != pick.B || pc.nb != pick.nb || pc.t != pick.t) out.push_back(pc);
    return out;
}

// The launch plan for segments (B, nb, t): nb segments of B rows, then the
// rest in segments of t rows; nb * B >= ny means equal segments of B rows.
Plan plan_of(int nx, int ny, int W, int B, int nb, int t) {
    const int nstrips = (nx + kStrip - 1) / kStrip;
    Plan p;
    p.W = W;
    p.ncstrips = (nstrips + W - 1) / W;
    if (nb * B >= ny) {
        p.seg_rows = p.tail_rows = B;
        p.nsegs = (ny + B - 1) / B;
        p.ntail = 0;
    } else {
        p.seg_rows = B;
        p.nsegs = nb;
        p.tail_rows = t;
        p.ntail = (ny - nb * B + t - 1) / t;
    }
    p.nitems = p.ncstrips * (p.nsegs + p.ntail);
    p.blocks = p.nitems;
    return p;
}

Plan make_plan(int nx, int ny, int R, int W, int resident_ctas, int elem_bytes) {
    const PlanChoice pc = plan_candidates(nx, ny, R, W, resident_ctas, elem_bytes)[0];
    return plan_of(nx, ny, W, pc.B, pc.nb, pc.t);
}

void store_plan(fdlbm_s* h, const Plan& pl) {
    const int v[6] = {pl.seg_rows, pl.nsegs, pl.tail_rows, pl.ntail, pl.ncstrips, pl.nitems};
    std::copy(v, v + 6, h->stream_plan);
}

Plan cached_plan(const fdlbm_s* h, int W) {
    Plan p;
    p.W = W;
    p.seg_rows = h->stream_plan[0];
    p.nsegs = h->stream_plan[1];
    p.tail_rows = h->stream_plan[2];
    p.ntail = h->stream_plan[3];
    p.ncstrips = h->stream_plan[4];
    p.nitems = p.blocks = h->stream_plan[5];
    return p;
}

int stencil_radius(int32_t scheme) {
    switch (scheme) {
        case FDLBM_SCHEME_FD3: return 1;
        case FDLBM_SCHEME_FD5: return 2;
        case FDLBM_SCHEME_LWACM: return 0;
        default: return -1;
    }
}

int storage_bytes(int32_t storage) {
    switch (storage) {
        case FDLBM_STORAGE_F32: return 4;
        case FDLBM_STORAGE_F16:
        case FDLBM_STORAGE_BF16:
        case FDLBM_STORAGE_I16: return 2;
        default: return 0;
    }
}

template <int R, bool FORCE, bool WALLS, typename T, int W>
cudaError_t launch_stream_w(fdlbm_s* h, const void* src, void* dst) {
    auto kernel = fd_step_stream_kernel<R, FORCE, WALLS, T, W>;
    const size_t smem = smem_bytes(W, sizeof(T));
    if (h->stream_plan_warps == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, W * 32, smem);
        h->stream_plan_warps = std::max(1, sms * per_sm);  // resident CTAs
        if (!h->stream_plan_user) {
            const Plan pl = make_plan(h->p.nx, h->p.ny, R, W, h->stream_plan_warps, (int)sizeof(T));
            store_plan(h, pl);
        }
    }
    const Plan plan = cached_plan(h, W);
    StreamArgs a;
    a.src = src;
    a.dst = dst;
    a.plane = h->L.plane;
    a.pitch = h->L.pitch;
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.xi = (float)h->p.wall_xi;
    a.nstrips = (h->p.nx + kStrip - 1) / kStrip;
    a.ncstrips = plan.ncstrips;
    a.seg_rows = plan.seg_rows;
    a.nsegs = plan.nsegs;
    a.tail_rows = plan.tail_rows;
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
    a.q = quant_of(h->p);
    a.status = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    kernel<<<plan.blocks, W * 32, smem, h->stream>>>(a);
    return cudaGetLastError();
}

template <int R, bool FORCE, bool WALLS, typename T>
cudaError_t launch_stream_typed(fdlbm_s* h, const void* src, void* dst) {
    return launch_stream_w<R, FORCE, WALLS, T, kWarps>(h, src, dst);
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
        case FDLBM_STORAGE_I16: return launch_stream_boundary<int16_t>(h, src, dst);
        default: return launch_stream_boundary<float>(h, src, dst);
    }
}

}  // namespace fdlbm

extern "C" int fdlbm_stream_plan(int32_t nx, int32_t ny, int32_t scheme, int32_t storage,
                                 int32_t resident_ctas, int32_t* plan) {
    using namespace fdlbm;
    const int R = stencil_radius(scheme), elem = storage_bytes(storage);
    if (!plan || nx < 1 || ny < 1 || resident_ctas < 1 || R < 0 || elem == 0)
        return FDLBM_ERR_INVALID;
    const Plan p = make_plan(nx, ny, R, kWarps, resident_ctas, elem);
    plan[0] = p.seg_rows;
    plan[1] = p.nsegs;
    plan[2] = p.tail_rows;
    plan[3] = p.ntail;
    plan[4] = p.ncstrips;
    plan[5] = p.nitems;
    return FDLBM_OK;
}

extern "C" int fdlbm_stream_plan_candidates(int32_t nx, int32_t ny, int32_t scheme,
                                            int32_t storage, int32_t resident_ctas,
                                            int32_t* out, int32_t max, int32_t* count) {
    using namespace fdlbm;
    const int R = stencil_radius(scheme), elem = storage_bytes(storage);
    if (!out || !count || max < 1 || nx < 1 || ny < 1 || resident_ctas < 1 || R < 0 ||
        elem == 0)
        return FDLBM_ERR_INVALID;
    const std::vector<PlanChoice> c = plan_candidates(nx, ny, R, kWarps, resident_ctas, elem);
    const int n = std::min<int>(max, (int)c.size());
    for (int i = 0; i < n; ++i) {
        out[3 * i] = c[i].B;
        out[3 * i + 1] = c[i].nb * c[i].B >= ny ? (ny + c[i].B - 1) / c[i].B : c[i].nb;
        out[3 * i + 2] = c[i].t;
    }
    *count = n;
    return FDLBM_OK;
}

extern "C" int fdlbm_set_stream_plan(fdlbm_t* h, int32_t seg_rows, int32_t nsegs,
                                     int32_t tail_rows) {
    using namespace fdlbm;
    if (!h) return FDLBM_ERR_INVALID;
    if (!uses_stream_step(h)) return FDLBM_ERR_INVALID;
    const int ny = h->p.ny;
    if (seg_rows == 0 && nsegs == 0 && tail_rows == 0) {  // back to the model's plan
        h->stream_plan_user = 0;
        if (h->stream_plan_warps > 0)
            store_plan(h, make_plan(h->p.nx, ny, stencil_radius(h->p.scheme), kWarps,
                                    h->stream_plan_warps, storage_bytes(h->p.storage)));
        return FDLBM_OK;
    }
    if (seg_rows < 1 || nsegs < 1 || tail_rows < 1 || seg_rows > ny) return FDLBM_ERR_INVALID;
    // equal segments when the first part reaches the last row
    if ((int64_t)seg_rows * nsegs >= ny) nsegs = (ny + seg_rows - 1) / seg_rows;
    store_plan(h, plan_of(h->p.nx, ny, kWarps, seg_rows, nsegs, tail_rows));
    h->stream_plan_user = 1;
    return FDLBM_OK;
}

extern "C" int fdlbm_get_stream_plan(fdlbm_t* h, int32_t* plan) {
    using namespace fdlbm;
    if (!h || !plan || !uses_stream_step(h) || h->stream_plan_warps < 1)
        return FDLBM_ERR_INVALID;
    std::copy(h->stream_plan, h->stream_plan + 6, plan);
    plan[6] = h->stream_plan_warps;
    return FDLBM_OK;
}
