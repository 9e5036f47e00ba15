// fd_batch.cu -- batched FD-LBM steps (Sec. 2, Eq. 2) for many independent
// lattices of any size (sides >= 16), each periodic or a channel with walls
// in y, advanced by persistent kernels (one per item list) per step; a run
// of steps is captured once in a CUDA graph and replayed.
//
// Storage.  Every slot lives in a caller-owned arena: two copies (ping-pong)
// of 3 planes (rho - 1, ux, uy), rows of `pitch` floats holding the logical
// columns -8 .. nx + 7 (physical column = logical + 8).  The 8 ghost columns
// on each side are periodic copies, refreshed by the lanes that own the
// first and last 8 columns when they store, so the streaming kernel's row
// windows never wrap and any nx works.  Walls in y are virtual rows: their
// density is that of the first fluid row and their velocity the linear
// extrapolation to zero at the wall (the same closure as the tiled kernel).
//
// Work.  An item is (slot, 120-column strip, row segment), processed by one
// warp exactly like the single-lattice streaming kernel; warps take items
// from an atomic counter (one counter per step of the captured run).  A
// lattice's last strip of at most 56 columns may run on 2-column lanes (a
// narrow strip); narrow items form a list of their own, advanced by a second
// kernel after the first in every step, so that no SM runs both forms' code
// at once (together they overflow the instruction cache).  A
// per-slot descriptor carries the slot's size, relaxation factors, force,
// which copy holds the state, and how many steps of the run the slot takes,
// so lattices of different viscosity and remaining step count share the
// launches.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "fd_stream_common.cuh"
#include "tma_ring.cuh"

namespace fdlbm {
namespace batch {

using namespace stream;

constexpr int kWarpsPerBlock = 1;  // one-warp CTAs, 16 resident per SM (128 registers)
constexpr int kMinBlocks = 16;
constexpr int kStrip = 120;
constexpr int kLoadCols = 136;
// Narrow strips (2-column lanes) for a lattice's last strip when it holds at
// most 56 columns: 64 columns in the lanes plus 8 staged for alignment.
constexpr int kNarrowStrip = 56;
constexpr int kNarrowCols = 72;
constexpr int kSlots = 8;
constexpr int kSlotMask = kSlots - 1;
constexpr int kGhost = 8;
constexpr int kMaxRun = 64;   // steps per captured graph
constexpr int kAlign = 32;    // floats (128 bytes)
constexpr int kRedBlocks = 256;

// Device descriptor of one slot.
struct Lat {
    long long off[2];  // element offsets of the two state copies in the arena
    int nx, ny, pitch, walls;
    int nstrips, seg_rows, nsegs;
    int stop;          // steps this slot takes in the current run (0: idle)
    int cur;           // copy holding the state at the start of the run
    float xi, pad;
    StreamCoeffs k;
};

struct Args {
    float* arena;
    const Lat* lats;
    const int2* items;  // (slot, strip + segment x strips): the wide list, then the narrow one
    const int* counts;  // device: items in the two lists (change without re-capture)
    int step;           // step index within the run
    int* counter;       // work counter of this step and list
    int* status;
};

struct Ring {
    float* slot_base;
    uint64_t* bars;
};

__device__ __forceinline__ float* slot_field(const Ring& ring, int slot, int field) {
    return ring.slot_base + (slot * 3 + field) * kLoadCols;
}

struct Item {
    int strip0, yb, ye, row_first, nrows;
    int nx, ny, pitch, walls;
    float xi;
    const float* src;
    float* dst;
    size_t plane;
    bool lane_stores;
    int cols;          // staged columns per field: kLoadCols, or kNarrowCols (narrow strip)
    uint32_t base;
};

// Rows feeding logical row r: (row of rho - 1, row of u, velocity factor).
// Periodic rows wrap; wall rows are virtual (Sec. 3-b, 3-c closure).
__device__ __forceinline__ void row_source(const Item& it, int r, int* rrho, int* ru,
                                           float* factor) {
    if (!it.walls) {
        if (r < 0) r += it.ny;
        if (r >= it.ny) r -= it.ny;
        *rrho = *ru = r;
        *factor = 1.f;
        return;
    }
    if (r >= 0 && r < it.ny) {
        *rrho = *ru = r;
        *factor = 1.f;
        return;
    }
    const bool below = r < 0;
    const int edge = below ? 0 : it.ny - 1;
    const int jref = it.xi >= 0.5f ? edge : (below ? 1 : it.ny - 2);
    const float ywall = below ? -it.xi : (float)(it.ny - 1) + it.xi;
    *rrho = edge;
    *ru = jref;
    *factor = ((float)r - ywall) / ((float)jref - ywall);
}

// Copy item rows k0 .. k0 + count - 1 (count <= 4) into their ring slots:
// lanes below count arm the slots' barriers, three lanes per row copy one
// field each.
__device__ __forceinline__ void issue_rows(const Ring& ring, const Item& it, int k0, int count,
                                           int lane) {
    if (lane < count) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&ring.bars[(it.base + k0 + lane) & kSlotMask],
                              3u * it.cols * sizeof(float));
    }
    __syncwarp();
    if (lane < 3 * count) {
        const int j = lane / 3;
        const int f = lane - 3 * j;
        const int slot = (it.base + k0 + j) & kSlotMask;
        int rrho, ru;
        float factor;
        row_source(it, it.row_first + k0 + j, &rrho, &ru, &factor);
        const int r = f == 0 ? rrho : ru;
        fence_proxy_async_smem();
        const float* rowp = it.src + f * it.plane + (size_t)r * it.pitch + it.strip0;
        tma_load_1d(slot_field(ring, slot, f), rowp, it.cols * sizeof(float), &ring.bars[slot]);
    }
}

__device__ __forceinline__ float row_factor(const Item& it, int r) {
    int a, b;
    float f;
    row_source(it, r, &a, &b, &f);
    return f;
}

// Rows before this one are the window's warm-up (no centre row yet, or the
// closed row is above the segment).
template <int R>
__host__ __device__ constexpr int warm_rows() {
    return 2 * R + 2;
}

__device__ __forceinline__ bool row_landed(const Ring& ring, const Item& it, int k) {
    const uint32_t pos = it.base + k;
    return mbar_wait_bounded(&ring.bars[pos & kSlotMask], (pos / kSlots) & 1u);
}

template <int R, bool FORCE>
struct BatchRowStep {
    // Row k (already landed); WARM: k may be below warm_rows<R>().
    template <bool WARM>
    static __device__ __forceinline__ void run(const Ring& ring, const Item& it,
                                               const StreamCoeffs& kc, int lane, int k,
                                               Win& fm2, Win& fm1, Win& dm3, Win& dm2,
                                               Acc& acc) {
        // five points: rows 0 and 1 of an item only wait in the ring for
        // the window update of rows 2 and 3
        if (WARM && R == 2 && k < R) return;
        const uint32_t pos = it.base + k;
        const int slot = pos & kSlotMask;
        const int col = 4 + 4 * lane;
        float2 nr[2], nux[2], nuy[2];
        Vec4<float>::load(slot_field(ring, slot, 0) + col, nr);
        Vec4<float>::load(slot_field(ring, slot, 1) + col, nux);
        Vec4<float>::load(slot_field(ring, slot, 2) + col, nuy);
        if (it.walls) {
            const float2 fac = sp(row_factor(it, it.row_first + k));
            nux[0] = mul2(nux[0], fac);
            nux[1] = mul2(nux[1], fac);
            nuy[0] = mul2(nuy[0], fac);
            nuy[1] = mul2(nuy[1], fac);
        }
        const int cslot = (pos - R) & kSlotMask;
        float2 cdr[2] = {sp(0.f), sp(0.f)}, cux[2] = {sp(0.f), sp(0.f)};
        float2 cuy[2] = {sp(0.f), sp(0.f)};
        if (!WARM || k >= R) {
            if (R == 2) Vec4<float>::load(slot_field(ring, cslot, 0) + col, cdr);
            Vec4<float>::load(slot_field(ring, cslot, 1) + col, cux);
            Vec4<float>::load(slot_field(ring, cslot, 2) + col, cuy);
            if (it.walls) {
                const float2 fac = sp(row_factor(it, it.row_first + k - R));
                cux[0] = mul2(cux[0], fac);
                cux[1] = mul2(cux[1], fac);
                cuy[0] = mul2(cuy[0], fac);
                cuy[1] = mul2(cuy[1], fac);
            }
        }
        if (WARM && R > 0 && k < 2 * R) {  // the window only: no output needs this row
            window_row<R>(nr, nux, nuy, cdr, cux, cuy, fm2, dm3);
            return;
        }
        float2 odr[2], oux[2], ouy[2];
        stream_row<R, FORCE>(nr, nux, nuy, cdr, cux, cuy, kc, fm2, fm1, dm3, dm2, acc, odr, oux,
                             ouy);
        if ((!WARM || k >= warm_rows<R>()) && it.lane_stores) {
            const int c0 = it.strip0 - 4 + 4 * lane;  // logical column of this lane
            const size_t row = (size_t)(it.yb + k - 2 * R - 2) * it.pitch;
            float* d0 = it.dst + row;
            Vec4<float>::store(d0 + c0 + kGhost, odr);
            Vec4<float>::store(d0 + it.plane + c0 + kGhost, oux);
            Vec4<float>::store(d0 + 2 * it.plane + c0 + kGhost, ouy);
            // periodic ghost columns of the destination copy
            if (c0 < kGhost || c0 + 4 > it.nx - kGhost) {
                const float v[3][4] = {{odr[0].x, odr[0].y, odr[1].x, odr[1].y},
                                       {oux[0].x, oux[0].y, oux[1].x, oux[1].y},
                                       {ouy[0].x, ouy[0].y, ouy[1].x, ouy[1].y}};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + j;
                    if (c >= it.nx) continue;
                    int gpos = -1;
                    if (c < kGhost) gpos = c + it.nx + kGhost;
                    if (c >= it.nx - kGhost) {
#pragma unroll
                        for (int f = 0; f < 3; ++f) d0[f * it.plane + c - it.nx + kGhost] = v[f][j];
                    }
                    if (gpos >= 0) {
#pragma unroll
                        for (int f = 0; f < 3; ++f) d0[f * it.plane + gpos] = v[f][j];
                    }
                }
            }
        }
    }
};

// The narrow-strip row step: lane L holds logical columns strip0 - 4 + 2L and
// the next one (ring columns 4 + 2L), lanes 2..29 store.
template <int R, bool FORCE>
struct BatchRowStep1 {
    template <bool WARM>
    static __device__ __forceinline__ void run(const Ring& ring, const Item& it,
                                               const StreamCoeffs& kc, int lane, int k,
                                               Win1& fm2, Win1& fm1, Win1& dm3, Win1& dm2,
                                               Acc1& acc) {
        if (WARM && R == 2 && k < R) return;
        const uint32_t pos = it.base + k;
        const int slot = pos & kSlotMask;
        const int col = 4 + 2 * lane;
        const float2 nr = *reinterpret_cast<const float2*>(slot_field(ring, slot, 0) + col);
        float2 nux = *reinterpret_cast<const float2*>(slot_field(ring, slot, 1) + col);
        float2 nuy = *reinterpret_cast<const float2*>(slot_field(ring, slot, 2) + col);
        if (it.walls) {
            const float2 fac = sp(row_factor(it, it.row_first + k));
            nux = mul2(nux, fac);
            nuy = mul2(nuy, fac);
        }
        const int cslot = (pos - R) & kSlotMask;
        float2 cdr = sp(0.f), cux = sp(0.f), cuy = sp(0.f);
        if (!WARM || k >= R) {
            if (R == 2) cdr = *reinterpret_cast<const float2*>(slot_field(ring, cslot, 0) + col);
            cux = *reinterpret_cast<const float2*>(slot_field(ring, cslot, 1) + col);
            cuy = *reinterpret_cast<const float2*>(slot_field(ring, cslot, 2) + col);
            if (it.walls) {
                const float2 fac = sp(row_factor(it, it.row_first + k - R));
                cux = mul2(cux, fac);
                cuy = mul2(cuy, fac);
            }
        }
        if (WARM && k < 2 * R) {  // the window only: no output needs this row
            window_row1<R>(nr, nux, nuy, cdr, cux, cuy, fm2, dm3);
            return;
        }
        float2 odr, oux, ouy;
        stream_row1<R, FORCE>(nr, nux, nuy, cdr, cux, cuy, kc, fm2, fm1, dm3, dm2, acc, odr, oux,
                              ouy);
        if ((!WARM || k >= warm_rows<R>()) && it.lane_stores) {
            const int c0 = it.strip0 - 4 + 2 * lane;  // logical column of this lane
            const size_t row = (size_t)(it.yb + k - 2 * R - 2) * it.pitch;
            float* d0 = it.dst + row;
            const float v[3][2] = {{odr.x, odr.y}, {oux.x, oux.y}, {ouy.x, ouy.y}};
            if (c0 + 1 < it.nx) {
#pragma unroll
                for (int f = 0; f < 3; ++f)
                    *reinterpret_cast<float2*>(d0 + f * it.plane + c0 + kGhost) =
                        make_float2(v[f][0], v[f][1]);
            } else {  // the lattice's last column is the pair's first
#pragma unroll
                for (int f = 0; f < 3; ++f) d0[f * it.plane + c0 + kGhost] = v[f][0];
            }
            // periodic ghost columns of the destination copy
            if (c0 < kGhost || c0 + 2 > it.nx - kGhost) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int c = c0 + j;
                    if (c >= it.nx) continue;
                    if (c >= it.nx - kGhost) {
#pragma unroll
                        for (int f = 0; f < 3; ++f) d0[f * it.plane + c - it.nx + kGhost] = v[f][j];
                    }
                    if (c < kGhost) {
#pragma unroll
                        for (int f = 0; f < 3; ++f) d0[f * it.plane + c + it.nx + kGhost] = v[f][j];
                    }
                }
            }
        }
    }
};

// The rows of one item for one warp, in the wide (4-column lanes) or the
// narrow form; false if a copy did not land in time.  `issued` counts the
// ring positions whose copies were issued, `k` returns the rows consumed.
template <int R, bool FORCE, bool NARROW>
__device__ __forceinline__ bool item_rows(const Ring& ring, const Item& it, const StreamCoeffs& kc,
                                          int lane, uint32_t& issued, int& k) {
    using W = typename std::conditional<NARROW, Win1, Win>::type;
    using A = typename std::conditional<NARROW, Acc1, Acc>::type;
    using Step = typename std::conditional<NARROW, BatchRowStep1<R, FORCE>,
                                           BatchRowStep<R, FORCE>>::type;
    W w0 = {}, w1 = {}, w2 = {}, w3 = {};
    A acc = {};
    k = 0;
    for (; k + 1 < it.nrows; k += 2) {
        const bool l0 = row_landed(ring, it, k), l1 = row_landed(ring, it, k + 1);
        if (!__all_sync(kFull, l0 && l1)) return false;
        if (k >= warm_rows<R>()) {
            Step::template run<false>(ring, it, kc, lane, k, w0, w1, w2, w3, acc);
            Step::template run<false>(ring, it, kc, lane, k + 1, w1, w0, w3, w2, acc);
        } else {
            Step::template run<true>(ring, it, kc, lane, k, w0, w1, w2, w3, acc);
            Step::template run<true>(ring, it, kc, lane, k + 1, w1, w0, w3, w2, acc);
        }
        // after every second pair: the rows read for the last time are
        // refilled four at a time, half the synchronisations of refilling
        // after every pair (4096 lattices 177.0 -> 183.9 GLUPS); a row is
        // still issued at least one pair before it is read
        if (k & 2) {
            __syncwarp();
            const int m1 = k + 1 - R;
            const int n0 = (int)(issued - it.base);
            const int cnt = min(m1 + kSlots + 1, it.nrows) - n0;
            if (m1 >= 0 && cnt > 0) {
                issue_rows(ring, it, n0, cnt, lane);
                issued += cnt;
            }
        }
    }
    if (k < it.nrows) {
        if (!__all_sync(kFull, row_landed(ring, it, k))) return false;
        Step::template run<true>(ring, it, kc, lane, k, w0, w1, w2, w3, acc);
        ++k;
    }
    return true;
}

template <int R, bool FORCE, bool NARROW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kMinBlocks) fd_batch_kernel(Args a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp_bytes = kSlots * 3 * kLoadCols * (int)sizeof(float);
    Ring ring;
    ring.slot_base = reinterpret_cast<float*>(smem + warp * warp_bytes);
    ring.bars = reinterpret_cast<uint64_t*>(smem + kWarpsPerBlock * warp_bytes) + warp * kSlots;
    if (lane == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(&ring.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t base = 0, issued = 0, consumed = 0;
    bool ok = true;
    while (ok) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.counts[NARROW ? 1 : 0]) break;
        const int2 e = a.items[(NARROW ? a.counts[0] : 0) + item];
        const Lat& L = a.lats[e.x];
        if (a.step >= L.stop) continue;
        Item it;
        const int strip = e.y % L.nstrips, seg = e.y / L.nstrips;
        it.nx = L.nx;
        it.ny = L.ny;
        it.pitch = L.pitch;
        it.walls = L.walls;
        it.xi = L.xi;
        it.plane = (size_t)L.ny * L.pitch;
        it.src = a.arena + L.off[(L.cur + a.step) & 1];
        it.dst = a.arena + L.off[(L.cur + a.step + 1) & 1];
        it.strip0 = strip * kStrip;
        it.yb = seg * L.seg_rows;
        it.ye = min(L.ny, it.yb + L.seg_rows);
        it.row_first = it.yb - 1 - R;
        it.nrows = it.ye - it.yb + 2 + 2 * R;
        it.cols = NARROW ? kNarrowCols : kLoadCols;
        it.lane_stores = NARROW
            ? lane >= 2 && lane <= 29 && (it.strip0 - 4 + 2 * lane) < L.nx
            : lane >= 1 && lane <= 30 && (it.strip0 - 4 + 4 * lane) < L.nx;
        it.base = base;
        const StreamCoeffs kc = L.k;
        __syncwarp();
        for (int k0 = 0; k0 < kSlots && k0 < it.nrows; k0 += 2)
            issue_rows(ring, it, k0, min(2, it.nrows - k0), lane);
        issued = base + min(kSlots, it.nrows);
        int k = 0;
        ok = item_rows<R, FORCE, NARROW>(ring, it, kc, lane, issued, k);
        consumed = base + k;
        base += it.nrows;
    }
    if (!ok) {
        if (lane == 0) atomicExch(a.status, FDLBM_ERR_TIMEOUT);
        for (uint32_t n = consumed; n < issued; ++n)
            mbar_wait_bounded(&ring.bars[n & kSlotMask], (n / kSlots) & 1u);
    }
}

// ---- per-slot auxiliary kernels ------------------------------------------------------

// contiguous (rho - 1, u) [ny][nx] -> both copies' planes of a slot, ghost columns included
__global__ void batch_init_kernel(const float* __restrict__ drho, const float* __restrict__ ux,
                                  const float* __restrict__ uy, float* __restrict__ state, int nx,
                                  int ny, int pitch) {
    const int pc = blockIdx.x * blockDim.x + threadIdx.x;  // physical column
    const int y = blockIdx.y;
    if (pc >= nx + 2 * kGhost) return;
    const int c = wrap_index(pc - kGhost, nx);
    const size_t i = (size_t)y * nx + c, o = (size_t)y * pitch + pc, plane = (size_t)ny * pitch;
    state[o] = drho[i];
    state[plane + o] = ux[i];
    state[2 * plane + o] = uy[i];
}

__global__ void batch_moments_kernel(const float* __restrict__ state, int nx, int ny, int pitch,
                                     float* __restrict__ drho, float* __restrict__ ux,
                                     float* __restrict__ uy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const size_t i = (size_t)y * nx + x, o = (size_t)y * pitch + x + kGhost;
    const size_t plane = (size_t)ny * pitch;
    drho[i] = state[o];
    ux[i] = state[plane + o];
    uy[i] = state[2 * plane + o];
}

__device__ __forceinline__ double bwarp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double bwarp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// FP64 reductions over one slot's logical region (see fdlbm_reduce)
__global__ void __launch_bounds__(256) batch_reduce_kernel(const float* __restrict__ state, int nx,
                                                          int ny, int pitch, int what, double m,
                                                          double n, double* __restrict__ partial) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const size_t plane = (size_t)ny * pitch;
    const int64_t total = (int64_t)nx * ny;
    double kx = 0.0, ky = 0.0, tx = 0.0, ty = 0.0;
    if (what == FDLBM_REDUCE_MODE) {
        kx = 2.0 * M_PI * m / nx;
        ky = 2.0 * M_PI * n / ny;
        const double kk = sqrt(kx * kx + ky * ky);
        tx = kk > 0.0 ? -ky / kk : 0.0;
        ty = kk > 0.0 ? kx / kk : 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * 256) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const size_t o = (size_t)y * pitch + x + kGhost;
        const float dr = state[o], vx = state[plane + o], vy = state[2 * plane + o];
        if (!(isfinite(dr) && isfinite(vx) && isfinite(vy))) {
            acc[3] += 1.0;
            continue;
        }
        const double rho = 1.0 + (double)dr;
        switch (what) {
            case FDLBM_REDUCE_MASS: acc[0] += dr; break;
            case FDLBM_REDUCE_MOMENTUM:
                acc[0] += rho * vx;
                acc[1] += rho * vy;
                break;
            case FDLBM_REDUCE_ENERGY: acc[0] += 0.5 * rho * ((double)vx * vx + (double)vy * vy); break;
            case FDLBM_REDUCE_MODE: {
                double sn, cs;
                sincos(kx * x + ky * y, &sn, &cs);
                const double ut = tx * vx + ty * vy;
                acc[0] += ut * cs;
                acc[1] -= ut * sn;
                break;
            }
            default:
                acc[0] = fmax(acc[0], sqrt((double)vx * vx + (double)vy * vy));
                acc[1] = fmax(acc[1], fabs((double)dr));
        }
    }
    __shared__ double sh[8][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        const bool mx = what == FDLBM_REDUCE_MAXABS && k < 2;
        const double v = mx ? bwarp_max(acc[k]) : bwarp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int k = threadIdx.x;
        const bool mx = what == FDLBM_REDUCE_MAXABS && k < 2;
        double v = sh[0][k];
        for (int w = 1; w < 8; ++w) v = mx ? fmax(v, sh[w][k]) : v + sh[w][k];
        partial[blockIdx.x * 4 + k] = v;
    }
}

__global__ void batch_reduce_final(const double* __restrict__ partial, int nb, int what,
                                   double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 4) return;
    const bool mx = what == FDLBM_REDUCE_MAXABS && k < 2;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v = mx ? fmax(v, partial[b * 4 + k]) : v + partial[b * 4 + k];
    out[k] = v;
}

}  // namespace batch
}  // namespace fdlbm

// ---- host side -------------------------------------------------------------------------

using namespace fdlbm;
using namespace fdlbm::batch;

struct SlotHost {
    bool used = false;
    fdlbm_params p;
    long long off[2] = {0, 0};  // element offsets
    long long elems = 0;        // elements of one copy
    int pitch = 0, cur = 0, nstrips = 0, seg_rows = 0, nsegs = 0;
};

struct fdlbm_batch_s {
    fdlbm_batch_params bp;
    cudaStream_t stream;
    int device;
    char* ws;
    size_t off_arena, off_lats, off_items, off_counters, off_status, off_staging, off_partial;
    long long arena_elems;
    int max_items;
    std::vector<SlotHost> slots;
    std::vector<std::pair<long long, long long>> free_list;  // (offset, elems), sorted
    std::vector<int2> items;  // the wide list, then the narrow one
    bool items_dirty = true;
    int nitems = 0;      // both lists
    int nnarrow = 0;     // items of the narrow list
    int seg_rows = 64;   // rows per work item (autotuned)
    int narrow = 0;      // last strips of <= 56 columns on 2-column lanes (autotuned)
    int grid = 0;        // persistent CTAs
    // captured runs: graph per (steps, force)
    cudaGraphExec_t exec[2][2][kMaxRun + 1];  // [force][narrow list non-empty][steps]
    int64_t launches = 0;
    char err[512];
};

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

static int berr(fdlbm_batch_t* b, int code, const char* msg) {
    if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
    return code;
}

static int bcuda(fdlbm_batch_t* b, cudaError_t e, const char* where) {
    if (b) snprintf(b->err, sizeof(b->err), "%s: %s", where, cudaGetErrorString(e));
    return FDLBM_ERR_CUDA;
}

static bool batch_layout(const fdlbm_batch_params* bp, size_t* offs, size_t* total,
                         long long* arena_elems, int* max_items) {
    if (!bp || bp->max_lattices < 1 || bp->arena_bytes < 1024 || bp->max_side < 16 ||
        bp->max_side > 65535 || (bp->scheme != FDLBM_SCHEME_FD3 && bp->scheme != FDLBM_SCHEME_FD5) ||
        bp->flags != 0)
        return false;
    const long long ms = bp->max_side;
    // items: each slot has at most ceil(ms / 120) strips and ceil(ms / 16) segments
    const long long per_slot = ((ms + kStrip - 1) / kStrip) * ((ms + 15) / 16);
    const long long items = std::min<long long>((long long)bp->max_lattices * per_slot, 1LL << 28);
    size_t o = 0;
    offs[0] = o;  // arena
    *arena_elems = bp->arena_bytes / 4 / kAlign * kAlign;
    o += al256((size_t)*arena_elems * 4);
    offs[1] = o;  // descriptors
    o += al256(sizeof(Lat) * bp->max_lattices);
    offs[2] = o;  // items: (slot, index) pairs, the wide list then the narrow one
    o += al256(sizeof(int2) * items);
    offs[3] = o;  // counters of the steps of a run (wide, then narrow), then the two counts
    o += al256(sizeof(int) * (2 * kMaxRun + 2));
    offs[4] = o;  // status
    o += 256;
    offs[5] = o;  // staging: 3 fields of the largest slot
    o += al256((size_t)3 * ms * ms * sizeof(float));
    offs[6] = o;  // reduction partials + result
    o += al256(sizeof(double) * (kRedBlocks + 1) * 4);
    *total = o;
    *max_items = (int)items;
    return true;
}

static void fill_coeffs(const fdlbm_params& p, int R, StreamCoeffs* k) {
    const double sc = (R == 1) ? 0.5 : 0.125;
    const double ae = (1.0 - 1.0 / p.s_e) * sc / 36.0;
    const double axx = (1.0 - 1.0 / p.s_xx) * sc;
    k->e6 = (float)(6.0 * ae);
    k->e2 = (float)(2.0 * ae);
    k->em2 = (float)(-2.0 * ae);
    k->xm23 = (float)(-2.0 / 3.0 * axx);
    k->x13 = (float)(axx / 3.0);
    k->hfx = (float)(0.5 * p.force_x);
    k->hfy = (float)(0.5 * p.force_y);
}

static int rebuild_items(fdlbm_batch_t* b) {
    b->items.clear();
    std::vector<int2> narrow;
    for (size_t s = 0; s < b->slots.size(); ++s) {
        SlotHost& sl = b->slots[s];
        if (!sl.used) continue;
        sl.seg_rows = std::min(b->seg_rows, sl.p.ny);
        sl.nsegs = (sl.p.ny + sl.seg_rows - 1) / sl.seg_rows;
        sl.nstrips = (sl.p.nx + kStrip - 1) / kStrip;
        const bool nar = b->narrow && sl.p.nx - (sl.nstrips - 1) * kStrip <= kNarrowStrip;
        for (int i = 0; i < sl.nstrips * sl.nsegs; ++i) {
            const int2 e = make_int2((int)s, i);
            if (nar && i % sl.nstrips == sl.nstrips - 1)
                narrow.push_back(e);
            else
                b->items.push_back(e);
        }
    }
    // Longest first: a warp's item costs its streamed rows whatever the
    // columns stored, so each list is ordered by rows, longest first (stable:
    // slot order among equals).  Warps take items in list order, so the long
    // ones start early and a run's steps end on short ones: 4096 lattices
    // 171.3 -> 178.5 GLUPS (the tuner then takes 128 rows), 1024 lattices
    // 158.4 -> 165.7 (64 rows).
    const int R = b->bp.scheme == FDLBM_SCHEME_FD3 ? 1 : 2;
    const auto rows_of = [&](const int2& e) {
        const SlotHost& sl = b->slots[e.x];
        const int seg = e.y / sl.nstrips;
        return std::min(sl.p.ny, (seg + 1) * sl.seg_rows) - seg * sl.seg_rows + 2 + 2 * R;
    };
    const auto longer = [&](const int2& x, const int2& y) { return rows_of(x) > rows_of(y); };
    std::stable_sort(b->items.begin(), b->items.end(), longer);
    std::stable_sort(narrow.begin(), narrow.end(), longer);
    const int nwide = (int)b->items.size();
    b->items.insert(b->items.end(), narrow.begin(), narrow.end());
    if ((int)b->items.size() > b->max_items) return berr(b, FDLBM_ERR_NOMEM, "too many work items");
    b->nitems = (int)b->items.size();
    b->nnarrow = (int)narrow.size();
    const int counts[2] = {nwide, b->nnarrow};
    cudaError_t e = cudaSuccess;
    if (b->nitems)
        e = cudaMemcpyAsync(b->ws + b->off_items, b->items.data(), sizeof(int2) * b->nitems,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ws + b->off_counters + sizeof(int) * 2 * kMaxRun, counts,
                            sizeof(counts), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "item upload");
    b->items_dirty = false;
    return FDLBM_OK;
}

// Upload every slot's descriptor with `stop` steps for the next run.
static int upload_lats(fdlbm_batch_t* b, const int* stop) {
    const int R = b->bp.scheme == FDLBM_SCHEME_FD3 ? 1 : 2;
    std::vector<Lat> L(b->slots.size());
    for (size_t s = 0; s < b->slots.size(); ++s) {
        const SlotHost& sl = b->slots[s];
        Lat& d = L[s];
        memset(&d, 0, sizeof(d));
        if (!sl.used) continue;
        d.off[0] = sl.off[0];
        d.off[1] = sl.off[1];
        d.nx = sl.p.nx;
        d.ny = sl.p.ny;
        d.pitch = sl.pitch;
        d.walls = sl.p.boundary == FDLBM_BOUNDARY_WALLS_Y;
        d.nstrips = sl.nstrips;
        d.seg_rows = sl.seg_rows;
        d.nsegs = sl.nsegs;
        d.stop = stop ? stop[s] : 0;
        d.cur = sl.cur;
        d.xi = (float)sl.p.wall_xi;
        fill_coeffs(sl.p, R, &d.k);
    }
    cudaError_t e = cudaMemcpyAsync(b->ws + b->off_lats, L.data(), sizeof(Lat) * L.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "descriptor upload");
    // the host buffer must stay valid until the copy has read it
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "descriptor upload sync");
    return FDLBM_OK;
}

// One step: the wide items' kernel, then (if the run carries narrow items)
// the narrow items' kernel, each with its own work counter.
template <int R, bool FORCE>
static cudaError_t launch_batch_step(fdlbm_batch_t* b, int step, bool narrow) {
    const size_t smem = kWarpsPerBlock * (kSlots * 3 * kLoadCols * sizeof(float) + kSlots * 8);
    Args a;
    a.arena = reinterpret_cast<float*>(b->ws + b->off_arena);
    a.lats = reinterpret_cast<const Lat*>(b->ws + b->off_lats);
    a.items = reinterpret_cast<const int2*>(b->ws + b->off_items);
    a.counts = reinterpret_cast<const int*>(b->ws + b->off_counters) + 2 * kMaxRun;
    a.step = step;
    a.counter = reinterpret_cast<int*>(b->ws + b->off_counters) + step;
    a.status = reinterpret_cast<int*>(b->ws + b->off_status);
    fd_batch_kernel<R, FORCE, false><<<b->grid, kWarpsPerBlock * 32, smem, b->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !narrow) return e;
    a.counter = reinterpret_cast<int*>(b->ws + b->off_counters) + kMaxRun + step;
    fd_batch_kernel<R, FORCE, true><<<b->grid, kWarpsPerBlock * 32, smem, b->stream>>>(a);
    return cudaGetLastError();
}

template <int R, bool FORCE, bool NARROW>
static cudaError_t prepare_one(fdlbm_batch_t* b, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(fd_batch_kernel<R, FORCE, NARROW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fd_batch_kernel<R, FORCE, NARROW>,
                                cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <int R, bool FORCE>
static cudaError_t prepare_kernel(fdlbm_batch_t* b) {
    const size_t smem = kWarpsPerBlock * (kSlots * 3 * kLoadCols * sizeof(float) + kSlots * 8);
    cudaError_t e = prepare_one<R, FORCE, false>(b, smem);
    if (e == cudaSuccess) e = prepare_one<R, FORCE, true>(b, smem);
    if (e != cudaSuccess) return e;
    if (b->grid == 0) {
        int sms = 0, per_sm = 0, per_sm_narrow = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fd_batch_kernel<R, FORCE, false>,
                                                      kWarpsPerBlock * 32, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_narrow,
                                                      fd_batch_kernel<R, FORCE, true>,
                                                      kWarpsPerBlock * 32, smem);
        b->grid = std::max(1, sms * std::min(per_sm, per_sm_narrow));
    }
    return cudaSuccess;
}

// One run of `steps` steps: memset of the counters and the kernels, as a
// captured graph (instantiated once per run length and force variant).
static int run_steps(fdlbm_batch_t* b, int steps, bool force) {
    const int R = b->bp.scheme == FDLBM_SCHEME_FD3 ? 1 : 2;
    cudaError_t e = (R == 1) ? (force ? prepare_kernel<1, true>(b) : prepare_kernel<1, false>(b))
                             : (force ? prepare_kernel<2, true>(b) : prepare_kernel<2, false>(b));
    if (e != cudaSuccess) return bcuda(b, e, "kernel attributes");
    const bool narrow = b->nnarrow > 0;
    cudaGraphExec_t& ex = b->exec[force ? 1 : 0][narrow ? 1 : 0][steps];
    if (!ex) {
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(b, e, "capture stream");
        cudaStream_t user = b->stream;
        b->stream = cap;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b->ws + b->off_counters, 0, sizeof(int) * 2 * kMaxRun, cap);
        for (int s = 0; s < steps && e == cudaSuccess; ++s)
            e = (R == 1) ? (force ? launch_batch_step<1, true>(b, s, narrow)
                                  : launch_batch_step<1, false>(b, s, narrow))
                         : (force ? launch_batch_step<2, true>(b, s, narrow)
                                  : launch_batch_step<2, false>(b, s, narrow));
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        b->stream = user;
        cudaStreamDestroy(cap);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ex = nullptr;
            return bcuda(b, e, "graph capture");
        }
    }
    e = cudaGraphLaunch(ex, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "graph launch");
    b->launches += (int64_t)steps * (narrow ? 2 : 1);
    return FDLBM_OK;
}

extern "C" {

size_t fdlbm_batch_workspace_size(const fdlbm_batch_params* bp) {
    size_t offs[7], total;
    long long ae;
    int mi;
    return batch_layout(bp, offs, &total, &ae, &mi) ? total : 0;
}

int fdlbm_batch_create(const fdlbm_batch_params* bp, void* workspace, size_t bytes, void* stream,
                       fdlbm_batch_t** out) {
    if (!out) return FDLBM_ERR_INVALID;
    *out = nullptr;
    size_t offs[7], total;
    long long ae;
    int mi;
    if (!batch_layout(bp, offs, &total, &ae, &mi)) return FDLBM_ERR_INVALID;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return FDLBM_ERR_INVALID;
    if (bytes < total) return FDLBM_ERR_NOMEM;
    fdlbm_batch_t* b = new (std::nothrow) fdlbm_batch_s();
    if (!b) return FDLBM_ERR_NOMEM;
    b->bp = *bp;
    b->stream = static_cast<cudaStream_t>(stream);
    b->ws = static_cast<char*>(workspace);
    b->off_arena = offs[0];
    b->off_lats = offs[1];
    b->off_items = offs[2];
    b->off_counters = offs[3];
    b->off_status = offs[4];
    b->off_staging = offs[5];
    b->off_partial = offs[6];
    b->arena_elems = ae;
    b->max_items = mi;
    b->slots.resize(bp->max_lattices);
    b->free_list.push_back({0, ae});
    memset(b->exec, 0, sizeof(b->exec));
    b->err[0] = 0;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return FDLBM_ERR_CUDA;
    }
    // zero the arena (ghost and padding columns hold finite values) and the status
    if (cudaMemsetAsync(b->ws + b->off_arena, 0, (size_t)ae * 4, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->ws + b->off_status, 0, sizeof(int), b->stream) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return FDLBM_ERR_CUDA;
    }
    *out = b;
    return FDLBM_OK;
}

void fdlbm_batch_destroy(fdlbm_batch_t* b) {
    if (!b) return;
    for (auto& by_force : b->exec)
        for (auto& row : by_force)
            for (auto& ex : row)
                if (ex) cudaGraphExecDestroy(ex);
    delete b;
}

int fdlbm_batch_add(fdlbm_batch_t* b, const fdlbm_params* p, int32_t* slot) {
    if (!b || !p || !slot) return FDLBM_ERR_INVALID;
    if (p->scheme != b->bp.scheme || p->storage != FDLBM_STORAGE_F32 || p->nx < 16 || p->ny < 16 ||
        p->nx > b->bp.max_side || p->ny > b->bp.max_side || !(p->s_xx > 0 && p->s_xx < 2) ||
        !(p->s_e > 0 && p->s_e < 2) ||
        (p->boundary != FDLBM_BOUNDARY_PERIODIC && p->boundary != FDLBM_BOUNDARY_WALLS_Y) ||
        (p->boundary == FDLBM_BOUNDARY_WALLS_Y && !(p->wall_xi > 0 && p->wall_xi <= 1)))
        return berr(b, FDLBM_ERR_INVALID, "batch_add: unsupported lattice parameters");
    int s = -1;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (!b->slots[i].used) {
            s = (int)i;
            break;
        }
    if (s < 0) return berr(b, FDLBM_ERR_NOMEM, "batch_add: no free slot");
    const int nstrips = (p->nx + kStrip - 1) / kStrip;
    int pitch = std::max(p->nx + 2 * kGhost, nstrips * kStrip + 2 * kGhost);
    pitch = (pitch + kAlign - 1) / kAlign * kAlign;
    const long long elems = 3LL * p->ny * pitch;
    // first fit of two copies
    long long offs[2];
    for (int c = 0; c < 2; ++c) {
        bool found = false;
        for (auto it = b->free_list.begin(); it != b->free_list.end(); ++it) {
            if (it->second >= elems) {
                offs[c] = it->first;
                it->first += elems;
                it->second -= elems;
                if (it->second == 0) b->free_list.erase(it);
                found = true;
                break;
            }
        }
        if (!found) {
            if (c == 1) {  // give the first copy back
                b->free_list.push_back({offs[0], elems});
                std::sort(b->free_list.begin(), b->free_list.end());
            }
            return berr(b, FDLBM_ERR_NOMEM, "batch_add: arena full");
        }
    }
    SlotHost& sl = b->slots[s];
    sl.used = true;
    sl.p = *p;
    sl.off[0] = offs[0];
    sl.off[1] = offs[1];
    sl.elems = elems;
    sl.pitch = pitch;
    sl.cur = 0;
    b->items_dirty = true;
    *slot = s;
    return FDLBM_OK;
}

int fdlbm_batch_remove(fdlbm_batch_t* b, int32_t slot) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return FDLBM_ERR_INVALID;
    SlotHost& sl = b->slots[slot];
    for (int c = 0; c < 2; ++c) b->free_list.push_back({sl.off[c], sl.elems});
    std::sort(b->free_list.begin(), b->free_list.end());
    std::vector<std::pair<long long, long long>> merged;
    for (auto& r : b->free_list) {
        if (!merged.empty() && merged.back().first + merged.back().second == r.first)
            merged.back().second += r.second;
        else
            merged.push_back(r);
    }
    b->free_list.swap(merged);
    sl = SlotHost();
    b->items_dirty = true;
    return FDLBM_OK;
}

int fdlbm_batch_init(fdlbm_batch_t* b, int32_t slot, const float* drho, const float* ux,
                     const float* uy) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used || !drho || !ux ||
        !uy)
        return FDLBM_ERR_INVALID;
    SlotHost& sl = b->slots[slot];
    float* arena = reinterpret_cast<float*>(b->ws + b->off_arena);
    dim3 grid((sl.p.nx + 2 * kGhost + 127) / 128, sl.p.ny);
    for (int c = 0; c < 2; ++c)
        batch_init_kernel<<<grid, 128, 0, b->stream>>>(drho, ux, uy, arena + sl.off[c], sl.p.nx,
                                                      sl.p.ny, sl.pitch);
    b->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "batch init");
    sl.cur = 0;
    return FDLBM_OK;
}

int fdlbm_batch_init_modes(fdlbm_batch_t* b, int32_t slot, int32_t n_modes, const double* modes,
                           double mean_ux, double mean_uy) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
        return FDLBM_ERR_INVALID;
    if (n_modes < 0 || n_modes > kMaxModes || (n_modes > 0 && !modes)) return FDLBM_ERR_INVALID;
    SlotHost& sl = b->slots[slot];
    const size_t n = (size_t)sl.p.nx * sl.p.ny;
    float* st = reinterpret_cast<float*>(b->ws + b->off_staging);
    // launch_modes_eval takes a handle; give it one that carries this stream and size
    fdlbm_s h;
    memset(&h, 0, sizeof(h));
    h.p = sl.p;
    h.stream = b->stream;
    cudaError_t e = launch_modes_eval(&h, n_modes, modes, mean_ux, mean_uy, st, st + n, st + 2 * n);
    b->launches += 1;
    if (e != cudaSuccess) return bcuda(b, e, "batch modes");
    return fdlbm_batch_init(b, slot, st, st + n, st + 2 * n);
}

int fdlbm_batch_step(fdlbm_batch_t* b, int64_t nsteps, const int64_t* slot_steps) {
    if (!b || nsteps < 0) return FDLBM_ERR_INVALID;
    if (nsteps == 0) return FDLBM_OK;
    if (b->items_dirty) {
        int rc = rebuild_items(b);
        if (rc != FDLBM_OK) return rc;
    }
    const int ns = (int)b->slots.size();
    std::vector<int64_t> left(ns, 0);
    bool force = false;
    for (int s = 0; s < ns; ++s) {
        if (!b->slots[s].used) continue;
        left[s] = slot_steps ? std::max<int64_t>(0, std::min<int64_t>(slot_steps[s], nsteps)) : nsteps;
        force = force || b->slots[s].p.force_x != 0.0 || b->slots[s].p.force_y != 0.0;
    }
    std::vector<int> stop(ns, 0);
    int64_t done = 0;
    while (done < nsteps) {
        const int run = (int)std::min<int64_t>(kMaxRun, nsteps - done);
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            stop[s] = (int)std::min<int64_t>(run, std::max<int64_t>(0, left[s] - done));
            any = any || stop[s] > 0;
        }
        if (!any) break;
        int rc = upload_lats(b, stop.data());
        if (rc != FDLBM_OK) return rc;
        rc = run_steps(b, run, force);
        if (rc != FDLBM_OK) return rc;
        for (int s = 0; s < ns; ++s)
            if (b->slots[s].used) b->slots[s].cur ^= (stop[s] & 1);
        done += run;
    }
    return FDLBM_OK;
}

int fdlbm_batch_moments(fdlbm_batch_t* b, int32_t slot, float* drho, float* ux, float* uy) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used || !drho || !ux ||
        !uy)
        return FDLBM_ERR_INVALID;
    SlotHost& sl = b->slots[slot];
    const float* arena = reinterpret_cast<const float*>(b->ws + b->off_arena);
    dim3 grid((sl.p.nx + 127) / 128, sl.p.ny);
    batch_moments_kernel<<<grid, 128, 0, b->stream>>>(arena + sl.off[sl.cur], sl.p.nx, sl.p.ny,
                                                     sl.pitch, drho, ux, uy);
    b->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FDLBM_OK : bcuda(b, e, "batch moments");
}

int fdlbm_batch_reduce(fdlbm_batch_t* b, int32_t slot, int32_t what, const double* args,
                       double* out) {
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used || !out ||
        what < FDLBM_REDUCE_MASS || what > FDLBM_REDUCE_MAXABS || (what == FDLBM_REDUCE_MODE && !args))
        return FDLBM_ERR_INVALID;
    SlotHost& sl = b->slots[slot];
    const float* arena = reinterpret_cast<const float*>(b->ws + b->off_arena);
    double* partial = reinterpret_cast<double*>(b->ws + b->off_partial);
    const int64_t total = (int64_t)sl.p.nx * sl.p.ny;
    const int nb = (int)std::min<int64_t>(kRedBlocks, (total + 255) / 256);
    batch_reduce_kernel<<<nb, 256, 0, b->stream>>>(arena + sl.off[sl.cur], sl.p.nx, sl.p.ny,
                                                   sl.pitch, what, args ? args[0] : 0.0,
                                                   args ? args[1] : 0.0, partial);
    batch_reduce_final<<<1, 32, 0, b->stream>>>(partial, nb, what, partial + kRedBlocks * 4);
    b->launches += 2;
    double host[4];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, partial + kRedBlocks * 4, sizeof(host), cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch reduce");
    const int nout = (what == FDLBM_REDUCE_MOMENTUM || what == FDLBM_REDUCE_MODE ||
                      what == FDLBM_REDUCE_MAXABS) ? 2 : 1;
    const double scale = what == FDLBM_REDUCE_MODE ? 1.0 / (double)total : 1.0;
    for (int k = 0; k < nout; ++k) out[k] = host[k] * scale;
    if (host[3] != 0.0) return berr(b, FDLBM_ERR_DIVERGED, "batch reduce: non-finite values");
    return FDLBM_OK;
}

int fdlbm_batch_sync(fdlbm_batch_t* b) {
    if (!b) return FDLBM_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch sync");
    int flag = 0;
    e = cudaMemcpy(&flag, b->ws + b->off_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "batch status");
    if (flag != 0) {
        cudaMemset(b->ws + b->off_status, 0, sizeof(int));
        return berr(b, flag, "batch kernel reported a device-side timeout");
    }
    return FDLBM_OK;
}

int fdlbm_batch_set_segment_rows(fdlbm_batch_t* b, int32_t rows) {
    if (!b || rows < 8 || rows > 65535) return FDLBM_ERR_INVALID;
    if (rows != b->seg_rows) {
        b->seg_rows = rows;
        b->items_dirty = true;
    }
    return FDLBM_OK;
}

int fdlbm_batch_set_narrow_strips(fdlbm_batch_t* b, int32_t on) {
    if (!b || (on != 0 && on != 1)) return FDLBM_ERR_INVALID;
    if (on != b->narrow) {
        b->narrow = on;
        b->items_dirty = true;  // the two item lists are rebuilt by the next step
    }
    return FDLBM_OK;
}

int fdlbm_batch_set_grid(fdlbm_batch_t* b, int32_t ctas) {
    if (!b || ctas < 0) return FDLBM_ERR_INVALID;
    if (ctas != b->grid) {
        b->grid = ctas;  // 0: back to one wave of resident CTAs
        for (auto& by_force : b->exec)
            for (auto& row : by_force)
                for (auto& ex : row)
                    if (ex) {
                        cudaGraphExecDestroy(ex);
                        ex = nullptr;
                    }
    }
    return FDLBM_OK;
}

const char* fdlbm_batch_last_error(const fdlbm_batch_t* b) { return b ? b->err : "NULL handle"; }

int64_t fdlbm_batch_launch_count(const fdlbm_batch_t* b) { return b ? b->launches : -1; }

int32_t fdlbm_batch_count(const fdlbm_batch_t* b) {
    if (!b) return -1;
    int n = 0;
    for (auto& s : b->slots) n += s.used ? 1 : 0;
    return n;
}

}  // extern "C"
