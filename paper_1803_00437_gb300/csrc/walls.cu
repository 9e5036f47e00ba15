// walls.cu -- curved walls for FD-LBM lattices (Sec. 3-b): the host builds,
// from the caller's geometry (node kinds and, per virtual node, a lattice
// link and the wall's distance xi along it), one closure entry per non-fluid
// node; a fill kernel writes those entries into the state before each step,
// so that the unchanged step kernels read the virtual fluid the closure
// defines.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "fdlbm_internal.cuh"
#include "fdlbm_walls.h"

namespace fdlbm {
namespace {

// One non-fluid node: element offsets (row * pitch + column) of the node, of
// the node whose velocity it extrapolates (-1: rest state) and of the node
// whose density it copies, and the extrapolation factor.
struct WallEntry {
    int32_t dst, src_u, src_rho;
    float factor;
};
static_assert(sizeof(WallEntry) == 16, "16-byte wall entries");

constexpr int kLinkX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kLinkY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int kMaxWalk = 16;

template <typename T>
__global__ void __launch_bounds__(256)
    walls_fill_kernel(const WallEntry* __restrict__ e, int64_t n, T* __restrict__ drho,
                      T* __restrict__ ux, T* __restrict__ uy) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const WallEntry w = e[t];
        float r = 0.f, vx = 0.f, vy = 0.f;
        if (w.src_u >= 0) {
            r = Storage<T>::load(drho + w.src_rho);
            vx = Storage<T>::load(ux + w.src_u) * w.factor;
            vy = Storage<T>::load(uy + w.src_u) * w.factor;
        }
        Storage<T>::store(drho + w.dst, r);
        Storage<T>::store(ux + w.dst, vx);
        Storage<T>::store(uy + w.dst, vy);
    }
}

template <typename T>
cudaError_t fill_typed(fdlbm_s* h, void* state) {
    T* s = static_cast<T*>(state);
    const size_t plane = h->L.plane;
    const int64_t n = h->walls_n;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    walls_fill_kernel<T><<<blocks, 256, 0, h->stream>>>(
        static_cast<const WallEntry*>(h->walls), n, s, s + plane, s + 2 * plane);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walls_fill(fdlbm_s* h, void* state) {
    switch (h->p.storage) {
        case FDLBM_STORAGE_F16: return fill_typed<__half>(h, state);
        case FDLBM_STORAGE_BF16: return fill_typed<__nv_bfloat16>(h, state);
        default: return fill_typed<float>(h, state);
    }
}

}  // namespace fdlbm

using namespace fdlbm;

static int walls_error(fdlbm_t* h, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" {

size_t fdlbm_walls_table_bytes(const fdlbm_params* p) {
    if (!p || p->nx < 1 || p->ny < 1) return 0;
    return (size_t)p->nx * (size_t)p->ny * sizeof(WallEntry);
}

int fdlbm_set_walls(fdlbm_t* h, const uint8_t* kind, int64_t nvirt, const int64_t* vnode,
                    const int8_t* vlink, const double* vxi, void* table, size_t table_bytes) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!kind) {
        h->walls = nullptr;
        h->walls_n = 0;
        return FDLBM_OK;
    }
    const fdlbm_params& p = h->p;
    if (p.scheme != FDLBM_SCHEME_FD3 && p.scheme != FDLBM_SCHEME_FD5 &&
        p.scheme != FDLBM_SCHEME_FD9)
        return walls_error(h, FDLBM_ERR_UNSUPPORTED, "set_walls: FD-LBM (FD3, FD5, FD9) only");
    if (p.boundary != FDLBM_BOUNDARY_PERIODIC)
        return walls_error(h, FDLBM_ERR_UNSUPPORTED, "set_walls: needs a periodic lattice");
    if (h->p.storage == FDLBM_STORAGE_I16)
        return walls_error(h, FDLBM_ERR_UNSUPPORTED, "set_walls: not with I16 storage");
    if (h->L.plane >= ((size_t)1 << 31))
        return walls_error(h, FDLBM_ERR_UNSUPPORTED, "set_walls: plane above 2^31 elements");
    const int nx = p.nx, ny = p.ny;
    const int64_t nodes = (int64_t)nx * ny;
    if (nvirt < 0 || nvirt > nodes || (nvirt > 0 && (!vnode || !vlink || !vxi)))
        return walls_error(h, FDLBM_ERR_INVALID, "set_walls: bad virtual-node arrays");
    if (!table || (reinterpret_cast<uintptr_t>(table) & 15u))
        return walls_error(h, FDLBM_ERR_INVALID, "set_walls: table must be 16-byte aligned");
    auto at = [&](int i, int j) {
        return kind[(int64_t)wrap_index(j, ny) * nx + wrap_index(i, nx)];
    };
    std::vector<int32_t> slot((size_t)nodes, -1);
    int64_t non_fluid = 0;
    for (int64_t n = 0; n < nodes; ++n) {
        if (kind[n] > 2) return walls_error(h, FDLBM_ERR_INVALID, "set_walls: kind %d", kind[n]);
        non_fluid += kind[n] != 0;
    }
    for (int64_t t = 0; t < nvirt; ++t) {
        const int64_t n = vnode[t];
        if (n < 0 || n >= nodes || kind[n] != 1 || slot[(size_t)n] >= 0)
            return walls_error(h, FDLBM_ERR_INVALID,
                               "set_walls: entry %lld is not a virtual node listed once",
                               (long long)t);
        if (vlink[t] < 1 || vlink[t] > 8 || !(vxi[t] > 0.0 && vxi[t] <= 1.0))
            return walls_error(h, FDLBM_ERR_INVALID, "set_walls: entry %lld: bad link or xi",
                               (long long)t);
        slot[(size_t)n] = (int32_t)t;
    }
    for (int64_t n = 0; n < nodes; ++n)
        if (kind[n] == 1 && slot[(size_t)n] < 0)
            return walls_error(h, FDLBM_ERR_INVALID, "set_walls: virtual node %lld not listed",
                               (long long)n);
    // every node the scheme reads for a fluid node must be fluid or virtual
    const int reach = (p.scheme == FDLBM_SCHEME_FD5 ? 2 : 1) + 1;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (kind[(int64_t)j * nx + i] != 0) continue;
            for (int dj = -reach; dj <= reach; ++dj)
                for (int di = -reach; di <= reach; ++di)
                    if (at(i + di, j + dj) == 2)
                        return walls_error(h, FDLBM_ERR_INVALID,
                                           "set_walls: node (%d, %d) is read by the scheme but "
                                           "unused", wrap_index(i + di, nx),
                                           wrap_index(j + dj, ny));
        }
    if (table_bytes < (size_t)non_fluid * sizeof(WallEntry))
        return walls_error(h, FDLBM_ERR_INVALID, "set_walls: table too small");
    const size_t pitch = h->L.pitch;
    auto offset = [&](int i, int j) {
        return (int32_t)((size_t)wrap_index(j, ny) * pitch + (size_t)wrap_index(i, nx));
    };
    std::vector<WallEntry> entries;
    entries.reserve((size_t)non_fluid);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const uint8_t k = kind[(int64_t)j * nx + i];
            if (k == 0) continue;
            WallEntry w{offset(i, j), -1, -1, 0.f};
            if (k == 1) {
                const int t = slot[(size_t)j * nx + i];
                const int a = vlink[t];
                const double xi = vxi[t];
                // first fluid node on the line, d links from the virtual node
                int d = 1;
                while (d <= kMaxWalk && at(i + d * kLinkX[a], j + d * kLinkY[a]) != 0) ++d;
                const int tref = xi >= 0.5 ? d : d + 1;
                if (d > kMaxWalk || at(i + tref * kLinkX[a], j + tref * kLinkY[a]) != 0)
                    return walls_error(h, FDLBM_ERR_INVALID,
                                       "set_walls: the line from (%d, %d) finds no fluid", i, j);
                // u = 0 at t_w = d - xi; linear through the node at t_ref
                const double tw = (double)d - xi;
                w.src_rho = offset(i + d * kLinkX[a], j + d * kLinkY[a]);
                w.src_u = offset(i + tref * kLinkX[a], j + tref * kLinkY[a]);
                w.factor = (float)(-tw / ((double)tref - tw));
            }
            entries.push_back(w);
        }
    cudaError_t e = cudaSuccess;
    if (!entries.empty())
        e = cudaMemcpyAsync(table, entries.data(), entries.size() * sizeof(WallEntry),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return walls_error(h, FDLBM_ERR_CUDA, "set_walls: %s", cudaGetErrorString(e));
    h->walls = table;
    h->walls_n = (int64_t)entries.size();
    return FDLBM_OK;
}

}  // extern "C"
