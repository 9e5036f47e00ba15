// reduce_static.cu -- fdlbm_reduce_fields_static: the FP64 reductions of
// fdlbm_reduce applied to caller-held fields, with no workspace.
//
// Why it exists: some callers cannot allocate device memory at all -- code
// running inside a memory pool they do not own, a driver or plug-in that is
// handed only the buffers it must fill, or a CUDA-graph region where any
// allocation is forbidden.  They cannot create a workspace for fdlbm_create,
// yet may want to check a field (mass, momentum, energy, a mode amplitude,
// the largest velocity) that they already hold on the device.
//
// How: the per-block partial sums that fdlbm_reduce keeps in the handle's
// workspace live here in one file-scope __device__ array of fixed size
// (kStaticBlocks partials of kStaticSlots doubles, 32 KiB).  Host code may
// not use that array's name as a device address (it names a host-side
// stand-in), so its address is obtained once per device with
// cudaGetSymbolAddress, the first time the entry point runs on that device.
//
// Sharing: every call on a device uses the same array, and the array keeps
// the last call's partials.  Each call writes every partial it later reads
// (nothing is assumed to start at zero), so consecutive calls on one stream
// are correct; calls that overlap on the GPU (different streams, or host
// threads without ordering) race on the array and give wrong results.
#include <mutex>

#include "fdlbm_internal.cuh"

namespace fdlbm {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticBlocks = 1024;
constexpr int kStaticSlots = 4;  // two results, spare, count of non-finite nodes
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[kStaticBlocks * kStaticSlots];

__device__ __forceinline__ double static_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double static_warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kStaticThreads)
    static_reduce_partial(const float* __restrict__ drho, const float* __restrict__ ux,
                          const float* __restrict__ uy, int nx, int ny, int what, double m,
                          double n, double* __restrict__ partial) {
    double acc[kStaticSlots] = {0.0, 0.0, 0.0, 0.0};
    const int64_t total = (int64_t)nx * ny;
    double kx = 0.0, ky = 0.0, tx = 0.0, ty = 0.0;
    if (what == FDLBM_REDUCE_MODE) {
        kx = 2.0 * M_PI * m / nx;
        ky = 2.0 * M_PI * n / ny;
        const double kk = sqrt(kx * kx + ky * ky);
        tx = kk > 0.0 ? -ky / kk : 0.0;
        ty = kk > 0.0 ? kx / kk : 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * kStaticThreads + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * kStaticThreads) {
        const float dr = drho[i], vx = ux[i], vy = uy[i];
        if (!(isfinite(dr) && isfinite(vx) && isfinite(vy))) {
            acc[3] += 1.0;
            continue;
        }
        const double rho = 1.0 + (double)dr;
        switch (what) {
            case FDLBM_REDUCE_MASS: acc[0] += (double)dr; break;
            case FDLBM_REDUCE_MOMENTUM:
                acc[0] += rho * vx;
                acc[1] += rho * vy;
                break;
            case FDLBM_REDUCE_ENERGY:
                acc[0] += 0.5 * rho * ((double)vx * vx + (double)vy * vy);
                break;
            case FDLBM_REDUCE_MODE: {
                const int x = (int)(i % nx), y = (int)(i / nx);
                const double ut = tx * vx + ty * vy;
                double sn, cs;
                sincos(kx * x + ky * y, &sn, &cs);
                acc[0] += ut * cs;
                acc[1] -= ut * sn;
                break;
            }
            default:
                acc[0] = fmax(acc[0], sqrt((double)vx * vx + (double)vy * vy));
                acc[1] = fmax(acc[1], fabs((double)dr));
        }
    }
    __shared__ double sh[kStaticThreads / 32][kStaticSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kStaticSlots; ++k) {
        const bool is_max = what == FDLBM_REDUCE_MAXABS && k < 2;
        const double v = is_max ? static_warp_max(acc[k]) : static_warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kStaticSlots) {
        const int k = threadIdx.x;
        const bool is_max = what == FDLBM_REDUCE_MAXABS && k < 2;
        double v = sh[0][k];
        for (int w = 1; w < kStaticThreads / 32; ++w) v = is_max ? fmax(v, sh[w][k]) : v + sh[w][k];
        partial[blockIdx.x * kStaticSlots + k] = v;
    }
}

__global__ void static_reduce_final(const double* __restrict__ partial, int nblocks, int what,
                                    double scale, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= kStaticSlots) return;
    const bool is_max = what == FDLBM_REDUCE_MAXABS && k < 2;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double p = partial[b * kStaticSlots + k];
        v = is_max ? fmax(v, p) : v + p;
    }
    out[k] = (k < 2) ? v * scale : v;
}

std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace fdlbm

extern "C" int fdlbm_reduce_fields_static(const float* drho, const float* ux, const float* uy,
                                          int32_t nx, int32_t ny, int32_t what,
                                          const double* args, double* out, void* stream) {
    using namespace fdlbm;
    if (!drho || !ux || !uy || !out) return FDLBM_ERR_INVALID;
    if (nx < 1 || ny < 1 || (int64_t)nx * ny > FDLBM_STATIC_REDUCE_MAX_NODES)
        return FDLBM_ERR_INVALID;
    if (what < FDLBM_REDUCE_MASS || what > FDLBM_REDUCE_MAXABS) return FDLBM_ERR_INVALID;
    if (what == FDLBM_REDUCE_MODE && !args) return FDLBM_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return FDLBM_ERR_CUDA;
    // The kernels run on the current device and read the fields and write
    // out there: each pointer must be device memory of that device (or
    // managed memory), never host memory or another GPU's memory.
    const void* ptrs[4] = {drho, ux, uy, out};
    for (const void* q : ptrs) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, q) != cudaSuccess) {
            cudaGetLastError();
            return FDLBM_ERR_INVALID;
        }
        const bool on_dev = attr.type == cudaMemoryTypeDevice && attr.device == dev;
        if (!on_dev && attr.type != cudaMemoryTypeManaged) return FDLBM_ERR_INVALID;
    }
    double* partial = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return FDLBM_ERR_CUDA;
            }
            g_static_ptr[dev] = static_cast<double*>(p);
        }
        partial = g_static_ptr[dev];
    }
    const int64_t total = (int64_t)nx * ny;
    const int blocks =
        (int)std::min<int64_t>(kStaticBlocks, (total + kStaticThreads - 1) / kStaticThreads);
    const double m = args ? args[0] : 0.0, n = args ? args[1] : 0.0;
    const double scale = (what == FDLBM_REDUCE_MODE) ? 1.0 / (double)total : 1.0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static_reduce_partial<<<blocks, kStaticThreads, 0, s>>>(drho, ux, uy, nx, ny, what, m, n,
                                                           partial);
    if (cudaGetLastError() != cudaSuccess) return FDLBM_ERR_CUDA;
    static_reduce_final<<<1, 32, 0, s>>>(partial, blocks, what, scale, out);
    if (cudaGetLastError() != cudaSuccess) return FDLBM_ERR_CUDA;
    return FDLBM_OK;
}
