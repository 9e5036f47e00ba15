// fdlbm_internal.cuh -- shared definitions of the CUDA library (not public).
//
// D2Q9 velocity set, in the order of the moment matrix of Sec. 1:
//   c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
// The state is held as deviations from the fluid at rest (rho = 1, u = 0):
// FD-LBM keeps (rho - 1, ux, uy); MRT keeps h_a = f_a - w_a.  With FP32
// storage this keeps the resolution of small perturbations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdlbm.h"  // include/ of the repository (-I)

namespace fdlbm {

// ---- storage types --------------------------------------------------------
//
// Every type is read into FP32 and written from FP32 (round to nearest).
// FDLBM_STORAGE_I16 is fixed point: a stored q stands for q * scale with
// scale = storage_range / 32767, written as q = RN(v * (1 / scale)) clamped
// to +-32767; a value outside the range (or not finite) saturates and the
// store reports it.  The floating-point types ignore the scale and never
// saturate.

struct Quant {
    float scale = 1.f;  // value of one fixed-point step
    float inv = 1.f;    // 1 / scale, rounded to FP32
};

template <typename T>
struct Storage;

template <>
struct Storage<float> {
    static __device__ __forceinline__ float load(const float* p) { return *p; }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
    static __device__ __forceinline__ float load(const float* p, Quant) { return *p; }
    static __device__ __forceinline__ bool store(float* p, float v, Quant) {
        *p = v;
        return false;
    }
};

template <>
struct Storage<__half> {
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float load(const __half* p, Quant) { return load(p); }
    static __device__ __forceinline__ bool store(__half* p, float v, Quant) {
        store(p, v);
        return false;
    }
};

template <>
struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, Quant) { return load(p); }
    static __device__ __forceinline__ bool store(__nv_bfloat16* p, float v, Quant) {
        store(p, v);
        return false;
    }
};

// Fixed-point step of a value: t = v / scale, rounded to the nearest integer
// (ties to even) by adding 1.5 * 2^23, which leaves the integer in the low
// mantissa bits; |t| is clamped to 32767 first.  Returns q; *sat is set when
// |t| > 32767 or t is not finite.
__device__ __forceinline__ int quantize16(float v, Quant q, bool* sat) {
    const float t = v * q.inv;
    *sat = !(fabsf(t) <= 32767.f);
    const float c = fminf(fmaxf(t, -32767.f), 32767.f);  // a NaN becomes -32767
    return __float_as_int(c + 12582912.f) - 0x4B400000;
}

template <>
struct Storage<int16_t> {
    static __device__ __forceinline__ float load(const int16_t* p, Quant q) {
        return (float)*p * q.scale;
    }
    static __device__ __forceinline__ bool store(int16_t* p, float v, Quant q) {
        bool sat;
        *p = (int16_t)quantize16(v, q, &sat);
        return sat;
    }
};

// ---- lattice ----------------------------------------------------------------

__host__ __device__ __forceinline__ int wrap_index(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Arguments of the FD-LBM step.  Planes are [ny][pitch] elements.
template <typename T>
struct FdState {
    T* drho;
    T* ux;
    T* uy;
};

struct FdCoeffs {
    float a_e;    // 1 - 1/s_e  (factor of theta_E)
    float a_xx;   // 1 - 1/s_xx (factor of theta_XX, theta_XY)
    float fx, fy; // body force
    float xi;     // wall offset
    Quant q;      // fixed-point scale (FDLBM_STORAGE_I16)
};

struct MrtCoeffs {
    float s_e, s_xx, s_q, s_eps;
    float fx, fy;
};

// ---- handle -------------------------------------------------------------------

struct Layout {
    size_t pitch;        // elements per stored row (multiple of 64)
    size_t plane;        // pitch * ny elements
    size_t elem;         // bytes per stored element
    int nplanes;         // 3 (FD-LBM) or 9 (MRT)
    size_t state_bytes;  // one copy of the state
    size_t off_state[2];
    size_t off_staging;  // 3 * nx * ny floats
    size_t off_reduce;   // reduction scratch (doubles)
    size_t reduce_bytes;
    size_t off_flag;     // device status word
    size_t total;
};

constexpr int kReduceBlocks = 1216;  // 8 x 152 SMs (full occupancy at 256 threads)
constexpr int kReduceSlots = 4;     // doubles per block partial

bool compute_layout(const fdlbm_params& p, Layout* L);

// Fixed-point scale of a lattice's storage (scale 1 unless FDLBM_STORAGE_I16).
Quant quant_of(const fdlbm_params& p);

// Record a saturated fixed-point store in the device status word (no other
// error is overwritten).
__device__ __forceinline__ void report_saturation(int* status) {
    atomicCAS(status, 0, FDLBM_ERR_RANGE);
}

}  // namespace fdlbm

struct fdlbm_s {
    fdlbm_params p;
    fdlbm::Layout L;
    cudaStream_t stream;
    int device;
    char* ws;
    int cur;  // index of the current state copy
    int64_t launches;
    int stream_plan_warps;  // resident CTAs of the streaming FD kernel (0: not queried)
    int stream_plan[6];     // its launch plan (see make_plan)
    int stream_plan_user;   // 1: the plan was set by fdlbm_set_stream_plan
    int fd_path;            // 0: automatic, 1: tiled FD kernel, 2: streaming where it qualifies
    const void* walls;      // curved walls: device table of closure entries (NULL: none)
    int64_t walls_n;        // its number of entries
    // page-locked host landing area for reduction results and the device
    // status word (one synchronisation per reduction); NULL if unavailable
    struct HostIO {
        double result[4];
        int flag;
        int pad;
    }* host_io;
    char err[512];
};

namespace fdlbm {

MrtCoeffs mrt_coeffs(const fdlbm_params& p);

// launchers (each returns cudaGetLastError() of its launch)
cudaError_t launch_fd_step(fdlbm_s* h, const void* src, void* dst);
cudaError_t launch_fd_step_tiled(fdlbm_s* h, const void* src, void* dst);
cudaError_t launch_fd_step_stream(fdlbm_s* h, const void* src, void* dst);
bool uses_stream_step(const fdlbm_s* h);
bool fd_stream_supported(const fdlbm_params& p);
cudaError_t launch_mrt_step(fdlbm_s* h, const void* src, void* dst);
cudaError_t launch_fd_init(fdlbm_s* h, const float* drho, const float* ux, const float* uy,
                           void* dst);
cudaError_t launch_mrt_init(fdlbm_s* h, const float* drho, const float* ux, const float* uy,
                            void* dst);
constexpr int kMaxModes = 64;
cudaError_t launch_modes_eval(fdlbm_s* h, int n_modes, const double* modes_host, double mean_ux,
                              double mean_uy, float* drho, float* ux, float* uy);
cudaError_t launch_moments(fdlbm_s* h, const void* state, float* drho, float* ux, float* uy);
cudaError_t launch_walls_fill(fdlbm_s* h, void* state);
cudaError_t launch_reduce(fdlbm_s* h, const void* state, int what, double a0, double a1,
                          double* partial, double* result);

}  // namespace fdlbm
