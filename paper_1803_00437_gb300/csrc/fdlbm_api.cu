// fdlbm_api.cu -- the extern "C" entry points declared in include/fdlbm.h.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "fdlbm_internal.cuh"
#include "tma_ring.cuh"

namespace fdlbm {
namespace {
// Failure-detection self test: one warp waits on a barrier whose arrival
// never comes, with a bound of `tries` polls, and reports the expiry through
// the status word as the step kernels do.  No copy is in flight, so the
// kernel ends cleanly after recording the error.
__global__ void selftest_wait_kernel(int* status, uint32_t tries) {
    __shared__ uint64_t bar;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool landed = __all_sync(0xffffffffu, mbar_wait_tries(&bar, 0, tries));
    __syncwarp();
    if (lane == 0) {
        if (!landed) atomicExch(status, FDLBM_ERR_TIMEOUT);
        mbar_inval(&bar);
    }
}
}  // namespace
}  // namespace fdlbm

namespace fdlbm {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static bool valid_rate(double s) { return s > 0.0 && s < 2.0; }

// Eq. sigsig (quartic condition, Sec. 3-b): (1/s_xx - 1/2)(1/s_q - 1/2) = 1/6.
// For s_xx in (0, 2) the result lies in (0, 2).
static double quartic_s_q(double s_xx) { return 1.0 / (1.0 / (6.0 * (1.0 / s_xx - 0.5)) + 0.5); }

// Parameters as the kernels use them: MRT's s_q resolved from the sentinel.
static fdlbm_params resolved_params(const fdlbm_params& p) {
    fdlbm_params r = p;
    if (r.scheme == FDLBM_SCHEME_MRT && r.s_q == FDLBM_S_Q_QUARTIC) r.s_q = quartic_s_q(r.s_xx);
    return r;
}

// Parameter check shared by workspace_size and create; writes a reason.
static int check_params(const fdlbm_params* p, char* why, size_t n) {
    auto fail = [&](int code, const char* msg) {
        if (why) snprintf(why, n, "%s", msg);
        return code;
    };
    if (!p) return fail(FDLBM_ERR_INVALID, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nx > 65535 || p->ny > 65535)
        return fail(FDLBM_ERR_INVALID, "nx and ny must lie in [1, 65535]");
    if (p->scheme != FDLBM_SCHEME_FD3 && p->scheme != FDLBM_SCHEME_FD5 &&
        p->scheme != FDLBM_SCHEME_FD9 && p->scheme != FDLBM_SCHEME_MRT &&
        p->scheme != FDLBM_SCHEME_LWACM)
        return fail(FDLBM_ERR_INVALID, "scheme must be FD3, FD5, FD9, MRT or LWACM");
    if (p->boundary != FDLBM_BOUNDARY_PERIODIC && p->boundary != FDLBM_BOUNDARY_WALLS_Y)
        return fail(FDLBM_ERR_INVALID, "boundary must be PERIODIC or WALLS_Y");
    if (p->storage != FDLBM_STORAGE_F32 && p->storage != FDLBM_STORAGE_F16 &&
        p->storage != FDLBM_STORAGE_BF16 && p->storage != FDLBM_STORAGE_I16)
        return fail(FDLBM_ERR_INVALID, "storage must be F32, F16, BF16 or I16");
    if (p->storage == FDLBM_STORAGE_I16 &&
        !(p->storage_range > 0.0 && p->storage_range < 1e30))
        return fail(FDLBM_ERR_INVALID, "I16 storage needs a finite storage_range > 0");
    if ((p->flags & ~(FDLBM_FLAG_TILED | FDLBM_FLAG_STREAM)) != 0)
        return fail(FDLBM_ERR_INVALID, "unknown flags");
    if ((p->flags & FDLBM_FLAG_TILED) && (p->flags & FDLBM_FLAG_STREAM))
        return fail(FDLBM_ERR_INVALID, "FDLBM_FLAG_TILED and FDLBM_FLAG_STREAM exclude each other");
    if (!valid_rate(p->s_xx) || !valid_rate(p->s_e))
        return fail(FDLBM_ERR_INVALID, "s_xx and s_e must lie in (0, 2)");
    if (p->scheme == FDLBM_SCHEME_MRT &&
        ((!valid_rate(p->s_q) && p->s_q != FDLBM_S_Q_QUARTIC) || !valid_rate(p->s_eps)))
        return fail(FDLBM_ERR_INVALID,
                    "MRT needs s_eps in (0, 2) and s_q in (0, 2) or FDLBM_S_Q_QUARTIC");
    if (p->scheme == FDLBM_SCHEME_MRT && p->storage != FDLBM_STORAGE_F32)
        return fail(FDLBM_ERR_UNSUPPORTED, "MRT supports FP32 storage only");
    if (p->boundary == FDLBM_BOUNDARY_WALLS_Y) {
        if (!(p->wall_xi > 0.0 && p->wall_xi <= 1.0))
            return fail(FDLBM_ERR_INVALID, "wall_xi must lie in (0, 1]");
        if (p->ny < 2) return fail(FDLBM_ERR_INVALID, "a channel needs ny >= 2");
        if (p->scheme == FDLBM_SCHEME_MRT && p->wall_xi != 0.5)
            return fail(FDLBM_ERR_UNSUPPORTED, "MRT bounce-back puts the wall at xi = 1/2");
    }
    if (!(p->force_x == p->force_x) || !(p->force_y == p->force_y))
        return fail(FDLBM_ERR_INVALID, "force is NaN");
    if (p->scheme == FDLBM_SCHEME_LWACM &&
        (p->boundary != FDLBM_BOUNDARY_PERIODIC || p->force_x != 0.0 || p->force_y != 0.0))
        return fail(FDLBM_ERR_UNSUPPORTED, "LWACM: periodic lattices without force only");
    if (p->scheme == FDLBM_SCHEME_FD9 && (p->flags & FDLBM_FLAG_STREAM))
        return fail(FDLBM_ERR_UNSUPPORTED, "FD9 runs on the tiled kernel only");
    return FDLBM_OK;
}

Quant quant_of(const fdlbm_params& p) {
    Quant q;
    if (p.storage == FDLBM_STORAGE_I16) {
        q.scale = (float)(p.storage_range / 32767.0);
        q.inv = 1.f / q.scale;
    }
    return q;
}

bool compute_layout(const fdlbm_params& p, Layout* L) {
    L->elem = (p.storage == FDLBM_STORAGE_F32) ? 4 : 2;
    L->nplanes = (p.scheme == FDLBM_SCHEME_MRT) ? 9 : 3;
    // rows padded to 256 bytes for aligned, vectorised row access
    L->pitch = align_up((size_t)p.nx, 256 / L->elem);
    L->plane = L->pitch * (size_t)p.ny;
    L->state_bytes = align_up(L->plane * L->elem * L->nplanes, 256);
    size_t off = 0;
    L->off_state[0] = off;
    off += L->state_bytes;
    L->off_state[1] = off;
    off += L->state_bytes;
    L->off_staging = off;
    off += align_up((size_t)3 * p.nx * p.ny * sizeof(float), 256);
    L->off_reduce = off;
    L->reduce_bytes = align_up(sizeof(double) * (kReduceBlocks + 1) * kReduceSlots, 256);
    off += L->reduce_bytes;
    L->off_flag = off;
    off += 256;
    L->total = off;
    return true;
}

}  // namespace fdlbm

using namespace fdlbm;

static int set_error(fdlbm_t* h, int code, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

static int cuda_fail(fdlbm_t* h, cudaError_t e, const char* where) {
    return set_error(h, FDLBM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static void* state_ptr(fdlbm_t* h, int which) { return h->ws + h->L.off_state[which]; }

static float* staging(fdlbm_t* h) { return reinterpret_cast<float*>(h->ws + h->L.off_staging); }

// Device of the handle current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static const char* device_error_text(int flag) {
    switch (flag) {
        case FDLBM_ERR_TIMEOUT: return "FDLBM_ERR_TIMEOUT (a bounded wait expired)";
        case FDLBM_ERR_RANGE:
            return "FDLBM_ERR_RANGE (a value outside storage_range was stored saturated)";
        default: return "an error";
    }
}

// Read (and clear) the device status word after the stream has drained.
static int device_status(fdlbm_t* h) {
    int flag = 0;
    int* dflag = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    cudaError_t e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (flag != 0) {
        cudaMemsetAsync(dflag, 0, sizeof(int), h->stream);
        return set_error(h, flag, "device reported %s", device_error_text(flag));
    }
    return FDLBM_OK;
}

extern "C" {

size_t fdlbm_workspace_size(const fdlbm_params* p) {
    if (check_params(p, nullptr, 0) != FDLBM_OK) return 0;
    Layout L;
    compute_layout(*p, &L);
    return L.total;
}

int fdlbm_create(const fdlbm_params* p, void* workspace, size_t bytes, void* stream,
                 fdlbm_t** out) {
    if (!out) return FDLBM_ERR_INVALID;
    *out = nullptr;
    char why[256] = {0};
    int rc = check_params(p, why, sizeof(why));
    if (rc != FDLBM_OK) return rc;
    Layout L;
    compute_layout(*p, &L);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return FDLBM_ERR_INVALID;
    if (bytes < L.total) return FDLBM_ERR_NOMEM;
    fdlbm_t* h = new (std::nothrow) fdlbm_s();
    if (!h) return FDLBM_ERR_NOMEM;
    h->p = resolved_params(*p);
    h->L = L;
    h->stream = static_cast<cudaStream_t>(stream);
    h->ws = static_cast<char*>(workspace);
    h->cur = 0;
    h->launches = 0;
    h->stream_plan_warps = 0;
    h->stream_plan_user = 0;
    h->fd_path = (p->flags & FDLBM_FLAG_TILED) ? 1 : (p->flags & FDLBM_FLAG_STREAM) ? 2 : 0;
    h->err[0] = 0;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return FDLBM_ERR_CUDA;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess ||
        (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        delete h;
        return FDLBM_ERR_INVALID;
    }
    if (cudaMemsetAsync(h->ws + h->L.off_flag, 0, sizeof(int), h->stream) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return FDLBM_ERR_CUDA;
    }
    h->host_io = nullptr;
    void* hio = nullptr;
    if (cudaHostAlloc(&hio, sizeof(fdlbm_s::HostIO), cudaHostAllocDefault) == cudaSuccess)
        h->host_io = static_cast<fdlbm_s::HostIO*>(hio);
    else
        cudaGetLastError();  // reductions then go through pageable memory
    *out = h;
    return FDLBM_OK;
}

void fdlbm_destroy(fdlbm_t* h) {
    if (h && h->host_io) cudaFreeHost(h->host_io);
    delete h;
}

int fdlbm_set_stream(fdlbm_t* h, void* stream) {
    if (!h) return FDLBM_ERR_INVALID;
    h->stream = static_cast<cudaStream_t>(stream);
    return FDLBM_OK;
}

static int init_from_device(fdlbm_t* h, const float* drho, const float* ux, const float* uy) {
    cudaError_t e;
    void* dst = state_ptr(h, 0);
    if (h->p.scheme == FDLBM_SCHEME_MRT)
        e = launch_mrt_init(h, drho, ux, uy, dst);
    else
        e = launch_fd_init(h, drho, ux, uy, dst);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    h->cur = 0;
    return FDLBM_OK;
}

int fdlbm_init(fdlbm_t* h, const float* drho, const float* ux, const float* uy) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!drho || !ux || !uy) return set_error(h, FDLBM_ERR_INVALID, "init: NULL field pointer");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    return init_from_device(h, drho, ux, uy);
}

int fdlbm_init_host(fdlbm_t* h, const float* drho, const float* ux, const float* uy) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!drho || !ux || !uy) return set_error(h, FDLBM_ERR_INVALID, "init: NULL field pointer");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const float* src[3] = {drho, ux, uy};
    // Page-locked host arrays are device-addressable: the init kernel reads
    // them in place over the host link (one pass, no staging copy).
    const float* mapped[3] = {nullptr, nullptr, nullptr};
    bool in_place = true;
    for (int k = 0; k < 3 && in_place; ++k) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, src[k]) != cudaSuccess) {
            cudaGetLastError();  // not a CUDA-known pointer: clear and stage
            in_place = false;
        } else if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
            mapped[k] = static_cast<const float*>(at.devicePointer);
        } else {
            in_place = false;
        }
    }
    if (in_place) {
        int rc = init_from_device(h, mapped[0], mapped[1], mapped[2]);
        if (rc != FDLBM_OK) return rc;
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "init_host sync");
        return FDLBM_OK;
    }
    float* st = staging(h);
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaMemcpyAsync(st + k * n, src[k], n * sizeof(float),
                                        cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "init_host copy");
    }
    int rc = init_from_device(h, st, st + n, st + 2 * n);
    if (rc != FDLBM_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init_host sync");
    return FDLBM_OK;
}

int fdlbm_init_modes(fdlbm_t* h, int32_t n_modes, const double* modes, double mean_ux,
                     double mean_uy) {
    if (!h) return FDLBM_ERR_INVALID;
    if (n_modes < 0 || n_modes > kMaxModes || (n_modes > 0 && !modes))
        return set_error(h, FDLBM_ERR_INVALID, "init_modes: need 0..%d modes", kMaxModes);
    for (int k = 0; k < n_modes; ++k)
        if (modes[4 * k] == 0.0 && modes[4 * k + 1] == 0.0)
            return set_error(h, FDLBM_ERR_INVALID, "init_modes: mode %d has k = 0", k);
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    float* st = staging(h);
    cudaError_t e = launch_modes_eval(h, n_modes, modes, mean_ux, mean_uy, st, st + n, st + 2 * n);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(h, e, "modes kernel");
    return init_from_device(h, st, st + n, st + 2 * n);
}

int fdlbm_step(fdlbm_t* h, int64_t nsteps) {
    if (!h) return FDLBM_ERR_INVALID;
    if (nsteps < 0) return set_error(h, FDLBM_ERR_INVALID, "step: nsteps < 0");
    if (nsteps == 0) return FDLBM_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    for (int64_t n = 0; n < nsteps; ++n) {
        void* src = state_ptr(h, h->cur);
        void* dst = state_ptr(h, 1 - h->cur);
        if (h->walls) {  // curved walls: the virtual fluid the step reads (Sec. 3-b)
            cudaError_t e = launch_walls_fill(h, src);
            h->launches += 1;
            if (e != cudaSuccess) return cuda_fail(h, e, "walls kernel");
        }
        cudaError_t e = (h->p.scheme == FDLBM_SCHEME_MRT) ? launch_mrt_step(h, src, dst)
                                                           : launch_fd_step(h, src, dst);
        h->launches += 1;
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur = 1 - h->cur;
    }
    if (h->walls) {
        cudaError_t e = launch_walls_fill(h, state_ptr(h, h->cur));
        h->launches += 1;
        if (e != cudaSuccess) return cuda_fail(h, e, "walls kernel");
    }
    return FDLBM_OK;
}

int fdlbm_moments(fdlbm_t* h, float* drho, float* ux, float* uy) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!drho || !ux || !uy) return set_error(h, FDLBM_ERR_INVALID, "moments: NULL pointer");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    cudaError_t e = launch_moments(h, state_ptr(h, h->cur), drho, ux, uy);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return FDLBM_OK;
}

int fdlbm_moments_host(fdlbm_t* h, float* drho, float* ux, float* uy) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!drho || !ux || !uy) return set_error(h, FDLBM_ERR_INVALID, "moments: NULL pointer");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    float* st = staging(h);
    cudaError_t e = launch_moments(h, state_ptr(h, h->cur), st, st + n, st + 2 * n);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    float* dst[3] = {drho, ux, uy};
    for (int k = 0; k < 3; ++k) {
        e = cudaMemcpyAsync(dst[k], st + k * n, n * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments_host copy");
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments_host sync");
    return FDLBM_OK;
}

int fdlbm_reduce(fdlbm_t* h, int32_t what, const double* args, double* out) {
    if (!h) return FDLBM_ERR_INVALID;
    if (!out || what < FDLBM_REDUCE_MASS || what > FDLBM_REDUCE_MAXABS)
        return set_error(h, FDLBM_ERR_INVALID, "reduce: bad 'what' or NULL out");
    if (what == FDLBM_REDUCE_MODE && !args)
        return set_error(h, FDLBM_ERR_INVALID, "reduce: MODE needs args = (m, n)");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    double* partial = reinterpret_cast<double*>(h->ws + h->L.off_reduce);
    double* result = partial + kReduceBlocks * kReduceSlots;
    const double a0 = args ? args[0] : 0.0, a1 = args ? args[1] : 0.0;
    cudaError_t e = launch_reduce(h, state_ptr(h, h->cur), what, a0, a1, partial, result);
    h->launches += 2;
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce kernel");
    double stack_host[kReduceSlots];
    double* host = h->host_io ? h->host_io->result : stack_host;
    e = cudaMemcpyAsync(host, result, sizeof(double) * kReduceSlots, cudaMemcpyDeviceToHost,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce copy");
    int* dflag = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    if (h->host_io) {  // the status word rides along: one synchronisation
        e = cudaMemcpyAsync(&h->host_io->flag, dflag, sizeof(int), cudaMemcpyDeviceToHost,
                            h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce sync");
    const int nout = (what == FDLBM_REDUCE_MOMENTUM || what == FDLBM_REDUCE_MODE ||
                      what == FDLBM_REDUCE_MAXABS) ? 2 : 1;
    const double scale =
        (what == FDLBM_REDUCE_MODE) ? 1.0 / ((double)h->p.nx * (double)h->p.ny) : 1.0;
    for (int k = 0; k < nout; ++k) out[k] = host[k] * scale;
    if (host[3] != 0.0)
        return set_error(h, FDLBM_ERR_DIVERGED, "reduce: %.0f nodes hold non-finite values",
                         host[3]);
    if (!h->host_io) return device_status(h);
    const int flag = h->host_io->flag;
    if (flag != 0) {
        cudaMemsetAsync(dflag, 0, sizeof(int), h->stream);
        return set_error(h, flag, "device reported %s", device_error_text(flag));
    }
    return FDLBM_OK;
}

int fdlbm_sync(fdlbm_t* h) {
    if (!h) return FDLBM_ERR_INVALID;
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    return device_status(h);
}

int fdlbm_selftest_wait_timeout(fdlbm_t* h, int32_t tries) {
    if (!h) return FDLBM_ERR_INVALID;
    if (tries < 0) return set_error(h, FDLBM_ERR_INVALID, "selftest: tries < 0");
    DeviceGuard g(h->device);
    if (!g.ok) return set_error(h, FDLBM_ERR_CUDA, "cannot select the handle's device");
    int* dflag = reinterpret_cast<int*>(h->ws + h->L.off_flag);
    fdlbm::selftest_wait_kernel<<<1, 32, 0, h->stream>>>(dflag, (uint32_t)tries);
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "selftest kernel");
    return FDLBM_OK;
}

const char* fdlbm_last_error(const fdlbm_t* h) { return h ? h->err : "NULL handle"; }

const char* fdlbm_status_string(int s) {
    switch (s) {
        case FDLBM_OK: return "FDLBM_OK";
        case FDLBM_ERR_INVALID: return "FDLBM_ERR_INVALID";
        case FDLBM_ERR_UNSUPPORTED: return "FDLBM_ERR_UNSUPPORTED";
        case FDLBM_ERR_NOMEM: return "FDLBM_ERR_NOMEM";
        case FDLBM_ERR_CUDA: return "FDLBM_ERR_CUDA";
        case FDLBM_ERR_DIVERGED: return "FDLBM_ERR_DIVERGED";
        case FDLBM_ERR_TIMEOUT: return "FDLBM_ERR_TIMEOUT";
        case FDLBM_ERR_RANGE: return "FDLBM_ERR_RANGE";
        default: return "FDLBM_UNKNOWN_STATUS";
    }
}

int64_t fdlbm_launch_count(const fdlbm_t* h) { return h ? h->launches : -1; }

}  // extern "C"

namespace fdlbm {
bool uses_stream_step(const fdlbm_s* h) {
    // the streaming kernel pays off once the lattice fills the GPU's warps
    constexpr int64_t kStreamMinNodes = 1 << 20;
    const bool big = (int64_t)h->p.nx * h->p.ny >= kStreamMinNodes;
    return h->p.scheme != FDLBM_SCHEME_MRT && h->p.scheme != FDLBM_SCHEME_FD9 &&
           h->fd_path != 1 && fd_stream_supported(h->p) && (big || h->fd_path == 2);
}

cudaError_t launch_fd_step(fdlbm_s* h, const void* src, void* dst) {
    if (uses_stream_step(h)) return launch_fd_step_stream(h, src, dst);
    return launch_fd_step_tiled(h, src, dst);
}
}  // namespace fdlbm
