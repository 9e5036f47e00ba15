// populations.cu -- read and write the nine population planes of an MRT
// lattice (its whole state), for exact checkpoints.  One pitched copy each
// way: the planes are contiguous, so the state is 9 * ny rows of `pitch`
// floats of which the first nx are used.
#include <stdio.h>

#include "fdlbm_internal.cuh"
#include "fdlbm_populations.h"

using namespace fdlbm;

static int populations_copy(fdlbm_t* h, void* dst, size_t dpitch, const void* src,
                            size_t spitch, const char* what) {
    const size_t width = (size_t)h->p.nx * sizeof(float);
    const size_t rows = (size_t)9 * h->p.ny;
    cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows,
                                      cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
        snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
        return FDLBM_ERR_CUDA;
    }
    return FDLBM_OK;
}

static int populations_check(fdlbm_t* h, const void* f, const char* what) {
    if (h->p.scheme != FDLBM_SCHEME_MRT) {
        snprintf(h->err, sizeof(h->err), "%s: MRT lattices only (the state of the others is "
                                         "the moments)", what);
        return FDLBM_ERR_UNSUPPORTED;
    }
    if (!f) {
        snprintf(h->err, sizeof(h->err), "%s: NULL pointer", what);
        return FDLBM_ERR_INVALID;
    }
    return FDLBM_OK;
}

extern "C" {

int fdlbm_get_populations(fdlbm_t* h, float* f) {
    if (!h) return FDLBM_ERR_INVALID;
    const int rc = populations_check(h, f, "get_populations");
    if (rc != FDLBM_OK) return rc;
    const char* state = h->ws + h->L.off_state[h->cur];
    return populations_copy(h, f, (size_t)h->p.nx * sizeof(float), state,
                            h->L.pitch * sizeof(float), "get_populations");
}

int fdlbm_set_populations(fdlbm_t* h, const float* f) {
    if (!h) return FDLBM_ERR_INVALID;
    const int rc = populations_check(h, f, "set_populations");
    if (rc != FDLBM_OK) return rc;
    char* state = h->ws + h->L.off_state[h->cur];
    return populations_copy(h, state, h->L.pitch * sizeof(float), f,
                            (size_t)h->p.nx * sizeof(float), "set_populations");
}

}  // extern "C"
