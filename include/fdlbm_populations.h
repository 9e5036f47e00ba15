/* fdlbm_populations.h -- the state of an MRT lattice (Sec. 1, 1-a).
 *
 * An FD-LBM or LW-ACM lattice keeps only (rho - 1, ux, uy) per node, which
 * fdlbm_moments reads and fdlbm_init writes, so those two calls checkpoint
 * and resume it exactly.  The MRT step keeps its nine populations, whose
 * non-equilibrium parts the moments do not carry; these two calls read and
 * write them, so that an MRT lattice can be checkpointed and resumed exactly
 * too.
 */
#ifndef FDLBM_POPULATIONS_H
#define FDLBM_POPULATIONS_H

#include "fdlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Copy the stored state of an MRT lattice into f (device memory, 9*nx*ny
 * floats, [9][ny][nx] row-major): h_a = f_a - w_a, a = 0..8 in the link
 * order of Sec. 1, the post-collision populations of the last step minus
 * their rest weights (4/9, 1/9 x 4, 1/36 x 4).  Asynchronous on the
 * handle's stream.  FDLBM_ERR_UNSUPPORTED for the other schemes (their
 * state is the moments), FDLBM_ERR_INVALID for a NULL pointer. */
int fdlbm_get_populations(fdlbm_t* h, float* f);

/* Replace the state of an MRT lattice by f (device memory, the layout and
 * meaning of fdlbm_get_populations).  Asynchronous on the handle's stream;
 * f must stay valid until the copy has run. */
int fdlbm_set_populations(fdlbm_t* h, const float* f);

#ifdef __cplusplus
}
#endif

#endif /* FDLBM_POPULATIONS_H */
