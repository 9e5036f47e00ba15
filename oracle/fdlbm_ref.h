/*
 * fdlbm_ref.h -- FP64 CPU oracle for the FD-LBM and MRT D2Q9 schemes of
 * Dubois, Lallemand, Obrecht, Tekitek, "Lattice Boltzmann model approximated
 * with finite difference expressions" (Computers & Fluids 155, 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * calls it.  It shares no code, header, table or constant with the CUDA
 * library: every constant here is written out again from the paper.
 *
 * Conventions
 *   - Fields are FP64, row-major [ny][nx]; node (i, j) sits at j*nx + i,
 *     i along x, j along y.
 *   - The FD-LBM state is (rho, ux, uy) with u the velocity that includes
 *     half of the body force: u = (J + F/2) / rho (Strang splitting, Sec. 1).
 *   - The MRT state is the 9 pre-collision populations f[a][ny][nx].
 *   - Velocity set (Sec. 1, moment table, with the signs of the Jx and Jy
 *     rows read from the qx/qy/XY rows):
 *       c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
 *
 * Every function returns 0 on success and a negative code on invalid input;
 * nothing aborts.  Buffers are owned by the caller.
 */
#ifndef FDLBM_REF_H
#define FDLBM_REF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* scheme: finite-difference stencil width of FD-LBM (Sec. 2), or MRT (Sec. 1-a) */
#define FDLBM_REF_FD3 3     /* three-point centred difference  */
#define FDLBM_REF_FD5 5     /* five-point centred difference   */
#define FDLBM_REF_FD9 9     /* nine-point D2Q9-footprint difference */
#define FDLBM_REF_MRT 100   /* multiple-relaxation-time D2Q9 LBM */
#define FDLBM_REF_LWACM 200 /* link-wise artificial compressibility method (Sec. 1-b) */

/* boundary */
#define FDLBM_REF_PERIODIC 0
#define FDLBM_REF_WALLS_Y 1 /* periodic in x, solid walls below row 0 and above row ny-1 */

#define FDLBM_REF_OK 0
#define FDLBM_REF_EINVAL (-1)
#define FDLBM_REF_ENOMEM (-3)

typedef struct {
    int32_t nx, ny;
    int32_t scheme;    /* FDLBM_REF_FD3 / FD5 / FD9 / MRT / LWACM */
    int32_t boundary;  /* FDLBM_REF_PERIODIC / WALLS_Y */
    double s_xx;       /* rate of XX and XY (shear viscosity) */
    double s_e;        /* rate of E (bulk viscosity) */
    double s_q;        /* rate of qx, qy (MRT only) */
    double s_eps;      /* rate of epsilon (MRT only) */
    double wall_xi;    /* wall offset: walls at y = -xi and y = ny-1+xi (0 < xi <= 1) */
    double force_x, force_y; /* uniform body force per node and time step */
} fdlbm_ref_params;

/* Set OpenMP threads used by the step loops (<= 0: library default). */
void fdlbm_ref_set_threads(int n);
int fdlbm_ref_get_threads(void);

/* The moment matrix M (Sec. 1) and its inverse, row-major 9x9. */
void fdlbm_ref_moment_matrix(double* M81, double* Minv81);

/* FD-LBM: advance (rho, ux, uy) in place by nsteps (Sec. 2). */
int fdlbm_ref_fd_step(const fdlbm_ref_params* p, double* rho, double* ux, double* uy,
                      int64_t nsteps);

/* FD-LBM: one step evaluated only at npts nodes idx[] (flat j*nx+i) of the
 * given state; out receives (rho, ux, uy) per point, out[3*t + 0..2]. */
int fdlbm_ref_fd_step_points(const fdlbm_ref_params* p, const double* rho, const double* ux,
                             const double* uy, int64_t npts, const int64_t* idx, double* out);

/* FD-LBM: the 9 reconstructed post-collision populations f* at node (i, j)
 * (j may be a ghost row -1 or ny when walls are present). */
int fdlbm_ref_fd_fstar(const fdlbm_ref_params* p, const double* rho, const double* ux,
                       const double* uy, int32_t i, int32_t j, double* fstar9);

/* FD-LBM with curved walls (Sec. 3-b) on a periodic lattice (boundary
 * PERIODIC).  kind[j*nx+i]: 0 fluid, 1 virtual, 2 unused.  The nvirt
 * virtual nodes are vnode[t] (flat index, kind 1, each listed once); the
 * straight line from vnode[t] along link vlink[t] (1..8, Sec. 1 order)
 * reaches the fluid, and the wall crosses it vxi[t] link lengths (0 < xi
 * <= 1) before the first fluid node on it.  A virtual node, whenever read,
 * takes rho of that first fluid node and u linearly extrapolated to zero at
 * the wall from the first fluid node (xi >= 1/2) or the second (xi < 1/2).
 * Only fluid nodes are advanced; the other entries of rho, ux, uy are left
 * as they are.  FDLBM_REF_EINVAL if the scheme would read an unused node,
 * if a line finds no fluid within 16 links or if the table is inconsistent. */
int fdlbm_ref_fd_step_walls(const fdlbm_ref_params* p, const uint8_t* kind, int64_t nvirt,
                            const int64_t* vnode, const int8_t* vlink, const double* vxi,
                            double* rho, double* ux, double* uy, int64_t nsteps);

/* MRT: populations at equilibrium for (rho, u) with J = rho*u - F/2, so that
 * the reported velocity at t = 0 equals u. */
int fdlbm_ref_mrt_init(const fdlbm_ref_params* p, const double* rho, const double* ux,
                       const double* uy, double* f);

/* MRT: collide (Eq. 1, Strang force) and propagate (Eq. 2), nsteps times. */
int fdlbm_ref_mrt_step(const fdlbm_ref_params* p, double* f, int64_t nsteps);

/* MRT: rho = sum f, u = (sum c f + F/2) / rho. */
int fdlbm_ref_mrt_moments(const fdlbm_ref_params* p, const double* f, double* rho, double* ux,
                          double* uy);

/* MRT: moments after one step from an equilibrium start at (rho, u),
 * evaluated only at npts nodes; out[3*t + 0..2] = (rho, ux, uy). */
int fdlbm_ref_mrt_step_points_from_eq(const fdlbm_ref_params* p, const double* rho,
                                      const double* ux, const double* uy, int64_t npts,
                                      const int64_t* idx, double* out);

/* LW-ACM (Sec. 1-b, Eq. 3): nsteps steps of the (rho, ux, uy) state in place.
 * Reconstruction at each node from the equilibria alone,
 *   f*_a(x) = feq_a(x) + Theta (feo_a(x + c_a) - feo_a(x)),
 * feo the odd part of feq, Theta = 1 - 6 nu with nu = (1/s_xx - 1/2) / 3,
 * then propagation f_a(x + c_a) <- f*_a(x) and the moments.  Periodic
 * lattices without force only (the paper gives neither walls nor a force
 * for this scheme); s_e is not used. */
int fdlbm_ref_lwacm_step(const fdlbm_ref_params* p, double* rho, double* ux, double* uy,
                         int64_t nsteps);

/* LW-ACM: one step evaluated only at the nodes idx[0..npts) (flat j*nx + i),
 * with the propagation substituted into the reconstruction:
 *   f_a(x) = feq_a(x - c_a) + Theta (feo_a(x) - feo_a(x - c_a)).
 * out[3 t + 0..2] = (rho, ux, uy) at idx[t]. */
int fdlbm_ref_lwacm_step_points(const fdlbm_ref_params* p, const double* rho, const double* ux,
                                const double* uy, int64_t npts, const int64_t* idx, double* out);

#ifdef __cplusplus
}
#endif
#endif
