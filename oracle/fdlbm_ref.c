/*
 * fdlbm_ref.c -- FP64 CPU oracle: FD-LBM (Sec. 2), MRT D2Q9 (Sec. 1-a) and the
 * link-wise artificial compressibility method LW-ACM (Sec. 1-b, Eq. 3).
 *
 * TEST INFRASTRUCTURE ONLY (see fdlbm_ref.h).  Written for a reader who
 * checks it against the paper by eye: the moment matrix M is the table of
 * Sec. 1, M^-1 is formed from it, equilibria are the table of Sec. 1-a, the
 * defects of conservation theta_E, theta_XX, theta_XY and the reconstructed
 * moments are those of Sec. 2, the finite differences are the three-, five-
 * and nine-point formulas of Sec. 2, and propagation is Eq. 2.  No step is
 * fused, reordered or specialised.
 *
 * Readings where the paper is ambiguous (all listed in the design notes):
 *   - Jx, Jy rows of M carry the minus signs implied by the qx, qy, XY rows.
 *   - theta_XY's linear part is (1/3)(d_x uy + d_y ux) (strain rate): it is
 *     the value of d_t m^eq + Lambda d m for the XY moment, Eq. theta.
 *   - E and epsilon use |J|^2 / rho (Sec. 1-a) where Sec. 2 prints v^2 / rho.
 *   - theta: the paper writes it for density close to 1 with d v and d(v v).
 *     Eq. theta defines it through derivatives of the moments, so the
 *     finite differences act on J = rho u and on the momentum flux J J / rho
 *     (then the v.grad(rho) terms are exactly those of d_t m^eq + Lambda d m);
 *     undifferentiated factors are v = J / rho.  With derivatives of u
 *     instead, up- and downstream sound waves in a mean flow are damped
 *     unequally at first order in V, and unstably at V = 0.2.
 *   - The finite differences are applied to the product fields themselves.
 *   - Force: Strang splitting on J only.  J' = J + F/2 enters the equilibria
 *     and theta; the post-collision momentum is J' + F/2; the stored velocity
 *     is u = J' / rho.
 *   - LW-ACM, Eq. 3: the odd part of the equilibrium f^eo(i0, j0) is taken
 *     at the node the link points to, (i0, j0) = (i, j) + c_a, before the
 *     propagation; after it, f_a(x) = feq_a(x - c_a) + Theta (feo_a(x) -
 *     feo_a(x - c_a)).  This placement gives the H(k) printed in Sec. 1-b
 *     (its (1,2) entry -6 i nu k); the upstream node would give
 *     -i k (1 + Theta) / 3.  The equilibrium is the second-order D2Q9 one in
 *     (rho, u); periodic, no force (the paper gives neither for it).
 *   - Walls (Sec. 3-b, 3-c): virtual nodes outside the fluid carry u linearly
 *     extrapolated to zero at the wall, from the first fluid row when
 *     xi >= 1/2 and from the second when xi < 1/2; rho is copied from the
 *     first fluid row.  MRT uses half-way bounce-back (wall at xi = 1/2).
 *   - Curved walls (Sec. 3-b): the same closure along a lattice link.  Each
 *     virtual node comes with the link along which its straight line reaches
 *     the fluid and the wall's distance xi before the first fluid node on it;
 *     u is extrapolated to zero at the wall from the first fluid node
 *     (xi >= 1/2) or the second (xi < 1/2), rho copied from the first.  For a
 *     straight channel this is the closure above.
 */
#include "fdlbm_ref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice constants (Sec. 1) ---------------------------------------- */

static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* rows: rho, Jx, Jy, E, XX, XY, qx, qy, epsilon */
static const double M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
};

/* M is orthogonal (Sec. 1), so M^-1 = M^T diag(1 / |row k|^2). */
static void inverse_moment_matrix(double Minv[9][9]) {
    for (int k = 0; k < 9; ++k) {
        double norm2 = 0.0;
        for (int a = 0; a < 9; ++a) norm2 += M[k][a] * M[k][a];
        for (int a = 0; a < 9; ++a) Minv[a][k] = M[k][a] / norm2;
    }
}

static int g_threads = 0;

void fdlbm_ref_set_threads(int n) { g_threads = n; }

int fdlbm_ref_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

void fdlbm_ref_moment_matrix(double* M81, double* Minv81) {
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            if (M81) M81[r * 9 + c] = M[r][c];
            if (Minv81) Minv81[r * 9 + c] = Minv[r][c];
        }
}

static int valid_params(const fdlbm_ref_params* p) {
    if (!p) return 0;
    if (p->nx < 1 || p->ny < 1) return 0;
    if (p->scheme != FDLBM_REF_FD3 && p->scheme != FDLBM_REF_FD5 && p->scheme != FDLBM_REF_FD9 &&
        p->scheme != FDLBM_REF_MRT && p->scheme != FDLBM_REF_LWACM)
        return 0;
    if (p->boundary != FDLBM_REF_PERIODIC && p->boundary != FDLBM_REF_WALLS_Y) return 0;
    if (!(p->s_xx > 0.0 && p->s_xx < 2.0)) return 0;
    if (!(p->s_e > 0.0 && p->s_e < 2.0)) return 0;
    if (p->scheme == FDLBM_REF_MRT) {
        if (!(p->s_q > 0.0 && p->s_q < 2.0)) return 0;
        if (!(p->s_eps > 0.0 && p->s_eps < 2.0)) return 0;
    }
    if (p->boundary == FDLBM_REF_WALLS_Y) {
        if (!(p->wall_xi > 0.0 && p->wall_xi <= 1.0)) return 0;
        if (p->ny < 2) return 0;
        if (p->scheme == FDLBM_REF_MRT && p->wall_xi != 0.5) return 0;
    }
    return 1;
}

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* ---- FD-LBM (Sec. 2) ------------------------------------------------------ */

typedef struct {
    const fdlbm_ref_params* p;
    const double* rho;
    const double* ux;
    const double* uy;
    /* curved walls (Sec. 3-b); kind == NULL without them */
    const uint8_t* kind;
    const int32_t* vslot;  /* per node: index into the virtual-node table, or -1 */
    const int8_t* vlink;
    const double* vxi;
    int* bad;              /* set when an unused node would be read */
} fields_t;

static void mark_bad(const fields_t* F) {
#pragma omp atomic write
    *F->bad = 1;
}

static int kind_at(const fields_t* F, int i, int j) {
    const int nx = F->p->nx, ny = F->p->ny;
    return F->kind[(int64_t)wrap(j, ny) * nx + wrap(i, nx)];
}

/* State of a node of a lattice with curved walls (Sec. 3-b).  Fluid nodes
 * hold their own state.  A virtual node lies outside the fluid, on a
 * straight line along link a that reaches the first fluid node after d
 * links; the wall crosses the line at t_w = d - xi (t counted in links from
 * the virtual node).  Its velocity is the linear extrapolation, through
 * u = 0 at t_w, of the velocity at t_ref = d (first fluid node, xi >= 1/2)
 * or t_ref = d + 1 (second, xi < 1/2): u(0) = u(t_ref) (0 - t_w) /
 * (t_ref - t_w).  Its density is that of the first fluid node. */
static void walled_node_state(const fields_t* F, int i, int j, double* r, double* vx,
                              double* vy) {
    const int nx = F->p->nx, ny = F->p->ny;
    i = wrap(i, nx);
    j = wrap(j, ny);
    const int64_t idx = (int64_t)j * nx + i;
    *r = 1.0;
    *vx = 0.0;
    *vy = 0.0;
    if (F->kind[idx] == 0) {
        *r = F->rho[idx];
        *vx = F->ux[idx];
        *vy = F->uy[idx];
        return;
    }
    if (F->kind[idx] != 1) {
        mark_bad(F);
        return;
    }
    const int t = F->vslot[idx];
    const int a = F->vlink[t];
    const double xi = F->vxi[t];
    int d = 1;
    while (d <= 16 && kind_at(F, i + d * CX[a], j + d * CY[a]) != 0) ++d;
    const int tref = (xi >= 0.5) ? d : d + 1;
    if (d > 16 || kind_at(F, i + tref * CX[a], j + tref * CY[a]) != 0) {
        mark_bad(F);
        return;
    }
    const double tw = (double)d - xi;
    const double factor = (0.0 - tw) / ((double)tref - tw);
    const int64_t first = (int64_t)wrap(j + d * CY[a], ny) * nx + wrap(i + d * CX[a], nx);
    const int64_t ref = (int64_t)wrap(j + tref * CY[a], ny) * nx + wrap(i + tref * CX[a], nx);
    *r = F->rho[first];
    *vx = F->ux[ref] * factor;
    *vy = F->uy[ref] * factor;
}

/* Primitive state at (i, j).  Rows outside 0..ny-1 are periodic images, or,
 * with walls, virtual fluid nodes whose velocity is the linear extrapolation
 * to zero at the wall (Sec. 3-b) and whose density is that of the first
 * fluid row. */
static void node_state(const fields_t* F, int i, int j, double* r, double* vx, double* vy) {
    if (F->kind) {
        walled_node_state(F, i, j, r, vx, vy);
        return;
    }
    const int nx = F->p->nx, ny = F->p->ny;
    i = wrap(i, nx);
    if (F->p->boundary == FDLBM_REF_PERIODIC) j = wrap(j, ny);
    if (j >= 0 && j < ny) {
        *r = F->rho[(int64_t)j * nx + i];
        *vx = F->ux[(int64_t)j * nx + i];
        *vy = F->uy[(int64_t)j * nx + i];
        return;
    }
    const double xi = F->p->wall_xi;
    int jref, jrho;
    double ywall;
    if (j < 0) {
        ywall = -xi;
        jref = (xi >= 0.5) ? 0 : 1;
        jrho = 0;
    } else {
        ywall = (double)(ny - 1) + xi;
        jref = (xi >= 0.5) ? ny - 1 : ny - 2;
        jrho = ny - 1;
    }
    const double factor = ((double)j - ywall) / ((double)jref - ywall);
    *r = F->rho[(int64_t)jrho * nx + i];
    *vx = F->ux[(int64_t)jref * nx + i] * factor;
    *vy = F->uy[(int64_t)jref * nx + i] * factor;
}

/* Fields that the finite differences act on.  Eq. theta defines theta_k
 * through derivatives of the moments: the density, the momentum J = rho u
 * and the momentum flux J J / rho.  The paper prints them for density close
 * to 1 as derivatives of v and v v; they are read here as derivatives of J
 * and of J J / rho, while the undifferentiated factors are v = J / rho. */
enum { Q_RHO, Q_JX, Q_JY, Q_JXJX, Q_JXJY, Q_JYJY };

static double field_q(const fields_t* F, int q, int i, int j) {
    double r, vx, vy;
    node_state(F, i, j, &r, &vx, &vy);
    switch (q) {
        case Q_RHO: return r;
        case Q_JX: return r * vx;
        case Q_JY: return r * vy;
        case Q_JXJX: return r * vx * vx;
        case Q_JXJY: return r * vx * vy;
        default: return r * vy * vy;
    }
}

/* Finite-difference estimate of the derivative of field q along axis
 * (0 = x, 1 = y) at (i, j): the three-, five- and nine-point formulas of
 * Sec. 2. */
static double deriv(const fields_t* F, int q, int axis, int i, int j) {
    const int di = (axis == 0), dj = (axis == 1);
#define FQ(a, b) field_q(F, q, (a), (b))
    switch (F->p->scheme) {
        case FDLBM_REF_FD3:
            return 0.5 * (FQ(i + di, j + dj) - FQ(i - di, j - dj));
        case FDLBM_REF_FD5:
            return 0.75 * (FQ(i + di, j + dj) - FQ(i - di, j - dj)) -
                   0.125 * (FQ(i + 2 * di, j + 2 * dj) - FQ(i - 2 * di, j - 2 * dj));
        default: /* nine points, D2Q9 footprint */
            if (axis == 0)
                return FQ(i + 1, j) - FQ(i - 1, j) -
                       0.25 * (FQ(i + 1, j + 1) - FQ(i - 1, j + 1) - FQ(i - 1, j - 1) +
                               FQ(i + 1, j - 1));
            return FQ(i, j + 1) - FQ(i, j - 1) -
                   0.25 * (FQ(i + 1, j + 1) - FQ(i + 1, j - 1) - FQ(i - 1, j - 1) +
                           FQ(i - 1, j + 1));
    }
#undef FQ
}

/* Reconstructed post-collision populations f* at (i, j): moments from Sec. 2
 * (equilibria of Sec. 1-a plus (1 - 1/s) theta, Eq. order2), then f* = M^-1 m*. */
static void fd_reconstruct(const fields_t* F, const double Minv[9][9], int i, int j,
                           double fstar[9]) {
    const fdlbm_ref_params* p = F->p;
    double r, vx, vy;
    node_state(F, i, j, &r, &vx, &vy);

    /* derivatives of rho, of J and of the momentum flux P = J J / rho
     * (the paper's d v and d(v v) for density close to 1) */
    const double drx = deriv(F, Q_RHO, 0, i, j), dry = deriv(F, Q_RHO, 1, i, j);
    const double dx_Jx = deriv(F, Q_JX, 0, i, j), dy_Jx = deriv(F, Q_JX, 1, i, j);
    const double dx_Jy = deriv(F, Q_JY, 0, i, j), dy_Jy = deriv(F, Q_JY, 1, i, j);
    const double dx_Pxx = deriv(F, Q_JXJX, 0, i, j);
    const double dy_Pxy = deriv(F, Q_JXJY, 1, i, j);
    const double dx_Pxy = deriv(F, Q_JXJY, 0, i, j);
    const double dy_Pyy = deriv(F, Q_JYJY, 1, i, j);

    /* defects of conservation (Sec. 2), density close to 1 */
    const double theta_E = (2.0 + 6.0 * (vx * vx + vy * vy)) * (dx_Jx + dy_Jy) -
                           2.0 * (vx * drx + vy * dry);
    const double theta_XX = (2.0 / 3.0) * (dx_Jx - dy_Jy) - (2.0 / 3.0) * (vx * drx - vy * dry) -
                            2.0 * (vx * (dx_Pxx + dy_Pxy) - vy * (dx_Pxy + dy_Pyy));
    const double theta_XY = (1.0 / 3.0) * (dx_Jy + dy_Jx) - (1.0 / 3.0) * (vx * dry + vy * drx) -
                            vx * (dx_Pxy + dy_Pyy) - vy * (dx_Pxx + dy_Pxy);

    const double Jx = r * vx, Jy = r * vy; /* J' = J + F/2 */
    const double J2 = Jx * Jx + Jy * Jy;
    double m[9];
    m[0] = r;
    m[1] = Jx + 0.5 * p->force_x;
    m[2] = Jy + 0.5 * p->force_y;
    m[3] = -2.0 * r + 3.0 * J2 / r + (1.0 - 1.0 / p->s_e) * theta_E;
    m[4] = (Jx * Jx - Jy * Jy) / r + (1.0 - 1.0 / p->s_xx) * theta_XX;
    m[5] = (Jx * Jy) / r + (1.0 - 1.0 / p->s_xx) * theta_XY;
    m[6] = -Jx;
    m[7] = -Jy;
    m[8] = r - 3.0 * J2 / r;

    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += Minv[a][k] * m[k];
        fstar[a] = s;
    }
}

int fdlbm_ref_fd_fstar(const fdlbm_ref_params* p, const double* rho, const double* ux,
                       const double* uy, int32_t i, int32_t j, double* fstar9) {
    if (!valid_params(p) || p->scheme == FDLBM_REF_MRT || !rho || !ux || !uy || !fstar9)
        return FDLBM_REF_EINVAL;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    fields_t F = {p, rho, ux, uy, NULL, NULL, NULL, NULL, NULL};
    fd_reconstruct(&F, Minv, i, j, fstar9);
    return FDLBM_REF_OK;
}

/* Moments of the populations arriving at (i, j) by Eq. 2, with f*_a(y)
 * supplied by fetch(); returns rho and u = (J + F/2) / rho. */
static void close_moments(const fdlbm_ref_params* p, const double f[9], double* r, double* vx,
                          double* vy) {
    double s = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        s += f[a];
        jx += CX[a] * f[a];
        jy += CY[a] * f[a];
    }
    *r = s;
    *vx = (jx + 0.5 * p->force_x) / s;
    *vy = (jy + 0.5 * p->force_y) / s;
}

int fdlbm_ref_fd_step(const fdlbm_ref_params* p, double* rho, double* ux, double* uy,
                      int64_t nsteps) {
    if (!valid_params(p) || p->scheme == FDLBM_REF_MRT || !rho || !ux || !uy || nsteps < 0)
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int walls = (p->boundary == FDLBM_REF_WALLS_Y);
    /* source rows: the fluid rows, plus one virtual row on each side when walls */
    const int jlo = walls ? -1 : 0, jhi = walls ? ny : ny - 1;
    const int nrows = jhi - jlo + 1;
    const int64_t plane = (int64_t)nrows * nx;
    double* fstar = (double*)malloc(sizeof(double) * 9 * (size_t)plane);
    if (!fstar) return FDLBM_REF_ENOMEM;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;

    for (int64_t n = 0; n < nsteps; ++n) {
        fields_t F = {p, rho, ux, uy, NULL, NULL, NULL, NULL, NULL};
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = jlo; j <= jhi; ++j) {
            for (int i = 0; i < nx; ++i) {
                double fs[9];
                fd_reconstruct(&F, Minv, i, j, fs);
                for (int a = 0; a < 9; ++a) fstar[a * plane + (int64_t)(j - jlo) * nx + i] = fs[a];
            }
        }
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                double f[9];
                for (int a = 0; a < 9; ++a) {
                    const int si = wrap(i - CX[a], nx);
                    int sj = j - CY[a];
                    if (!walls) sj = wrap(sj, ny);
                    f[a] = fstar[a * plane + (int64_t)(sj - jlo) * nx + si];
                }
                double r, vx, vy;
                close_moments(p, f, &r, &vx, &vy);
                rho[(int64_t)j * nx + i] = r;
                ux[(int64_t)j * nx + i] = vx;
                uy[(int64_t)j * nx + i] = vy;
            }
        }
    }
    free(fstar);
    return FDLBM_REF_OK;
}

int fdlbm_ref_fd_step_walls(const fdlbm_ref_params* p, const uint8_t* kind, int64_t nvirt,
                            const int64_t* vnode, const int8_t* vlink, const double* vxi,
                            double* rho, double* ux, double* uy, int64_t nsteps) {
    if (!valid_params(p) || p->scheme == FDLBM_REF_MRT || p->scheme == FDLBM_REF_LWACM ||
        p->boundary != FDLBM_REF_PERIODIC || !kind || !rho || !ux || !uy || nsteps < 0 ||
        nvirt < 0 || (nvirt > 0 && (!vnode || !vlink || !vxi)))
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int64_t nodes = (int64_t)nx * ny;
    int32_t* vslot = (int32_t*)malloc(sizeof(int32_t) * (size_t)nodes);
    double* fstar = (double*)malloc(sizeof(double) * 9 * (size_t)nodes);
    uint8_t* source = (uint8_t*)calloc((size_t)nodes, 1); /* fluid nodes and their neighbours */
    if (!vslot || !fstar || !source) {
        free(vslot);
        free(fstar);
        free(source);
        return FDLBM_REF_ENOMEM;
    }
    int bad = 0;
    for (int64_t n = 0; n < nodes; ++n) {
        vslot[n] = -1;
        if (kind[n] > 2) bad = 1;
    }
    for (int64_t t = 0; t < nvirt && !bad; ++t) {
        if (vnode[t] < 0 || vnode[t] >= nodes || kind[vnode[t]] != 1 || vslot[vnode[t]] >= 0 ||
            vlink[t] < 1 || vlink[t] > 8 || !(vxi[t] > 0.0 && vxi[t] <= 1.0))
            bad = 1;
        else
            vslot[vnode[t]] = (int32_t)t;
    }
    for (int64_t n = 0; n < nodes && !bad; ++n)
        if (kind[n] == 1 && vslot[n] < 0) bad = 1;
    /* the nodes whose populations propagate into a fluid node (Eq. 2) */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (kind[(int64_t)j * nx + i] == 0)
                for (int a = 0; a < 9; ++a)
                    source[(int64_t)wrap(j - CY[a], ny) * nx + wrap(i - CX[a], nx)] = 1;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
    for (int64_t step = 0; step < nsteps && !bad; ++step) {
        fields_t F = {p, rho, ux, uy, kind, vslot, vlink, vxi, &bad};
        /* reconstruction (Sec. 2) at the fluid nodes and the virtual nodes
         * next to them */
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const int64_t n = (int64_t)j * nx + i;
                double fs[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                if (source[n]) fd_reconstruct(&F, Minv, i, j, fs);
                for (int a = 0; a < 9; ++a) fstar[a * nodes + n] = fs[a];
            }
        }
        /* propagation (Eq. 2) into the fluid nodes; their sources must not
         * be unused nodes */
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const int64_t n = (int64_t)j * nx + i;
                if (kind[n] != 0) continue;
                double f[9];
                for (int a = 0; a < 9; ++a) {
                    const int64_t src = (int64_t)wrap(j - CY[a], ny) * nx + wrap(i - CX[a], nx);
                    if (kind[src] == 2) mark_bad(&F);
                    f[a] = fstar[a * nodes + src];
                }
                double r, vx, vy;
                close_moments(p, f, &r, &vx, &vy);
                rho[n] = r;
                ux[n] = vx;
                uy[n] = vy;
            }
        }
    }
    free(vslot);
    free(fstar);
    free(source);
    return bad ? FDLBM_REF_EINVAL : FDLBM_REF_OK;
}

int fdlbm_ref_fd_step_points(const fdlbm_ref_params* p, const double* rho, const double* ux,
                             const double* uy, int64_t npts, const int64_t* idx, double* out) {
    if (!valid_params(p) || p->scheme == FDLBM_REF_MRT || !rho || !ux || !uy || npts < 0 ||
        (npts > 0 && (!idx || !out)))
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int walls = (p->boundary == FDLBM_REF_WALLS_Y);
    for (int64_t t = 0; t < npts; ++t)
        if (idx[t] < 0 || idx[t] >= (int64_t)nx * ny) return FDLBM_REF_EINVAL;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    fields_t F = {p, rho, ux, uy, NULL, NULL, NULL, NULL, NULL};
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthr)
    for (int64_t t = 0; t < npts; ++t) {
        const int i = (int)(idx[t] % nx), j = (int)(idx[t] / nx);
        double f[9];
        for (int a = 0; a < 9; ++a) {
            const int si = wrap(i - CX[a], nx);
            int sj = j - CY[a];
            if (!walls) sj = wrap(sj, ny);
            double fs[9];
            fd_reconstruct(&F, Minv, si, sj, fs);
            f[a] = fs[a];
        }
        close_moments(p, f, &out[3 * t], &out[3 * t + 1], &out[3 * t + 2]);
    }
    return FDLBM_REF_OK;
}

/* ---- MRT D2Q9 (Sec. 1, Sec. 1-a) ------------------------------------------ */

/* Equilibrium values of the non-conserved moments (Sec. 1-a table). */
static void mrt_equilibrium(double r, double Jx, double Jy, double meq[9]) {
    const double J2 = Jx * Jx + Jy * Jy;
    meq[0] = r;
    meq[1] = Jx;
    meq[2] = Jy;
    meq[3] = -2.0 * r + 3.0 * J2 / r;
    meq[4] = (Jx * Jx - Jy * Jy) / r;
    meq[5] = Jx * Jy / r;
    meq[6] = -Jx;
    meq[7] = -Jy;
    meq[8] = r - 3.0 * J2 / r;
}

/* Collision (Eq. 1) with half of the force before and half after (Sec. 1). */
static void mrt_collide(const fdlbm_ref_params* p, const double Minv[9][9], const double f[9],
                        double fstar[9]) {
    double m[9];
    for (int k = 0; k < 9; ++k) {
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += M[k][a] * f[a];
        m[k] = s;
    }
    const double r = m[0];
    const double Jx = m[1] + 0.5 * p->force_x;
    const double Jy = m[2] + 0.5 * p->force_y;
    double meq[9];
    mrt_equilibrium(r, Jx, Jy, meq);
    const double rate[9] = {0, 0, 0, p->s_e, p->s_xx, p->s_xx, p->s_q, p->s_q, p->s_eps};
    double ms[9];
    ms[0] = r;
    ms[1] = Jx + 0.5 * p->force_x;
    ms[2] = Jy + 0.5 * p->force_y;
    for (int k = 3; k < 9; ++k) ms[k] = m[k] + rate[k] * (meq[k] - m[k]);
    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += Minv[a][k] * ms[k];
        fstar[a] = s;
    }
}

static void mrt_eq_populations(const fdlbm_ref_params* p, const double Minv[9][9], double r,
                               double vx, double vy, double f[9]) {
    double meq[9];
    mrt_equilibrium(r, r * vx - 0.5 * p->force_x, r * vy - 0.5 * p->force_y, meq);
    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += Minv[a][k] * meq[k];
        f[a] = s;
    }
}

int fdlbm_ref_mrt_init(const fdlbm_ref_params* p, const double* rho, const double* ux,
                       const double* uy, double* f) {
    if (!valid_params(p) || p->scheme != FDLBM_REF_MRT || !rho || !ux || !uy || !f)
        return FDLBM_REF_EINVAL;
    const int64_t plane = (int64_t)p->nx * p->ny;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    for (int64_t n = 0; n < plane; ++n) {
        double fe[9];
        mrt_eq_populations(p, Minv, rho[n], ux[n], uy[n], fe);
        for (int a = 0; a < 9; ++a) f[a * plane + n] = fe[a];
    }
    return FDLBM_REF_OK;
}

int fdlbm_ref_mrt_step(const fdlbm_ref_params* p, double* f, int64_t nsteps) {
    if (!valid_params(p) || p->scheme != FDLBM_REF_MRT || !f || nsteps < 0)
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int walls = (p->boundary == FDLBM_REF_WALLS_Y);
    const int64_t plane = (int64_t)nx * ny;
    double* fs = (double*)malloc(sizeof(double) * 9 * (size_t)plane);
    if (!fs) return FDLBM_REF_ENOMEM;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
    for (int64_t n = 0; n < nsteps; ++n) {
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int64_t c = 0; c < plane; ++c) {
            double fl[9], fo[9];
            for (int a = 0; a < 9; ++a) fl[a] = f[a * plane + c];
            mrt_collide(p, Minv, fl, fo);
            for (int a = 0; a < 9; ++a) fs[a * plane + c] = fo[a];
        }
        /* propagation (Eq. 2); a link whose source lies in a wall is bounced
         * back half-way: it receives the opposite population of the node itself */
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                for (int a = 0; a < 9; ++a) {
                    const int si = wrap(i - CX[a], nx);
                    int sj = j - CY[a];
                    double v;
                    if (!walls) {
                        sj = wrap(sj, ny);
                        v = fs[a * plane + (int64_t)sj * nx + si];
                    } else if (sj < 0 || sj >= ny) {
                        v = fs[OPP[a] * plane + (int64_t)j * nx + i];
                    } else {
                        v = fs[a * plane + (int64_t)sj * nx + si];
                    }
                    f[a * plane + (int64_t)j * nx + i] = v;
                }
            }
        }
    }
    free(fs);
    return FDLBM_REF_OK;
}

int fdlbm_ref_mrt_moments(const fdlbm_ref_params* p, const double* f, double* rho, double* ux,
                          double* uy) {
    if (!valid_params(p) || p->scheme != FDLBM_REF_MRT || !f || !rho || !ux || !uy)
        return FDLBM_REF_EINVAL;
    const int64_t plane = (int64_t)p->nx * p->ny;
    for (int64_t n = 0; n < plane; ++n) {
        double fl[9];
        for (int a = 0; a < 9; ++a) fl[a] = f[a * plane + n];
        close_moments(p, fl, &rho[n], &ux[n], &uy[n]);
    }
    return FDLBM_REF_OK;
}

int fdlbm_ref_mrt_step_points_from_eq(const fdlbm_ref_params* p, const double* rho,
                                      const double* ux, const double* uy, int64_t npts,
                                      const int64_t* idx, double* out) {
    if (!valid_params(p) || p->scheme != FDLBM_REF_MRT || !rho || !ux || !uy || npts < 0 ||
        (npts > 0 && (!idx || !out)))
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int walls = (p->boundary == FDLBM_REF_WALLS_Y);
    for (int64_t t = 0; t < npts; ++t)
        if (idx[t] < 0 || idx[t] >= (int64_t)nx * ny) return FDLBM_REF_EINVAL;
    double Minv[9][9];
    inverse_moment_matrix(Minv);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthr)
    for (int64_t t = 0; t < npts; ++t) {
        const int i = (int)(idx[t] % nx), j = (int)(idx[t] / nx);
        double f[9];
        for (int a = 0; a < 9; ++a) {
            int si = wrap(i - CX[a], nx), sj = j - CY[a], pa = a;
            if (!walls) {
                sj = wrap(sj, ny);
            } else if (sj < 0 || sj >= ny) {
                si = i;
                sj = j;
                pa = OPP[a];
            }
            const int64_t s = (int64_t)sj * nx + si;
            double fe[9], fo[9];
            mrt_eq_populations(p, Minv, rho[s], ux[s], uy[s], fe);
            mrt_collide(p, Minv, fe, fo);
            f[a] = fo[pa];
        }
        close_moments(p, f, &out[3 * t], &out[3 * t + 1], &out[3 * t + 2]);
    }
    return FDLBM_REF_OK;
}

/* ---- LW-ACM (Sec. 1-b) ------------------------------------------------------ */

/* D2Q9 weights of the equilibrium (Sec. 1, the f^eq identity). */
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Second-order equilibrium of population a for density r and velocity (vx, vy). */
static double lw_feq(int a, double r, double vx, double vy) {
    const double cu = CX[a] * vx + CY[a] * vy;
    const double u2 = vx * vx + vy * vy;
    return W[a] * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
}

/* Odd part of the equilibrium: (feq(r, u) - feq(r, -u)) / 2. */
static double lw_feo(int a, double r, double vx, double vy) {
    return 0.5 * (lw_feq(a, r, vx, vy) - lw_feq(a, r, -vx, -vy));
}

static int lw_valid(const fdlbm_ref_params* p) {
    return valid_params(p) && p->scheme == FDLBM_REF_LWACM &&
           p->boundary == FDLBM_REF_PERIODIC && p->force_x == 0.0 && p->force_y == 0.0;
}

/* Theta = 1 - 2 nu / c_s^2 = 1 - 6 nu, nu = (1/s_xx - 1/2) / 3 */
static double lw_theta(const fdlbm_ref_params* p) {
    const double nu = (1.0 / p->s_xx - 0.5) / 3.0;
    return 1.0 - 6.0 * nu;
}

static void lw_moments(const double f[9], double* r, double* vx, double* vy) {
    double s = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        s += f[a];
        jx += CX[a] * f[a];
        jy += CY[a] * f[a];
    }
    *r = s;
    *vx = jx / s;
    *vy = jy / s;
}

int fdlbm_ref_lwacm_step(const fdlbm_ref_params* p, double* rho, double* ux, double* uy,
                         int64_t nsteps) {
    if (!lw_valid(p) || !rho || !ux || !uy || nsteps < 0) return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    const int64_t plane = (int64_t)nx * ny;
    double* fstar = (double*)malloc(sizeof(double) * 9 * (size_t)plane);
    if (!fstar) return FDLBM_REF_ENOMEM;
    const double theta = lw_theta(p);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
    for (int64_t n = 0; n < nsteps; ++n) {
        /* reconstruction at every node, from the equilibria of the node and of
           the node each link points to */
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const int64_t o = (int64_t)j * nx + i;
                for (int a = 0; a < 9; ++a) {
                    const int64_t d = (int64_t)wrap(j + CY[a], ny) * nx + wrap(i + CX[a], nx);
                    fstar[a * plane + o] =
                        lw_feq(a, rho[o], ux[o], uy[o]) +
                        theta * (lw_feo(a, rho[d], ux[d], uy[d]) - lw_feo(a, rho[o], ux[o], uy[o]));
                }
            }
        }
        /* propagation and moments */
#pragma omp parallel for schedule(static) num_threads(nthr)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                double f[9];
                for (int a = 0; a < 9; ++a)
                    f[a] = fstar[a * plane + (int64_t)wrap(j - CY[a], ny) * nx + wrap(i - CX[a], nx)];
                const int64_t o = (int64_t)j * nx + i;
                lw_moments(f, &rho[o], &ux[o], &uy[o]);
            }
        }
    }
    free(fstar);
    return FDLBM_REF_OK;
}

int fdlbm_ref_lwacm_step_points(const fdlbm_ref_params* p, const double* rho, const double* ux,
                                const double* uy, int64_t npts, const int64_t* idx, double* out) {
    if (!lw_valid(p) || !rho || !ux || !uy || npts < 0 || (npts > 0 && (!idx || !out)))
        return FDLBM_REF_EINVAL;
    const int nx = p->nx, ny = p->ny;
    for (int64_t t = 0; t < npts; ++t)
        if (idx[t] < 0 || idx[t] >= (int64_t)nx * ny) return FDLBM_REF_EINVAL;
    const double theta = lw_theta(p);
    const int nthr = fdlbm_ref_get_threads();
    (void)nthr;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthr)
    for (int64_t t = 0; t < npts; ++t) {
        const int i = (int)(idx[t] % nx), j = (int)(idx[t] / nx);
        const int64_t x = idx[t];
        double f[9];
        for (int a = 0; a < 9; ++a) {
            const int64_t y = (int64_t)wrap(j - CY[a], ny) * nx + wrap(i - CX[a], nx);
            f[a] = lw_feq(a, rho[y], ux[y], uy[y]) +
                   theta * (lw_feo(a, rho[x], ux[x], uy[x]) - lw_feo(a, rho[y], ux[y], uy[y]));
        }
        lw_moments(f, &out[3 * t], &out[3 * t + 1], &out[3 * t + 2]);
    }
    return FDLBM_REF_OK;
}
