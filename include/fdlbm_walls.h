/* fdlbm_walls.h -- curved walls for FD-LBM lattices (Sec. 3-b).
 *
 * The lattice stays periodic; solid regions inside it are described per
 * node.  Nodes outside the fluid that the scheme reads are "virtual": their
 * state is estimated from the fluid by linear extrapolation using u = 0 on
 * the wall (Sec. 3-b), along a lattice link, with the expression chosen by
 * where the wall cuts the line between the last fluid node and the first
 * solid one: the wall xi link lengths before the first fluid node on the
 * line (0 < xi <= 1), u extrapolated from that node when xi >= 1/2 and from
 * the next one along the line when xi < 1/2, rho copied from the first.  A
 * straight channel written this way is the channel closure of
 * FDLBM_BOUNDARY_WALLS_Y (Sec. 3-c).
 */
#ifndef FDLBM_WALLS_H
#define FDLBM_WALLS_H

#include <stddef.h>
#include <stdint.h>

#include "fdlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of device memory the wall table of a lattice needs: 16 per node;
 * 0 if the parameters are invalid. */
size_t fdlbm_walls_table_bytes(const fdlbm_params* p);

/* Give an FD-LBM lattice (FDLBM_SCHEME_FD3, FD5 or FD9, boundary
 * FDLBM_BOUNDARY_PERIODIC) solid regions with curved walls.
 *   kind  : host, nx*ny bytes, row-major: 0 fluid, 1 virtual, 2 unused.
 *   nvirt : number of virtual nodes; vnode[t] (host) is the flat index
 *           j*nx + i of one (each kind-1 node listed exactly once),
 *           vlink[t] (host) the link 1..8 (order: (1,0), (0,1), (-1,0),
 *           (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)) along which the
 *           straight line from it reaches the fluid, vxi[t] (host) the
 *           distance of the wall before the first fluid node on that line,
 *           in link lengths, in (0, 1].
 *   table : caller-owned device memory of at least table_bytes =
 *           fdlbm_walls_table_bytes(p) bytes, 16-byte aligned, kept until
 *           the handle is destroyed or the walls are removed.
 * kind == NULL removes the walls (the other arguments are then ignored).
 * From then on, before every step and after the last step of each
 * fdlbm_step call, the library writes into the current state: at each
 * virtual node the closure's (rho - 1, ux, uy), at each unused node rest
 * (0, 0, 0).  Only fluid nodes follow the scheme; fdlbm_moments and
 * fdlbm_reduce still cover every node.  The host arrays are read during
 * the call only; the table is written on the handle's stream, and the call
 * returns once the copy has read the host data.
 * Returns FDLBM_ERR_INVALID for an inconsistent table: a kind other than
 * 0, 1, 2; a virtual node listed twice or not at all; a link outside 1..8;
 * xi outside (0, 1]; a line that meets no fluid within 16 links or whose
 * reference node is not fluid; an unused node within Chebyshev distance
 * R + 1 of a fluid node (R = 2 for FD5, 1 for FD3 and FD9), which the
 * scheme would read; a table smaller than needed.  FDLBM_ERR_UNSUPPORTED
 * for MRT, LW-ACM, FDLBM_BOUNDARY_WALLS_Y or a lattice above 2^31
 * elements per plane. */
int fdlbm_set_walls(fdlbm_t* h, const uint8_t* kind, int64_t nvirt, const int64_t* vnode,
                    const int8_t* vlink, const double* vxi, void* table, size_t table_bytes);

#ifdef __cplusplus
}
#endif

#endif /* FDLBM_WALLS_H */
