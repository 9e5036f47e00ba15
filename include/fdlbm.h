/*
 * fdlbm.h -- C ABI of the GB300 (sm_103a) FD-LBM / MRT / LW-ACM D2Q9 library.
 *
 * The schemes are those of Dubois, Lallemand, Obrecht, Tekitek, "Lattice
 * Boltzmann model approximated with finite difference expressions"
 * (Computers & Fluids 155, 2017):
 *   - FD-LBM (Sec. 2): only the primitive moments (rho, ux, uy) are kept per
 *     node.  Each step rebuilds the 9 populations at every node from the
 *     equilibria of Sec. 1-a plus (1 - 1/s) theta (Eq. order2), with the
 *     defects theta_E, theta_XX, theta_XY estimated by three- or five-point
 *     finite differences, maps them to populations with M^-1 (Sec. 1) and
 *     propagates them one link (Eq. 2).
 *   - MRT D2Q9 (Sec. 1, 1-a): collision of the non-conserved moments towards
 *     their equilibria (Eq. 1) and propagation (Eq. 2).
 *   - LW-ACM (Sec. 1-b, Eq. 3): the same (rho, ux, uy) state, every link
 *     rebuilt from equilibria alone (no finite differences) and propagated.
 *   - Body force: Strang splitting, half before and half after the
 *     collision (Sec. 1).  Walls (Sec. 3-b, 3-c): FD-LBM extrapolates the
 *     velocity linearly to zero at walls placed xi outside the first and
 *     last fluid rows; MRT uses half-way bounce-back (xi = 1/2).
 *
 * Conventions shared by all entry points
 *   - Fields are row-major [ny][nx], node (i, j) at j*nx + i, i along x.
 *   - Density is passed as the deviation drho = rho - 1, so that FP32 keeps
 *     the resolution of small perturbations.  Velocities are u = (J + F/2) /
 *     rho, the physical velocity at the middle of the force splitting.
 *   - Device pointers are CUDA device (or managed) pointers on the device
 *     that was current at fdlbm_create.  Host pointers are ordinary host
 *     memory; pinned memory makes the copies asynchronous.
 *   - Every call is enqueued on the stream given at creation (or set with
 *     fdlbm_set_stream) and returns without waiting, except fdlbm_reduce,
 *     the *_host variants and fdlbm_sync, which wait for the stream.
 *   - The caller owns the workspace and every buffer.  The library owns only
 *     the small host-side handle; it never calls cudaMalloc or cudaFree.
 *   - Errors: every int-returning call returns FDLBM_OK (0) or a negative
 *     fdlbm_status.  Nothing aborts or throws.  The text of the last error on
 *     a handle is available from fdlbm_last_error.  A device-side wait that
 *     ran out (FDLBM_ERR_TIMEOUT) is reported by the next fdlbm_sync or
 *     fdlbm_reduce; non-finite values by fdlbm_reduce (FDLBM_ERR_DIVERGED);
 *     a saturated fixed-point store (FDLBM_ERR_RANGE) by fdlbm_sync or
 *     fdlbm_reduce.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef FDLBM_H
#define FDLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FDLBM_OK 0
#define FDLBM_ERR_INVALID (-1)     /* bad argument or parameter            */
#define FDLBM_ERR_UNSUPPORTED (-2) /* valid but not implemented combination */
#define FDLBM_ERR_NOMEM (-3)       /* workspace too small                   */
#define FDLBM_ERR_CUDA (-4)        /* a CUDA runtime call failed            */
#define FDLBM_ERR_DIVERGED (-5)    /* non-finite values found on the device */
#define FDLBM_ERR_TIMEOUT (-6)     /* a bounded device-side wait expired    */
#define FDLBM_ERR_RANGE (-7)       /* a value beyond storage_range (I16 storage)
                                      was stored saturated                   */

/* ---- scheme, boundary, storage ----------------------------------------- */
#define FDLBM_SCHEME_FD3 3   /* FD-LBM, three-point differences (Sec. 2)   */
#define FDLBM_SCHEME_FD5 5   /* FD-LBM, five-point differences (Sec. 2)    */
#define FDLBM_SCHEME_MRT 100 /* multiple-relaxation-time D2Q9 (Sec. 1-a)  */
/* FD-LBM with the nine-point differences of Sec. 2 (D2Q9 footprint):
 * d_x f = f(i+1,j) - f(i-1,j) - [f(i+1,j+1) - f(i-1,j+1) + f(i+1,j-1)
 * - f(i-1,j-1)] / 4, d_y alike.  Same state, storage, walls and force as the
 * other FD-LBM stencils; always the tiled kernel (FDLBM_FLAG_STREAM is
 * FDLBM_ERR_UNSUPPORTED).  Linearly unstable at short wavelengths for small
 * viscosities (Sec. 3-a; max |z| about 1.2 at nu = 0.01, 1 near nu = 0.15). */
#define FDLBM_SCHEME_FD9 9
/* Link-wise artificial compressibility method (Sec. 1-b, Eq. 3): every link
 * rebuilt from equilibria alone, f_a(x) = feq_a(x - c_a) + Theta (feo_a(x) -
 * feo_a(x - c_a)), feo the odd part of feq, Theta = 1 - 6 nu, nu from s_xx as
 * for the other schemes; s_e is not used.  Same (rho - 1, ux, uy) state,
 * storage options and kernel choice (FDLBM_FLAG_*) as FD-LBM.  Periodic
 * lattices without force (FDLBM_ERR_UNSUPPORTED otherwise). */
#define FDLBM_SCHEME_LWACM 200

#define FDLBM_BOUNDARY_PERIODIC 0 /* periodic in x and y                  */
#define FDLBM_BOUNDARY_WALLS_Y 1  /* periodic in x; walls below row 0 and
                                     above row ny-1 (channel, Sec. 3-c)    */

#define FDLBM_STORAGE_F32 0  /* state stored in FP32                      */
#define FDLBM_STORAGE_F16 1  /* FD-LBM only: (rho-1, ux, uy) in FP16, FP32 math */
#define FDLBM_STORAGE_BF16 2 /* FD-LBM only: (rho-1, ux, uy) in BF16, FP32 math */
/* FD-LBM only: (rho-1, ux, uy) in 16-bit fixed point, FP32 math.  A value v
 * is stored as q = round_to_nearest(v * 32767 / storage_range), |q| <= 32767,
 * and read as q * storage_range / 32767: a uniform spacing of
 * storage_range / 32767 instead of FP16's 2^-11 relative spacing, which the
 * slow per-step change of the fields (nu k^2 of their value) needs.  A value
 * beyond +-storage_range (or not finite) is stored saturated at the bound and
 * reported as FDLBM_ERR_RANGE by the next fdlbm_sync or fdlbm_reduce; the
 * caller chooses storage_range above the largest |rho - 1|, |ux|, |uy| the
 * flow will reach.  Curved walls (fdlbm_set_walls) are not supported with
 * it. */
#define FDLBM_STORAGE_I16 3

/* Kernel choice for FD-LBM lattices.  By default a lattice that qualifies
 * for the streaming kernel (periodic or channel, nx % 8 == 0, nx >= 256,
 * ny >= 16) and holds at least 2^20 nodes uses it; smaller or other
 * lattices use the general tiled kernel, which spreads small lattices over
 * more of the GPU (the streaming kernel walks each strip row by row and has
 * a latency floor of ~18 us per step).  FDLBM_FLAG_TILED forces the tiled
 * kernel; FDLBM_FLAG_STREAM forces the streaming kernel whenever the lattice
 * qualifies (both give the same results up to FP32 rounding; used to
 * cross-check the two).  Setting both is invalid. */
#define FDLBM_FLAG_TILED 1
#define FDLBM_FLAG_STREAM 2

/* Parameters of one lattice.  Relaxation rates lie in (0, 2).
 *   s_xx : rate of XX and XY; shear viscosity nu = (1/s_xx - 1/2)/3 (Sec. 1-a)
 *   s_e  : rate of E; bulk viscosity zeta = (1/s_e - 1/2)/3 (Sec. 1-a)
 *   s_q  : rate of qx, qy (MRT only; FD-LBM sets q = -J, Sec. 2).  For MRT,
 *          s_q = FDLBM_S_Q_QUARTIC (0) asks the library for the rate of the
 *          quartic condition (Eq. sigsig, Sec. 3-b): (1/s_xx - 1/2)(1/s_q - 1/2)
 *          = 1/6, which makes the shear hyperviscosity isotropic; any other
 *          value must lie in (0, 2).
 *   s_eps: rate of epsilon (MRT only; FD-LBM sets epsilon to equilibrium)
 *   wall_xi: walls at y = -xi and y = ny-1+xi in lattice units, 0 < xi <= 1
 *            (FD-LBM); MRT requires xi = 1/2.  Ignored when periodic.
 *   force_x, force_y: uniform body force per node and time step.
 *   storage_range: FDLBM_STORAGE_I16 only, the largest |value| representable
 *            (> 0); ignored by the other storage types. */
#define FDLBM_S_Q_QUARTIC 0.0
typedef struct fdlbm_params {
    int32_t nx, ny;
    int32_t scheme;   /* FDLBM_SCHEME_*   */
    int32_t boundary; /* FDLBM_BOUNDARY_* */
    int32_t storage;  /* FDLBM_STORAGE_*  */
    int32_t flags;    /* 0, or FDLBM_FLAG_* bits */
    double s_xx, s_e, s_q, s_eps;
    double wall_xi;
    double force_x, force_y;
    double storage_range;
} fdlbm_params;

typedef struct fdlbm_s fdlbm_t;

/* Bytes of device workspace that fdlbm_create needs for these parameters:
 * two copies of the state (ping-pong), a staging area for host transfers
 * and reduction scratch.  Returns 0 if the parameters are invalid. */
size_t fdlbm_workspace_size(const fdlbm_params* params);

/* Create a handle on the current CUDA device.  workspace: device memory of
 * at least fdlbm_workspace_size bytes, 256-byte aligned, owned by the caller
 * and kept alive until fdlbm_destroy.  stream: a cudaStream_t (NULL = the
 * legacy default stream).  On success *out receives the handle.  The state
 * is undefined until fdlbm_init* is called. */
int fdlbm_create(const fdlbm_params* params, void* workspace, size_t workspace_bytes,
                 void* stream, fdlbm_t** out);

/* Release the host-side handle (and its 48-byte page-locked landing area for
 * reduction results, allocated by fdlbm_create).  Never touches the
 * workspace. */
void fdlbm_destroy(fdlbm_t* h);

/* Change the stream that later calls are enqueued on. */
int fdlbm_set_stream(fdlbm_t* h, void* stream);

/* Load the initial state from device arrays drho, ux, uy (nx*ny floats
 * each, row-major).  For MRT the populations are set to the equilibria of
 * Sec. 1-a at (rho, J = rho u - F/2), so the reported velocity is u. */
int fdlbm_init(fdlbm_t* h, const float* drho, const float* ux, const float* uy);

/* Same, from host arrays; waits until the state is initialised.  Arrays in
 * page-locked host memory (cudaHostAlloc / cudaHostRegister, e.g. torch's
 * pin_memory) are read in place by the init kernel over the host link;
 * other host arrays are copied through the workspace staging area first.
 * The arrays are only read, and may be reused once the call returns. */
int fdlbm_init_host(fdlbm_t* h, const float* drho, const float* ux, const float* uy);

/* Initial state rho = 1 and u = V + sum of transverse plane waves
 * A cos(k.x + phase) (-ky, kx)/|k| with k = 2 pi (m / nx, n / ny)
 * (shear waves, Sec. 3-a), evaluated on the device.  modes: host array of
 * n_modes records {m, n, A, phase} (4 doubles each). */
int fdlbm_init_modes(fdlbm_t* h, int32_t n_modes, const double* modes, double mean_ux,
                     double mean_uy);

/* Advance nsteps >= 0 time steps (asynchronous).  nsteps = 0 is a no-op. */
int fdlbm_step(fdlbm_t* h, int64_t nsteps);

/* The launch plan of the streaming step (the time step of Sec. 2, and
 * LW-ACM's of Sec. 1-b) for an nx x ny lattice when resident_ctas CTAs of it
 * fit on the device at once (fdlbm_step queries that occupancy itself and
 * computes the plan once per handle).  A CTA covers a 240-column strip of one
 * row segment.  The rows are cut into a first part of long segments followed
 * by short ones (the finite-difference steps, where this measured faster),
 * or into segments of one length (LW-ACM, and wherever the cost model finds
 * that cheaper); the model counts the rows a segment streams beyond its own,
 * the launch's tail, and the spread of the long segments' finishing times
 * that the short ones must absorb.  scheme: FDLBM_SCHEME_FD3, _FD5 or
 * _LWACM; storage: FDLBM_STORAGE_*.  plan (host, 6 int32): rows per long
 * segment, long segments, rows per short segment, short segments (0 when all
 * are equal), CTA strips, CTAs.  Host-only: needs no device.
 * FDLBM_ERR_INVALID for a NULL plan, a size or resident_ctas below 1, or
 * another scheme or storage. */
int fdlbm_stream_plan(int32_t nx, int32_t ny, int32_t scheme, int32_t storage,
                      int32_t resident_ctas, int32_t* plan);

/* Candidate launch plans of the streaming step, for measuring which is
 * fastest on the device at hand (the cost model ranks plans whose step times
 * differ by a few per cent, below its accuracy).  Same arguments as
 * fdlbm_stream_plan; out (host, 3 * max int32) receives per candidate the
 * rows per long segment, the long segments, and the rows per short segment
 * (equal to the first entry when all segments are equal), the model's plan
 * first and the rest cheapest first by the model; *count the number written
 * (1 <= *count <= max).  FDLBM_ERR_INVALID as for fdlbm_stream_plan, or for
 * max < 1 or a NULL count. */
int fdlbm_stream_plan_candidates(int32_t nx, int32_t ny, int32_t scheme, int32_t storage,
                                 int32_t resident_ctas, int32_t* out, int32_t max,
                                 int32_t* count);

/* Use the given row segments for this lattice's streaming step instead of the
 * model's plan: nsegs segments of seg_rows rows, then the remaining rows in
 * segments of tail_rows rows (equal segments of seg_rows rows if nsegs *
 * seg_rows >= ny).  (0, 0, 0) returns to the model's plan.  Any plan gives
 * the same lattice bit for bit; only the step time changes.  FDLBM_ERR_INVALID
 * for a value below 1 (other than all three 0), seg_rows > ny, or a lattice
 * whose steps do not run on the streaming kernel (MRT, nine points, the tiled
 * kernel). */
int fdlbm_set_stream_plan(fdlbm_t* h, int32_t seg_rows, int32_t nsegs, int32_t tail_rows);

/* The launch plan this lattice's streaming step uses: plan (host, 7 int32)
 * receives the six entries of fdlbm_stream_plan, then the resident CTAs the
 * device holds (the count the model's plan was computed for).  Known once the
 * lattice has stepped: FDLBM_ERR_INVALID before its first step, for a NULL
 * plan, or for a lattice whose steps do not run on the streaming kernel. */
int fdlbm_get_stream_plan(fdlbm_t* h, int32_t* plan);

/* Write the current drho, ux, uy into device arrays (nx*ny floats each). */
int fdlbm_moments(fdlbm_t* h, float* drho, float* ux, float* uy);

/* Same into host arrays; waits for the copies. */
int fdlbm_moments_host(fdlbm_t* h, float* drho, float* ux, float* uy);

/* FP64 reductions over the lattice, computed on the device and returned in
 * the host array out (waits for the stream):
 *   FDLBM_REDUCE_MASS     out[0] = sum drho
 *   FDLBM_REDUCE_MOMENTUM out[0..1] = sum rho ux, sum rho uy
 *   FDLBM_REDUCE_ENERGY   out[0] = sum rho |u|^2 / 2
 *   FDLBM_REDUCE_MODE     args[0..1] = (m, n); out[0..1] = real and imaginary
 *                         parts of (1/(nx ny)) sum u_t exp(-i k.x), u_t the
 *                         velocity component along (-ky, kx)/|k|: the
 *                         correlation A(t) of Sec. 3-a (A/2 e^{i phase} for
 *                         one wave of amplitude A)
 *   FDLBM_REDUCE_MAXABS   out[0] = max |u|, out[1] = max |drho|
 * A non-finite value anywhere makes the call return FDLBM_ERR_DIVERGED. */
#define FDLBM_REDUCE_MASS 0
#define FDLBM_REDUCE_MOMENTUM 1
#define FDLBM_REDUCE_ENERGY 2
#define FDLBM_REDUCE_MODE 3
#define FDLBM_REDUCE_MAXABS 4
int fdlbm_reduce(fdlbm_t* h, int32_t what, const double* args, double* out);

/* ---- batches of lattices ------------------------------------------------------
 *
 * Many independent lattices (periodic, or channels with walls in y) of any
 * size (16 <= nx, ny <= max_side), each with its own relaxation rates and
 * force, stepped together by persistent FD-LBM kernels (the scheme of Sec. 2
 * with the streaming data path; a second kernel per step takes the lattices'
 * narrow last strips, see fdlbm_batch_set_narrow_strips); runs of up to 64
 * steps are captured once in a CUDA graph and replayed.  FP32 storage.  Slots are
 * added and removed between calls (continuous batching); each slot's state
 * lives in a caller-owned arena with 8 periodic ghost columns per row side.
 * Results equal those of a single-lattice handle with the same parameters
 * up to FP32 rounding. */
typedef struct fdlbm_batch_s fdlbm_batch_t;

typedef struct fdlbm_batch_params {
    int32_t scheme;        /* FDLBM_SCHEME_FD3 or FDLBM_SCHEME_FD5 (all slots)      */
    int32_t max_lattices;  /* number of slots                                      */
    int64_t arena_bytes;   /* device bytes for the slots' states (2 copies each)   */
    int32_t max_side;      /* largest nx or ny of a slot (sizes work lists, staging) */
    int32_t flags;         /* must be 0                                            */
} fdlbm_batch_params;

/* Workspace bytes for a batch (arena + descriptors + work list + staging),
 * 0 if the parameters are invalid. */
size_t fdlbm_batch_workspace_size(const fdlbm_batch_params* bp);

/* Create a batch on the current device; workspace is caller-owned device
 * memory (256-byte aligned, fdlbm_batch_workspace_size bytes), kept until
 * fdlbm_batch_destroy; stream: a cudaStream_t. */
int fdlbm_batch_create(const fdlbm_batch_params* bp, void* workspace, size_t workspace_bytes,
                       void* stream, fdlbm_batch_t** out);
/* Free the batch's host state and its captured graphs; never frees the
 * workspace (the caller's).  NULL is ignored. */
void fdlbm_batch_destroy(fdlbm_batch_t* b);

/* Reserve a slot for a lattice (p->scheme must be the batch's, storage F32);
 * *slot receives its index.  FDLBM_ERR_NOMEM if no slot or arena space. */
int fdlbm_batch_add(fdlbm_batch_t* b, const fdlbm_params* p, int32_t* slot);
/* Release a slot and its arena space. */
int fdlbm_batch_remove(fdlbm_batch_t* b, int32_t slot);
/* Initial state of a slot from device fields (as fdlbm_init) or modes (as
 * fdlbm_init_modes). */
int fdlbm_batch_init(fdlbm_batch_t* b, int32_t slot, const float* drho, const float* ux,
                     const float* uy);
int fdlbm_batch_init_modes(fdlbm_batch_t* b, int32_t slot, int32_t n_modes, const double* modes,
                           double mean_ux, double mean_uy);
/* Advance every slot by nsteps, or slot s by min(slot_steps[s], nsteps) when
 * slot_steps (host array of max_lattices counts) is given. */
int fdlbm_batch_step(fdlbm_batch_t* b, int64_t nsteps, const int64_t* slot_steps);
/* A slot's drho, ux, uy into device arrays (nx*ny floats each). */
int fdlbm_batch_moments(fdlbm_batch_t* b, int32_t slot, float* drho, float* ux, float* uy);
/* FP64 reductions of one slot, as fdlbm_reduce (host out; waits). */
int fdlbm_batch_reduce(fdlbm_batch_t* b, int32_t slot, int32_t what, const double* args,
                       double* out);
/* Wait for the batch's stream; reports a device-side timeout. */
int fdlbm_batch_sync(fdlbm_batch_t* b);
/* Tuning knobs (chosen by the autotuner in the Python layer): rows per work
 * item (>= 8), persistent CTAs (0 = one wave of resident CTAs), and the strip
 * form of each lattice's last strip: with narrow strips on (1) a last strip
 * of at most 56 columns runs on lanes of 2 columns (a warp covers 56 output
 * columns) instead of 4 (120), in a second kernel per step, so that fewer
 * columns are computed for the ones stored; off (0, the default): every strip
 * on 4-column lanes, one kernel per step.
 * Both forms compute the same populations in the same order (Sec. 2, Eq. 2).
 * Settings apply from the next fdlbm_batch_step.  FDLBM_ERR_INVALID for a
 * NULL handle or an out-of-range value. */
int fdlbm_batch_set_segment_rows(fdlbm_batch_t* b, int32_t rows);
int fdlbm_batch_set_grid(fdlbm_batch_t* b, int32_t ctas);
int fdlbm_batch_set_narrow_strips(fdlbm_batch_t* b, int32_t on);
/* Message of the batch's last failed call (owned by the batch; "NULL handle"
 * for b == NULL). */
const char* fdlbm_batch_last_error(const fdlbm_batch_t* b);
/* Kernel launches the batch has enqueued since creation (-1 for NULL). */
int64_t fdlbm_batch_launch_count(const fdlbm_batch_t* b);
/* Number of occupied slots (-1 for NULL). */
int32_t fdlbm_batch_count(const fdlbm_batch_t* b);

/* fdlbm_reduce_fields_static -- the reductions of fdlbm_reduce for callers
 * that cannot allocate device memory.
 *
 * The paper has no counterpart; this is a convenience of the library.  Some
 * callers may not call cudaMalloc at all (code that runs inside a memory
 * pool it does not own, a plug-in that is only handed the buffers it must
 * fill, a region being captured into a CUDA graph), so they cannot provide
 * the workspace that fdlbm_create needs.  This entry point takes fields they
 * already hold on the device -- drho, ux, uy, nx*ny floats each, row-major,
 * for instance written by fdlbm_moments -- and computes the same FP64 sums
 * as fdlbm_reduce without any handle, workspace or allocation.
 *
 *   what, args: as for fdlbm_reduce (FDLBM_REDUCE_*; args = (m, n) for MODE).
 *   out: DEVICE pointer to 4 doubles, written asynchronously on `stream`:
 *        out[0..1] as fdlbm_reduce's out, out[2] = 0, out[3] = number of
 *        nodes holding a non-finite value (the caller checks it).
 *   stream: a cudaStream_t (NULL = the legacy default stream).
 *
 * Scratch: the per-block partial sums live in one fixed 32 KiB device array
 * inside the library; every GPU on which the library is loaded keeps it
 * until the process exits.  The first call on each device looks up that
 * array's device address (cudaGetSymbolAddress), so make the first call on a
 * device before capturing its stream into a CUDA graph.  All calls on a
 * device share the array and it keeps the last call's contents: calls
 * ordered on one stream are correct, calls that overlap on the GPU (other
 * streams, unordered host threads) race on it and give wrong results.
 * Device: the work runs on the current CUDA device; drho, ux, uy and out
 * must be device memory of that device (or managed memory), else the call
 * returns FDLBM_ERR_INVALID before any work is enqueued.
 * Limits: nx, ny >= 1 and nx*ny <= FDLBM_STATIC_REDUCE_MAX_NODES; anything
 * else returns FDLBM_ERR_INVALID before any work is enqueued.  Returns
 * FDLBM_ERR_CUDA if a launch fails.  Never calls cudaMalloc or cudaFree. */
#define FDLBM_STATIC_REDUCE_MAX_NODES (1LL << 30)
int fdlbm_reduce_fields_static(const float* drho, const float* ux, const float* uy, int32_t nx,
                               int32_t ny, int32_t what, const double* args, double* out,
                               void* stream);

/* Wait for all work enqueued by this handle. */
int fdlbm_sync(fdlbm_t* h);

/* Text of the last error on this handle ("" if none); valid until the next
 * call on the handle.  fdlbm_status_string maps a status code to its name. */
/* Failure-detection self test (the paper has no counterpart): enqueue one
 * warp that waits on a device barrier nothing will complete, bounded by
 * `tries` polls (a poll may suspend the warp for a hardware-defined slice;
 * 1000 polls take well under a second).  On expiry it records
 * FDLBM_ERR_TIMEOUT in the handle's status word, as a step kernel does when
 * a bulk copy does not land in time, and returns; the next fdlbm_sync or
 * fdlbm_reduce returns FDLBM_ERR_TIMEOUT and clears the word.  Nothing is in
 * flight when the warp gives up, so the device stays usable.  Returns
 * FDLBM_OK once enqueued, FDLBM_ERR_INVALID for tries < 0. */
int fdlbm_selftest_wait_timeout(fdlbm_t* h, int32_t tries);

/* Message of the handle's last failed call (owned by the handle, valid
 * until its next call or destruction; "NULL handle" for h == NULL). */
const char* fdlbm_last_error(const fdlbm_t* h);
/* Name of a status code ("FDLBM_OK", "FDLBM_ERR_INVALID", ...; a static
 * string, "FDLBM_UNKNOWN_STATUS" for other values). */
const char* fdlbm_status_string(int status);

/* Number of kernel launches this handle has enqueued since creation. */
int64_t fdlbm_launch_count(const fdlbm_t* h);

#ifdef __cplusplus
}
#endif
#endif /* FDLBM_H */
