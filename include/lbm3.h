/*
 * lbm3.h -- C ABI of the GB300 (sm_103a) three-phase MRT colour-gradient lattice Boltzmann
 * step with the characteristic-line wetting condition on curved walls
 * (arXiv:2102.04709, Section II).
 *
 * One handle owns one D2Q9 simulation on one GPU.  Every call that touches the GPU is
 * enqueued on the handle's CUDA stream; calls that return host data synchronise that
 * stream.  Plain pointers and sizes only.  All functions return an int status:
 *   0 = OK, > 0 = warning (the call did its work), < 0 = error (see lbm3_last_error).
 *
 * Layout conventions (all host arrays, row-major, node index i = y * nx + x):
 *   solid mask       uint8  [ny][nx]            1 = solid node (the paper's C_S), 0 = fluid (C_F)
 *   wall angles      double [ny][nx][3]         (theta_01, theta_20, theta_12) in degrees, i.e.
 *                                               the paper's (theta_rg, theta_br, theta_gb) of Eq.(17);
 *                                               theta_kl is measured inside fluid k; only values at
 *                                               solid nodes that touch fluid (C_SB) are read
 *   densities        double [3][ny][nx]         rho_k of fluids 0, 1, 2 (the paper's red, green, blue)
 *   velocity         double [2][ny][nx]         (u_x, u_y)
 * Fluid indices 0, 1, 2 are the paper's r, g, b.  Pure-fluid densities are 1 (the method is
 * limited to equal densities, Section II.A).
 */
#ifndef LBM3_H
#define LBM3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3 lbm3;

/* status codes */
#define LBM3_OK 0
#define LBM3_WARN_YOUNG 1        /* wall angles violate Eq.(18) by more than 1e-6 (work done) */
#define LBM3_ERR_INVALID (-1)    /* bad argument or unsupported geometry */
#define LBM3_ERR_CUDA (-2)       /* a CUDA call failed */
#define LBM3_ERR_OOM (-3)        /* device allocation failed */
#define LBM3_ERR_DIVERGED (-4)   /* non-finite or non-positive density found by lbm3_diag */
#define LBM3_ERR_STATE (-5)      /* call out of order (e.g. lbm3_step before lbm3_set_fields) */
#define LBM3_ERR_TOO_LARGE (-6)  /* grid larger than lbm3_diag_fields accepts */

/* x boundary (bc_x) */
#define LBM3_BC_PERIODIC 0       /* periodic */
#define LBM3_BC_MODPER 1         /* modified periodic, Section III.C: populations and phase
                                    fields crossing the x seam swap fluids 0 and 2;
                                    requires sigma_01 == sigma_12 */
#define LBM3_BC_ZOUHE 2          /* Zou-He velocity inlet (u_in, 0) at x = 0 and pressure outlet
                                    rho = rho_out at x = nx-1, Section III.D; requires periodic y
                                    and no solid node in the first/last 4 columns */
#define LBM3_BC_WALLS 3          /* columns 0 and nx-1 must be solid */

/* population storage (precision) */
#define LBM3_FP32 0              /* 27 FP32 populations per node */
#define LBM3_FP16 1              /* per fluid: FP32 rho_k + 8 FP16 offsets f_ak - w_a rho_k */
#define LBM3_BF16 2              /* per fluid: FP32 rho_k + 8 BF16 offsets f_ak - w_a rho_k */

typedef struct lbm3_grid {
    int32_t nx, ny;        /* grid size, nx >= 8, ny >= 8, 27 * nx * ny < 2^31 */
    int32_t periodic_y;    /* 1: periodic in y; 0: rows 0 and ny-1 must be solid */
    int32_t bc_x;          /* LBM3_BC_* */
    double u_in;           /* inlet velocity for LBM3_BC_ZOUHE (|u_in| < 0.3) */
    double rho_out;        /* outlet density for LBM3_BC_ZOUHE (> 0) */
    int32_t precision;     /* LBM3_FP32 / LBM3_FP16 / LBM3_BF16 */
} lbm3_grid;

/* Create a simulation.  Classifies nodes into C_FI, C_FB, C_SB, C_SI (Section II.B, any of the
 * 8 D2Q9 neighbours counts as contact), computes the outward solid normal at every C_SB node
 * with the eighth-order isotropic stencil of Eq.(19)-(20), builds the compact wall list and
 * allocates device memory (owned by the handle).  All host inputs are copied.
 *   sigma  = (sigma_01, sigma_02, sigma_12), interfacial tensions of Eq.(10), > 0
 *   nu     = kinematic viscosity of each pure fluid, > 0 (mixture by Eq.(7))
 *   beta0  = reference segregation parameter of Eq.(14) (the paper uses 0.7)
 *   stream = cudaStream_t (NULL = legacy default stream) on which all work is enqueued
 * Returns LBM3_WARN_YOUNG if an angle triple at a C_SB node violates Eq.(18); *out is valid
 * for any status >= 0 and NULL otherwise. */
int lbm3_create(lbm3** out, const lbm3_grid* grid, const uint8_t* solid_mask,
                const double* wall_angles_deg, const double sigma[3], const double nu[3],
                double beta0, void* stream);

/* Initialise every fluid node at rest: f_ak = w_a rho_k (Eq.3 with u = 0), as a post-streaming
 * state (open boundaries completed by Zou-He).  The wall values that Eq.(21) reads in the first
 * step are the w-weighted means of each C_SB node's fluid neighbours.  rho: host [3][ny][nx]. */
int lbm3_set_fields(lbm3* h, const double* rho);

/* Advance nsteps >= 0 timesteps (Eq.1-22), asynchronously on the handle's stream.  Each step is
 * the wetting pass over the C_SB list (Eq.21-22) and the fused step kernel (Eq.1-16: densities,
 * gradients, interfacial force, MRT collision, recolouring, streaming with halfway bounce-back
 * and the x boundary).  Tiles with no solid node within 3 nodes run concurrently with the wetting
 * pass on the handle's stream (through bulk tensor copies when nx is a multiple of 4, on the SMs
 * that the other tiles' share of the work leaves); the other tiles follow the wetting pass on an
 * internal higher-priority stream that is joined back before the call's work completes.  The
 * velocity of the last collision of the call is recorded for lbm3_fields / lbm3_diag.  A bulk
 * copy that does not complete within its wait limit is reported by the next lbm3_diag.  While more
 * than 8 steps remain, blocks of 8 steps are launched as one CUDA graph, captured on an internal
 * stream the first time it is needed (one graph per starting population buffer) and replayed on
 * the handle's stream: the same kernels in the same order, so the results do not depend on how
 * steps are split between calls.  If a capture fails the steps are launched one by one. */
int lbm3_step(lbm3* h, int32_t nsteps);

/* lbm3_step with per-launch timing: CUDA events are recorded around every launch on the stream
 * it runs on; after the last step the call synchronises and writes the summed times in ms:
 * ms_out[0] = wetting pass, ms_out[1] = fused step kernel on the pure tiles (no solid within
 * 3 nodes; main stream), ms_out[2] = fused step kernel on the other tiles (side stream, after the
 * wetting pass).  The pure-tile launch overlaps the other two. */
int lbm3_step_timed(lbm3* h, int32_t nsteps, double ms_out[3]);

/* lbm3_step_timed with the other tiles split by kind: ms_out[0] = wetting pass, ms_out[1] = pure
 * tiles, ms_out[2] = wall tiles (solids within 3 nodes, halo inside the domain), ms_out[3] = edge
 * tiles (halo crossing the domain edge; on a second internal stream, those with no solid within
 * 3 nodes from the start of the step, the others once the wetting pass is done), summed over the
 * steps in ms, and ms_out[4] = the device time of the whole run, from the event before the first
 * step's first launch to one recorded after the last step (the host's read-back of the events
 * after the run is outside it).  Synchronises.  lbm3_step_timed's ms_out[2] is the sum of
 * ms_out[2] and ms_out[3]. */
int lbm3_step_timed_detail(lbm3* h, int32_t nsteps, double ms_out[5]);

/* Copy the current post-streaming densities rho_k (host [3][ny][nx], 0 at solid nodes) and the
 * velocity of the most recent collision, Eq.(11) (host [2][ny][nx], may be NULL).  Synchronises.
 * Returns LBM3_ERR_CUDA (with the arrays filled) if a step kernel gave up on a bulk copy since the
 * error was last reported (see lbm3_set_copy_wait_limit). */
int lbm3_fields(lbm3* h, double* rho_out, double* u_out);

/* Diagnostics of the current state, accumulated in FP64 on the GPU:
 * out[0..2] = sum of rho_k over fluid nodes, out[3] = sum x rho_0, out[4] = sum y rho_0,
 * out[5] = max |u| of the last collision, out[6] = min rho, out[7] = count of non-finite rho_k.
 * Returns LBM3_ERR_DIVERGED (with out filled) if out[7] > 0 or out[6] <= 0, and LBM3_ERR_CUDA if
 * a step kernel gave up on a bulk copy since the error was last reported.  Synchronises. */
int lbm3_diag(lbm3* h, double out[8]);

/* Number of C_SB nodes (the wall list) and their node indices, in increasing order
 * (cap = capacity of idx; returns the count or a negative status). */
int lbm3_n_wall(const lbm3* h);
int lbm3_wall_nodes(const lbm3* h, int32_t* idx, int32_t cap);

/* Wall values C_0, C_1, C_2 at the C_SB nodes (in lbm3_wall_nodes order) as of the last wetting
 * pass (before any step: the initial fluid-neighbour means); c: host [cap][3].  Returns the
 * number of wall nodes or a negative status.  Synchronises. */
int lbm3_wall_values(lbm3* h, double* c, int32_t cap);

/* Checkpoint / resume.  The state of a simulation is its post-streaming populations
 * f_post [3][9][ny][nx] (fluid k, direction a; 0 at solid nodes) and the wall values
 * wall_c [3][ny][nx] that the next wetting pass reads in Eq.(21) (used at C_SB nodes only).
 * lbm3_get_state copies both to host memory (synchronises); lbm3_set_state replaces the state
 * (the populations of directions entering from an open side are recomputed by Zou-He). */
int lbm3_get_state(lbm3* h, double* f_post, double* wall_c);
int lbm3_set_state(lbm3* h, const double* f_post, const double* wall_c);

/* Replace the wall-angle triples (theta_01, theta_20, theta_12) in degrees of every C_SB node,
 * host [n_wall][3] in lbm3_wall_nodes order (each in (0, 180)). */
int lbm3_set_wall_angles(lbm3* h, const double* angles_deg);

/* Replace the Zou-He inlet velocity (|u_in| < 0.3; LBM3_BC_ZOUHE only).  A new value drops the
 * captured CUDA graphs of lbm3_step and of the adjoint (they hold it); the same value keeps them. */
int lbm3_set_inflow(lbm3* h, double u_in);

/* Adjoint (reverse-mode) gradient.  Runs nsteps timesteps from the current state, evaluates
 * J = sum_x x rho_0(x) / sum_x rho_0(x), the x-centroid of fluid 0 over the post-streaming fluid
 * nodes of the final state, and returns dJ/d(theta_01, theta_20, theta_12) for every C_SB node
 * (host [n_wall][3], lbm3_wall_nodes order) and dJ/du_in (0 unless LBM3_BC_ZOUHE).  The states
 * at every checkpoint_every-th step are kept on the device, and the forward pass keeps every
 * state of the last segment; each other segment is recomputed forward by the step kernels from
 * its checkpoint, and every segment is then traversed backward by the adjoint kernels
 * (vector-Jacobian products of Eq.1-16, 21, 22 and the characteristic lines, FP32 with FP64
 * accumulators).  checkpoint_every >= nsteps keeps every state and recomputes nothing.
 * FP32 storage only, not with LBM3_BC_MODPER.  On return the simulation holds its final state.
 * Device memory: about nsteps / checkpoint_every + min(checkpoint_every, nsteps) states (132 B
 * per node each) plus ~300 B per node of work arrays, allocated by the first call that needs
 * them and kept in the handle for later calls that need no more (an optimisation loop calls it
 * once per iteration); lbm3_adjoint_release or lbm3_destroy releases it.  The first call of a
 * given nsteps / checkpoint_every also records the whole sweep as a CUDA graph, which later such
 * calls replay (dropped with the store, or when lbm3_set_inflow / lbm3_set_copy_wait_limit
 * change a captured parameter).  Synchronises. */
int lbm3_adjoint_centroid(lbm3* h, int32_t nsteps, int32_t checkpoint_every, double* J_out,
                          double* dJ_dangles, double* dJ_du);

/* Release the device memory that lbm3_adjoint_centroid keeps in the handle (nothing if none).
 * Synchronises. */
int lbm3_adjoint_release(lbm3* h);

/* Size facts: out[0] = fluid nodes, out[1] = C_SB nodes, out[2] = algorithmic HBM bytes of the
 * fused step per timestep (216 B per fluid node with FP32 storage, 120 B with 16-bit offsets,
 * + 1 class byte per node), out[3] = fused-step launches per timestep, out[4] = wetting launches
 * per timestep, out[5] = device bytes held by the handle, out[6] = algorithmic bytes of the
 * pure-tile launch, out[7] = nodes in pure tiles, out[8] = how the pure tiles move their
 * populations: 0 plain loads, 1 bulk tensor copies with two blocks per SM, 2 bulk tensor copies
 * through the warp-specialised ring (FP32 storage; LBM3_PURE_KERNEL=tma in the environment at
 * lbm3_create selects 1 instead).  Bulk copies need nx a multiple of 4 (FP32) or 8 (16-bit
 * offsets) and are disabled by LBM3_DISABLE_TMA=1. */
int lbm3_info(const lbm3* h, int64_t out[9]);

/* Change the stream used by later calls (cudaStream_t).  Work already enqueued by the handle
 * on the old stream is ordered before the work of later calls on the new one (an event recorded
 * on the old stream that the new stream waits for). */
int lbm3_set_stream(lbm3* h, void* stream);

/* Failure detection.  The pure-tile kernels move each tile's populations with bulk tensor copies
 * that complete on an mbarrier; a block polls it at most `polls` times (default 4194304, a few
 * seconds; polls < 0 restores the default) before it gives up: it sets an error bit, waits (with
 * the full default limit) for the copies it has in flight and returns without writing its
 * tiles.  lbm3_fields, lbm3_diag and lbm3_adjoint_centroid then return LBM3_ERR_CUDA once (the
 * bit is cleared when reported, and by lbm3_set_fields / lbm3_set_state, which replace the state
 * whose tiles were skipped).  polls = 0 makes every wait give up at once, which is how the error
 * path is tested without faulting or hanging anything.  The paper has no counterpart. */
int lbm3_set_copy_wait_limit(lbm3* h, int32_t polls);

/* Block until all work enqueued by the handle is done. */
int lbm3_sync(lbm3* h);

/* Release all device memory of the handle (NULL is ignored). */
void lbm3_destroy(lbm3* h);

/* Allocation-free diagnostics of caller-owned device fields.  The paper has no counterpart:
 * this is the reduction of lbm3_diag (same out[0..7], same FP64 accumulation) applied to fields
 * that the caller already holds on the device, for callers that must not allocate at the call:
 * a monitor running inside a host framework whose caching allocator has reserved the device's
 * memory (a cudaMalloc there can fail, and a cudaFree synchronises the device), or a loop that
 * must not synchronise.  The call allocates nothing on the device or the host: the block
 * partials live in one fixed device array of LBM3_DIAG_FIELDS_MAX_BLOCKS x 8 doubles (64 KiB)
 * inside the library, and the reduction strides over the grid with at most that many blocks,
 * so any grid up to LBM3_DIAG_FIELDS_MAX_NODES nodes fits; larger grids return
 * LBM3_ERR_TOO_LARGE without launching anything.  Nothing in that array has to start at zero
 * (each block writes its partials before the final pass reads them).
 *   rho    device float [3][ny][nx]  densities rho_k (e.g. lbm3_fields' output, in FP32)
 *   u      device float [2][ny][nx]  velocity (u_x, u_y)
 *   solid  device uint8 [ny][nx]     1 = solid node (skipped), 0 = fluid
 *   out    device double [8]         written when the enqueued work completes
 *   stream cudaStream_t (NULL = legacy default stream) of the current device, which must be the
 *          device holding the four buffers
 * The call only enqueues two kernels and returns: it does not synchronise and does not check
 * the results for divergence.  Ownership of every buffer stays with the caller.  The first call
 * on each device looks up the address of the fixed array (cudaGetSymbolAddress) once, with that
 * device current; callers that begin stream capture make that first call before the capture
 * starts.  Calls that overlap in time on the same device (on different streams, or from
 * different threads without ordering) share the array and race; calls ordered on one stream do
 * not.  Returns LBM3_ERR_INVALID for a NULL pointer or nx, ny <= 0, LBM3_ERR_TOO_LARGE for
 * nx * ny > LBM3_DIAG_FIELDS_MAX_NODES, LBM3_ERR_CUDA if the lookup or a launch fails. */
#define LBM3_DIAG_FIELDS_MAX_BLOCKS 1024
#define LBM3_DIAG_FIELDS_MAX_NODES 2147483647LL
int lbm3_diag_fields(const float* rho, const float* u, const uint8_t* solid, int32_t nx,
                     int32_t ny, double* out, void* stream);

/* Text of the last error or warning of the handle (or of the last failed lbm3_create when
 * h == NULL). Valid until the next call on the same handle. */
const char* lbm3_last_error(const lbm3* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM3_H */
