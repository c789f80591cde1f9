/*
 * dugks.h -- C ABI of the GB300 (sm_103a) two-phase DUGKS library.
 *
 * The library advances the discrete unified gas-kinetic scheme for immiscible
 * two-phase flows of Zhang, Yang & Guo (arXiv:1802.02868): two D2Q9 kinetic
 * equations, f for pressure and momentum and g for the Cahn-Hilliard order
 * parameter phi (Sec. 2.2, Eqs. bgkf, bgkg), on tensor-product finite-volume
 * meshes with per-column and per-row spacings.
 *
 * Conventions for every call:
 *  - All calls return an int status (dugks_status); nothing aborts or exits.
 *  - Host arrays are caller-owned, read or written during the call, and never
 *    retained.  Cell fields are row-major [ny][nx] doubles (x fastest); for a
 *    batch, instance k's cells follow those of instance k-1.
 *  - Device memory is owned by the library (cudaMalloc at create time, freed
 *    by dugks_destroy).  The stream is the caller's; all device work of a
 *    simulation is enqueued on it.
 *  - Argument errors return DUGKS_ERR_ARG before any device work.  CUDA errors
 *    return DUGKS_ERR_CUDA.  A single simulation whose state became non-finite
 *    is reported as DUGKS_ERR_NONFINITE by the next synchronising call.  In a
 *    batch, an instance that becomes non-finite is masked (its tiles are
 *    skipped from the next step on) and reported by dugks_batch_status only;
 *    the other instances continue.
 */
#ifndef DUGKS_H
#define DUGKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DUGKS_OK = 0,
    DUGKS_ERR_ARG = -1,
    DUGKS_ERR_CUDA = -2,
    DUGKS_ERR_NONFINITE = -3,
    DUGKS_ERR_OOM = -4,
    DUGKS_ERR_TIMEOUT = -5,
    DUGKS_ERR_UNSUPPORTED = -6
} dugks_status;

/* Boundary condition per axis: periodic, or bounce-back no-slip walls at both
   ends of the axis (Sec. 3.2 "no-slip", Sec. 3.4 "bounce-back"). */
typedef enum { DUGKS_BC_PERIODIC = 0, DUGKS_BC_WALL = 1 } dugks_bc;

/* Storage and arithmetic precision of the distributions. */
typedef enum { DUGKS_FP64 = 0, DUGKS_FP32 = 1 } dugks_precision;

/* Tensor-product mesh: dx[nx] column widths, dy[ny] row heights, all > 0
   (Sec. 2.2, cell volume |V| = dx*dy; Sec. 3.2 non-uniform mesh).  Copied at
   create time.  Wall axes need at least 2 cells. */
typedef struct {
    int nx, ny;
    const double *dx, *dy;
    int bc_x, bc_y; /* dugks_bc */
} dugks_mesh;

/* Model parameters (Sec. 2.1-2.2):
 *  phiA, phiB  order parameter of bulk fluids A and B (phiA != phiB);
 *  rhoA, rhoB  densities (Eq. oderrho), > 0;
 *  nuA, nuB    kinematic viscosities, mixed by Eq. mixvis, > 0;
 *  mobility    lambda of Eq. CH0, >= 0;  tau_g relaxation time of g (> 0),
 *              eta = lambda / (c_s^2 tau_g) (Eq. kineticandmobility);
 *  beta, kappa free-energy coefficients (Eqs. doublewell, chemicalpotential);
 *  gx, gy      body-force acceleration; F_b = (rho - rho_ref) (gx, gy);
 *  cfl         alpha of Eq. cfl, in (0, 1]; dt = cfl * min(dx, dy) / sqrt(2);
 *  precision   dugks_precision. */
typedef struct {
    double phiA, phiB, rhoA, rhoB, nuA, nuB, mobility, tau_g, beta, kappa, gx, gy, rho_ref, cfl;
    int precision;
} dugks_params;

typedef struct dugks_sim dugks_sim; /* opaque, library-owned */

/* Device memory from the caller: a caller that manages device memory itself
   (for instance through PyTorch's caching allocator) supplies the library's
   device memory.  The paper has no counterpart.  alloc(bytes, stream, ctx) returns device memory of at
   least `bytes` bytes, aligned to 256 bytes, usable on `stream` (the stream
   the sim was created with), or NULL; release(ptr, stream, ctx) returns it.
   The pair applies to the sims created after the call, for their whole life:
   their planes and tables, and the temporary buffers of dugks_autotune,
   dugks_adjoint and the diagnostics.  NULL, NULL restores cudaMalloc and
   cudaFree.  Passing only one of the two is DUGKS_ERR_ARG.  An alloc that
   returns NULL makes the call that needed the memory fail with
   DUGKS_ERR_OOM.  The setting is process-wide and not synchronised: set it
   before creating sims from several threads. */
typedef void *(*dugks_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dugks_free_fn)(void *ptr, void *stream, void *ctx);
int dugks_set_allocator(dugks_alloc_fn alloc, dugks_free_fn release, void *ctx);

/* Create one simulation on the current CUDA device; stream may be NULL (the
   legacy default stream).  Validates the mesh and parameters (ERR_ARG),
   allocates device state (ERR_OOM on failure) and uploads the geometry. */
int dugks_create(const dugks_mesh *mesh, const dugks_params *params, void *cuda_stream, dugks_sim **out);

/* Create a batch of n independent instances (uneven sizes allowed) advanced
   together, one launch per kernel per step.  All instances share the
   precision of params[0]. */
int dugks_batch_create(int n, const dugks_mesh *meshes, const dugks_params *params, void *cuda_stream,
                       dugks_sim **out);

void dugks_destroy(dugks_sim *sim);

/* Step 1 of the procedure (Sec. 2.2): set phi, u, p at the cell centres and
   the tracked distributions tilde = eq - dt/2 F (Eq. auxf a with the original
   distribution at equilibrium).  Host arrays of all cells; ux, uy, p may be
   NULL (zero).  Copies host -> device on the sim's stream and synchronises. */
int dugks_init(dugks_sim *sim, const double *phi, const double *ux, const double *uy, const double *p);

/* Steps 2-7 repeated nsteps times (Sec. 2.2; Eqs. relations1/2, fbar_h,
   original-function, microfluxf, updatef).  Asynchronous on the sim's stream;
   a non-finite state is reported by the next synchronising call. */
int dugks_step(dugks_sim *sim, long nsteps);

/* Macroscopic fields at the cell centres from the current state (Eqs. phi,
   oderrho, u, P).  Host outputs of all cells, each may be NULL.  Synchronises. */
int dugks_moments(dugks_sim *sim, double *phi, double *rho, double *ux, double *uy, double *p);

/* FP64 volume-weighted sums of phi and rho per instance (Eq. locallyconserved);
   arrays of n_instances doubles.  Synchronises. */
int dugks_conservation(dugks_sim *sim, double *sum_phi, double *sum_rho);

/* The sums of dugks_conservation without a synchronisation: enqueues the
   reduction and its copy on the sim's stream and returns.  When the stream
   has reached them, sums[2k] = sum |V| phi and sums[2k + 1] = sum |V| rho of
   instance k (a host array of 2 n_instances doubles).  `sums` must be
   page-locked (cudaHostAlloc or cudaHostRegister; pageable memory gives
   DUGKS_ERR_ARG, since its copy could not be asynchronous) and must not be
   read or freed before dugks_conservation_wait returns.  Steps enqueued
   after the call run behind it on the stream, so a caller can enqueue step
   k + 1 and then wait for the sums of step k while the GPU works.  The first
   call creates an event and a small page-locked status buffer, which
   dugks_destroy frees. */
int dugks_conservation_async(dugks_sim *sim, double *sums);

/* Wait (on an event, not the whole stream) until the sums of the latest
   dugks_conservation_async have landed; DUGKS_OK at once when none is
   pending.  A single simulation whose state was non-finite at that point
   returns DUGKS_ERR_NONFINITE, as dugks_conservation does. */
int dugks_conservation_wait(dugks_sim *sim);

/* Per-instance status (DUGKS_OK or DUGKS_ERR_NONFINITE) since creation or the
   last init; array of n_instances ints.  Synchronises. */
int dugks_batch_status(dugks_sim *sim, int *per_instance_status);

/* Hold instances of a batch still: paused[k] != 0 pauses instance k,
   0 resumes it (host array of n_instances ints).  A paused instance keeps its
   state through dugks_step while the others advance; dugks_moments,
   dugks_conservation and the diagnostics still report it.  dugks_init resumes
   every instance; dugks_adjoint refuses a batch with a paused instance
   (DUGKS_ERR_ARG).  Synchronises. */
int dugks_batch_set_paused(dugks_sim *sim, const int *paused);

/* Advance instance k by nsteps[k] >= 0 steps (host array of n_instances
   longs): the batch steps max(nsteps) times, each instance pausing once its
   count is reached, so that instances with different time steps (a CFL
   sweep) can be brought to the same time.  Instances paused before the call
   stay paused and keep their pause afterwards.  Synchronises between the
   segments of equal counts. */
int dugks_batch_step_each(dugks_sim *sim, const long *nsteps);

/* Time step dt of instance k (Eq. cfl). */
int dugks_dt(const dugks_sim *sim, int instance, double *dt);

/* Sizes: number of instances, total cells, and the state size in bytes. */
int dugks_info(const dugks_sim *sim, int *n_instances, long *n_cells, size_t *state_bytes);

/* Checkpoint: copy the tracked state (tilde f and g, all instances, FP64) to a
   host buffer of *bytes bytes ([2][9][cells] doubles, f first) or restore it.
   With buf == NULL, dugks_save only reports the size.  Synchronises. */
int dugks_save(dugks_sim *sim, void *buf, size_t *bytes);
int dugks_load(dugks_sim *sim, const void *buf, size_t bytes);

/* Adjoint (reverse-mode gradient) of L = sum over all cells of
   (phi_T - phi_target)^2, phi_T the order parameter after nsteps steps from
   the last dugks_init inputs (the forward step is Sec. 2.2's procedure, the
   gradient is its exact transpose).
   The forward run is replayed from the saved init inputs with a checkpoint of
   the state every ckpt_every steps; each segment is recomputed and swept
   backwards.  Outputs (host, each may be NULL): loss[n_instances],
   dL_dphi0[cells] (the gradient with respect to the initial phi field, u0 and
   p0 held fixed), dL_dkappa[n_instances], dL_dlambda[n_instances] (lambda =
   the mobility).  phi_target: host array of all cells.  Allocates its
   checkpoints and work planes for the duration of the call and synchronises;
   the simulation is left at the final forward state.  ERR_ARG if the sim was
   never initialised or an instance is paused (dugks_batch_set_paused). */
int dugks_adjoint(dugks_sim *sim, long nsteps, int ckpt_every, const double *phi_target, double *loss,
                  double *dL_dphi0, double *dL_dkappa, double *dL_dlambda);

/* Counts kernel launches issued by this sim (for the caller's accounting). */
int dugks_launch_count(const dugks_sim *sim, long *count);

/* Per-kernel timing with CUDA events on the sim's stream: enable (1) or
   disable (0).  While enabled every launch is bracketed by events; read the
   accumulated milliseconds and launch counts per kernel with
   dugks_kernel_times (arrays of DUGKS_NUM_KERNELS entries, names by
   dugks_kernel_name).  Synchronises on read. */
#define DUGKS_NUM_KERNELS 8
int dugks_set_timing(dugks_sim *sim, int enable);
int dugks_kernel_times(dugks_sim *sim, double *ms, long *launches);
const char *dugks_kernel_name(int k);

/* Algorithmic bytes one launch of kernel k moves per cell (for roofline
   accounting), for this sim's precision. */
int dugks_kernel_bytes_per_cell(const dugks_sim *sim, int k, double *bytes);

/* Shapes of the fused step.  Tiles, one tile of cells per thread block:
   0 = 32x8 cells on 256 threads, 1 = 32x4 on 128 threads,
   2 = 32x12 on 384 threads, 3 = 32x8 on 352 threads with the face fluxes in
   their own shared memory (two blocks per SM).  Strips, one thread block of
   288 threads marching up 32 columns in blocks of 32x8 cells (two blocks per
   SM): 4 = strips of 8 blocks, 5 = 16 blocks, 6 = 32 blocks.  Every shape
   computes the same scheme: on uniform periodic meshes the results agree bit
   for bit, elsewhere to rounding.  A new fused-step sim starts with shape 5
   when its meshes give at least 3 strips of 16 blocks per resident strip slot
   (2 per SM in FP32, 1 in FP64), else shape 4 when they give at least 2
   strips of 8 blocks per slot, else shape 0; a sim on the four-kernel step
   reports shape 0.  dugks_autotune times every shape on the sim's current state for
   `steps` steps each (CUDA events on the sim's stream), restores the state and
   the per-instance status after each trial, keeps the fastest shape and
   returns its index and time per step.  It allocates a temporary snapshot of
   the state (cudaMalloc) for the duration of the call and synchronises. */
#define DUGKS_NUM_TILE_SHAPES 7
int dugks_autotune(dugks_sim *sim, int steps, int *chosen, double *ms_per_step);
int dugks_set_tile_shape(dugks_sim *sim, int shape);
/* The shape a new fused-step sim of these meshes starts with (the rule above),
   without a device: nx, ny are host arrays of n_instances mesh sizes, n_sm the
   device's multiprocessor count (152 on GB300).  DUGKS_ERR_ARG for a null
   pointer, a size or count below 1, or an unknown precision. */
int dugks_default_tile_shape(const int *nx, const int *ny, int n_instances, int precision, int n_sm, int *shape);
int dugks_tile_shape(const dugks_sim *sim, int *shape, int *bx, int *by);
const char *dugks_tile_shape_name(int shape);

/* Number of instances that take the fused step's uniform periodic path: both
   axes periodic and every spacing of an axis equal (bit for bit).  Their
   geometry is one record per axis, so that path skips the per-position
   geometry reads and the wall branches; its results equal the general path's
   bit for bit.  A batch holding both kinds launches one kernel per kind each
   step.  Setting DUGKS_GENERAL_ONLY=1 in the environment before creation sends
   every instance through the general path. */
int dugks_uniform_instances(const dugks_sim *sim, int *n);

/* Diagnostics of the current state of every instance, computed on the device
   (the paper's test quantities; c = (phi - phiB)/(phiA - phiB)).  FP64 sims
   work in FP64; FP32 sims form the cell quantities and each 32 x 64 strip's
   sums in FP32 and add the strips in FP64; the results are FP64:
     mass        total volume of the cells with c > 1/2: the droplet mass of
                 Sec. 3.1, Table A1 (a cell count on a unit mesh)
     xc, yc      centroid of that region (coordinates with the low faces at
                 0, no unwrapping across periodic boundaries), Sec. 3.3
     ux, uy      its volume-weighted mean velocity (the rise velocity of a
                 bubble), Sec. 3.3
     p_bulk_A/B  volume-weighted mean of the Laplace pressure P over the cells
                 with c > 0.9 / c < 0.1; their difference is the pressure jump
                 of Laplace's law, Sec. 3.1
     front_y, tip_y  highest and lowest height at which c crosses 1/2 going up
                 a column (c < 1/2 below, >= 1/2 above, linear interpolation
                 between the two centres; pairs across a periodic y boundary
                 excluded): with fluid A on top, the bubble front and the spike
                 tip of the Rayleigh-Taylor instability, Sec. 3.4
   Undefined entries (an empty region, no crossing, a masked instance) are
   NaN.  out holds n_instances entries (host memory).  Allocates a small
   device buffer on the first call; synchronises. */
typedef struct {
    double mass, xc, yc, ux, uy, p_bulk_A, p_bulk_B, front_y, tip_y;
} dugks_diag;
int dugks_diagnostics(dugks_sim *sim, dugks_diag *out);

/* The Laplace pressure field of Sec. 3.1, P = p0 - kappa phi lap(phi)
   + kappa |grad phi|^2 / 2 + p with p0 = phi psi' - psi and
   psi = beta (phi - phiA)^2 (phi - phiB)^2, on the device in the sim's
   precision (returned as FP64); the gradients use the stencils of Eqs.
   (nonphi), (nonphi2) with mirror ghosts at walls.  P (host) holds all instances' cells, row-major, in instance
   order.  Synchronises. */
int dugks_laplace_pressure(dugks_sim *sim, double *P);

const char *dugks_status_str(int status);

/* Arithmetic throughput of the current device, for roofline accounting of the
   fused step.  The paper has no counterpart.  Runs three FMA-only kernels on
   cuda_stream (8 blocks of 256 threads per SM, 8 independent FMA chains per
   thread): FP32 scalar FMAs for iters_f32 rounds, FP32 packed two-lane FMAs
   (the form the step uses for its f/g pairs) for iters_f32 / 2 rounds, FP64
   FMAs for iters_f64 rounds.  Each kernel runs twice and the second launch is
   timed with CUDA events; FMA = 2 flop.  Outputs (host): TFLOP/s of each.
   Allocates no device memory and writes none; synchronises.  ERR_ARG for
   iteration counts below 1 or NULL outputs. */
int dugks_measure_alu_peaks(int iters_f32, int iters_f64, double *fp32_tflops, double *fp32x2_tflops,
                            double *fp64_tflops, void *cuda_stream);

/* Allocation-free FP64 conservation sums of one mesh.  The paper has no
   counterpart; this exists for callers that cannot allocate device memory,
   such as a host loop under a device-memory budget owned by another allocator
   (a cudaMalloc there can fail or fragment that allocator's pool) or a
   latency-critical loop that cannot accept the device synchronisation of
   cudaMalloc/cudaFree.
   Inputs, all device pointers owned by the caller: phi[ny][nx] (dense, x
   fastest), dx[nx], dy[ny]; phiA, phiB, rhoA, rhoB as in dugks_params.
   Output: out[0] = sum |V| phi, out[1] = sum |V| rho(phi) (device pointer to
   two doubles), written on cuda_stream (NULL = legacy default stream).
   The call allocates nothing: its scratch (one partial pair per 4096 cells) is
   a file-scope device array of DUGKS_STATIC_MAX_CELLS / 4096 pairs (64 KiB)
   that every GPU loading this library holds until the process exits.  Meshes
   with more than DUGKS_STATIC_MAX_CELLS cells are rejected with DUGKS_ERR_ARG
   before any device work.  The first call on a device looks up the scratch
   array's device address (cudaGetSymbolAddress, with that device current);
   make that first call before any stream capture.  The address is kept for
   the life of the process: after a cudaDeviceReset (which unloads this
   library's device code from that device) it is stale, so do not call this
   entry point on a device that was reset since its first call.  Every call overwrites the
   scratch slots it uses, so no state carries over, but all calls share the one
   array: calls whose kernels overlap on the GPU (different streams, or
   different host threads) race and must be serialised by the caller. */
#define DUGKS_STATIC_MAX_CELLS 16777216
int dugks_conservation_static(const double *phi, const double *dx, const double *dy, int nx, int ny, double phiA,
                              double phiB, double rhoA, double rhoB, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DUGKS_H */
