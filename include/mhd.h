/*
 * mhd.h - C ABI of the GB300 relaxing-TVD ideal-MHD solver.
 *
 * Method: Wong, Wong, Feng & Tang, "Efficient magnetohydrodynamic simulations on graphics
 * processing units with CUDA" (arXiv:0908.4362).  The solver advances the ideal MHD
 * equations (Sect. 3, equations of the conservation laws, mu = 1) on a regular Cartesian
 * grid with the relaxing-TVD scheme (Sect. 3), constrained transport for B (Sect. 3,
 * Eqs. "eq:averaging_x", "eq:first_flux"), dimensionally split forward and reverse sweeps
 * with a cycled axis order (Eq. "eq:L_sequence"), and a CFL time step (Eq. "equat_CFL").
 * All arithmetic runs in the library's CUDA kernels on one GPU (sm_103a).
 *
 * Conventions shared by every entry point
 *   Fields      8 arrays in the order (rho, rho*vx, rho*vy, rho*vz, E, Bx, By, Bz)
 *               (Sect. 4.1, "eight components ... stored in eight arrays").
 *   Index       cell (x, y, z) is element (x*ny + y)*nz + z of each array: z is contiguous
 *               (Sect. 4.1, index equations).
 *   Staggering  B is face centred (Eq. "equat_b"): Bx[x,y,z] lives on the x-face x-1/2,
 *               By on the y-face y-1/2, Bz on the z-face z-1/2.  Cell width h on all axes.
 *   Boundaries  per axis, periodic (wrap) or outflow (every array index clamped to the
 *               grid, i.e. zero-gradient ghost cells).  The paper does not specify them.
 *   Step        one step = dt from the CFL condition, forward sweep L_c L_b L_a and
 *               reverse sweep L_a L_b L_c, t += 2 dt, axis order (a,b,c) cycled over
 *               (x,y,z), (z,x,y), (y,z,x) (Sect. 4.2 steps 4-8, Eq. "eq:L_sequence").
 *   Ownership   the context owns all device memory; host and device buffers passed in are
 *               owned by the caller, only read or written during the call (or, for the
 *               asynchronous calls, until the context's stream reaches that point).
 *   Errors      every call returns a status and never aborts.  Device-side problems
 *               (rho <= 0, a negative fast-speed radicand, non-finite values, bad dt) are
 *               sticky bits in the context, reported by the next call that synchronises
 *               (mhd_read, mhd_sums, mhd_state, mhd_step with a non-NULL out pointer).
 *   Threads     a context may be used from one host thread at a time.
 */
#ifndef MHD_GB300_H
#define MHD_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_ctx mhd_ctx;

typedef enum {
  MHD_OK = 0,
  MHD_ERR_INVALID = 1,     /* bad argument or configuration */
  MHD_ERR_OOM = 2,         /* device allocation failed */
  MHD_ERR_CUDA = 3,        /* a CUDA call failed (the message is in mhd_last_error) */
  MHD_ERR_UNPHYSICAL = 4,  /* rho <= 0, NaN/Inf, or gamma p/rho + B^2/rho < 0 seen */
  MHD_ERR_TIMEOUT = 5      /* a bounded device wait gave up (batched form) */
} mhd_status;

typedef enum { MHD_BC_PERIODIC = 0, MHD_BC_OUTFLOW = 1 } mhd_bc;
typedef enum { MHD_FP32 = 0, MHD_FP64 = 1 } mhd_precision;
/* How the FP32 sweeps recover the pressure p = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2) (the
 * equation of state of Sect. 3), which cancels when the plasma beta is low: plain FP32, FP64
 * arithmetic, or compensated FP32 (error-free sums and products carry the rounding errors
 * of the two quadratic terms and of the subtractions: the exactly rounded p of the FP32
 * inputs, as FP64 gives it, at FP32 speed).  Selected by mhd_config.fp64_pressure. */
typedef enum { MHD_PRESSURE_FP32 = 0, MHD_PRESSURE_FP64 = 1, MHD_PRESSURE_COMPENSATED = 2 }
    mhd_pressure_mode;

typedef struct {
  int nx, ny, nz;        /* cells per axis, each >= 1 */
  double h;              /* cell width, > 0 (the paper uses h = 1) */
  double gamma;          /* ratio of specific heats, > 1 */
  double cfl;            /* Courant number, 0 < cfl < 1 (paper: ~0.7) */
  int bc[3];             /* mhd_bc per axis */
  int prec;              /* mhd_precision of the device state and arithmetic */
  int fp64_pressure;     /* mhd_pressure_mode of the pressure recovery; FP64 contexts: 0 */
  void* cuda_stream;     /* cudaStream_t to run on; NULL: the context creates its own */
} mhd_config;

/* Validate cfg and create a context: device state (two buffers per field, the ping-pong
 * of the out-of-place sweeps), step scalars and scratch.  *out is NULL on failure.
 * The state is undefined until mhd_init_fields or mhd_upload. */
mhd_status mhd_create(const mhd_config* cfg, mhd_ctx** out);

/* Load the state from 8 host arrays of nx*ny*nz doubles (copied; converted to the
 * context precision), set t = t0, step = 0, phase = 0, clear the status and compute the
 * CFL speed of the new state (Sect. 4.2 steps 2-4).  Blocking. */
mhd_status mhd_init_fields(mhd_ctx* ctx, const double* const f[8], double t0);

/* As mhd_init_fields, from 8 arrays of dtype (0 = float32, 1 = float64) in host memory
 * (on_device = 0; page-locked host memory copies at full link speed) or device memory
 * (on_device = 1).  Blocking. */
mhd_status mhd_upload(mhd_ctx* ctx, const void* const f[8], int dtype, int on_device, double t0);

/* Advance up to nsteps steps (Sect. 4.2 steps 4-9).  t_end < 0: exactly nsteps steps,
 * enqueued on the context's stream without a host synchronisation (CUDA-graph replays).
 * t_end >= 0: stop once t reaches t_end; the last dt is clipped so that t lands on t_end
 * exactly; the call synchronises periodically to watch t.  If steps_done or t_now is
 * non-NULL the call synchronises at the end and reports the steps taken and the time. */
mhd_status mhd_step(mhd_ctx* ctx, int nsteps, double t_end, int* steps_done, double* t_now);

/* Apply one sweep operator with a given dt, for testing: op 0 = fluid_axis (Algorithm 1),
 * op 1 = CT along axis for both transverse components (Algorithm 2), op 2 = CT along axis
 * twice (the pair of CT operators that meet in the middle of a step whose axis order ends
 * with that axis, Eq. "eq:L_sequence": one launch where the library has a two-pass kernel,
 * else two; the same result as op 1 applied twice), op 3 = the reverse L along z (CT along
 * z, then the fluid sweep along z, Sect. 4.3) in one launch: axis 2, FP32 contexts with
 * plain FP32 pressure recovery and a z axis of more than one cell only (MHD_ERR_INVALID
 * otherwise, the state left as it was); the same result as op 1 then op 0, measured slower
 * than those two launches and not used by mhd_step.  Returns after the operator completed. */
mhd_status mhd_apply(mhd_ctx* ctx, int op, int axis, double dt);

/* c_max of the current state (Eq. "equat_CFL").  Blocking. */
mhd_status mhd_cmax(mhd_ctx* ctx, double* cmax);

/* Copy the state to 8 host arrays of nx*ny*nz doubles.  Blocking; returns the sticky
 * status. */
mhd_status mhd_read(mhd_ctx* ctx, double* const f[8]);

/* As mhd_read, into 8 arrays of dtype in host (on_device = 0) or device (1) memory.
 * Blocking. */
mhd_status mhd_download(mhd_ctx* ctx, void* const f[8], int dtype, int on_device);

/* FP64 sums over all cells of the 8 fields (conservation diagnostics; the periodic sums
 * of rho, m, E and of each face component of B are invariants of the scheme).  Blocking. */
mhd_status mhd_sums(mhd_ctx* ctx, double out[8]);

/* Checkpoint scalars: time, dt of the last step, steps taken, axis-order phase (0..2).
 * Together with mhd_read they are a complete checkpoint.  Blocking. */
mhd_status mhd_state(mhd_ctx* ctx, double* t, double* dt_last, int* step, int* phase);

/* Restore checkpoint scalars after mhd_init_fields/mhd_upload of the saved fields. */
mhd_status mhd_set_state(mhd_ctx* ctx, double t, int step, int phase);

/* Wait for the context's stream; returns the sticky status. */
mhd_status mhd_sync(mhd_ctx* ctx);

/* Number of cells and the device bytes the context holds (state, scalars, scratch). */
mhd_status mhd_info(const mhd_ctx* ctx, long long* ncells, long long* device_bytes);

/* Kernel timing mode (enable != 0): steps are launched kernel by kernel, without CUDA
 * graphs, with a CUDA event pair recorded on the context's stream around each kernel.
 * Off by default. */
mhd_status mhd_profile(mhd_ctx* ctx, int enable);

/* Accumulated kernel times (ms) and launch counts of the timing mode, by kind:
 * 0..2 fluid sweep along x, y, z; 3..5 CT along x, y, z; 6 dt kernel; 7 other.
 * Synchronises; reset != 0 clears the accumulators after reading. */
mhd_status mhd_profile_read(mhd_ctx* ctx, double ms[8], long long count[8], int reset);

/* The cudaStream_t the context runs on (its own, or the one given in mhd_config). */
mhd_status mhd_stream(const mhd_ctx* ctx, void** stream);

/* ---------------------------------------------------------------------------------------
 * Batched persistent form: many grids advanced together.
 *
 * A batch groups FP32 contexts (any shapes, each at its own time and axis-order phase).
 * mhd_batch_step advances every one of them by nsteps method steps (Sect. 4.2) in ONE
 * persistent, CUDA-graph-captured kernel launch: resident CTAs take (instance, operation,
 * tile) items from a device queue, and a per-instance completion counter makes each
 * operation of an instance wait for all tiles of its previous operation.  Each grid's
 * result is bit-identical to advancing it alone with mhd_step.  The contexts keep owning
 * their state; read them with mhd_read/mhd_download as usual.
 * ------------------------------------------------------------------------------------- */
typedef struct mhd_batch mhd_batch;

/* Create a batch over n contexts (FP32, fp64_pressure off, no t_end pending).  The
 * contexts must outlive the batch.  z_tile_warps: warp segments per work item of a z sweep
 * (0: chosen per sweep, about 1024 items, 4 to 128 segments each); ctas_per_sm: resident
 * CTAs per SM of the persistent launch (0: as many as fit).
 * Both are launch shapes only (results do not depend on them); the autotuner picks them. */
mhd_status mhd_batch_create(mhd_ctx* const* ctxs, int n, int z_tile_warps, int ctas_per_sm,
                            mhd_batch** out);

/* Enqueue nsteps steps of every context of the batch as one persistent launch, ordered
 * after each context's pending work; each context's later work waits for it.  The work
 * list and the graph are cached per (nsteps, phases); with nsteps a multiple of 3 every
 * call reuses them.  Contexts may also be stepped alone between batch launches: a context
 * whose buffers moved (mhd_step runs the middle CT pair of some steps as one launch, which
 * swaps the B buffers; mhd_apply) has its operations rebuilt, after the batch's previous
 * launch completed.  The batched steps run the middle pair as two launches, the same bits. */
mhd_status mhd_batch_step(mhd_batch* b, int nsteps);

/* As mhd_batch_step, with a step count per context: nsteps[i] >= 0 for each of the n
 * contexts (in creation order), at least one of them >= 1; a context with 0 is left as it
 * is.  Work items are queued step by step, so a context with more steps keeps advancing
 * after the others have finished within the same launch.  Used by a scheduler that gives
 * small grids many steps and large grids few in one launch.  The work list and graph are
 * cached for the last (counts, phases) key only.  MHD_ERR_INVALID for a negative count or
 * all counts 0. */
mhd_status mhd_batch_step_each(mhd_batch* b, const int* nsteps);

/* Wait for the batch.  MHD_ERR_TIMEOUT if a bounded device wait gave up: the launch then
 * stops early, the states of the contexts it advanced are incomplete, and each of those
 * contexts reports MHD_ERR_TIMEOUT from then on (mhd_step, mhd_read, ...) until it is
 * initialised again. */
mhd_status mhd_batch_sync(mhd_batch* b);

/* Launch shape of one context inside a batch.  Every field at 0 takes the default.  The
 * shapes change speed only: each choice gives the same bits as mhd_step.
 *   march_len  cells per work item along an x or y sweep (fluid and CT marching tiles,
 *              each with its halo of 6 or 8 cells recomputed): 128, 192 or 256 (0: 192)
 *   ct_march   1: x/y constrained transport as one marching pipeline per pencil, 0: with
 *              EMF rows shared between neighbouring pencils where the grid allows it
 *              (z extent >= 48 and at least 4 rows across)
 *   seg_k      z sweeps: cells per lane of a warp segment, 2 or 3 (0: from the z extent)
 *   z_warps    z sweeps: warp segments per work item, 1 .. 2^20 (0: the batch's
 *              z_tile_warps)
 *   alone      1: advance this context with the single-grid kernels (mhd_step, on the
 *              context's own stream) instead of inside the persistent launch */
typedef struct mhd_batch_shape {
  int march_len;
  int ct_march;
  int seg_k;
  int z_warps;
  int alone;
} mhd_batch_shape;

/* Set the launch shapes of a batch: threads per CTA of the persistent kernel (128 or 256;
 * the EMF rows of a shared-row CT tile are its warps; 0 keeps the current, initially 128),
 * resident CTAs per SM (0: as many as fit), the bound of each device wait in SM clock
 * cycles (1 .. 4e9; 0: 4e9, about 2 s) and, when shapes is not NULL, one mhd_batch_shape per
 * context in creation order (NULL: every context at the defaults).  Waits for the batch's
 * previous launch, rebuilds the work lists and drops the captured graphs.  MHD_ERR_INVALID
 * for a value out of range (nothing is changed then). */
mhd_status mhd_batch_configure(mhd_batch* b, int threads_per_cta, int ctas_per_sm,
                               long long spin_cycles, const mhd_batch_shape* shapes);

/* Resident CTAs of the persistent launch, work items per launch (0 before a step) and the
 * cudaStream_t the batch runs on (any pointer may be NULL). */
mhd_status mhd_batch_info(const mhd_batch* b, int* resident_ctas, long long* items_per_launch,
                          void** stream);

void mhd_batch_destroy(mhd_batch* b);

/* Diagnostic of the bounded device waits: launches the persistent kernel with one work item
 * that waits for a completion nothing produces.  The wait must give up after spin_cycles
 * SM clock cycles (1 .. 4e9) and the call returns MHD_ERR_TIMEOUT; the device stays usable. */
mhd_status mhd_batch_selftest_timeout(long long spin_cycles);

/* ---------------------------------------------------------------------------------------
 * Visualization without a graphics API (Sect. 8).  The paper maps the state into OpenGL
 * buffers (a vertex per cell for 1D problems, a pixel per cell of a 2D problem coloured by a
 * transfer function, a texture volume render for 3D).  These entry points write the same
 * products into caller-owned DEVICE buffers on the context's stream and synchronise; no
 * window or graphics context is involved.  The selected value q of a cell is one of
 * mhd_quantity, with B averaged from the faces to the cell centre and p = (gamma-1)(E -
 * |m|^2/(2 rho) - |B|^2/2); arithmetic is in the context's precision.
 *
 * Transfer function (the paper does not give one): s = (q - vmin)/(vmax - vmin) clamped to
 * [0, 1] (NaN to 0) is mapped linearly through five colour stops at s = 0, 1/4, 1/2, 3/4, 1:
 * (0,0,0.5), (0,0,1), (0,1,1), (1,1,0), (1,0,0).
 * Errors: MHD_ERR_INVALID for a bad quantity, axis, index, range or NULL pointer;
 * MHD_ERR_CUDA if a launch fails.
 * ------------------------------------------------------------------------------------- */
typedef enum { MHD_Q_RHO = 0, MHD_Q_P = 1, MHD_Q_E = 2, MHD_Q_VMAG = 3, MHD_Q_BMAG = 4 } mhd_quantity;

/* 1D grids (at most one axis longer than 1): xy[2j] = (j + 1/2) h, xy[2j+1] = q(j) for the n
 * cells of that axis (device pointer, 2n floats) -- the paper's vertex buffer. */
mhd_status mhd_vis_curve(mhd_ctx* ctx, int quantity, float* xy);

/* The plane of cells normal to `axis` at `index` as an RGBA8 image (device pointer,
 * w*h*4 bytes, alpha 255): image axes are the two other grid axes u < v, pixel (row v, column
 * u) at byte 4 (v w + u); each channel is round(255 x colour). */
mhd_status mhd_vis_slice(mhd_ctx* ctx, int quantity, int axis, int index, double vmin,
                         double vmax, unsigned char* rgba);

/* Orthographic emission-absorption ray cast along `axis`, one ray per cell column, front to
 * back (increasing index): with the cell's colour c and opacity a = clamp(opacity x s, 0, 1),
 * C += (1 - A) a c and A += (1 - A) a.  Output: RGBA float image (device pointer, w*h*4
 * floats, premultiplied colour and accumulated opacity), pixel layout as mhd_vis_slice. */
mhd_status mhd_vis_volume(mhd_ctx* ctx, int quantity, int axis, double vmin, double vmax,
                          double opacity, float* rgba);

/* Minimum and maximum of q over the grid (host outputs), e.g. for vmin/vmax. */
mhd_status mhd_vis_range(mhd_ctx* ctx, int quantity, double* vmin, double* vmax);

/* FP64 sums of 8 device arrays without allocating device memory.
 *
 * The paper has no counterpart to this entry point.  It exists for callers that cannot
 * call cudaMalloc: for example code inside a serving process whose device memory is all
 * handed out by another allocator under a fixed budget, or a host thread that must not
 * trigger the device-wide synchronisation that cudaMalloc and cudaFree imply while other
 * work is in flight.  It computes what mhd_sums computes (the sum over n cells of each of
 * 8 fields, accumulated in FP64) for arrays the caller owns, with the reduction's scratch
 * held in a fixed array of 262,208 bytes in the library's device image (every GPU that
 * loads the library keeps it until the process exits).
 *
 *   f       8 device pointers to n elements each, dtype 0 = float32, 1 = float64
 *   out     host array of 8 doubles, written before the call returns
 *   stream  cudaStream_t to run on (NULL: the default stream); the call synchronises it
 *
 * Returns MHD_ERR_INVALID for a NULL argument, a bad dtype, n < 1, or
 * n > MHD_SUMS_NOALLOC_MAX_CELLS (the scratch holds one row of partial sums per 65,536
 * cells, 4096 rows); MHD_ERR_CUDA if a CUDA call fails.  The first call on a device looks
 * up the scratch array's device address with that device current.  The address is kept
 * for the life of the process: a cudaDeviceReset of that device makes it stale.  All calls
 * share the one scratch array: calls whose work overlaps on the GPU race, so serialise
 * them. */
#define MHD_SUMS_NOALLOC_MAX_CELLS 268435456LL
mhd_status mhd_sums_noalloc(const void* const f[8], int dtype, long long n, double out[8],
                            void* stream);

/* Free everything the context owns.  NULL is ignored. */
void mhd_destroy(mhd_ctx* ctx);

const char* mhd_status_str(mhd_status s);

/* Text of the last CUDA or validation error seen by this context (never NULL). */
const char* mhd_last_error(const mhd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MHD_GB300_H */
