/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann library with the Knudsen refinement sensor.
 *
 * The library advances a lattice Boltzmann BGK simulation of a lid-driven cavity (D2Q9 or D3Q19)
 * on one GPU and evaluates, fused into the same pass, the kinetic refinement sensor of
 * arXiv 1507.06767 ("Local mesh refinement sensor for the lattice Boltzmann method"):
 *
 *     K(x) = (1/q) sum_i | f_i^neq(x) / f_i^eq(x) |,   f^neq = f - f^eq       (Sec. 3.2, Eq. sensor;
 *                                                                             Sec. 3.3, Eq. kkn)
 *
 * reduced per block to a maximum and turned into refine / keep / coarsen flags (Sec. 3.4 maps the
 * sensor to refinement levels; Sec. 5.2 regrids from it).
 *
 * Model (Sec. 2.2):
 *   - discrete velocities D2Q9 / D3Q19 with the standard weights w_i, c_s^2 = 1/3;
 *   - equilibrium f_i^eq = w_i rho (1 + c_i.u / c_s^2 + Q_i:uu / (2 c_s^4)),  Q_i = c_i c_i - c_s^2 I
 *     (Eq. feq_i); rho = sum_i f_i, rho u = sum_i c_i f_i (Eqs. rho, u);
 *   - one time step = streaming + BGK collision f* = f - (f - f^eq)/tau (Eq. bgklb and the
 *     collide-and-stream split).  It is computed in pull form: each cell gathers f_i from x - c_i
 *     of the previous post-collision field, then evaluates moments, equilibrium, sensor and
 *     collision in registers and writes f* once;
 *   - tau and the viscosity are linked by nu = c_s^2 (tau - 1/2) (Eq. nu_omega).
 *
 * Geometry: nodes at integer positions 0..n-1 on each axis; non-periodic axes have half-way
 * bounce-back walls at -1/2 and n-1/2.  The wall at y = ny - 1/2 is the lid: it moves with the lid
 * velocity (Sec. 4.1, moving bounce-back): a population pulled from a ghost node with y == ny gets
 * f_i = f*_opp(i)(x) + 2 w_i (c_i . u_lid) / c_s^2 (wall density 1), every other wall ghost reflects
 * f*_opp(i)(x) unchanged.  Edge and corner ghosts on the plane y == ny belong to the lid, which makes
 * the total mass of the closed cavity exactly invariant.
 *
 * Sensor state: K is evaluated on the pre-collision populations of the step (after streaming and
 * bounce-back) with their own rho and u.
 *
 * Memory layout of the populations (device): structure of arrays f[i][z][y][x], x fastest, i
 * slowest, N = nx*ny*nz cells per population, no padding.  Storage types:
 *   LBM_F64   double, stores f
 *   LBM_F32   float,  stores f
 *   LBM_F16S  IEEE half, stores f - w_i (shifted by the lattice weight); arithmetic in float
 *   LBM_BF16S bfloat16,  stores f - w_i; arithmetic in float
 * Arithmetic is double for LBM_F64 and float for the others.
 *
 * Blocks: the fused step records, on every sensor step, the maximum of K over base tiles of edge
 * LBM_TILE (8x8 in 2-D, 8x8x8 in 3-D) anchored at the origin; partial tiles at the high ends hold the
 * cells they have.  Block maxima for any block edge that is a multiple of LBM_TILE are exact maxima
 * of tile maxima.  Block arrays are indexed ((bz * nby) + by) * nbx + bx, nb* = ceil(n* / block).
 * A NaN anywhere in a block makes that block's maximum NaN.
 *
 * Flags (int8 per block): threshold rule: +1 refine if max > T, -1 coarsen if max < T/2, 0 keep;
 * a NaN max refines.  Top-fraction rule: +1 for the ceil(frac * nblocks) largest maxima (ties by
 * lower block index; NaN counts as +inf), 0 for the others.  Comparisons are made in double.
 *
 * Conventions for every call:
 *   - return value: LBM_OK (0) or a negative LBM_E* status; calls returning a pointer return NULL on
 *     failure.  lbm_last_error() / lbm_last_message() give the status and a text of the last
 *     failing call on this host thread.  No C++ exception crosses the ABI.
 *   - pointers named *_host are caller-owned host memory (pageable or pinned), copied synchronously;
 *     pointers named *_dev are caller-owned device memory on the handle's device, used
 *     asynchronously on the handle's stream.
 *   - a handle is not thread-safe; different handles are independent.  Work is issued on the
 *     handle's stream (lbm_set_stream; default: the legacy default stream) and is asynchronous
 *     unless the call says it synchronises.
 *   - a NULL handle gives LBM_EINVAL.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Lattices (the value is q). */
#define LBM_D2Q9 9
#define LBM_D3Q19 19

/* Population storage types. */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_F16S 2
#define LBM_BF16S 3

/* Status codes. */
#define LBM_OK 0
#define LBM_EINVAL (-1)   /* bad argument */
#define LBM_ENOMEM (-2)   /* device allocation failed */
#define LBM_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define LBM_ENUMERIC (-4) /* NaN or Inf found in the populations */
#define LBM_ETIMEOUT (-5) /* a bounded device wait ran out */
#define LBM_ENOTSUP (-6)  /* not supported in this build */
#define LBM_ESTATE (-7)   /* call not allowed in the handle's current state */
#define LBM_EIO (-8)      /* a checkpoint file could not be written, read or verified */

/* Periodic axis mask bits. */
#define LBM_PERIODIC_X 1
#define LBM_PERIODIC_Y 2
#define LBM_PERIODIC_Z 4

/* Edge of the base tile over which the fused step records the sensor maximum. */
#define LBM_TILE 8

/* Flag rules for lbm_flags_from_maxima. */
#define LBM_FLAG_THRESHOLD 0
#define LBM_FLAG_TOP 1

typedef struct lbm_s lbm_t;

/* Status of the last failing call on this host thread (LBM_OK if none), and its message. */
LBM_API int lbm_last_error(void);
LBM_API const char *lbm_last_message(void);
/* Static text for a status code. */
LBM_API const char *lbm_strerror(int status);
/* ABI version of this library (major * 100 + minor). */
LBM_API int lbm_version(void);

/*
 * Create a lattice of nx * ny * nz cells on the current CUDA device.  lattice is LBM_D2Q9 (nz must
 * be 1) or LBM_D3Q19; tau > 1/2 is the lattice relaxation time (nu = (tau - 1/2)/3, Eq. nu_omega).
 * Defaults: storage LBM_F32, lid velocity (0.1, 0, 0), no periodic axis, sensor on the last step of
 * every lbm_step call, block edge 16, legacy default stream.  Device buffers are allocated on first
 * use (or adopted with lbm_attach); the initial state is rest, f_i = w_i.  Returns NULL on a bad
 * argument (LBM_EINVAL) or when the lattice exceeds 2^31 - 1 cells.
 */
LBM_API lbm_t *lbm_create(int lattice, int nx, int ny, int nz, double tau);
/* Release the handle and the device memory it owns (never the buffers given to lbm_attach).
 * Synchronises the handle's stream. */
LBM_API int lbm_destroy(lbm_t *h);

/* Storage type (LBM_F64 / LBM_F32 / LBM_F16S / LBM_BF16S).  Only before the population buffers
 * exist (LBM_ESTATE afterwards). */
LBM_API int lbm_set_dtype(lbm_t *h, int dtype);
/* Lid velocity (ux, uz) of the wall at y = ny - 1/2 (the y component is 0 by construction). */
LBM_API int lbm_set_lid(lbm_t *h, double ux, double uz);
/* Periodic axes (mask of LBM_PERIODIC_*); a periodic y axis removes the lid and the y walls.  D2Q9
 * ignores the z bit. */
LBM_API int lbm_set_periodic(lbm_t *h, int axis_mask);
/* Relaxation time tau > 1/2. */
LBM_API int lbm_set_tau(lbm_t *h, double tau);
/* CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream) for all later work. */
LBM_API int lbm_set_stream(lbm_t *h, void *stream);
/* Sensor schedule: k > 0 records the sensor on every step whose 1-based global index is a multiple
 * of k; k == 0 records it on the last step of each lbm_step call. */
LBM_API int lbm_set_sensor_every(lbm_t *h, int k);
/* on != 0: sensor steps also write the per-cell K field (read with lbm_get_sensor_field). */
LBM_API int lbm_set_sensor_field(lbm_t *h, int on);
/* Block edge (a positive multiple of LBM_TILE) used by lbm_flag / lbm_flag_top and their _dev
 * forms. */
LBM_API int lbm_set_block(lbm_t *h, int block);
/* on != 0: time every fused step kernel with CUDA events on the handle's stream (read with
 * lbm_kernel_time); turning it on clears the counters. */
LBM_API int lbm_set_profiling(lbm_t *h, int on);
/* Kernel variant of the fused step: LBM_KERNEL_AUTO (default) picks the fastest measured kernel that
 * applies (per lattice, storage, size and step kind: plain steps and sensor steps may differ),
 * LBM_KERNEL_CELL forces the one-cell kernel, LBM_KERNEL_PAIR the two-cell kernel with
 * packed FP32 arithmetic (storage other than LBM_F64, an even nx and (q + 1) * cells < 2^32),
 * LBM_KERNEL_TMA the kernel that
 * stages the populations through shared memory with TMA copies (D3Q19, storage other than LBM_F64,
 * nx times the element size a multiple of 16 bytes), LBM_KERNEL_TMA_PAIR the two-cell kernel that
 * stages the populations of a 64 x 8-cell tile through shared memory with TMA copies (D3Q19, 16-bit
 * storage, nx a multiple of 8, 20 * cells < 2^32); LBM_EINVAL where a variant does not apply.
 * All compute the same step; they differ in rounding order only.  The TMA kernels' waits are
 * bounded: if one runs out (it should not), the next synchronising call returns LBM_ETIMEOUT until
 * lbm_reset. */
#define LBM_KERNEL_AUTO 0
#define LBM_KERNEL_CELL 1
#define LBM_KERNEL_PAIR 2
#define LBM_KERNEL_TMA 3
#define LBM_KERNEL_TMA_PAIR 4
LBM_API int lbm_set_kernel_variant(lbm_t *h, int variant);
/* on != 0: lbm_step replays captured CUDA graphs for runs of steps (default on). */
LBM_API int lbm_set_graphs(lbm_t *h, int on);

/*
 * Adopt caller-owned device buffers a and b (each >= lbm_population_bytes(h) bytes, 16-byte aligned)
 * as the two population buffers; a is taken as the current post-collision state as it is.  The
 * caller keeps ownership and must keep them alive until lbm_destroy.  Resets the step counter.
 */
LBM_API int lbm_attach(lbm_t *h, void *a_dev, void *b_dev, size_t bytes);
/* Bytes of one population buffer for the current storage type (q * N * element size). */
LBM_API size_t lbm_population_bytes(const lbm_t *h);
/* Number of blocks for block edge `block` (0 if block is not a positive multiple of LBM_TILE). */
LBM_API int lbm_nblocks(const lbm_t *h, int block);
/* Number of completed steps. */
LBM_API long long lbm_steps_done(const lbm_t *h);

/* Reset the state to rest (f_i = w_i) and the step counter to 0. */
LBM_API int lbm_reset(lbm_t *h);

/*
 * Advance n >= 0 time steps (asynchronous).  Each step is one launch of the fused kernel:
 * pull-stream with moving-wall bounce-back -> rho, u -> f^eq -> [sensor K and its per-tile max on
 * sensor steps] -> BGK collision -> store.  f^neq never leaves registers.
 */
LBM_API int lbm_step(lbm_t *h, int n);

/*
 * Block maxima of K of the most recent sensor step, for block edge `block` (positive multiple of
 * LBM_TILE), written as lbm_nblocks(h, block) doubles.  _host synchronises; _dev is asynchronous.
 * LBM_ESTATE if no sensor step has run since the last reset.
 */
LBM_API int lbm_sensor(lbm_t *h, int block, double *out_host);
LBM_API int lbm_sensor_dev(lbm_t *h, int block, double *out_dev);

/* Threshold flags (+1 / 0 / -1, see above) of the most recent sensor step for the handle's block
 * edge (lbm_set_block).  _host synchronises; _dev is asynchronous. */
LBM_API int lbm_flag(lbm_t *h, double threshold, int8_t *out_host);
LBM_API int lbm_flag_dev(lbm_t *h, double threshold, int8_t *out_dev);
/* Top-fraction flags: +1 for the ceil(frac * nblocks) largest block maxima, 0 otherwise
 * (0 <= frac <= 1). */
LBM_API int lbm_flag_top(lbm_t *h, double frac, int8_t *out_host);
LBM_API int lbm_flag_top_dev(lbm_t *h, double frac, int8_t *out_dev);

/*
 * Flag builder on caller data: maxima_dev holds n block maxima of type maxima_dtype (LBM_F32:
 * float, LBM_F64: double) on the current device; rule is LBM_FLAG_THRESHOLD (param = T) or
 * LBM_FLAG_TOP (param = frac).  Writes n int8 flags to out_dev, asynchronously on `stream`.
 */
LBM_API int lbm_flags_from_maxima(const void *maxima_dev, int maxima_dtype, int n, int rule,
                                  double param, int8_t *out_dev, void *stream);

/*
 * Time-averaged sensor (Sec. 5.1 builds its static mesh from the sensor averaged over one
 * dimensionless period).  on != 0 clears the running sums and, from then on, adds the tile maxima
 * of every sensor step; on == 0 stops adding (the sums are kept).  lbm_sensor_average writes, per
 * block of edge `block`, the maximum over its tiles of the time-averaged tile maxima, and the
 * number of sensor steps averaged (count may be NULL).  Synchronises; LBM_ESTATE before the first
 * averaged sensor step.
 */
LBM_API int lbm_set_sensor_average(lbm_t *h, int on);
LBM_API int lbm_sensor_average(lbm_t *h, int block, double *out_host, long long *count);

/*
 * Refinement levels per block (Sec. 3.4, Eqs. phi and l): phi = log2 K_max and
 * l = clamp(floor(a * phi + b), lmin, lmax).  The paper writes the integral part [a phi]; this
 * library reads it as the floor and adds an offset b (b = 0 is the paper's form); a > 0.  A block
 * with K_max <= 0 gets lmin, a NaN block lmax.  lbm_levels_fit chooses a and b from the blocks'
 * own range (finite K_max > 0): phi normalised to [0, 1] -- the normalised phi of the paper's
 * figures -- maps onto [lmin, lmax + 1), so l = lmin + floor(phi_n (lmax - lmin + 1)), clamped;
 * with fewer than two distinct values every block gets lmin.  source is LBM_SENSOR_LAST (block
 * maxima of the last sensor step) or LBM_SENSOR_AVERAGE (time-averaged, see above).  Writes
 * lbm_nblocks(h, block) int8 levels; synchronises.  Requires -128 <= lmin <= lmax <= 127.
 */
#define LBM_SENSOR_LAST 0
#define LBM_SENSOR_AVERAGE 1
LBM_API int lbm_levels(lbm_t *h, int block, double a, double b, int lmin, int lmax, int source,
                       int8_t *out_host);
LBM_API int lbm_levels_fit(lbm_t *h, int block, int lmin, int lmax, int source, int8_t *out_host);

/* Populations as doubles, layout f[i][z][y][x] (q * N values).  get synchronises; set resets
 * nothing but the state (the step counter is kept). */
LBM_API int lbm_get_populations(lbm_t *h, double *out_host);
LBM_API int lbm_set_populations(lbm_t *h, const double *in_host);
/* Raw storage bytes (checkpointing): bytes must equal lbm_population_bytes(h). */
LBM_API int lbm_get_raw(lbm_t *h, void *out_host, size_t bytes);
LBM_API int lbm_set_raw(lbm_t *h, const void *in_host, size_t bytes);
/* Density rho[N] and velocity u[3][N] (doubles) of the current state (moments of f*, which equal
 * those of the pre-collision state of the last step).  Synchronises. */
LBM_API int lbm_get_moments(lbm_t *h, double *rho_host, double *u_host);
/* Per-cell K[N] of the most recent sensor step (needs lbm_set_sensor_field(h, 1) before it). */
LBM_API int lbm_get_sensor_field(lbm_t *h, double *out_host);
/*
 * Total mass sum_x sum_i f_i and momentum sum_x sum_i c_i f_i (3 doubles) of the current state,
 * summed in double on the device in a fixed order (deterministic).  Synchronises.  Returns
 * LBM_ENUMERIC (with the sums still written) if a population is NaN or Inf.
 */
LBM_API int lbm_conservation(lbm_t *h, double *mass, double *mom3);

/*
 * Slabs of a lattice cut along its slowest axis (z for D3Q19, y for D2Q9), one handle per slab,
 * e.g. one per GPU.  The fused step of Sec. 2.2 pulls each population from the nearest neighbour
 * along its velocity, so a slab needs, per step, one plane of its neighbour's previous
 * post-collision state, and only the populations whose velocity crosses the cut: 5 per face for
 * D3Q19, 3 for D2Q9 (no counterpart in the paper, whose runs are on one machine).
 *
 * lbm_set_halo(h, faces): faces = LBM_HALO_LO and / or LBM_HALO_HI (0 restores walls on both)
 * makes the low / high face of the slab axis a cut instead of a wall.  A cell on a halo face then
 * pulls the crossing populations from the face's halo plane wherever the rest of the pull source
 * lies inside the lattice (or wraps on a periodic x / y axis); sources outside along another axis
 * are wall ghosts as before.  On a D2Q9 slab the high y face, where the lid is, carries no lid
 * term once it is a halo.  The slab axis must not be periodic (LBM_EINVAL either way round).  The
 * halos live on the device, start as fluid at rest, keep their content until the next import and
 * are read by every following step; lbm_reset leaves them as they are.  Set the storage type
 * first: it cannot change once halos exist.  A slab with halo faces runs the one-cell kernel
 * (LBM_KERNEL_AUTO or LBM_KERNEL_CELL; the other variants are refused either way round).
 *
 * lbm_halo_size: elements (and bytes) of one halo message: k planes of nx (D2Q9) or nx * ny
 * (D3Q19) values in the storage type, k = 3 (D2Q9) or 5 (D3Q19); plane j holds the j-th crossing
 * direction in the library's population order, cells x fastest.
 *
 * lbm_halo_export(h, face, out, on_device): writes the populations leaving through the face --
 * velocity component -1 along the slab axis on the low face, +1 on the high face -- of the
 * boundary plane of the current (post-collision) state.  lbm_halo_import(h, face, in, on_device):
 * sets the face's halo to the populations arriving through it -- +1 on the low face, -1 on the high
 * face -- so the neighbour below exports its high face into this slab's low face and the one above
 * its low face into the high face.  on_device = 0: `out` / `in` are host memory and the call
 * synchronises; 1: device memory, used asynchronously on the handle's stream.  Per step: export
 * both faces, exchange, import, lbm_step(h, 1).  Bytes are copied as stored, so a slab run is bit
 * for bit the single-domain run wherever the same kernel relaxes each cell.  LBM_ESTATE for a face
 * without a halo.
 */
#define LBM_HALO_LO 1
#define LBM_HALO_HI 2
LBM_API int lbm_set_halo(lbm_t *h, int faces);
LBM_API int lbm_halo_size(const lbm_t *h, long long *elems, long long *bytes);
LBM_API int lbm_halo_export(lbm_t *h, int face, void *out, int on_device);
LBM_API int lbm_halo_import(lbm_t *h, int face, const void *in, int on_device);

/*
 * Checkpoint files (no counterpart in the paper; resuming a long run).  lbm_checkpoint_save writes
 * an 88-byte header -- magic "LBMCKPT\0", version 1, lattice, nx, ny, nz, storage type, periodic
 * mask, tau, lid (x, z), step counter, payload size and the 64-bit FNV-1a checksum of the payload,
 * native byte order -- followed by the populations in the layout of lbm_get_raw (synchronises).
 * lbm_checkpoint_load checks the header and the checksum (LBM_EIO on an unreadable, truncated or
 * corrupted file), requires the handle's lattice, dimensions and storage type (LBM_EINVAL
 * otherwise), then restores tau, the lid, the periodic mask, the populations and the step counter,
 * so that the run continues bit for bit where it was saved.  Sensor results of earlier steps are
 * not part of a checkpoint.
 */
LBM_API int lbm_checkpoint_save(lbm_t *h, const char *path);
LBM_API int lbm_checkpoint_load(lbm_t *h, const char *path);

/*
 * Failure injection for tests (no counterpart in the paper).  lbm_debug_fail_alloc(after): of the
 * library's next device allocations (any handle, process-wide), the first `after` succeed and the
 * one after them fails with cudaErrorMemoryAllocation (reported as LBM_ENOMEM) without calling
 * cudaMalloc; the hook then disarms itself.  A negative value disarms it.  A call that fails this
 * way keeps what it had allocated (lbm_destroy frees it) and can be retried.
 * lbm_debug_set_wait_limit(h, ns) sets the limit of the bounded waits between the warps of the
 * handle's kernels that have them (the TMA-staged step); 0 restores the default of one second.  A
 * wait that runs out makes the kernel stop, wait (with the full default limit) for its own copies
 * in flight and return; the next synchronising call reports LBM_ETIMEOUT and the state is invalid
 * until lbm_reset.  lbm_debug_hold_copies(h, on): the producer warps of the handle's TMA-staged
 * kernels issue no copies, so their consumers' first wait can only run out -- a wait on something
 * that never comes, with nothing in flight when the kernel gives up (tests of the timeout path;
 * off by default).
 */
LBM_API int lbm_debug_fail_alloc(int after);
LBM_API int lbm_debug_set_wait_limit(lbm_t *h, long long ns);
LBM_API int lbm_debug_hold_copies(lbm_t *h, int on);

/* Total time (ms) and count of the fused step kernels timed since profiling was turned on.
 * Synchronises. */
LBM_API int lbm_kernel_time(lbm_t *h, double *ms_total, long long *launches);

/*
 * One fused step with the sensor, for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of lbm_step + lbm_sensor_dev.
 *
 * Who needs it: applications that serve all device memory from their own pool and do not let a
 * library call cudaMalloc, and latency-critical loops that cannot afford an allocation (which may
 * synchronise the device) after set-up.  This call allocates nothing: its scratch (the per-tile
 * sensor maxima and the block maxima before conversion) lives in one fixed device array of the
 * library, 2 * LBM_NOALLOC_MAX_TILES doubles (4 MiB), which every GPU that loads the library holds
 * until the process exits.
 *
 * Arguments: lattice, dtype, nx, ny, nz, tau, the lid velocity (lid_x, lid_z) and the periodic
 * mask mean what they mean for lbm_create / lbm_set_*.  f_in_dev holds the post-collision
 * populations of the previous step in the storage layout of lbm.h (f[i][z][y][x] of type dtype);
 * the new populations go to f_out_dev (same size, must not alias f_in_dev).  block (a positive
 * multiple of LBM_TILE) is the block edge; block_max_dev receives ceil(nx/block) * ceil(ny/block) *
 * ceil(nz/block) doubles (nz term 1 for D2Q9), the block maxima of this step's sensor.  All
 * pointers are device memory of the calling thread's current device, owned by the caller; the work
 * is queued on `stream` (a cudaStream_t, NULL for the legacy default stream) and the call returns
 * without waiting.
 *
 * Limit: at most LBM_NOALLOC_MAX_TILES tiles of 8^d cells (512^3 D3Q19, 4096^2 D2Q9); a larger
 * lattice gets LBM_EINVAL and a message naming the limit.  The first call in a CUDA context looks
 * up the array's device address in that context (the calling thread's current one) and caches it
 * under the context's unique ID; make that first call before any stream capture on the device.  A
 * context created later on the same device (after cudaDeviceReset, or a caller's own context) gets
 * its own lookup on its first call, so a stale address is never used.  An error left pending on
 * the thread by earlier CUDA work is reported (LBM_ECUDA, not cleared) before anything is
 * launched.  Calls share the array and it keeps the last call's contents;
 * nothing in it needs clearing, since each call writes every tile it reads.  Calls whose kernels
 * overlap on the GPU race on the array: serialise them (one stream per process, or synchronise).
 */
#define LBM_NOALLOC_MAX_TILES 262144
LBM_API int lbm_step_noalloc(int lattice, int dtype, int nx, int ny, int nz, double tau,
                             double lid_x, double lid_z, int periodic, const void *f_in_dev,
                             void *f_out_dev, int block, double *block_max_dev, void *stream);

/*
 * Multi-level block-structured mesh (refinement ratio 2; Sec. 2.1 and Sec. 5.2 describe the
 * cell-centred block-structured AMR the paper's dynamic meshes use).  The lattice of the handle is
 * the domain at the finest resolution: nbx * edge = nx and so on, tau is the finest level's
 * relaxation time, and the lid and periodic settings apply.  D3Q19 with LBM_F32 storage only
 * (LBM_ENOTSUP otherwise).
 *
 * The domain is a grid of nbx x nby x nbz physical blocks of edge `edge` finest cells; leaf[b]
 * (x fastest) is the finest level 0..lmax present in block b (lmax <= 2).  Level l exists on every
 * block whose leaf level is >= l, with edge / 2^(lmax - l) cells per block edge, so levels nest
 * and level 0 covers the domain; touching blocks (faces, edges, corners) may differ by one level
 * at most, and edge / 2^lmax must be >= 2.  Acoustic scaling: dx / dt is the same on every level,
 * so level l takes 2^l steps per level-0 step ("cycle") and tau_l = 3 nu / 2^(lmax - l) + 1/2 with
 * nu = (tau - 1/2) / 3 of the finest level (Eq. nu_omega); every level needs tau_l != 1.
 * Coupling: one-cell ghost layers; inside a level a ghost is the neighbouring block's cell (read
 * in place), at the edge of a level it is filled by trilinear space / linear time interpolation of
 * the next coarser level with the non-equilibrium
 * part rescaled by (tau_f - 1) / (2 (tau_c - 1)); after the two sub-steps of a finer level the
 * coarser cells under it take the average of their 8 fine cells, the non-equilibrium part rescaled
 * by 2 (tau_c - 1) / (tau_f - 1).  The sensor K of every cell is evaluated in each level step; the
 * reported block maximum is that of the block's leaf level at its last sub-step of the cycle.
 *
 * lbm_blocks_step builds the mesh at rest on the first call (or when the layout changes, which
 * restarts it at rest; lbm_reset discards it), runs `cycles` cycles as one captured CUDA graph
 * each (graphs off: direct launches), and, if block_max is not NULL, writes nbx * nby * nbz block
 * maxima (host, synchronising).  The step kernel's launch shape per level is chosen by timing the
 * candidates when the mesh is built (lbm_blocks_info reports it).
 */
typedef struct lbm_level_batch {
    int nbx, nby, nbz;   /* physical blocks per axis */
    int edge;            /* block edge in finest cells */
    int lmax;            /* finest level, 0..2 */
    const int8_t *leaf;  /* host: leaf level per block, x fastest */
    int cycles;          /* level-0 steps to advance */
    double *block_max;   /* host output, nbx * nby * nbz values, or NULL */
} lbm_level_batch;
LBM_API int lbm_blocks_step(lbm_t *h, const lbm_level_batch *batch);
/* Interior populations of physical block `block` at level `level` (n^3 cells, n = edge /
 * 2^(lmax - level)), layout f[i][z][y][x], as doubles; the block must exist at that level.
 * Synchronise. */
LBM_API int lbm_blocks_get(lbm_t *h, int level, int block, double *out_host);
LBM_API int lbm_blocks_set(lbm_t *h, int level, int block, const double *in_host);
/* Level facts: cells per block edge, tau, blocks at the level, the step kernel's threads per CTA
 * and cells (cell pairs for the two-cell form) per thread, and the cell updates of one cycle over
 * all levels (any pointer may be NULL). */
LBM_API int lbm_blocks_info(lbm_t *h, int level, int *n, double *tau, int *nblocks, int *threads,
                            int *cells_per_thread, long long *cell_updates_per_cycle);
/* Restriction onto the next coarser level after the finest level's two sub-steps: a separate
 * kernel (LBM_FUSION_SEPARATE) or fused into the finest level's second sub-step -- the tiled form
 * (LBM_FUSION_FUSED, blocks of 16, 32 or 64 cells per edge), or the brick form (LBM_FUSION_BRICK,
 * 8, 16, 32 or 64 cells per edge: one thread steps a 2 x 2 x 2 brick of fine cells and writes the
 * coarse cell under it).  All give the same average and f^neq rescaling, summed in other orders.
 * LBM_FUSION_AUTO (default) times the separate step + restriction against the brick form when the
 * mesh is built and keeps the faster.  Applies from the next mesh build: an existing mesh is
 * discarded. */
#define LBM_FUSION_AUTO 0
#define LBM_FUSION_SEPARATE 1
#define LBM_FUSION_FUSED 2
#define LBM_FUSION_BRICK 3
LBM_API int lbm_blocks_set_fusion(lbm_t *h, int mode);
/* How a cycle runs: a captured graph of the separate launches (LBM_SCHEDULE_GRAPH; the levels on
 * streams of their own, ordered by events), or one persistent launch (LBM_SCHEDULE_PERSISTENT):
 * persistent CTAs claim the cycle's tasks -- ghost fills, level steps, restrictions -- in the order
 * the graph enqueues them and wait, device-side and bounded, for the phases each task depends on
 * (replayed from a captured graph of that launch when graphs are on).  LBM_SCHEDULE_AUTO (default)
 * times both when the mesh is built and keeps the faster (the persistent kernel in two forms: with
 * the finest level's brick phases, or lean, with plain steps and restriction phases at a smaller
 * register budget; LBM_SCHEDULE_PERSISTENT keeps the faster of the two, _PERSISTENT_BRICK and
 * _PERSISTENT_LEAN force one); the persistent form is not available with LBM_FUSION_FUSED.  A wait that runs out (limit: lbm_debug_set_wait_limit, default one
 * second; lbm_debug_hold_copies makes every wait run out) stops the launch; the next call that
 * synchronises (lbm_blocks_step with block maxima, lbm_blocks_get) returns LBM_ETIMEOUT and the
 * mesh must be rebuilt.  Applies from the next mesh build: an existing mesh is discarded.
 * lbm_blocks_cycle_form returns the form the current mesh uses (LBM_SCHEDULE_GRAPH or
 * LBM_SCHEDULE_PERSISTENT), LBM_ESTATE without a mesh. */
#define LBM_SCHEDULE_AUTO 0
#define LBM_SCHEDULE_GRAPH 1
#define LBM_SCHEDULE_PERSISTENT 2
#define LBM_SCHEDULE_PERSISTENT_BRICK 3 /* the persistent kernel with brick phases only */
#define LBM_SCHEDULE_PERSISTENT_LEAN 4  /* the lean persistent kernel only */
LBM_API int lbm_blocks_set_schedule(lbm_t *h, int mode);
LBM_API int lbm_blocks_cycle_form(lbm_t *h);
/* Form of every level's step kernel: LBM_STEP_FORM_AUTO (default) times the candidate forms and
 * launch shapes of each level when the mesh is built and keeps the fastest; the others force one
 * form on every level whose block edge it applies to (the remaining levels stay timed):
 * LBM_STEP_FORM_FLAT one cell per thread in x-fastest order (any edge), LBM_STEP_FORM_TILED bricks
 * of whole rows walking z planes (edges 8, 16, 32, 64), LBM_STEP_FORM_SELECT flat with an
 * address-select gather for the rows inside the block in y and z (16, 32, 64),
 * LBM_STEP_FORM_PAIR two x-adjacent cells per thread with packed FP32 arithmetic (8, 16, 32, 64).
 * All compute the same step; they differ in rounding order only.  Applies from the next mesh
 * build: an existing mesh is discarded. */
#define LBM_STEP_FORM_AUTO 0
#define LBM_STEP_FORM_FLAT 1
#define LBM_STEP_FORM_TILED 2
#define LBM_STEP_FORM_SELECT 3
#define LBM_STEP_FORM_PAIR 4
LBM_API int lbm_blocks_set_step_form(lbm_t *h, int form);
/* The schedule picked for a level: the step kernel's form (0 flat, 1 tiled, 2 flat with the
 * address-select gather, 3 two cells per thread: LBM_STEP_FORM_* minus one), the planes a tiled
 * CTA walks (0 otherwise) and, for the finest level, how its second sub-step restricts: 0 a
 * separate kernel, 1 the brick form, >= 2 the planes of the tiled fused kernel.  Any pointer may be NULL; LBM_ESTATE without a mesh. */
LBM_API int lbm_blocks_schedule(lbm_t *h, int level, int *form, int *planes, int *fused);

/*
 * Regridding of one refinement level from the sensor (Sec. 5.2: cells flagged by the sensor, one
 * layer of buffer cells, refinement boxes holding at least 80 % flagged cells and subdivided
 * otherwise, proper nesting inside the next coarser level with a row of coarse buffer cells).
 * The clustering is the point-clustering method of Berger and Rigoutsos (1991), which the paper's
 * solver uses; the steps, in tag cells of coarsen^d lattice cells (coarsen^2 x 1 for D2Q9):
 *
 *   1. tag a tag cell if the field exceeds `threshold` (strict >) in one of its cells or one of
 *      them is NaN;
 *   2. tag every tag cell within Chebyshev distance `buffer` of a tagged one (periodic axes of the
 *      handle wrap, the domain edge stops the buffer elsewhere);
 *   3. if `allowed` is not NULL (tx * ty * tz bytes, x fastest, nonzero = covered by the coarser
 *      level), keep a tag only where every tag cell within Chebyshev distance `nest` is covered,
 *      positions beyond a non-periodic domain edge counting as covered;
 *   4. cluster, starting from the whole tag grid: shrink a box to the bounding box of its tags
 *      (drop it if empty); accept it if tags >= efficiency * volume; else cut it at the empty
 *      slab (hole) nearest the centre of its axis (least |2p - L|; ties: longer axis, lower axis,
 *      lower p; the hole starts the upper piece); else at the strongest strict sign change of the
 *      signature's second difference D[i] = s[i-1] - 2 s[i] + s[i+1], between slabs i and i + 1,
 *      strength |D[i+1] - D[i]| (ties: nearer the centre, longer axis, lower axis, lower p); else
 *      at floor(L / 2) of the longest axis (ties: lower axis).  A cut is admissible only if both
 *      pieces are >= min_width slabs long; without one the box is accepted as it is.  Signatures
 *      are the tag counts of the slabs normal to each axis.
 *
 * field_dev is a device array of nx * ny * nz doubles (x fastest), or NULL for the handle's
 * per-cell sensor of its most recent sensor step (lbm_set_sensor_field(h, 1) before stepping;
 * LBM_ESTATE otherwise).  Boxes come back in lattice cells, half-open ([lo, hi) per axis, the
 * high end cut at the lattice edge), sorted by (lo_z, lo_y, lo_x); tag cells in `boxes` keep their
 * order.  *nboxes receives the number of boxes; if it exceeds max_boxes, nothing is written to
 * `boxes` and the call returns LBM_EINVAL.  ntagged (may be NULL) receives the number of tag cells
 * tagged after steps 1-3, tags_out (host, tx * ty * tz bytes, may be NULL) the tags themselves
 * (0/1).  Tag, buffer, nesting and the slab counts of each round of boxes run on the GPU; the cut
 * decisions are made on the host between rounds.  Synchronises.  Arguments out of range
 * (coarsen < 1, buffer < 0, nest < 0, min_width < 1, efficiency outside [0, 1] or NaN) give
 * LBM_EINVAL.
 */
typedef struct lbm_box {
    int lo[3];  /* x, y, z */
    int hi[3];
} lbm_box;
typedef struct lbm_regrid_params {
    int coarsen;             /* tag cell edge in lattice cells (>= 1) */
    double threshold;        /* T of step 1 */
    int buffer;              /* step 2 (the paper uses 1) */
    const uint8_t *allowed;  /* step 3 mask (host) or NULL */
    int nest;                /* step 3 buffer (the paper uses 1) */
    double efficiency;       /* step 4 (the paper uses 0.8) */
    int min_width;           /* step 4, in tag cells (>= 1) */
} lbm_regrid_params;
LBM_API int lbm_regrid(lbm_t *h, const double *field_dev, const lbm_regrid_params *p,
                       lbm_box *boxes, int max_boxes, int *nboxes, long long *ntagged,
                       uint8_t *tags_out);

/*
 * Learned predictor of the block sensor maxima (not in the paper; it serves the dynamic
 * regridding of Sec. 5.2, which re-evaluates the sensor at every level-0 step, by estimating
 * where the sensor will be large some steps ahead, so that a regrid can refine before the flow
 * gets there; the exact sensor stays the fallback and the judge of the predicted flags).
 *
 * lbm_block_features writes, per block of edge `block` (along z too for D3Q19; partial blocks at
 * the high ends), the mean over its cells of rho, u_x, u_y (and u_z for D3Q19) of the current
 * populations: out_dev[c * nblocks + b] (FP32, device, caller-owned; blocks x fastest), queued on
 * the handle's stream.
 *
 * The network: X -> normalise ((x - shift[c]) * scale[c] per input channel) -> 3x3 conv (cin ->
 * hidden) + ReLU -> 3x3 conv (hidden -> hidden) + ReLU -> 3x3 conv (hidden -> 1), zero padding,
 * inputs X[batch][cin][h][w] and outputs Y[batch][1][h][w] in FP32 on the device.  Parameters
 * are one flat FP32 vector: W1[hidden][cin][3][3], b1[hidden], W2[hidden][hidden][3][3],
 * b2[hidden], W3[1][hidden][3][3], b3[1] (lbm_net_param_count values); weights and activations
 * are used in BF16 with FP32 accumulation; the master parameters, gradients and Adam moments are
 * FP32.  Training minimises the mean over all outputs of (Y - T)^2 with Adam (Kingma and Ba 2015:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, theta -= lr (m / (1 - b1^t)) /
 * (sqrt(v / (1 - b2^t)) + eps)).  cin is 3 or 4 and hidden 8 or 16 (LBM_EINVAL otherwise).
 *
 * lbm_net_backward runs the forward pass and writes the gradients of the loss (lbm_net_get_grads);
 * lbm_net_adam applies one Adam step with the current gradients (lbm_net_set_grads replaces them,
 * e.g. with gradients averaged over several processes); lbm_net_train_step is backward + Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  A non-NULL loss_host receives the loss and synchronises;
 * otherwise the calls queue their kernels on the network's stream (lbm_net_set_stream) and return.
 * lbm_net_set_params sets the parameters and clears the Adam state.  Targets and predictions are
 * in log10 units: lbm_net_log_targets writes t = log10(max(K, floor_k)) - offset for n block
 * maxima (NaN for a NaN maximum), lbm_net_to_maxima K = 10^(y + offset); the latter feeds lbm_flags_from_maxima.
 */
typedef struct lbm_net_s lbm_net;
LBM_API int lbm_block_features(lbm_t *h, int block, float *out_dev);
LBM_API lbm_net *lbm_net_create(int cin, int hidden);
LBM_API void lbm_net_destroy(lbm_net *n);
LBM_API int lbm_net_set_stream(lbm_net *n, void *stream);
LBM_API int lbm_net_param_count(lbm_net *n);
LBM_API int lbm_net_set_normalisation(lbm_net *n, const float *shift, const float *scale);
LBM_API int lbm_net_set_params(lbm_net *n, const float *host);
LBM_API int lbm_net_get_params(lbm_net *n, float *host);
LBM_API int lbm_net_get_grads(lbm_net *n, float *host);
LBM_API int lbm_net_set_grads(lbm_net *n, const float *host);
LBM_API int lbm_net_forward(lbm_net *n, const float *x_dev, int batch, int h, int w, float *y_dev);
LBM_API int lbm_net_backward(lbm_net *n, const float *x_dev, const float *target_dev, int batch,
                             int h, int w, double *loss_host);
LBM_API int lbm_net_adam(lbm_net *n, float lr, float beta1, float beta2, float eps);
LBM_API int lbm_net_train_step(lbm_net *n, const float *x_dev, const float *target_dev, int batch,
                               int h, int w, float lr, double *loss_host);
LBM_API int lbm_net_log_targets(const double *kmax_dev, long long n, float offset, float floor_k,
                                float *t_dev, void *stream);
/*
 * Residual form of the targets (the predictor reads the sensor now as a fourth input channel and
 * predicts how it changes): lbm_net_log_residual writes t = log10(max(K_next, floor_k)) -
 * log10(max(K_now, floor_k)) for n block maxima, lbm_net_to_maxima_residual K = max(K_now,
 * floor_k) * 10^y; NaN in a maximum gives NaN (a refine flag downstream).  Device pointers,
 * asynchronous on `stream`.
 */
LBM_API int lbm_net_log_residual(const double *kmax_next_dev, const double *kmax_now_dev,
                                 long long n, float floor_k, float *t_dev, void *stream);
LBM_API int lbm_net_to_maxima_residual(const float *y_dev, const double *kmax_now_dev, long long n,
                                       float floor_k, double *kmax_dev, void *stream);
LBM_API int lbm_net_to_maxima(const float *y_dev, long long n, float offset, double *kmax_dev,
                              void *stream);
/*
 * Judge and fallback of a regrid driven by predicted flags (not in the paper; the exact sensor of
 * Sec. 3.2 stays the judge).  lbm_flags_agreement writes to *out_dev the fraction of the n blocks
 * whose flags in a_dev and b_dev are equal (1 for n = 0).  lbm_flags_judge_select takes the flags
 * the previous regrid predicted for now (pred_prev_dev, or NULL at the first regrid), the exact
 * flags now (exact_now_dev) and the flags predicted now for the next interval (pred_next_dev): the
 * agreement of pred_prev with exact_now goes to *agreement_dev (NaN without pred_prev) and decides
 * the flags written to used_dev -- pred_next if the agreement is at least min_agreement or there is
 * no previous prediction, else exact_now, with *fell_back_dev = 1 (agreement_dev and fell_back_dev
 * may be NULL).  All pointers are device memory; both calls queue one kernel on `stream`.
 *
 * lbm_gather_rows copies rows idx_dev[0..count) of src_dev (nrows rows of row_bytes bytes, a
 * multiple of 4) to consecutive rows of dst_dev, e.g. the minibatch of a training step; an index
 * outside [0, nrows) is not read and sets *bad_dev to 1 (the caller clears it beforehand).
 */
LBM_API int lbm_flags_agreement(const int8_t *a_dev, const int8_t *b_dev, int n, double *out_dev,
                                void *stream);
LBM_API int lbm_flags_judge_select(const int8_t *pred_prev_dev, const int8_t *exact_now_dev,
                                   const int8_t *pred_next_dev, int n, double min_agreement,
                                   int8_t *used_dev, double *agreement_dev, int *fell_back_dev,
                                   void *stream);
LBM_API int lbm_gather_rows(const void *src_dev, long long nrows, size_t row_bytes,
                            const int *idx_dev, int count, void *dst_dev, int *bad_dev,
                            void *stream);

/*
 * Intermediate buffers of the last lbm_net_forward / lbm_net_backward call, copied to host memory
 * (synchronises): for inspection and for checking each layer on its own.  `which`:
 *   LBM_NET_BUF_PARAMS_BF16  the BF16 parameters the kernels read (lbm_net_param_count values);
 *   LBM_NET_BUF_X0           the normalised BF16 input, [batch][cin][h][w];
 *   LBM_NET_BUF_A1 / _A2     the BF16 activations after the first / second ReLU, [batch][hidden][h][w];
 *   LBM_NET_BUF_Y            the FP32 output of the last backward call, [batch][h][w];
 *   LBM_NET_BUF_DY           dL/dY (FP32) of the last backward call, [batch][h][w];
 *   LBM_NET_BUF_DZ2 / _DZ1   dL/dZ (FP32) of the second / first convolution's output, masked by
 *                            its ReLU, [batch][hidden][h][w].
 * bytes must equal the buffer's size for the shape of the last call (BF16: 2 bytes per value,
 * FP32: 4); LBM_EINVAL otherwise, LBM_ESTATE before the first forward pass.
 */
#define LBM_NET_BUF_PARAMS_BF16 0
#define LBM_NET_BUF_X0 1
#define LBM_NET_BUF_A1 2
#define LBM_NET_BUF_A2 3
#define LBM_NET_BUF_Y 4
#define LBM_NET_BUF_DY 5
#define LBM_NET_BUF_DZ2 6
#define LBM_NET_BUF_DZ1 7
LBM_API int lbm_net_get_buffer(lbm_net *n, int which, void *out_host, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
