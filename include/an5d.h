/*
 * an5d.h -- C ABI of a GB300 (sm_103a) library for iterated star/box
 * Jacobi stencil sweeps with high-degree N.5D temporal blocking.
 *
 * Method: AN5D (Matsumura, Zohouri, Wahib, Endo, Matsuoka, CGO 2020).
 *   - Stencils (Section 2.1, Table 4): star (axis neighbours only) or box
 *     (full (2R+1)^d cube) of radius R, constant per-offset coefficients,
 *     one array, one statement, on 2D or 3D grids.
 *   - N.5D blocking (Section 2.3, Fig. 1; Section 3.1): tile all axes but the
 *     slowest one, stream along it, and fuse bT time steps per pass over
 *     global memory with overlapped halo tiles (2 * bT * R per tiled axis).
 *   - Host code (Section 3.3): one kernel pass per bT steps, a final pass
 *     with a reduced degree when T is not a multiple of bT, buffers swapped
 *     so that the result lands in the caller's output.
 *
 * Data layout (all entry points): a grid with interior extents dims[]
 * (C order, slowest first, x = last axis contiguous) is stored as a dense
 * padded array of (dims[i] + 2R) elements per axis, C order, no row pitch.
 * The R-wide halo holds fixed (Dirichlet) boundary values: it is read,
 * never updated.  Device pointers must be 16-byte aligned.
 *
 * Per-point update, for every interior point p (coefficient k multiplies
 * offset o_k in the canonical order below):
 *     acc = c[0] * u[p + o_0];  acc = fma(c[k], u[p + o_k], acc), k = 1..n-1
 * in the run's precision, each operation rounded once.  Canonical order
 * (Table 4's sums; box streaming axis outermost as in the per-sub-plane
 * partial sums of Section 3.1):
 *     star: centre, then for i = -R..-1, 1..R: (dx=i), (dy=i)[, (dz=i)]
 *     box : for dz = -R..R (3D), dy = -R..R, dx = -R..R
 * The plain FP32 and FP64 methods are bit-exact to this definition.
 *
 * Errors: functions returning int return an AN5D_* status (0 = success).
 * Functions returning a pointer return NULL on failure.  The reason of the
 * last failure on the calling thread is available from an5d_last_error()
 * and an5d_last_status().  Device-side failures (a bounded wait that gave
 * up) are recorded in the plan and read by an5d_plan_status() after the
 * work has finished.  No entry point aborts the process.
 *
 * Ownership: a plan owns its device coefficient copy, its scratch buffers
 * and its tuned configuration.  The caller owns every in/out buffer and
 * every stream.  All device work is enqueued on the caller's stream
 * (a cudaStream_t passed as void*; NULL = the legacy default stream) and
 * is asynchronous unless stated.
 */
#ifndef AN5D_H
#define AN5D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct an5d_plan an5d_plan;

/* Stencil shape (Section 2.1). */
typedef enum { AN5D_STAR = 0, AN5D_BOX = 1 } an5d_shape;

/* Arithmetic of a run.
 *   AN5D_F32             FP32 storage and FP32 plain chain (bit-exact).
 *   AN5D_F64             FP64 storage and FP64 plain chain (bit-exact).
 *   AN5D_F16S_F32C       binary16 storage, FP32 chain, every time level
 *                        rounded to binary16 (nearest-even).
 *   AN5D_F32_COMPENSATED FP32 storage, per-point sum by Dot2 (Ogita, Rump,
 *                        Oishi 2005, Algorithm 5.3) in the canonical order.
 * The paper itself evaluates FP32 and FP64 with fast-math (Section 5.2);
 * the last two forms have no counterpart in the paper. */
typedef enum {
    AN5D_F32 = 0,
    AN5D_F64 = 1,
    AN5D_F16S_F32C = 2,
    AN5D_F32_COMPENSATED = 3
} an5d_dtype;

/* Status codes. */
enum {
    AN5D_OK = 0,
    AN5D_ERR_INVALID_ARG = -1, /* NULL pointer, bad extent, T < 0, misaligned pointer */
    AN5D_ERR_UNSUPPORTED = -2, /* ndim, shape, radius or dtype not built into the library */
    AN5D_ERR_ALIAS = -3,       /* out overlaps in */
    AN5D_ERR_CUDA = -4,        /* a CUDA runtime call failed (message in an5d_last_error) */
    AN5D_ERR_OOM = -5,         /* device allocation failed */
    AN5D_ERR_TIMEOUT = -6      /* a bounded device wait gave up (plan status) */
};

/* Chosen blocking of a plan (Section 3.1 / 3.2 parameters).
 *   bT          time steps fused per pass
 *   tile_x      tile extent along x in cells, overlap included (b_S1)
 *   tile_y      3D: tile extent along y in cells, overlap included (b_S2); 2D: 1
 *   stream_axis index of the streamed axis in dims[] (0 = slowest)
 *   hsn         streamed cells per stream block (h_SN, Section 3.2)
 *   warps_per_cta, ctas   launch shape of one pass (ctas of all its launches)
 *   launches_per_pass     kernel launches of one full-degree pass: 1, or 2
 *               when a 3D pass runs its ragged last tile column on a narrow
 *               kernel (32 or 64 cells wide, same tile rows)
 *   model_gcells      analytic roofline prediction, GCell-updates/s
 *   measured_gcells   timed throughput of this config during tuning (0 if untimed) */
typedef struct {
    int bT;
    int tile_x;
    int tile_y;
    int stream_axis;
    int hsn;
    int warps_per_cta;
    int ctas;
    int launches_per_pass;
    double model_gcells;
    double measured_gcells;
} an5d_config;

/* Number of coefficients of a stencil: star 2*ndim*R+1, box (2R+1)^ndim
 * (Table 4).  Returns a negative AN5D_* status for unsupported input. */
int an5d_coeff_count(int ndim, an5d_shape shape, int radius);

/* Create a plan for one stencil on one grid size (Section 3.3 host code).
 *   ndim    2 or 3
 *   shape   AN5D_STAR or AN5D_BOX
 *   radius  1..4 (star, and box in 2D and 3D; high-order boxes run at bT 1-2)
 *   coeffs  host array of an5d_coeff_count(...) doubles in canonical order,
 *           rounded once to the run's compute precision here
 *   dtype   see an5d_dtype
 *   dims    host array of ndim interior extents (each >= 1), slowest first;
 *           the padded array must have fewer than 2^31 elements
 * Picks the blocking with the library's analytic model (no GPU timing; see
 * an5d_plan_tune).  Allocates the plan's scratch buffer (one padded grid)
 * on the current device, and for 3D a second CUDA stream and two events
 * (see an5d_run); an5d_plan_destroy releases them.  Returns NULL on failure. */
an5d_plan *an5d_plan_create(int ndim, an5d_shape shape, int radius, const double *coeffs,
                            an5d_dtype dtype, const int64_t *dims);

/* Per-step operation of a division-type stencil (Table 4: j2d5pt, j2d9pt,
 * j2d9pt-gol, j3d27pt divide the weighted sum by a constant c0 every step).
 *   AN5D_POST_DIV      one IEEE division by the divisor (correctly rounded)
 *   AN5D_POST_MUL_RCP  one multiplication by the divisor's reciprocal, itself
 *                      rounded once to the compute precision (Section 6's
 *                      remedy for slow division: "/N" becomes "*(1/N)") */
typedef enum { AN5D_POST_DIV = 1, AN5D_POST_MUL_RCP = 2 } an5d_post;

/* Create a plan for a division-type stencil: every step computes the plain
 * chain of an5d_plan_create's stencil and then applies `post` with
 * `divisor` (rounded once to the compute precision).  Same arguments,
 * ownership and errors as an5d_plan_create, plus:
 *   divisor  finite and nonzero, with a nonzero finite reciprocal
 *   post     AN5D_POST_DIV or AN5D_POST_MUL_RCP
 *   dtype    AN5D_F32 or AN5D_F64 (AN5D_ERR_UNSUPPORTED otherwise)
 * Built: 2D star radius 1-2, 2D box radius 1, 3D box radius 1 (Table 4's
 * division-type rows).  an5d_run_adjoint rejects these plans. */
an5d_plan *an5d_plan_create_div(int ndim, an5d_shape shape, int radius, const double *coeffs,
                                double divisor, an5d_post post, an5d_dtype dtype,
                                const int64_t *dims);

/* Advance T time steps: out = S^T(in).
 *   in, out  device pointers to padded arrays of the storage type
 *            (FP32: float, FP64: double, F16S: binary16, COMPENSATED: float);
 *            in is never written; out must not overlap in (AN5D_ERR_ALIAS);
 *            out's halo is set to in's halo
 *   T        >= 0; T == 0 copies in to out
 *   stream   cudaStream_t as void*
 * Enqueues ceil(T / bT) passes plus a halo copy; returns after enqueueing.
 * A 3D pass whose last tile column runs on the narrow kernel forks that
 * launch onto the plan's own second stream after an event recorded on
 * `stream` and joins it back into `stream` before the next pass, so all of
 * the run's work is ordered on `stream` (also under stream capture).
 * Not thread-safe per plan: one run of a plan at a time (its scratch
 * buffer is shared by all runs). */
int an5d_run(an5d_plan *plan, const void *in, void *out, int64_t T, void *stream);

/* Same as an5d_run on HOST buffers (pageable or pinned): copies in to the
 * plan's device staging buffers, runs, copies the result back into out,
 * and synchronises the stream before returning.  Allocates the staging
 * buffers on first use. */
int an5d_run_host(an5d_plan *plan, const void *in_host, void *out_host, int64_t T,
                  void *stream);

/* Release the plan and its device memory.  NULL-safe.  Synchronises the
 * device work the plan has enqueued first. */
void an5d_plan_destroy(an5d_plan *plan);

/* Copy the plan's current configuration into *cfg. */
int an5d_plan_config(const an5d_plan *plan, an5d_config *cfg);

/* Force a configuration (bT, hsn; 0 = keep the current value).  Other
 * fields are derived.  Returns AN5D_ERR_UNSUPPORTED for a bT not built.
 * If the plan's tile variant does not build bT, the plan returns to the
 * default variant. */
int an5d_plan_set_config(an5d_plan *plan, int bT, int hsn);

/* Kernel launches that an5d_run enqueues for T steps with the plan's
 * current configuration: the halo copies plus one launch per pass, two for
 * a 3D pass that runs its last tile column on the narrow kernel (0 for
 * T = 0, which is a plain copy).  Negative AN5D_* status on bad input. */
int64_t an5d_plan_launches(const an5d_plan *plan, int64_t T);

/* Select the sweep kernel's tile variant: 0 = the default width (128 cells
 * along x), else a tile width along x for which a variant is built
 * (2D FP32: 192 cells, 6 per lane, for the radius-1 star at bT 4-6, also in
 * both division forms, the radius-2 star at bT 2-3, the radius-3 star at
 * bT 2 and the radius-1 box at bT 3-5: less overlap per tile at a lower
 * degree; 3D: 64 cells, 2 per lane, on 4-row warps, for the FP32 radius-1
 * star at bT 2-4, the FP32 radius-1 box at bT 1-3, the Dot2 and binary16
 * radius-1 stars at bT 1-3 and the FP64 radius-2 star at bT 1: taller tiles
 * with less overlap in y).  Keeps bT and hsn; a remainder pass whose
 * degree the variant does not build runs on the default kernel.  Returns
 * AN5D_ERR_UNSUPPORTED if no variant of that width exists for the plan's
 * stencil and current bT.  cfg.tile_x reports the width in use. */
int an5d_plan_set_tile(an5d_plan *plan, int tile_x);

/* Replace the plan's coefficients (n doubles in the canonical offset order,
 * rounded to the plan's precision as at creation; Section 5.1's constant
 * coefficients become kernel arguments).  Keeps the stencil, the grid, the
 * configuration and every buffer the plan owns, so a training loop that
 * updates the coefficients every step reuses one plan instead of creating
 * one per step.  Host-side only: the coefficients travel by value in each
 * launch's arguments, so work already enqueued keeps the coefficients it
 * was launched with.  AN5D_ERR_INVALID_ARG on a NULL plan or coeffs. */
int an5d_plan_set_coeffs(an5d_plan *plan, const double *coeffs);

/* Autotune (Section 5.3's "Tuned" procedure with this library's model):
 * rank every built bT and stream-block length of every tile variant with
 * the analytic model, time each variant's top `topk` candidates on the
 * plan's scratch buffers for
 * `T_probe` steps on `stream`, then time up to five more stream-block
 * lengths around the fastest one's (0.5x to 2x its block count), and keep
 * the fastest of all.  Synchronous.  Results are cached per (stencil,
 * dtype, division, dims, device) for the process. */
int an5d_plan_tune(an5d_plan *plan, int topk, int64_t T_probe, void *stream);

/* Fault injection for tests of the failure path (2D plans): while enabled,
 * warp 0 of every pass waits for 16 bytes that are never delivered.  The
 * bounded wait gives up after about one second, the warp waits (bounded)
 * for its real copies in flight and returns, and an5d_plan_status reports
 * AN5D_ERR_TIMEOUT; the CUDA context stays usable.  Nothing traps or hangs.
 * (No counterpart in the paper.) */
int an5d_plan_inject_stall(an5d_plan *plan, int enable);

/* Device-side status of the plan's finished work: AN5D_OK or
 * AN5D_ERR_TIMEOUT.  Synchronises the device.  Clears the status. */
int an5d_plan_status(an5d_plan *plan);

/* Allocation-free variant of an5d_run.  The paper has no counterpart: it is
 * an interface for callers that cannot call cudaMalloc, such as frameworks
 * that hand all device memory to their own pool or caching allocator (an
 * allocation outside it can fail against its budget or fragment it), and
 * loops that must not stall (cudaMalloc and cudaFree may synchronise the
 * device).  It takes the stencil description of an5d_plan_create and the
 * buffers of an5d_run, picks the blocking as an5d_plan_create would, and
 * runs T steps with the same kernels and the same bits as an5d_run.
 *
 * It allocates no device memory: the ping-pong buffer and the status word
 * live in one file-scope device array of AN5D_NOALLOC_MAX_BYTES (+256)
 * bytes that every GPU loading this library holds until the process exits.
 * Grids whose padded array is larger than AN5D_NOALLOC_MAX_BYTES are
 * rejected with AN5D_ERR_INVALID_ARG.
 *
 * The first call on a device looks up the array's device address on that
 * device (set-up, once per device); make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) after that first call is not
 * supported, as for plans: the address kept from the first call would no
 * longer name the array.  Every call shares the array: calls whose GPU work
 * overlaps (from other host threads or on other streams) race and give wrong
 * results.  Synchronous: enqueues on `stream`, reads the status word back
 * and waits for the stream, and returns AN5D_ERR_TIMEOUT if a bounded device
 * wait gave up.  A call that fails after it has enqueued work still waits
 * for the stream before it returns, so the array is idle whenever the call
 * returns. */
#define AN5D_NOALLOC_MAX_BYTES (32u << 20)
int an5d_run_noalloc(int ndim, an5d_shape shape, int radius, const double *coeffs,
                     an5d_dtype dtype, const int64_t *dims, const void *in, void *out, int64_t T,
                     void *stream);

/* Error norms of a run against an FP64 reference, over the interior of a
 * padded grid.  The precision forms are measured against an FP64 evaluation
 * of the same sweep; FP64 arithmetic on the GPU is otherwise used only by
 * the FP64 plain method.  (No counterpart in the paper, which reports no
 * accuracy figures.)
 *   u     device array of the storage type of `dtype`, padded layout
 *   ref   device FP64 array of the same padded shape
 *   out   host array of 3 doubles: max |u - ref|, sum (u - ref)^2, sum ref^2
 * FP64 accumulation over a fixed partition: deterministic for a given grid.
 * Allocates and frees a small device buffer; synchronous on `stream`. */
int an5d_error_norms(int ndim, int radius, const int64_t *dims, an5d_dtype dtype, const void *u,
                     const double *ref, double *out, void *stream);

/* Adjoint (reverse-mode gradient) of an5d_run for 2D FP32 plans of radius
 * 1-2.  For a loss L of u_T = S^T(u0):
 *   u0        device, the forward input (padded FP32)
 *   gT        device, dL/du_T (padded FP32; its halo is ignored)
 *   grad_u0   device output, dL/du0 on the interior, 0 on the halo (the
 *             halo is boundary data, not a parameter)
 *   grad_coeffs host output, dL/dc_k, k in canonical order (FP64)
 * g_t = S^T g_{t+1} is the transposed stencil (offsets -o_k, zero halo);
 * dL/dc_k = sum_t sum_p g_{t+1}[p] u_t[p + o_k].  Checkpoints every bT
 * steps (bT = min(plan degree, 4)); each block recomputes its states from
 * its checkpoint and runs the transposed stencil over the block as one
 * temporally blocked pass.  Its work memory (T/bT + 2 bT grids) is owned by
 * the plan, grown on demand and reused; synchronous.  (No counterpart in the
 * paper.) */
int an5d_run_adjoint(an5d_plan *plan, const void *u0, const void *gT, void *grad_u0,
                     double *grad_coeffs, int64_t T, void *stream);

/* Halo-deepened domain split (Section 2.3's overlapped tiling applied to
 * slabs of the grid; the per-device step of a multi-GPU decomposition).
 * The slowest axis (y in 2D, z in 3D) of the interior is cut into nsub
 * slabs as evenly as possible (the first extent % nsub slabs own one plane
 * more).  Slab k owns interior planes [a, b) (0-based interior index) and
 * holds the padded planes [lo, hi) = [a - bT R, b + bT R + 2R) clipped to
 * the padded array: bT R ghost planes beyond its owned planes and R outer
 * planes that act as a fixed halo during a pass.
 *
 * an5d_split_geometry: host only (no device needed).  out: host array of 4
 *   int64, receives {a, b, lo, hi} of slab k.  AN5D_ERR_INVALID_ARG on bad
 *   arguments; AN5D_ERR_UNSUPPORTED if a slab would own fewer than
 *   bT R + R planes (its ghost planes would reach past its neighbour).
 *
 * an5d_run_split: the plan's sweep of T steps (its degree bT and stream
 *   block length) run as nsub slabs on the calling device: per pass of
 *   degree d <= bT, every slab runs one pass of its own padded array; then
 *   every plane a slab holds but does not own is copied from the slab that
 *   owns it (the one exchange per pass), and at the end the owned planes are
 *   gathered into `out`.  in, out as for an5d_run (device, padded, plan
 *   dtype; `in` is not written).  The result is bit for bit that of
 *   an5d_run.  Allocates nsub slab plans and 2 nsub slab buffers for the
 *   call and frees them before returning; synchronous on `stream`.  Plain
 *   stencils (no per-step division) only: AN5D_ERR_UNSUPPORTED otherwise.
 *   nsub = 1 or T = 0 is an5d_run.  (The paper's host code runs one grid on
 *   one device; the exchange between devices is not built: one GPU.) */
int an5d_split_geometry(int ndim, const int64_t *dims, int radius, int bt, int nsub, int k,
                        int64_t *out);
int an5d_run_split(an5d_plan *plan, int nsub, const void *in, void *out, int64_t T, void *stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent 2D FP32 grids of uneven size, stencil and
 * length in one persistent launch replayed as a CUDA graph.  (No counterpart
 * in the paper; each grid gets exactly the bits of an5d_run on that grid.)
 * ------------------------------------------------------------------------ */

/* One grid of a batch. */
typedef struct {
    an5d_shape shape;
    int radius;            /* 1 or 2 */
    const double *coeffs;  /* host, an5d_coeff_count(2, shape, radius) values, canonical order */
    int64_t ny, nx;        /* interior extents (padded: +2R each) */
    int64_t T;             /* time steps of this grid, >= 0 */
} an5d_grid_desc;

typedef struct an5d_batch_plan an5d_batch_plan;

typedef struct {
    int grids;
    int ctas;              /* persistent CTAs (resident capacity of the device) */
    int64_t items;         /* (grid, x tile, stream block, pass) work items */
    double cell_updates;   /* sum over grids of ny * nx * T */
    int class_bt[4];       /* degree per class: star R1, star R2, box R1, box R2 */
    int class_tile_x[4];   /* tile width per class in cells (128, or 192 with the class's wide degree) */
} an5d_batch_info_t;

/* Create a batch plan: copies descs and coefficients, allocates one scratch
 * grid per grid, the work-item list and the tile pass counters on the
 * current device.  Degrees start at 8/4/4/2 (star R1/R2, box R1/R2).
 * Returns NULL on failure (message: an5d_batch_last_error). */
an5d_batch_plan *an5d_batch_plan_create(int n, const an5d_grid_desc *descs);

/* Pick each class's degree among the built ones {1,4,8} (radius 1) and
 * {1,2,4} (radius 2), and its tile width (128 cells, or 192 cells at the
 * class's wide degree: 4 for radius 1, 2 for radius 2), by timing whole
 * runs of the batch (Section 5.3's tuning by measurement; coordinate
 * descent over the classes, at most two sweeps).  an5d_batch_tune runs on temporary zero-filled buffers of every
 * grid (allocated and freed here); an5d_batch_tune_run on the caller's ins
 * and outs (same contract as an5d_batch_run; outs are overwritten).
 * Synchronous. */
int an5d_batch_tune(an5d_batch_plan *bp, void *stream);
int an5d_batch_tune_run(an5d_batch_plan *bp, const void *const *ins, void *const *outs, void *stream);

/* Force the degree of each class (class_bt[4], values from the built menu). */
int an5d_batch_set_degrees(an5d_batch_plan *bp, const int *class_bt);

/* Force the tile width of each class (class_tile_x[4]: 128 or 192 cells).
 * A width of 192 takes effect while the class runs at its wide degree (4
 * for radius 1, 2 for radius 2; the remaining T mod bT steps then run at
 * degree 1 on the same tiles); at other degrees the class uses 128-cell
 * tiles.  Tiles of every width give the same bits.  AN5D_ERR_UNSUPPORTED
 * for other widths. */
int an5d_batch_set_tiles(an5d_batch_plan *bp, const int *class_tile_x);

/* Advance every grid i by its T: outs[i] = S_i^{T_i}(ins[i]).  ins/outs are
 * host arrays of n device pointers to padded FP32 grids (16-byte aligned,
 * out must not overlap in).  Asynchronous on `stream`: one CUDA-graph launch
 * (counter reset, halo copies, the persistent kernel).  Not thread-safe per
 * plan.  Device-side failures: an5d_batch_status. */
int an5d_batch_run(an5d_batch_plan *bp, const void *const *ins, void *const *outs, void *stream);

/* AN5D_OK or AN5D_ERR_TIMEOUT for the finished batch runs.  Synchronises. */
int an5d_batch_status(an5d_batch_plan *bp);

int an5d_batch_info(const an5d_batch_plan *bp, an5d_batch_info_t *info);

/* Fault injection for tests: while enabled, the last work item waits for a
 * pass count that is never reached; its bounded wait gives up after about
 * one second, the batch aborts, and an5d_batch_status returns
 * AN5D_ERR_TIMEOUT.  Nothing traps or hangs. */
int an5d_batch_inject_stall(an5d_batch_plan *bp, int enable);
const char *an5d_batch_last_error(void);
void an5d_batch_plan_destroy(an5d_batch_plan *bp);

/* Peak rates used by the library's analytic model and by roofline reports.
 *   hbm_gbs      device copy bandwidth, read + write bytes, GB/s
 *   fp32_gflops  FP32 fma throughput, 2 flops per fma, GFLOP/s
 *   fp64_gflops  FP64 fma throughput, GFLOP/s
 *   smem_gbs     shared-memory load bandwidth, GB/s
 *   sm_clock_mhz peak SM clock of the device attribute (nominal figures)
 *   sms          streaming multiprocessors
 *   measured     1 if the figures come from an5d_measure_peaks, 0 if nominal
 * The paper measures its memory peaks with micro-benchmarks and takes the
 * compute peak from the FMA rate (Section 4); so does this library. */
typedef struct {
    double hbm_gbs;
    double fp32_gflops;
    double fp64_gflops;
    double smem_gbs;
    double sm_clock_mhz;
    int sms;
    int measured;
} an5d_peaks;

/* Run the copy (2 x 1 GiB), FP32 fma, FP64 fma and shared-memory load
 * micro-benchmarks on the current device and `stream`, store the result as
 * the model's peaks for this device and copy it to *out (may be NULL).
 * Synchronous; allocates and frees 2 GiB of device memory. */
int an5d_measure_peaks(an5d_peaks *out, void *stream);

/* The paper's analytic performance model (Section 4), evaluated on the host
 * for the paper's own kernel design: one thread per cell of a spatial block
 * bS[0] x ... (x first), threads classed as out-of-bound, boundary, redundant
 * or valid; global-memory traffic one read per in-grid thread at level 0 and
 * one write per valid thread at level bT; shared-memory traffic one write per
 * thread and level below bT plus Table 3's practical reads per computing or
 * boundary thread; compute over the region of valid computation of each
 * level (bS - 2tR per axis); time = max(compute / (peak x eff_ALU), global /
 * peak, shared / peak) / eff_SM.  It is independent of this library's
 * kernels (whose own model ranks the tuner's candidates) and needs no GPU.
 *   st     stencil: ndim, shape, radius, word bytes, and its operations per
 *          cell-update as FMA / MUL / ADD / other (star and box: n-1 FMA and
 *          one MUL; eff_ALU = (2 FMA + MUL + ADD + other) / (2 x all))
 *   dims   ndim interior extents, slowest (streamed) first
 *   bT     temporal degree (>= 1); bS: ndim-1 block sizes, x first, each
 *          greater than 2 bT R; hSN: planes per stream block (>= 1)
 *   dev    peaks: compute (GFLOP/s of the dtype), global and shared memory
 *          throughput (GB/s), SM count, resident threads per SM
 *   out    thread counts and totals of one pass (bT steps) over the grid,
 *          the three times and the model time (seconds), and the predicted
 *          useful rate (GCell-updates/s and GFLOP/s at the stencil's flops)
 * Returns AN5D_OK or AN5D_ERR_INVALID_ARG. */
typedef struct {
    int ndim;
    an5d_shape shape;
    int radius;
    int word_bytes;
    int op_fma, op_mul, op_add, op_other;
} an5d_paper_stencil;
typedef struct {
    double peak_comp_gflops;
    double peak_gm_gbs;
    double peak_sm_gbs;
    int sm_count;
    int max_threads_per_sm;
} an5d_paper_device;
typedef struct {
    double th_comp, th_sm_read, th_sm_write, th_gm_read, th_gm_write;
    double total_comp, total_gm, total_sm;  /* flop, bytes, bytes per pass */
    double eff_alu, eff_sm;
    double time_comp, time_gm, time_sm, time_model;
    double gcells, gflops;
    int64_t n_tb;                           /* thread blocks per pass */
    int bound;                              /* 0 compute, 1 global memory, 2 shared memory */
} an5d_paper_model_result;
int an5d_paper_model(const an5d_paper_stencil *st, const int64_t *dims, int bT, const int *bS,
                     int hSN, const an5d_paper_device *dev, an5d_paper_model_result *out);

/* Current peaks of the current device: measured if an5d_measure_peaks ran
 * in this process, else nominal figures from the device attributes. */
int an5d_get_peaks(an5d_peaks *out);

/* ------------------------------------------------------------------------
 * Batched adjoint: dL/du_0 and dL/dc for many independent 2D FP32 grids
 * (the grids of an an5d_grid_desc batch) in persistent launches replayed
 * as one CUDA graph.  (No counterpart in the paper: the adjoint follows from
 * differentiating the time loop of Section 3.3.)  Per grid, with block
 * degree nb (4 for radius 1, 2 for radius 2) and M = ceil(T / nb) blocks:
 * forward passes store checkpoints u_{m nb}; then for each block, last
 * first, one pass recomputes the block's states from its checkpoint and
 * stores them, and one temporally blocked pass of the transposed stencil
 * (offsets -o_k, zero halo) takes g through the block while adding
 * g_{t+1}[p] u_t[p + o_k] to the coefficient gradient in registers.
 * g_t = S^T g_{t+1}; dL/dc_k = sum_t sum_p g_{t+1}[p] u_t[p + o_k].
 * ------------------------------------------------------------------------ */

typedef struct an5d_adjoint_batch an5d_adjoint_batch;

typedef struct {
    int grids;
    int waves;             /* persistent launches per run (work memory within the budget) */
    int ctas;              /* persistent CTAs per launch */
    int64_t items;         /* (grid, x tile, stream block, pass) work items, all waves */
    double cell_updates;   /* sum over grids of ny * nx * T */
    size_t work_bytes;     /* device work memory owned by the batch (the largest wave's) */
    int class_nb[4];       /* block degree per class: star R1, star R2, box R1, box R2 */
} an5d_adjoint_batch_info_t;

/* Create: copies descs and coefficients (rounded to FP32), plans the work
 * items, and splits the grids, in order, into waves whose work memory
 * (T/nb checkpoints, nb - 1 level grids, one g grid and per-tile partial
 * sums per grid) fits budget_bytes (0: 48 GiB); a grid larger than the
 * budget gets a wave of its own.  Allocates the largest wave's work memory
 * on the current device.  Returns NULL on failure (message:
 * an5d_adjoint_batch_last_error). */
an5d_adjoint_batch *an5d_adjoint_batch_create(int n, const an5d_grid_desc *descs, size_t budget_bytes);

/* Run: u0s[i] device, grid i's forward input (padded FP32, halo = the
 * Dirichlet boundary); gTs[i] device, dL/du_T (padded; its halo is
 * ignored); grad_u0s[i] device output, dL/du_0 on the interior and 0 on the
 * halo (must not overlap u0s[i] or gTs[i]); grad_coeffs host output, n rows
 * of 25 doubles, row i holding grid i's dL/dc_k in canonical order (the
 * rest zero).  The coefficient gradient is summed in FP32 per warp over a
 * fixed partition and in FP64 across warps and tiles, in a fixed order:
 * deterministic.  The first call with a set of buffers captures the graph
 * (later calls with the same buffers replay it).  Synchronous on `stream`.
 * AN5D_ERR_TIMEOUT if a bounded device wait gave up (the context stays
 * usable).  Every wait is bounded; nothing traps or hangs. */
int an5d_adjoint_batch_run(an5d_adjoint_batch *ab, const void *const *u0s, const void *const *gTs,
                           void *const *grad_u0s, double *grad_coeffs, void *stream);
int an5d_adjoint_batch_info(const an5d_adjoint_batch *ab, an5d_adjoint_batch_info_t *info);
void an5d_adjoint_batch_destroy(an5d_adjoint_batch *ab);
const char *an5d_adjoint_batch_last_error(void);

/* Message and status of the last failure on the calling thread. */
const char *an5d_last_error(void);
int an5d_last_status(void);

/* Library version string. */
const char *an5d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AN5D_H */
