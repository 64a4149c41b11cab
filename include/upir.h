/*
 * upir.h — C ABI of the B300 runtime for offloaded UPIR regions.
 *
 * The calls follow the parallel constructs of UPIR (Unified Parallel
 * Intermediate Representation, arXiv 2209.10643):
 *   - data mapping to / from / tofrom / allocate ........ §4.1, Fig. "data attributes"
 *   - SPMD region with num_teams x num_units ............. §3.1, Fig. "SPMD parallelism"
 *   - canonical loop (lowerBound, upperBound, step,
 *     collapse) with worksharing schedule(static|dynamic,
 *     chunk) distributed over teams and units ........... §3.2, Fig. "data parallelism"
 *   - sync: reduction (operation + data), barrier,
 *     taskwait ........................................... §5, Fig. "synchronization"
 *
 * Every function returns a upir_status (0 = UPIR_OK, negative = error).  No
 * function throws, aborts or exits the process.  After an error the per-context
 * text of upir_last_error() says what was wrong.  Handles are not thread-safe:
 * use one context per host thread.
 *
 * Memory ownership.  The caller owns every host buffer it maps; a host buffer
 * must stay valid until the matching upir_data_unmap() returns.  Device memory
 * of mapped buffers and of the runtime's workspace belongs to the library and is
 * obtained through the allocator given to upir_init() (cudaMalloc / cudaFree
 * when none is given).  Device memory handed
 * in with upir_data_map_device() stays owned by the caller.
 *
 * Work is enqueued on the context's CUDA stream and runs in submission order.
 * Host/device copies of a mapping happen on that stream; upir_data_unmap() and
 * UPIR_SYNC_TASKWAIT block the host until the stream has drained.
 */
#ifndef UPIR_H
#define UPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */

typedef int32_t upir_status;

#define UPIR_OK            0
#define UPIR_EINVAL       (-1) /* bad argument: step 0, trip overflow, bad enum, sizes      */
#define UPIR_ENOTMAPPED   (-2) /* a buffer handle that is not (or no longer) mapped           */
#define UPIR_EBUSY        (-3) /* object still in use (e.g. unmap of a buffer a live region uses) */
#define UPIR_ENOMEM       (-4) /* the allocator returned NULL                                  */
#define UPIR_ECUDA        (-5) /* a CUDA runtime call failed                                   */
#define UPIR_ETIMEDOUT    (-6) /* a bounded device-side wait ran out (device error word set)  */
#define UPIR_EUNSUPPORTED (-7) /* valid request this library does not execute (e.g. K % 8 != 0 on tensor cores) */

/* Static text for a status code; never NULL. */
const char* upir_status_string(upir_status s);

/* ----------------------------------------------------------------- handles -- */

typedef struct upir_ctx_s*    upir_ctx;
typedef struct upir_buf_s*    upir_buf;
typedef struct upir_region_s* upir_region;
typedef struct upir_batch_s*  upir_batch;
typedef struct upir_event_s*  upir_event;

/* Device allocator callback.  alloc returns device memory of at least `bytes`
 * bytes, 256-byte aligned, usable in stream order on `stream`, or NULL.
 * free releases it in stream order. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void  (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} upir_allocator;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to
 * enqueue on (NULL: the context creates and owns its own non-blocking stream).
 * `allocator` may be NULL (cudaMalloc/cudaFree).  The context owns a
 * small device workspace (reduction partials, counters, the device error word).
 * Errors: EINVAL (out == NULL, bad device), ECUDA, ENOMEM. */
upir_status upir_init(upir_ctx* out, int32_t device, void* cuda_stream,
                      const upir_allocator* allocator);

/* Wait for the stream, free every buffer still mapped (no copy back), every
 * region and batch, and the context.  A NULL context is a no-op. */
upir_status upir_finalize(upir_ctx ctx);

/* Text describing the last error on `ctx` (valid until the next call on it). */
const char* upir_last_error(upir_ctx ctx);

/* ------------------------------------------------------------ data mapping -- */
/* §4.1: the data-mapping property of a data item is to, from, tofrom or
 * allocate. */

typedef enum {
    UPIR_MAP_TO     = 0, /* allocate + host->device copy at map; no copy back at unmap     */
    UPIR_MAP_FROM   = 1, /* allocate (contents undefined) at map; device->host at unmap    */
    UPIR_MAP_TOFROM = 2, /* host->device at map; device->host at unmap                     */
    UPIR_MAP_ALLOC  = 3  /* allocate only (contents undefined); no copies                  */
} upir_map_kind;

/* Map `bytes` bytes at host address `host` with mapping `kind`.  The copy for
 * TO/TOFROM is enqueued on the context stream (asynchronous with respect to the
 * host when `host` is page-locked).  bytes == 0 gives a valid empty mapping.
 * Errors: EINVAL (NULL out, NULL host with bytes > 0 for TO/FROM/TOFROM, bad
 * kind), ENOMEM, ECUDA. */
upir_status upir_data_map(upir_ctx ctx, void* host, size_t bytes, int32_t kind,
                          upir_buf* out);

/* Wrap caller-owned device memory (e.g. a resident torch tensor) as a mapped
 * buffer: no allocation, no copy, and unmap neither copies nor frees it. */
upir_status upir_data_map_device(upir_ctx ctx, void* device_ptr, size_t bytes,
                                 upir_buf* out);

/* Explicit data movement of a mapped buffer (§4.2, data_update):
 * direction UPIR_MAP_TO copies host->device, UPIR_MAP_FROM device->host and
 * waits for it.  EINVAL for a device-wrapped buffer or another direction. */
upir_status upir_data_update(upir_ctx ctx, upir_buf buf, int32_t direction);

/* End a mapping: for FROM/TOFROM enqueue the device->host copy, wait for the
 * stream, then release the device memory.  EBUSY if a live region or batch
 * still refers to the buffer (destroy those first); ENOTMAPPED for a stale
 * handle. */
upir_status upir_data_unmap(upir_ctx ctx, upir_buf buf);

/* Device address and size of a mapped buffer. */
upir_status upir_buf_device_ptr(upir_buf buf, void** device_ptr, size_t* bytes);

/* ----------------------------------------------- asynchronous data movement --
 * §4 leaves data movement to the runtime so that copies can overlap and be
 * pipelined with the computation.  These calls put the copies on the
 * context's copy streams and return at once.  A buffer's copy is ordered
 * after the buffer's previous copies and after the submitted work that uses
 * the buffer (the regions and batches submitted with it, device-side copies,
 * synchronous copies to it), not after unrelated work; a later submission
 * that uses the buffer waits (on the device) for the copy.  Overlap with computation needs
 * page-locked host memory (pageable memory still works, without overlap).
 *
 * Host->device and device->host copies use separate streams, so both copy
 * directions and the computation can overlap; one buffer's copies stay in
 * the order they were issued.
 * upir_data_map_async: like upir_data_map; TO/TOFROM copy host->device
 *   asynchronously (the host memory must stay unchanged until the copy is
 *   done: upir_buf_wait or a later submission that uses the buffer).
 * upir_data_update_async: like upir_data_update; FROM copies device->host
 *   asynchronously: read the host memory only after upir_buf_wait.
 * upir_buf_wait: the host waits for the buffer's pending copy (if any).
 * upir_data_unmap and upir_ctx_wait also wait for pending copies.
 * Errors as for the synchronous calls. */
upir_status upir_data_map_async(upir_ctx ctx, void* host, size_t bytes, int32_t kind, upir_buf* out);
upir_status upir_data_update_async(upir_ctx ctx, upir_buf buf, int32_t direction);
upir_status upir_buf_wait(upir_ctx ctx, upir_buf buf);

/* Device-side copy between mapped buffers (the device-to-device case of the
 * data movement of §4.2): the first src->bytes bytes of dst become those of
 * src, on the context's compute stream, after both buffers' pending
 * asynchronous copies and the work submitted so far; later submissions and
 * copies see the result.  Returns at once.  Use: one host array that seeds
 * two device buffers (the two grids of a Jacobi iteration) crosses the host
 * link once.  EINVAL if dst is smaller than src; ENOTMAPPED for a stale
 * handle; dst == src or an empty src does nothing. */
upir_status upir_buf_copy(upir_ctx ctx, upir_buf dst, upir_buf src);

/* ------------------------------------------------------ two-step sync steps --
 * §5: a sync is an arrive-compute step (a unit reaches the sync point and its
 * part of the work is issued) and a wait-release step (it waits for everyone
 * and is released); the asynchronous form splits them so that work can go
 * between.  Here the work is what a context has submitted:
 * upir_ctx_arrive: arrive-compute; *out marks everything submitted to the
 *   context so far (an event on its stream).
 * upir_event_query: UPIR_OK when that work has completed, UPIR_EBUSY if not.
 * upir_event_wait: wait-release on the host (blocks until completion).
 * upir_ctx_wait_event: wait-release on the device: work later submitted to
 *   `ctx` starts after the event's work (also across contexts on one device).
 * upir_event_destroy: release the event (after waits that use it). */
upir_status upir_ctx_arrive(upir_ctx ctx, upir_event* out);
upir_status upir_event_query(upir_event ev);
upir_status upir_event_wait(upir_event ev);
upir_status upir_ctx_wait_event(upir_ctx ctx, upir_event ev);
upir_status upir_event_destroy(upir_event ev);

/* ------------------------------------------------------------- SPMD region -- */
/* §3.1: an SPMD region runs num_teams teams of num_units units each.  Here a
 * team is a CUDA thread block and a unit a thread, so the launch geometry is
 * exactly <<<num_teams, num_units>>> (1 <= num_units <= 1024).  0 for either
 * lets the planner choose it per loop.  The returned region is empty; loops and
 * syncs are recorded into it and run by upir_region_submit().  A region can be
 * submitted any number of times. */
upir_status upir_spmd_region(upir_ctx ctx, int32_t num_teams, int32_t num_units,
                             upir_region* out);

/* --------------------------------------------------------- worksharing loop -- */

/* Schedule policies of §3.2 (worksharing schedule static | dynamic | guided |
 * runtime | auto, and the taskloop parallelization).  W = the loop's workers.
 *  STATIC    see upir_loop_desc.
 *  DYNAMIC   chunks of `chunk` iterations (0 means 1), in increasing order, to
 *            whichever worker asks next.
 *  GUIDED    like DYNAMIC, but each chunk holds max(chunk, ceil(R / W))
 *            iterations, R being those not yet handed out (chunk 0 means 1).
 *  RUNTIME   the context's run schedule (upir_ctx_set_run_schedule; default
 *            STATIC with chunk 0, or the UPIR_SCHEDULE environment variable
 *            "static|dynamic|guided[,chunk]" read by upir_init).
 *  AUTO      the runtime chooses: with a cost model installed
 *            (upir_ctx_set_cost_model) the candidate schedule and units per
 *            team it predicts fastest (AXPY, JACOBI5, MATVEC and GEMM_F32
 *            bodies; the others take STATIC), else STATIC with the planner's
 *            geometry.
 *  TASKLOOP  the iterations are cut into tasks (hints GRAINSIZE g: max(1,
 *            trip / g) tasks; NUM_TASKS n: min(n, trip) tasks; with both the
 *            smaller count; with neither 8 tasks per SM, 1184), contiguous,
 *            the first (trip mod tasks) one iteration longer, which the
 *            workers claim dynamically.  chunk must be 0.
 * Tiled bodies (tiled JACOBI5, JACOBI5_TB, FILTER7, GEMM_F32) schedule their
 * tiles: chunks, tasks and W count tiles and teams there.  The tensor-core
 * GEMM takes STATIC (and RUNTIME / AUTO resolving to it) only. */
typedef enum {
    UPIR_SCHED_STATIC = 0, UPIR_SCHED_DYNAMIC = 1, UPIR_SCHED_GUIDED = 2, UPIR_SCHED_RUNTIME = 3,
    UPIR_SCHED_AUTO = 4, UPIR_SCHED_TASKLOOP = 5
} upir_sched;

typedef enum {
    UPIR_RED_NONE = 0, UPIR_RED_ADD = 1, UPIR_RED_MUL = 2, UPIR_RED_MAX = 3, UPIR_RED_MIN = 4
} upir_red_op;

typedef enum { UPIR_F32 = 0, UPIR_I64 = 1 } upir_dtype;

/* Loop bodies (hand-written sm_103a kernels).  Buffers (bufs[]) and scalars
 * (scalars[]) per body; all arrays are dense, row-major, FP32 unless stated.
 *
 *  AXPY      bufs x[n], y[n]; scalars a [, imod_mul, imod_mod].
 *            y[iv] = fma(a, x[iv], y[iv]) for every induction value iv  (§6 AXPY)
 *  IMOD      no bufs; scalars imod_mul, imod_mod.  Empty body: only reduction
 *            terms over iv.
 *  COVERAGE  bufs owner[trip] (int64), count[trip] (int64) [; scalars imod_mul,
 *            imod_mod].  owner[k] = flattened worker id (team*units + unit) that
 *            ran logical iteration k, count[k] += 1: schedule instrumentation.
 *  JACOBI5   bufs u_in[rows*cols], u_out[rows*cols]; scalars rows, cols.
 *            collapse(2) over interior rows [lb, ub) (1 <= lb, ub <= rows-1, step 1)
 *            and all interior columns: u_out = 0.25*((N+S)+(W+E)), rounded per
 *            operation, no contraction.  Other points of u_out are not written.
 *  MATVEC    bufs A[rows*cols], x[cols], y[rows]; scalars rows, cols.
 *            y[r] = sum_j A[r][j] x[j] for rows r of the loop (§6 matvec).
 *  GEMM_F32  bufs A[M*K], B[K*N], C[M*N]; scalars M, N, K.  C = A B, FP32 SIMT.
 *  GEMM_BF16 bufs A[M*K] bf16, Bt[N*K] bf16 (B transposed, K contiguous),
 *            C[M*N] FP32; scalars M, N, K.  Tensor cores (tcgen05), FP32 accumulate.
 *  GEMM_BF16X3 bufs A_hi, A_lo [M*K] bf16, Bt_hi, Bt_lo [N*K] bf16, C[M*N];
 *            scalars M, N, K.  C = A_hi B_hi + A_hi B_lo + A_lo B_hi on tensor cores.
 *  SPLIT_BF16 bufs src[rows*cols] FP32, hi, lo (bf16) ; scalars rows, cols,
 *            transpose (0/1).  hi = bf16(src), lo = bf16(src - hi) (round to
 *            nearest even); with transpose the outputs are [cols*rows].
 *
 *  JACOBI5_TB bufs u_in[rows*cols], u_out[rows*cols]; scalars rows, cols,
 *            sweeps (1..8).  collapse(2) like JACOBI5; the loop carries `sweeps`
 *            successive JACOBI5 sweeps of u_in in which only rows [lb, ub) of
 *            the interior columns change and every other point keeps its u_in
 *            value; u_out receives the last sweep's values on those points (no
 *            other point is written).  Each sweep's arithmetic is JACOBI5's, so
 *            when the buffers agree on the fixed points the result equals
 *            `sweeps` JACOBI5 loops.  A TERM_RESID max/min reduction reduces
 *            sweep k into element index + k (k < sweeps) of its variable.
 *            Needs cols % 4 == 0 and 16-byte aligned buffers (EUNSUPPORTED).
 *  FILTER7   bufs x_in[rows*cols], x_out[rows*cols]; scalars rows, cols, then
 *            the 49 weights w[i][j] of the 7 x 7 window, row-major (the size-7
 *            filter of the §6 stencil evaluation).  collapse(2) over rows
 *            [lb, ub) (3 <= lb, ub <= rows-3, step 1) and columns [3, cols-3):
 *            x_out[r][c] = sum over i, j of w[i][j] x_in[r+i-3][c+j-3], an FP32
 *            fused multiply-add chain from 0 in row-major (i, then j) order.
 *            No reductions; cols % 4 == 0 and 16-byte aligned buffers.
 *
 *  GEMM bodies: the loop runs over rows [lb, ub) of C with collapse 2 (all N
 *  columns); tensor-core bodies need K % 8 == 0 (EUNSUPPORTED otherwise).
 */
typedef enum {
    UPIR_BODY_AXPY = 0, UPIR_BODY_IMOD = 1, UPIR_BODY_JACOBI5 = 2, UPIR_BODY_MATVEC = 3,
    UPIR_BODY_GEMM_F32 = 4, UPIR_BODY_GEMM_BF16 = 5, UPIR_BODY_GEMM_BF16X3 = 6,
    UPIR_BODY_COVERAGE = 7, UPIR_BODY_SPLIT_BF16 = 8, UPIR_BODY_JACOBI5_TB = 9,
    UPIR_BODY_FILTER7 = 10
} upir_body;

/* Value each iteration contributes to a reduction.
 *   TERM_Y     AXPY: the updated y[iv];  MATVEC: y[r]
 *   TERM_XY    AXPY: x[iv] * y[iv] (after the update; "AXPY + dot")
 *   TERM_IMOD  (imod_mul * iv) mod imod_mod, 64-bit wrap, remainder in [0, mod)
 *   TERM_IV    the induction value iv itself
 *   TERM_RESID JACOBI5: |u_out - u_in| at the point                          */
typedef enum {
    UPIR_TERM_Y = 0, UPIR_TERM_XY = 1, UPIR_TERM_IMOD = 2, UPIR_TERM_IV = 3, UPIR_TERM_RESID = 4
} upir_term;

/* A reduction clause (§5: sync "reduction" with an operation and its data).
 * The variable is element `index` of mapped buffer `var` (FP32 or int64).  Its
 * value before the loop is combined exactly once with the iterations' terms.
 * FP32 "+" is compensated (TwoSum) and, like FP32 "*", combined in a fixed tree
 * order over per-team (static) or per-chunk (dynamic) partials, so results are
 * bit-identical from run to run.  max/min (FP32: NaN operands ignored) and
 * int64 +, *, max, min (two's-complement wrap) are exact in any order. */
typedef struct {
    int32_t  op;     /* upir_red_op */
    int32_t  dtype;  /* upir_dtype  */
    int32_t  term;   /* upir_term   */
    int32_t  reserved;
    upir_buf var;
    int64_t  index;
} upir_reduction;

/* Tuning hints (§2.4 "UPIR extension": key-value pairs).  Unknown keys: EINVAL.
 * UPIR_HINT_VARIANT values: JACOBI5 1 = the per-point kernel (a unit per
 * point) instead of the tiled one (2D TMA boxes, or one TMA copy per halo row
 * for widths that are not a multiple of 4); GEMM_BF16 1 = one SM per 128 x 256
 * tile, 2 = CTA pairs (tcgen05 cta_group::2, 256 x 256 tiles; EUNSUPPORTED
 * with explicit teams, a chunk, a TILE_M hint or when no two-CTA cluster
 * fits), 0 = the planner's choice (pairs when every resident cluster gets a
 * tile); GEMM_F32 1 = the kernel that stages loads through registers (the
 * default, TMA-fed kernel needs K and N multiples of 4 and 16-byte aligned
 * buffers, and gives the same result bit for bit); FILTER7: each thread
 * computes strips of 4 output rows (0, 2) or 8 (1, 3; TILE_M then a multiple
 * of 8), two rows of a strip sharing one paired FMA (fma.rn.f32x2, each half
 * rounded once; 0, 1) or one FMA per output (2, 3), all four with the same
 * result bit for bit.  UPIR_HINT_STAGES also sets FILTER7's TMA ring depth
 * (2, the default, or 3). */
typedef enum {
    UPIR_HINT_VARIANT   = 1, /* kernel variant of the body (body-specific, 0 = default)       */
    UPIR_HINT_TILE_M    = 2, /* tile rows (JACOBI5 tiled variant, GEMM)                       */
    UPIR_HINT_TILE_N    = 3, /* tile cols                                                     */
    UPIR_HINT_VEC       = 4, /* iterations per worker the planner aims for (1, 4, 8, 16, 32) */
    UPIR_HINT_STAGES    = 5, /* shared-memory pipeline depth (tiled JACOBI5: 1..4; FILTER7: 2, 3) */
    UPIR_HINT_GRAINSIZE = 6, /* taskloop grainsize (>= 1; schedule TASKLOOP only)             */
    UPIR_HINT_NUM_TASKS = 7, /* taskloop num_tasks (>= 1; schedule TASKLOOP only)             */
    UPIR_HINT_TILE_ORDER = 8 /* tiled JACOBI5: 0 = planner's choice, 1 = ascending, 2 = descending */
} upir_hint_key;

/* UPIR_HINT_TILE_ORDER: under a blocked static schedule (chunk 0) each team
 * owns a contiguous run of tiles; the order it walks them in is not part of
 * the schedule (the sweep's iterations are independent and its max/min
 * residual is exact in any order), so the result is the same bit for bit
 * either way.  With 0 (the default) a tiled JACOBI5 loop whose input is the
 * output of the loop just before it in the region (a tiled JACOBI5 loop that
 * walked its tiles ascending) walks its own tiles descending: the sweep then
 * starts on the rows the previous sweep wrote last, which are still in L2.
 * 1 keeps every team ascending; 2 makes every team walk descending (for a
 * caller that runs each sweep as a region of its own and alternates the
 * order itself).  Schedules other than blocked static walk ascending; other
 * bodies ignore the hint. */

/* The canonical loop with its worksharing parallelization (§3.2).
 * Iterations: iv = lb, lb+step, ... while iv < ub (step > 0) or iv > ub
 * (step < 0); trip = ceil((ub-lb)/step) or 0; step 0 is EINVAL.
 * sched/chunk: static chunk c > 0 gives logical chunk j (iterations
 * [j c, min((j+1) c, trip))) to worker j mod W; static chunk 0 splits the
 * iterations into W contiguous blocks, the first (trip mod W) one longer;
 * dynamic chunk c (0 means 1) hands out chunks in increasing order to whichever
 * worker asks next.  W = teams * units for element bodies; the MATVEC worker is
 * a warp and the tiled JACOBI5 / GEMM worker is a team (the loop is tiled and
 * the tile loop workshared).  nowait drops the implicit barrier at the loop's
 * end (§5): the next loop may run beside this one; it completes only after
 * this one, so the implicit barrier after it (or any later barrier) covers
 * both.
 * Validation is eager: upir_loop() checks every field, buffer size and index
 * range against the mapped buffers and returns EINVAL/ENOTMAPPED/EUNSUPPORTED
 * without recording anything on error. */
typedef struct {
    int64_t lb, ub, step;
    int32_t collapse;      /* 1, or 2 for JACOBI5 / GEMM_* */
    int32_t sched;         /* upir_sched */
    int64_t chunk;         /* >= 0 */
    int32_t body;          /* upir_body */
    int32_t nbufs;
    const upir_buf* bufs;
    int32_t nscalars;
    int32_t nreductions;   /* 0..2 */
    const double* scalars;
    const upir_reduction* reductions;
    int32_t nowait;
    int32_t nhints;        /* number of (key, value) pairs */
    const int64_t* hints;  /* key0, value0, key1, value1, ... */
} upir_loop_desc;

upir_status upir_loop(upir_region region, const upir_loop_desc* loop);

/* -------------------------------------------------------------------- sync -- */

typedef enum { UPIR_SYNC_BARRIER = 0, UPIR_SYNC_TASKWAIT = 1 } upir_sync_kind; /* §5 subset */

/* BARRIER records an explicit barrier after the last recorded loop (redundant
 * with an implicit one, which the runtime then elides).  TASKWAIT blocks the
 * host until everything submitted on the context has finished and reports a
 * device-side error (ETIMEDOUT) if one was raised. */
upir_status upir_sync(upir_region region, int32_t kind);

/* ----------------------------------------------------------------- execute -- */

#define UPIR_SUBMIT_GRAPH 1  /* capture the region's launches in a CUDA graph once, replay it */

/* Enqueue every recorded loop of the region on the context stream, in order.
 * Asynchronous: returns once enqueued.  Buffers are resolved at submit time
 * (ENOTMAPPED if one was unmapped since). */
upir_status upir_region_submit(upir_region region, int32_t flags);

/* Free a region (waits for nothing: its launches already hold what they need). */
upir_status upir_region_destroy(upir_region region);

/* Many independent regions at once.
 *   LAUNCHES   : one launch per loop, regions one after another on the stream
 *   GRAPH      : the same launches captured once in a CUDA graph and replayed
 *   PERSISTENT : one persistent kernel over a work list of (region, tile)
 *                items, largest regions first, claimed one by one from an
 *                atomic counter by as many teams as the GPU holds at once;
 *                each region's FP32 "+" reduction is finalized by its last
 *                tile, folding the tile partials in tile order.  The launch
 *                is captured in a CUDA graph.
 * PERSISTENT accepts regions holding exactly one loop: AXPY (step 1, at most
 * one FP32 "+" clause over TERM_Y or TERM_XY), JACOBI5 (at most one max/min
 * residual clause) or MATVEC (step 1); others give EUNSUPPORTED.  Results are
 * those of the regions run alone (FP32 sums to rounding order).  A region in
 * a batch cannot take more loops or be destroyed until the batch is (EBUSY). */
typedef enum { UPIR_BATCH_LAUNCHES = 0, UPIR_BATCH_GRAPH = 1, UPIR_BATCH_PERSISTENT = 2 } upir_batch_mode;

upir_status upir_batch_create(upir_ctx ctx, const upir_region* regions, int32_t n,
                              int32_t mode, upir_batch* out);
upir_status upir_batch_submit(upir_batch batch);
upir_status upir_batch_destroy(upir_batch batch);

/* Autotune the tile shapes of a PERSISTENT batch: every candidate (AXPY
 * iterations per tile 4096..32768, Jacobi rows per tile 8..32, matvec rows
 * per tile 8..32 for rows wider than 64 columns, narrower rows going 256 to a
 * tile whatever the choice) is run `reps` times after one warm-up and timed with CUDA
 * events; the shapes with the least median time are kept.  The batch really
 * runs each time, so loops that update in place (AXPY) see every run.
 * tiles_out (may be NULL) receives the chosen {axpy_tile, jacobi_rows,
 * matvec_rows}.  Blocks the host.  EINVAL for other modes or reps < 1. */
upir_status upir_batch_autotune(upir_batch batch, int32_t reps, int64_t* tiles_out);

/* Taskwait at context level: wait for the stream, then read and clear the
 * device error word (ETIMEDOUT if a bounded wait ran out).  On ETIMEDOUT the
 * outputs of the launches in flight are undefined, and the scheduling
 * counters of every live region's loops are cleared, so regions can be
 * submitted again. */
upir_status upir_ctx_wait(upir_ctx ctx);

/* ------------------------------------------------------------ diagnostics -- */

/* Launch records: when enabled, every kernel launch of a submitted loop is
 * bracketed by CUDA events on the context stream.  upir_ctx_timings() waits
 * for the stream and returns up to `cap` per-launch durations (ms) recorded
 * since the last call, with the body of each; *count gets the number written. */
upir_status upir_ctx_set_timing(upir_ctx ctx, int32_t enable);
upir_status upir_ctx_timings(upir_ctx ctx, float* ms, int32_t* body, int32_t cap,
                             int32_t* count);

/* Launch geometry the planner chose for loop `loop_index` of a region (after
 * upir_loop): teams (grid) and units (block) of its main kernel. */
/* Schedule the planner settled on for loop `loop_index` (RUNTIME and AUTO
 * resolved): *sched (STATIC, DYNAMIC, GUIDED or TASKLOOP), *chunk, and
 * *nchunks, the number of chunks or tasks handed out dynamically (0 for
 * STATIC).  Any output pointer may be NULL. */
upir_status upir_region_loop_schedule(upir_region region, int32_t loop_index, int32_t* sched,
                                      int64_t* chunk, int64_t* nchunks);

upir_status upir_region_loop_geometry(upir_region region, int32_t loop_index,
                                      int32_t* teams, int32_t* units);

/* Bounded-wait self test: launches one block that waits on an mbarrier phase
 * nothing will complete, with the same bounded-spin helper the tensor-core
 * GEMM uses, giving up after `spin_limit` polls.  The wait ends, the device
 * error word is set and the next upir_ctx_wait() returns UPIR_ETIMEDOUT; the
 * context stays usable. */
upir_status upir_selftest_bounded_wait(upir_ctx ctx, int64_t spin_limit);

/* Spin budget (polls) of every bounded device-side wait; default 2^26, also
 * settable with the environment variable UPIR_SPIN_LIMIT. */
upir_status upir_ctx_set_spin_limit(upir_ctx ctx, int64_t spin_limit);

/* The run schedule that loops with UPIR_SCHED_RUNTIME take when they are
 * recorded: sched STATIC, DYNAMIC or GUIDED with chunk >= 0.  EINVAL
 * otherwise. */
upir_status upir_ctx_set_run_schedule(upir_ctx ctx, int32_t sched, int64_t chunk);

/* Install the learned cost model that UPIR_SCHED_AUTO consults when a loop is
 * recorded: `params` are the UPIR_MLP_NPARAM FP32 parameters of the
 * 12 -> 64 -> 64 -> 1 MLP (layout of upir_mlp_forward), `feat_mean` and
 * `feat_std` the 12 feature means and standard deviations the inputs are
 * standardised with (std <= 0 counts as 1).  All host pointers, copied.  The
 * features of a candidate are: body one-hot (AXPY, JACOBI5, MATVEC, GEMM),
 * log2 trip (JACOBI5: interior points; GEMM_F32: output elements), bytes and
 * flops per iteration (AXPY 12, 4; JACOBI5 8, 6; MATVEC 4 cols, 2 cols;
 * GEMM_F32 K / 16, 2 K), schedule one-hot (static, dynamic), log2(chunk + 1),
 * log2 units, log2 teams: the teams the planner launches the candidate with
 * (found by planning the loop without device scratch when it is recorded).
 * The prediction uses bfloat16-rounded weights and FP32 arithmetic on the
 * host.  params NULL removes the model. */
upir_status upir_ctx_set_cost_model(upir_ctx ctx, const float* params, const float* feat_mean,
                                    const float* feat_std);

/* Host-only helpers of the auto schedule (no GPU needed).
 * upir_auto_candidates: the candidate (sched, chunk, units) triples the cost
 *   model ranks for a body (AXPY, JACOBI5, MATVEC, GEMM_F32; none for the
 *   others);
 *   *count gets their number, at most `cap` are written (arrays may be NULL).
 * upir_auto_features: the 12 features of one candidate; trip is the loop's
 *   trip count (rows for JACOBI5 and MATVEC; output elements, rows x N, for
 *   GEMM_F32), cols the grid / matrix width (K for GEMM_F32).
 * upir_auto_pick: the candidate the model (params, feat_mean, feat_std as for
 *   upir_ctx_set_cost_model; params NULL: none) predicts fastest, restricted
 *   to `units` when non-zero, every candidate scored with the same `teams`
 *   feature (no loop is planned here); *units_out is its units (0 when fixed
 *   or when no candidate applies, the schedule then being STATIC with chunk 0).
 * EINVAL for bad pointers or sizes. */
upir_status upir_auto_candidates(int32_t body, int32_t* sched, int64_t* chunk, int32_t* units, int32_t cap,
                                 int32_t* count);
upir_status upir_auto_features(int32_t body, int64_t trip, int64_t cols, int32_t sched, int64_t chunk,
                               int32_t units, int32_t teams, float* out);
upir_status upir_auto_pick(const float* params, const float* feat_mean, const float* feat_std, int32_t body,
                           int64_t trip, int64_t cols, int32_t units, int32_t teams, int32_t* sched,
                           int64_t* chunk, int32_t* units_out);

/* ------------------------------------------- allocation-free AXPY variant -- */
/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: code whose device memory is fully reserved by its
 * own pool, latency-critical paths where a cudaMalloc would synchronize the
 * device, and embedders that cannot create a context (upir_init allocates) or
 * hand the library an allocator.
 *
 * y[i] = fma(a, x[i], y[i]) for 0 <= i < n, then
 *   *sum_y    += sum of the updated y[i]        (FP32, compensated, fixed order)
 *   *imod_sum += sum of (imod_mul * i) mod imod_mod  (int64, exact)
 * with the same kernels as an AXPY loop recorded through upir_loop with a
 * static schedule, chunk 0 and those two reduction clauses, on teams of 256
 * units with 8 iterations per unit: y and *imod_sum are identical to that
 * loop's; *sum_y may differ in its last bits when the loop runs in another
 * geometry (the fixed summation order follows the teams).  x, y, sum_y and imod_sum are device
 * pointers owned by the caller; the work is enqueued on `cuda_stream` (NULL:
 * the legacy default stream) of the current device and the call returns
 * without waiting.  Nothing is allocated: the reduction scratch is one fixed
 * array of about 512 KiB inside the library's device image, which every GPU
 * that loads the library holds until the process exits.
 *
 * Limits and errors: n <= 67,108,864 (2^26) and 1 <= imod_mod < 2^62 with
 * |imod_mul| * (n - 1) < 2^62, else UPIR_EINVAL; NULL pointers: UPIR_EINVAL;
 * n == 0 leaves the variables unchanged.  The first call on a device looks up
 * the array's device address (once per device, with that device current), so
 * make that first call before any stream capture.  That address is kept for
 * the life of the process, so do not use this call across a device reset
 * (cudaDeviceReset or a reset of the primary context), which moves the
 * array.  Every call shares the one
 * array: calls whose work overlaps on the GPU (other streams, other threads)
 * race and give wrong results; serialize them. */
upir_status upir_axpy_reduce_noalloc(const float* x, float* y, int64_t n, float a,
                                     int64_t imod_mul, int64_t imod_mod, float* sum_y,
                                     int64_t* imod_sum, void* cuda_stream);

/* ------------------------------------------------------ learned cost model -- */
/* A 12 -> 64 -> 64 -> 1 ReLU MLP predicting log2 of a loop's time from its
 * features; weights used in bfloat16, FP32 accumulation and FP32 master
 * weights.  Parameter block layout (FP32, contiguous, 5,121 floats):
 *   W1[64][12], b1[64], W2[64][64], b2[64], W3[1][64], b3[1].
 * All pointers are device pointers; calls are enqueued on the context stream. */

#define UPIR_MLP_IN     12
#define UPIR_MLP_HIDDEN 64
#define UPIR_MLP_NPARAM (64 * 12 + 64 + 64 * 64 + 64 + 64 + 1)

/* pred[b] for b < batch; x is [batch][12]. */
upir_status upir_mlp_forward(upir_ctx ctx, const float* params, const float* x,
                             int32_t batch, float* pred);

/* Mean-squared-error loss against target[batch] and its gradient with respect
 * to every parameter (same layout as params).  loss may be NULL. */
upir_status upir_mlp_backward(upir_ctx ctx, const float* params, const float* x,
                              const float* target, int32_t batch, float* grad,
                              float* loss);

/* params -= lr * grad, elementwise. */
upir_status upir_mlp_sgd(upir_ctx ctx, float* params, const float* grad, float lr);

#ifdef __cplusplus
}
#endif

#endif /* UPIR_H */
