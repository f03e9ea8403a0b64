/*
 * omprt.h - C ABI of a GB300-native (sm_103a) OpenMP device-runtime hot path.
 *
 * The paper ("Experience Report: Writing A Portable GPU Runtime with OpenMP
 * 5.1", arXiv 2106.03219) describes the LLVM OpenMP device runtime: the
 * routines an offloaded region calls on the GPU, among them the division of
 * loop iterations (Sec. 1, Sec. 2), __kmpc_alloc_shared (Sec. 2.1, Listing 1),
 * team-shared state with one team per thread block (Sec. 3.1, "Global Shared
 * Variables"), the flush and the five atomics (Sec. 3.1, Listings 2-3) and
 * synchronisation / thread hierarchy (Sec. 3.2).  This library provides the
 * data-parallel subset of those routines that a
 *     #pragma omp target teams distribute parallel for [reduction(...)]
 * loop spends its time in, as hand-written CUDA kernels, behind plain C calls.
 * The host launch call plays the role of the host runtime's target-launch
 * entry (Sec. 2.2: kernel id, base pointers, argument count).
 *
 * Conventions for every call:
 *   - Pointers named *_dev or held in descriptors are DEVICE pointers owned
 *     by the caller; the library never frees them.  Pointers named *_host are
 *     host memory.  The context (omprt_ctx) owns only its own scratch.
 *   - stream is a CUDA stream handle (cudaStream_t / CUstream) passed as
 *     void*; NULL means the legacy default stream.  Every launch is
 *     asynchronous on that stream.
 *   - Host-side argument errors return a non-OK status immediately and launch
 *     nothing.  Errors detected on the device set bits in a sticky device
 *     status word that omprt_sync_status reads and clears.  No call throws or
 *     traps.
 *   - Calls that launch work allocate nothing after omprt_init (and after
 *     omprt_batch_create for the batch call), so they may be captured in a
 *     CUDA graph.
 *   - A context's scratch (cross-team partials, tickets, dispatch counters)
 *     is handed out from a ring of OMPRT_SLOTS slots, one per launch; up to
 *     OMPRT_SLOTS launches from one context may be in flight at once on
 *     different streams.  Replays of a captured graph reuse the slots baked
 *     into it, so one captured graph must not be replayed concurrently with
 *     itself.
 */
#ifndef OMPRT_H_
#define OMPRT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OMPRT_SLOTS 64
/* teams of a launch that reduces or uses dynamic dispatch */
#define OMPRT_MAX_RED_TEAMS 16384
/* fallback-pool bytes per team for the shared-memory stack */
#define OMPRT_POOL_BYTES_PER_TEAM 4096

typedef enum {
    OMPRT_OK = 0,
    OMPRT_ERR_INVALID = 1,      /* bad argument; nothing launched */
    OMPRT_ERR_NOMEM = 2,        /* device allocation failed (init / batch create) */
    OMPRT_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    OMPRT_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    OMPRT_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement */
    OMPRT_ERR_NOT_INIT = 6,     /* NULL context */
    OMPRT_ERR_DEVICE = 7        /* the sticky device status word is non-zero */
} omprt_status;

/* Device status bits (sticky, OR-ed by kernels, read by omprt_sync_status). */
#define OMPRT_DEV_STACK_NOMEM 0x1u  /* shared stack and its pool were exhausted */
#define OMPRT_DEV_STACK_ORDER 0x2u  /* free of a block that is not on top */
#define OMPRT_DEV_TIMEOUT 0x4u      /* a bounded wait gave up */
#define OMPRT_DEV_BAD_ARG 0x8u      /* a kernel saw an argument it cannot honour */

/* Loop schedules (OpenMP loop-schedule semantics; the paper puts the
 * division of loop iterations in the runtime, Sec. 1 and Sec. 2). */
typedef enum {
    OMPRT_SCHED_STATIC = 0,         /* chunk 0: one contiguous piece per thread;
                                       chunk c > 0: same as STATIC_CHUNKED */
    OMPRT_SCHED_STATIC_CHUNKED = 1, /* chunks of c, round robin over threads */
    OMPRT_SCHED_DYNAMIC = 2,        /* chunks of c claimed at run time from a
                                       per-team counter in global memory */
    OMPRT_SCHED_AUTO = 3,           /* mapping left to the runtime: grid-stride
                                       over 32-byte vectors */
    OMPRT_SCHED_LEARNED = 4,        /* schedule, chunk and teams chosen by the
                                       context's cost model (see
                                       omprt_set_cost_model), else the heuristic */
    OMPRT_SCHED_GUIDED = 5,         /* each request takes max(c, ceil(r / 2T)) of
                                       the r iterations of the team's block not yet
                                       handed out (chunk c, 0 = 1); a warp claims 32
                                       such chunks with one compare-and-swap on a
                                       per-team counter (bounded retries; giving up
                                       sets OMPRT_DEV_TIMEOUT) */
    OMPRT_SCHED_NONMONOTONIC = 6    /* schedule(nonmonotonic: dynamic, c): chunks of
                                       c handed out at run time in any order.  The
                                       team's groups of 32 chunks are split evenly
                                       among its warps; a warp claims its own groups
                                       first (a counter in shared memory), then
                                       takes groups left to other warps.  Lane l of
                                       a claim runs chunk 32 g + l in full; a
                                       thread's chunks need not increase */
} omprt_sched;

typedef enum {
    OMPRT_I32 = 0, OMPRT_U32 = 1, OMPRT_I64 = 2, OMPRT_U64 = 3,
    OMPRT_F32 = 4, OMPRT_BF16 = 5, OMPRT_F64 = 6
} omprt_dtype;

typedef enum { OMPRT_OP_SUM = 0, OMPRT_OP_MAX = 1, OMPRT_OP_MIN = 2 } omprt_op;

/* Accumulation precision of floating-point sums. */
typedef enum {
    OMPRT_PREC_COMP_F64 = 0,  /* compensated fp32 per thread and per team,
                                 cross-team combine in fp64 (default) */
    OMPRT_PREC_COMP_F32 = 1,  /* compensated fp32 throughout, fp32 combine */
    OMPRT_PREC_NAIVE_F32 = 2  /* plain fp32 adds throughout */
} omprt_precision;

/* Loop bodies the executors run for each logical iteration i in [0, n). */
typedef enum {
    OMPRT_BODY_MAP_RECORD = 0, /* out: int32[n] owner id g*T + t;
                                  y: int32[n] execution counters, incremented
                                     atomically (NULL: skipped);
                                  x: int32[G*T] per-thread "last" flags
                                     (NULL: skipped) */
    OMPRT_BODY_AXPY = 1,       /* y[i] = alpha*x[i] + y[i]; data_type F32
                                  (single fma) or I32 (wrapping); reduces the
                                  new y[i] */
    OMPRT_BODY_STENCIL1D3 = 2, /* F32, out of place x -> out; interior
                                  out[i] = fma(c1, x[i-1]+x[i+1], c0*x[i]),
                                  end points copied; reduces out[i] */
    OMPRT_BODY_STENCIL2D5 = 3, /* F32 ny x nx row major, x -> out; interior
                                  out = fma(c1, (N+S)+(E+W), c0*C),
                                  boundary copied; n must equal nx*ny */
    OMPRT_BODY_DOT = 4,        /* F32, value x[i]*y[i] (rounded fp32 product)
                                  fed to the reduction; writes nothing */
    OMPRT_BODY_NONE = 5        /* value x[i] of data_type fed to the reduction */
} omprt_body;

/*
 * A worksharing loop  for (v = lb; incr > 0 ? v <= ub : v >= ub; v += incr).
 * Its trip count n is computed in the loop variable's type idx_type
 * (I32/U32/I64/U64; bounds given as 64-bit patterns and checked to lie in the
 * type; incr != 0).  Logical iteration i (v = lb + i*incr) touches element i
 * of the data arrays.  Data arrays are device pointers; 32-byte alignment
 * enables the 256-bit vector path, any 4-byte alignment is correct.
 */
typedef struct {
    int64_t lb, ub, incr;
    int32_t idx_type;          /* omprt_dtype, integer types only */
    int32_t body;              /* omprt_body */
    int32_t data_type;         /* omprt_dtype of x / y / out elements */
    int32_t reserved;          /* must be 0 */
    void *x, *y, *out;         /* device pointers, meaning per body */
    double alpha;              /* AXPY scale (rounded to fp32 or int32) */
    double c0, c1;             /* stencil weights (rounded to fp32) */
    int64_t nx, ny;            /* STENCIL2D5 grid */
    int32_t *seq;              /* MAP_RECORD only (NULL: skipped): int32[n];
                                  seq[i] = how many iterations the thread that
                                  ran i had run before it in this launch, so a
                                  thread's iterations sorted by seq are in the
                                  order it ran them.  Other bodies: NULL. */
} omprt_loop_desc;

/* reduction(op: var) clause of a region.  result_dev: 8 bytes of device
 * memory receiving a double (floating data) or an int64 (integer data);
 * sums of int32 data are widened to int64 and wrap modulo 2^64. */
typedef struct {
    int32_t op;                /* omprt_op */
    int32_t precision;         /* omprt_precision (floating sums only) */
    void *result_dev;
} omprt_reduce_desc;

typedef struct omprt_ctx omprt_ctx;

/* Create a context on a CUDA device: allocates the status word, the slot
 * ring (partials, tickets, dispatch counters) and the stack fallback pool.
 * All scratch starts zeroed and is left zeroed by every kernel, so no launch
 * needs a memset (explicit initialisation of uninitialised team state,
 * Sec. 3.1, "loader_uninitialized").  Returns OMPRT_ERR_CUDA / _NOMEM on
 * failure with *ctx untouched. */
omprt_status omprt_init(int device, omprt_ctx **ctx);

/* Free what omprt_init allocated: the context's scratch on the device (the
 * runtime's per-device state, Sec. 3.1) and the context itself.  The caller
 * must have synchronised its streams; ctx is invalid afterwards.  NULL is
 * OMPRT_ERR_NOT_INIT. */
omprt_status omprt_finalize(omprt_ctx *ctx);

/* Reserve the per-team shared-memory stack capacity S for later launches
 * (__kmpc_alloc_shared, Sec. 2.1, Listing 1).  S is rounded up to 16 and must
 * not exceed 200 KiB.  The runtime's own per-launch temporaries (reduction
 * scratch) are taken from this stack, so S below 1 KiB sends them to the
 * global fallback pool.  Default after init: 4 KiB. */
omprt_status omprt_alloc_shared(omprt_ctx *ctx, size_t bytes_per_team);

/* Per-team shared memory that dynamic and static schedules of streaming bodies
 * (axpy, dot, value reductions, the stencils) may use to stage their chunks.  The dispatch
 * and the ownership are unchanged (each warp takes 32 consecutive chunks of c,
 * lane l runs chunk base + l in full, Sec. 3.1 worksharing); the range is
 * moved through shared memory by bulk copies, P chunks per pass, with
 * P = min(32, bytes / (warps * arrays * c * element size)).  Schedules:
 * dynamic(c); static(c), where warp w's k-th set is chunks k*T + 32w + lane;
 * static without chunk when n = teams * threads * c' exactly (c' per thread).
 * A launch is staged when c * element size is a multiple of 16 and at least
 * 256, and P >= 16 (loops without a reduction), or P = 32 and c * element
 * size summed over the arrays is at most 512 (loops with one).  The
 * stencils (no reduction, n and nx multiples of 4) stage an input window that
 * reaches one element / one row beyond the pass, when the chunk is at most
 * 512 bytes and the two halos at most a quarter of the pass.  A claim of 32
 * chunks runs in equal passes.  Other launches, and teams whose block does
 * not start on a 16-byte boundary, run the plain form.  The 2-D stencil under
 * static(c) with c in [4, 8) or [32, 128] (fp32, no reduction, nx a multiple of
 * 4, n < 2^32, 16-byte-aligned pointers) instead walks each team's block in
 * passes of two rows through a six-row ring in shared memory (six rows of nx
 * floats, which must fit the device's per-block shared memory, whatever
 * `bytes`); every thread still runs exactly its own chunks.  bytes is rounded
 * down to 16; 0 turns every staged form, the row ring included, off; more than
 * the device's per-block shared memory is OMPRT_ERR_INVALID.  Default after
 * init: 32 KiB. */
omprt_status omprt_set_stage_bytes(omprt_ctx *ctx, int64_t bytes_per_team);

/* Shared memory per CTA that the 2-D stencil (fp32, no reduction) may use
 * under dynamic(c) and static(1) to stream its input.  A launch has at most as
 * many CTAs as fit the device at once; CTA k plays the consecutive teams
 * [k G / P, (k + 1) G / P) (OpenMP does not make teams run at the same time)
 * and reads their range of the grid, plus one row on each side, once, through
 * a ring of row-sized segments in shared memory filled by bulk copies (the
 * team-shared state of Sec. 3.1, "Global Shared Variables"): a producer warp
 * refills a slot as soon as every team group has released it.  The CTA's
 * threads form groups of thread_limit, each playing one team at a time; every
 * thread runs exactly the iterations the schedule gives it (Sec. 1, Sec. 2
 * worksharing), reading its operands from the ring.  Dynamic chunks are
 * claimed from the team's counter in shared memory, 32 per warp, lane l
 * running chunk base + l; a thread's claims increase.  The form applies when
 * nx is a multiple of 4, n < 2^32, both pointers are 16-byte aligned,
 * thread_limit <= 512 and the ring holds one team's rows with room to spare;
 * other launches run the forms of omprt_set_stage_bytes.  bytes is rounded
 * down to 16; 0 turns this form off, and with it the slab, band and column-ring
 * forms of omprt_set_stencil_slab_shape and the row ring of
 * dynamic(c) (those size their buffers from the device's shared memory);
 * more than the device's per-block shared memory is OMPRT_ERR_INVALID.
 * Default after init: 226 KiB. */
omprt_status omprt_set_stencil_stage_bytes(omprt_ctx *ctx, int64_t bytes_per_cta);

/* The slab form of the 2-D stencil (static(c) and dynamic(c) with c a
 * multiple of the slab line dividing nx, team blocks of whole rows, and
 * nx / c a multiple or a divisor of 32; on when stencil stage bytes are
 * non-zero): each warp takes its 32 chunks in slabs, one tensor copy a slab
 * (Sec. 3.1's team-shared staging, per warp), every thread running exactly
 * its own iterations.  slab_floats: floats of each chunk a slab holds, 16 or
 * 32; buffers: slabs a warp holds, 2 .. 4 (buffers - 1 copies in flight).
 * buffers also sets the band form of static(1) (team size dividing nx, team
 * blocks of whole rows: each warp's strips a band of rows at a time from
 * tensor copies) and the column ring (teams of 32 threads whose blocks are
 * the 32 / m rows holding 32 chunks, m = nx / c < 32: the CTA's warps play
 * adjacent teams from one tensor copy a step).  0 for either takes the
 * measured default (slabs: about 24 KB of buffers a warp; bands: 2; column
 * ring: 3).  Other values: OMPRT_ERR_INVALID, nothing changed. */
omprt_status omprt_set_stencil_slab_shape(omprt_ctx *ctx, int32_t slab_floats, int32_t buffers);

/* Whether the regions this context launches may overlap the tail of the
 * previous kernel on their stream.  On (non-zero, the default after init),
 * every executor kernel is launched with programmatic stream serialisation:
 * its blocks may be scheduled while the kernel before it on the stream
 * drains, and each block waits, before its first global memory access, until
 * that kernel has completed and its writes are visible, so results and
 * stream order are the same as with plain launches.  A region launched right
 * after another on the same stream then starts without the launch gap (a
 * 4096 x 4096 copy-sized launch saves about 2.4 us).  A launch asking for at
 * least 16 KiB less dynamic shared memory than the previous one on its stream
 * (made by this library on the same host thread), where blocks of both fit
 * one SM, is made plain: blocks started early beside the previous grid's
 * would run with that grid's small L1.  An event recorded between two
 * launches orders them as before.  omprt_reduce_noalloc, which takes no
 * context, always launches this way.  Off (0): plain launches. */
omprt_status omprt_set_launch_overlap(omprt_ctx *ctx, int32_t on);

/*
 * Run one "target teams distribute parallel for" region:
 *   level 1: the n logical iterations are split among num_teams teams in
 *            contiguous balanced blocks (the first n % G blocks one longer);
 *   level 2: each team's block is split among its thread_limit threads by
 *            `sched` with chunk `chunk` (chunk numbering restarts at the
 *            block start); AUTO ignores both levels and maps 32-byte vectors
 *            grid-stride.
 * num_teams: 1..2^31-1 (<= OMPRT_MAX_RED_TEAMS with a reduction, DYNAMIC or GUIDED),
 *            0 = runtime choice; thread_limit: multiple of 32 in [32, 1024],
 *            0 = 256; chunk >= 1 for STATIC_CHUNKED / DYNAMIC, 0 for STATIC
 *            without chunk.  red may be NULL (no reduction clause).
 * A reduction is finished inside the same launch: each team writes a partial,
 * fences (the flush of Sec. 3.1, Listing 2) and takes a ticket with atomic
 * inc (Sec. 3.1); the team drawing the last ticket combines all partials in
 * team order and writes red->result_dev.  The ticket wraps to 0 by itself.
 */
omprt_status omprt_launch_region(omprt_ctx *ctx, const omprt_loop_desc *desc, int32_t sched,
                                 int64_t chunk, int32_t num_teams, int32_t thread_limit,
                                 const omprt_reduce_desc *red, void *stream);

/* The same region with dist_schedule(static, dist_chunk) at the team level:
 * distribute chunk j = iterations [j*d, min((j+1)*d, n)) goes to team
 * j mod num_teams, and inside each distribute chunk the team's threads split
 * it by `sched` (STATIC with chunk 0 = one piece per thread, or
 * STATIC_CHUNKED / STATIC with chunk c), chunk numbering restarting at the
 * distribute chunk (OpenMP composite construct; the paper's runtime divides
 * these iterations, Sec. 1, Sec. 2).  dist_chunk = thread_limit with chunk 1
 * is the mapping iteration i -> team (i / T) mod G, thread i mod T.  When
 * dist_chunk = chunk * thread_limit with chunk a multiple of 8, every thread's
 * piece is whole 32-byte vectors.  Other schedules return
 * OMPRT_ERR_UNSUPPORTED; dist_chunk < 1 returns OMPRT_ERR_INVALID. */
omprt_status omprt_launch_region_dist(omprt_ctx *ctx, const omprt_loop_desc *desc,
                                      int64_t dist_chunk, int32_t sched, int64_t chunk,
                                      int32_t num_teams, int32_t thread_limit,
                                      const omprt_reduce_desc *red, void *stream);

/* Generic-mode (non-SPMD) regions over segments: the runtime's main-thread /
 * worker state machine and __kmpc_alloc_shared for the variables the
 * sequential code shares with its parallel regions (Sec. 2.1, Listing 1).
 * teams distribute (static, balanced) over the nseg segments; for each of its
 * segments s = [seg_dev[s], seg_dev[s+1]) the team's main thread (thread 0)
 * runs the sequential code of `program`, and for each parallel region in it
 * publishes a work descriptor in team-shared memory (the outlined region's
 * id, its loop bounds, its arguments: the scale and a pointer to the
 * globalised reduction variable) and releases the waiting workers; every
 * thread dispatches on the id and runs the region's parallel for (the
 * default schedule: static with a chunk of one 32-byte vector) with a
 * compensated reduction into the variable; a join barrier returns control to
 * the main thread.  Globalised variables live on the team stack of capacity
 * S (omprt_alloc_shared), overflowing to the team's 4 KiB pool slice (teams
 * below OMPRT_MAX_RED_TEAMS); a request that does not fit sets
 * OMPRT_DEV_STACK_NOMEM and the team stops (its remaining results are not
 * written).
 *   OMPRT_GENERIC_REDUCE: one region per segment, v = 0;
 *     parallel for reduction(+: v) with desc's body: DOT v += x[i]*y[i], or
 *     AXPY y[i] = alpha*x[i] + y[i], v += y[i]; result_dev[s] = v.
 *   OMPRT_GENERIC_DOT_AXPY: two regions per segment, the second using the
 *     first's result: v = sum x[i]*y[i] (region 1); a = (float)v * alpha
 *     (sequential, fp32 product); y[i] = a*x[i] + y[i] with w = sum of the
 *     new y[i] (region 2); result_dev[3s .. 3s+2] = v, a, w.
 * desc: data_type F32, x / y device arrays of its trip count n, which bounds
 * the offsets (0 <= seg_dev[s] <= seg_dev[s+1] <= n, else the team stops and
 * OMPRT_DEV_BAD_ARG is set); alpha as above.  seg_dev: int64[nseg + 1] device;
 * result_dev: double[nseg] or double[3 nseg] device.  num_teams 0 = SMs;
 * thread_limit 0 = 256. */
#define OMPRT_GENERIC_REDUCE 0
#define OMPRT_GENERIC_DOT_AXPY 1
omprt_status omprt_launch_generic(omprt_ctx *ctx, const int64_t *seg_dev, int64_t nseg,
                                  const omprt_loop_desc *desc, int32_t program,
                                  double *result_dev, int32_t num_teams, int32_t thread_limit,
                                  void *stream);

/* reduction(op) over n elements of dtype (F32, BF16, I32, I64) at data_dev:
 * omprt_launch_region with BODY_NONE and schedule AUTO, the reduction clause of
 * the worksharing loop the runtime divides (Sec. 1, Sec. 2); team partials
 * cross teams through the flush of Listing 2 and the atomic inc of Listing 3
 * (Sec. 3.1).  data_dev and result_dev are device pointers the caller owns;
 * result_dev: 8 bytes (double for F32/BF16, int64 for integers), written by
 * the launch (n = 0 writes the operation's identity in that type).
 * precision: omprt_precision.  teams 0: two a SM; threads 0: 512 (every
 * team resident at once).  Bad arguments return OMPRT_ERR_INVALID and
 * launch nothing. */
omprt_status omprt_reduce(omprt_ctx *ctx, int32_t op, int32_t dtype, int32_t precision,
                          const void *data_dev, int64_t n, void *result_dev,
                          int32_t num_teams, int32_t thread_limit, void *stream);

/* Write, from device code, the static worksharing tuple that every thread of
 * a composite launch would get (the __kmpc_for_static_init role, Sec. 1,
 * Sec. 2): table_dev is int64[G*T][8], row g*T+t = team LB, UB, stride, last,
 * thread LB, UB, stride, last, in user index space (64-bit two's complement
 * on the widened bounds; an empty piece has LB = one step past the block,
 * UB = LB - incr).  chunk 0 = no chunk. */
omprt_status omprt_static_init_table(omprt_ctx *ctx, const omprt_loop_desc *desc, int64_t chunk,
                                     int32_t num_teams, int32_t thread_limit, int64_t *table_dev,
                                     void *stream);

/* Host-only: the trip count n of desc's loop, the iterations the runtime's
 * worksharing routines divide (Sec. 2).  Rule above: bounds compared in
 * the loop variable's signedness, distance in unsigned 64-bit arithmetic;
 * a 32-bit index type takes |incr| <= 2^31 - 1.
 * Returns OMPRT_ERR_INVALID for a bad type, bound or incr == 0 and
 * OMPRT_ERR_UNSUPPORTED for 2^63 or more iterations.  Needs no device. */
omprt_status omprt_loop_trip_count(const omprt_loop_desc *desc, uint64_t *n_host);

/* Synchronise `stream`, then read and clear the sticky device status word.
 * *bits_host (may be NULL) receives the OMPRT_DEV_* bits.  Returns
 * OMPRT_ERR_DEVICE if any bit was set, OMPRT_ERR_CUDA if the sync failed.
 * Not a routine of the paper's runtime: this library's way to report what
 * its device code checks (bounded waits, stack overflow, bad arguments). */
omprt_status omprt_sync_status(omprt_ctx *ctx, void *stream, uint32_t *bits_host);

/* Static description of a status code. */
const char *omprt_status_str(omprt_status s);

/* Number of SMs of the context's device (0 for a NULL context).  A query of
 * this library, not a routine of the paper's runtime. */
int32_t omprt_sm_count(const omprt_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Reduction without any allocation                                    */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart to this call.  It exists for callers of this
 * library that cannot allocate device memory: code inside a stream callback
 * or an allocator hook, code holding a lock that cudaMalloc could need, or a
 * process whose device memory is owned and budgeted by another component.
 * It needs no context.
 *
 * Same operation and arguments as omprt_reduce (AUTO mapping, value body),
 * but the per-team partials and the ticket live in one scratch array
 * compiled into the library (256 bytes + 16 bytes per team, so 64.25 KiB at
 * the maximum of OMPRT_NOALLOC_MAX_TEAMS teams) that every GPU which loads
 * the library keeps until the process exits.  num_teams > OMPRT_NOALLOC_MAX_TEAMS
 * returns OMPRT_ERR_INVALID; num_teams 0 means the maximum, thread_limit 0
 * means 512.  The call never calls cudaMalloc, cudaFree or any allocating
 * routine.
 *  - The first call on a device looks up the array's device address for
 *    that device (cudaGetSymbolAddress, with that device current) and keeps
 *    it for the life of the process.  The kept address is invalid after
 *    cudaDeviceReset on that device: do not call this entry point after
 *    such a reset.
 *  - Every call shares the one array and clears its ticket on `stream`
 *    before launching, so calls that overlap on the GPU (on different
 *    streams) race and give wrong results.  Calls ordered on one stream are
 *    safe.
 *  - The array keeps the last call's partials; nothing reads them later.
 *  - No device status word is reported, and none is needed: the team stack
 *    is fixed at 4 KiB, which always holds the call's 512 bytes of
 *    temporaries (checked when the library is compiled), and the value loop
 *    has no bounded waits. */
#define OMPRT_NOALLOC_MAX_TEAMS 4096
omprt_status omprt_reduce_noalloc(int32_t op, int32_t dtype, int32_t precision,
                                  const void *data_dev, int64_t n, void *result_dev,
                                  int32_t num_teams, int32_t thread_limit, void *stream);

/* ------------------------------------------------------------------ */
/* Batched regions: many small target regions in one persistent kernel */
/* ------------------------------------------------------------------ */
/* The host calls omprt_batch_create once (it copies the region table to the
 * device and sizes the work queue); omprt_launch_batch then runs every region
 * in one persistent kernel whose CTAs claim (region, chunk) work items with
 * an atomic add on a queue head (the paper's atomic add, Sec. 3.1).  Regions
 * with a reduction combine their chunk partials in chunk order in the CTA
 * that finishes the region's last chunk (ticket by atomic add).  The queue
 * head and the tickets are reset by the last CTA to leave, so the launch can
 * be replayed from a CUDA graph without a memset.
 * Supported bodies: AXPY (F32), DOT (F32, needs red), STENCIL1D3 (F32);
 * inside a work item the CTA's threads take 32-byte vectors grid-stride
 * (the auto mapping); desc[i].lb = 0, incr = 1 (n = ub + 1).
 * chunk_elems: elements per work item (multiple of 256, or 0 = 8192).
 * reds may be NULL; reds[i].result_dev NULL means no reduction for region i. */
typedef struct omprt_batch omprt_batch;
omprt_status omprt_batch_create(omprt_ctx *ctx, const omprt_loop_desc *descs_host,
                                const omprt_reduce_desc *reds_host, int32_t nregions,
                                int64_t chunk_elems, omprt_batch **batch);
/* Run the batch: every region in one persistent launch (the many short
 * target regions of Sec. 4.3 as one launch; the work queue is claimed with the
 * atomic add of Sec. 3.1).  num_ctas 0 = SMs x resident CTAs per SM; threads:
 * multiple of 32 in [64, 1024], 0 = 256.  omprt_batch_destroy frees the
 * batch's device table and queue (the caller has synchronised its streams);
 * NULL is OMPRT_ERR_INVALID. */
omprt_status omprt_launch_batch(omprt_batch *batch, int32_t num_ctas, int32_t threads,
                                void *stream);
omprt_status omprt_batch_destroy(omprt_batch *batch);
/* Number of work items (chunks) in the batch; 0 for NULL.  The batch is the
 * many-short-regions case of Sec. 4.3 (miniQMC's target regions launched tens
 * of thousands of times), run as one launch. */
int64_t omprt_batch_items(const omprt_batch *batch);

/* ------------------------------------------------------------------ */
/* Runtime self-tests run on the device (atomics, barrier, stack)      */
/* ------------------------------------------------------------------ */
/* Atomics of Sec. 3.1 (add, inc, max, exchange, cas) on one 32-bit word per
 * op: num_teams x thread_limit threads each apply the op `reps` times.
 *   words_dev: uint32[5] initial values in, final values out
 *              [0] add 1, [1] inc with bound e, [2] max of the global thread
 *              id, [3] exchange with the global thread id, [4] cas(expected =
 *              thread id, desired = thread id + 1);
 *   returned_dev: uint32[G*T*reps] the values the inc op returned (may be
 *              NULL). */
omprt_status omprt_test_atomics(omprt_ctx *ctx, int32_t num_teams, int32_t thread_limit,
                                int32_t reps, uint32_t e, uint32_t *words_dev,
                                uint32_t *returned_dev, void *stream);

/* Team barrier check (Sec. 3.2, synchronisation): for `rounds` rounds each
 * thread writes the round number to its shared slot, waits at the barrier,
 * checks every slot, waits again.  sub_threads (multiple of 32, dividing
 * thread_limit, or 0) also runs the same test with named barriers over
 * sub-teams of that size.  errors_dev: uint32[1], += mismatches seen. */
omprt_status omprt_test_barrier(omprt_ctx *ctx, int32_t num_teams, int32_t thread_limit,
                                int32_t sub_threads, int32_t rounds, uint32_t *errors_dev,
                                void *stream);

/* Bounded device wait, the synchronization the target-specific part provides
 * (Sec. 3.2), with a limit (the runtime has no unbounded wait): thread 0 of each
 * of num_teams teams waits until *flag_dev == expect or timeout_us
 * microseconds (1 .. 2,000,000) pass on the GPU timer; out_dev[g] = 1 if the
 * value was seen, 0 if the wait gave up, in which case OMPRT_DEV_TIMEOUT is
 * set in the status word.  The context stays usable after a timeout. */
omprt_status omprt_test_wait(omprt_ctx *ctx, int32_t num_teams, const uint32_t *flag_dev,
                             uint32_t expect, int64_t timeout_us, int32_t *out_dev, void *stream);

/* Replay an alloc/free trace through the team shared-memory stack of every
 * team (__kmpc_alloc_shared, Sec. 2.1, Listing 1).  ops_dev: int64[nops][2]
 * (kind, arg): kind 0 = alloc(arg bytes), kind 1 = free of the block that
 * op number arg (an earlier alloc) returned.  out_dev: int64[num_teams][nops][2]: alloc -> (region 0 shared /
 * 1 pool / 2 failed, byte offset from that region's base), free -> (status
 * bits raised, 0).  stack_bytes: S for this test (<= 200 KiB);
 * pool_bytes: fallback bytes per team (<= OMPRT_POOL_BYTES_PER_TEAM).
 * status_dev: int64[num_teams] OR of the bits per team.  nops <= 4096. */
omprt_status omprt_test_stack(omprt_ctx *ctx, int32_t num_teams, int64_t stack_bytes,
                              int64_t pool_bytes, const int64_t *ops_dev, int64_t nops,
                              int64_t *out_dev, int64_t *status_dev, void *stream);

/* ------------------------------------------------------------------ */
/* Learned schedule: MLP cost model 16 -> 64 -> 64 -> 12 (fp32)        */
/* ------------------------------------------------------------------ */
/* Not a routine of the paper's runtime: a learned choice of schedule, chunk,
 * teams and threads for the loops the runtime divides (Sec. 2), added by this
 * library.  Every entry point below takes device pointers the caller owns
 * (params, inputs, gradients, Adam moments) unless it says host; bad sizes or
 * NULL pointers return OMPRT_ERR_INVALID and launch nothing.
 * Parameter vector layout (float32, 6028 values): W1[64][16], b1[64],
 * W2[64][64], b2[64], W3[12][64], b3[12], row-major W[out][in].
 * h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3. */
#define OMPRT_MLP_IN 16
#define OMPRT_MLP_HID 64
#define OMPRT_MLP_OUT 12
#define OMPRT_MLP_NPARAM 6028

/* y_dev[B][12] = model(x_dev[B][16]) (learned schedule: this library's own,
 * not a routine of the paper's runtime). */
omprt_status omprt_mlp_forward(omprt_ctx *ctx, const float *params_dev, const float *x_dev,
                               int32_t batch, float *y_dev, void *stream);
/* (Learned schedule: this library's own, not a routine of the paper's
 * runtime.)  Mean-squared-error loss over the batch and the 12 outputs and its gradient:
 * grad_dev[6028] = d loss / d params (overwritten), loss_dev[1] (may be NULL).
 * batch in [1, 16384]; the per-sample activations go to context scratch, so
 * calls on one context must not overlap on the device. */
omprt_status omprt_mlp_loss_grad(omprt_ctx *ctx, const float *params_dev, const float *x_dev,
                                 const float *target_dev, int32_t batch, float *grad_dev,
                                 float *loss_dev, void *stream);
/* (Learned schedule: this library's own, not a routine of the paper's
 * runtime.)  One bias-corrected Adam step (Kingma & Ba 2015) at step number t >= 1 on
 * params_dev, with moment buffers m_dev, v_dev (zero before step 1). */
omprt_status omprt_mlp_adam(omprt_ctx *ctx, float *params_dev, const float *grad_dev,
                            float *m_dev, float *v_dev, int32_t n, int32_t t, float lr,
                            float beta1, float beta2, float eps, void *stream);

/* (Learned schedule: this library's own, not a routine of the paper's
 * runtime.)  Configuration table: index k in [0, 12) of the model's
 * output is configuration k: sched_host[k], chunk_host[k], teams_per_sm_host[k]
 * (num_teams = teams_per_sm * SMs) and threads_host[k]; any pointer may be NULL. */
omprt_status omprt_learned_configs(int32_t *sched_host, int64_t *chunk_host,
                                   int32_t *teams_per_sm_host, int32_t *threads_host);

/* (Learned schedule: this library's own, not a routine of the paper's
 * runtime.)  Install (params_host != NULL) or remove (NULL) the cost model used by
 * OMPRT_SCHED_LEARNED, with the feature standardisation (mean_host[16],
 * std_host[16]).  The model is copied; inference runs on the host at launch
 * time, takes the argmin of the 12 predicted log-times, and falls back to the
 * heuristic when no model is installed or an output is not finite. */
omprt_status omprt_set_cost_model(omprt_ctx *ctx, const float *params_host,
                                  const float *mean_host, const float *std_host);

/* (Learned schedule: this library's own, not a routine of the paper's
 * runtime.)  Features (16 floats) the cost model sees for a loop, and the
 * configuration index the installed model (or, without one, the heuristic)
 * picks, for the loop the runtime divides (Sec. 2).  Host pointers; NULL ctx
 * is OMPRT_ERR_NOT_INIT, a NULL output OMPRT_ERR_INVALID.  omprt_loop_features
 * returns the trip count's error for a bad descriptor; omprt_choose_config
 * reads the descriptor only when a model is installed (without one it returns
 * the heuristic's index, and a launch validates the descriptor itself). */
omprt_status omprt_loop_features(const omprt_ctx *ctx, const omprt_loop_desc *desc,
                                 int32_t has_reduction, float *features_host);
omprt_status omprt_choose_config(const omprt_ctx *ctx, const omprt_loop_desc *desc,
                                 int32_t has_reduction, int32_t *config_host);

#ifdef __cplusplus
}
#endif

#endif /* OMPRT_H_ */
