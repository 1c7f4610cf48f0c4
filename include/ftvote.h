/*
 * ftvote.h -- C ABI of the B300 heterogeneity-aware majority voter.
 *
 * The voter is the one of Sec. IV.D of Kicherer & Karl, "Heterogeneity-aware
 * Fault Tolerance using a Self-Organizing Runtime System": the results of R
 * redundant executions of a task are compared element by element and the
 * presumable correct result is selected.  Integer values are compared bit by
 * bit; floating-point values are equal when they differ by at most a
 * programmer-set maximum (Sec. IV.D), so that a CPU-vs-GPU rounding difference
 * is not taken for a fault.  The element type plays the part of the value type
 * that the paper's dls_register_data() attaches to a buffer (Sec. IV.E).
 *
 * Semantics of one vote of n elements of R replicas x_0..x_{R-1}:
 *   eq(a,b)   integers: equal bit patterns.
 *             floats (computed in the element's own precision, IEEE
 *             round-to-nearest, no FMA, no flush-to-zero): equal bit patterns,
 *             else not equal if either is NaN or +-Inf, else
 *             |a-b| <= abs_tol  or  |a-b| <= rel_tol * max(|a|,|b|),
 *             with both tolerances rounded once to the element type.
 *   support   s_r = #{q : eq(x_r, x_q)}, q = r included.
 *   winner    w = smallest r with maximal s_r; out[i] = bit copy of x_w[i].
 *   majority  2 * s_w > R; elements without one are counted in no_majority
 *             and still receive x_w[i].
 *   mismatch[r]        #{i : not eq(x_r[i], out[i])}; first_mismatch[r] the
 *                      smallest such i, -1 if none.  These per-replica counts
 *                      are the observed fault rates that the paper's
 *                      fault-aware runtime estimate F_i = R_i / (1 - p_i)
 *                      consumes (Sec. IV.B).
 *   block_crc[b]       CRC32C (Castagnoli, reflected 0x82F63B78, init and final
 *                      XOR 0xFFFFFFFF) of bytes [4096 b, min(4096 (b+1), nbytes))
 *                      of out, blocks independent; the digest lets a memory
 *                      manager skip transfers of unchanged data (Sec. IV.A).
 *
 * Conventions for every entry point:
 *   - All data pointers are DEVICE pointers owned by the caller unless stated
 *     otherwise; descriptors are read from host memory during the call only.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  The return code reports
 *     argument validation and launch errors; results are valid once the
 *     stream reaches the work.
 *   - No entry point throws, aborts or falls back to the CPU.
 *   - ft_vote, ft_digest, ft_vote_many, ft_vote_batched, the registry and the
 *     rating functions may be called from several host threads at once.  A
 *     plan, a server or a checkpoint context is used by one thread at a time,
 *     except ft_submit / ft_submit_many / ft_poll / ft_poll_many /
 *     ft_server_info / ft_server_pause, which any thread may call
 *     concurrently.
 */
#ifndef FTVOTE_H
#define FTVOTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (all negative except FT_OK) ---- */
#define FT_OK          0
#define FT_EINVAL     -1   /* bad argument: dtype, R, NULL, misalignment, aliasing, tolerance */
#define FT_ENOMEM     -2   /* a library-owned allocation failed                               */
#define FT_EAGAIN     -3   /* server: over the memory budget / slot limit, or not done yet    */
#define FT_ETIMEDOUT  -4   /* server: the wait ran out before the request completed           */
#define FT_ECUDA      -5   /* a CUDA call failed; ft_last_cuda_error() gives the cudaError_t  */
#define FT_ENOTFOUND  -6   /* server: unknown or already collected ticket                      */

#define FT_MAX_R        8
#define FT_BLOCK_BYTES  4096u

/* element types; integer types compare bit-wise, tolerances are ignored */
typedef enum ft_dtype {
    FT_I32 = 0, FT_U32 = 1, FT_I64 = 2, FT_U64 = 3, FT_U8 = 4, FT_F32 = 5, FT_F64 = 6
} ft_dtype;

typedef void *ft_stream;   /* cudaStream_t */

/* Per-vote statistics, written by the vote (device memory, 8-byte aligned). */
typedef struct ft_stats {
    uint64_t mismatch[FT_MAX_R];        /* entries >= R are written as 0            */
    int64_t  first_mismatch[FT_MAX_R];  /* -1 = none; entries >= R are written -1   */
    uint64_t no_majority;
    int64_t  first_no_majority;         /* -1 = none                                 */
} ft_stats;

/* One vote.
 *   replicas[0..R-1]  device pointers, each n * sizeof(dtype) bytes, 16-byte
 *                     aligned; unused entries are ignored.  Two entries may
 *                     point to the same buffer.
 *   out               device, n * sizeof(dtype) bytes, 16-byte aligned; must
 *                     not overlap any replica.
 *   block_crc         device, ceil(n * sizeof(dtype) / 4096) uint32 entries,
 *                     4-byte aligned, or NULL when no digest is wanted (the
 *                     vote is not faster without it).
 *   stats             device, one ft_stats, 8-byte aligned (required).
 *   abs_tol, rel_tol  float dtypes: 0 <= rel_tol <= 1 and 0 <= abs_tol with
 *                     abs_tol finite once rounded to the element type (a
 *                     relative tolerance above 100% has no use in a vote);
 *                     ignored for integer dtypes.                          */
typedef struct ft_vote_desc {
    const void *replicas[FT_MAX_R];
    int32_t     R;          /* 2..8 */
    int32_t     dtype;      /* ft_dtype */
    uint64_t    n;          /* elements per replica; 0 is allowed (no work) */
    double      abs_tol;
    double      rel_tol;
    void       *out;
    uint32_t   *block_crc;
    ft_stats   *stats;
} ft_vote_desc;

/* Vote one task (Sec. IV.D) with the persistent voter kernel (128-bit
 * coalesced loads of all R replicas, vote, store, warp-ballot statistics and
 * the fused per-block CRC32C).  Normally one launch on `stream`: the
 * statistics are gathered in a library-owned slot (a pool per device, created
 * by the first call on it) and copied to desc->stats by the kernel's last CTA.
 * While `stream` is being captured into a graph, or when every slot is in use,
 * a statistics reset kernel runs first and the voter adds into desc->stats
 * directly.  The voter lets the next kernel on the stream start early under
 * programmatic dependent launch: a kernel launched after ft_vote with
 * programmatic stream serialization must call cudaGridDependencySynchronize()
 * before it reads the vote's results.
 * Returns FT_OK, FT_EINVAL or FT_ECUDA. */
int ft_vote(const ft_vote_desc *desc, ft_stream stream);

/* The same vote on buffers of mixed residency: each of desc->replicas[r],
 * out, block_crc (or NULL) and stats may be host memory (pinned makes the
 * copies direct DMA; pageable works, slower) or memory of the current device
 * (device or managed allocation), with ft_vote's alignment and overlap rules;
 * another device's memory is FT_EINVAL.  The vote runs on the current device
 * in chunks of chunk_bytes (0 = 64 MiB; a multiple of 4096): chunk k's
 * host-resident replicas are uploaded while chunk k-1 is voted and chunk k-2's
 * voted bytes and digests are downloaded, on the library's own streams;
 * device-resident replicas are read in place and a device-resident out or
 * block_crc is written in place.  The call is ordered after no stream: work
 * producing a device-resident replica must be complete when it is made.
 * Synchronous: returns when out, block_crc and stats hold the result, which
 * is the one ft_vote gives (statistics combined over the chunks).
 * The library keeps 2 * (R + 1) * chunk_bytes of device staging per device
 * between calls; calls on one device run one at a time.
 * Returns FT_OK, FT_EINVAL or FT_ECUDA. */
int ft_vote_host(const ft_vote_desc *desc, uint64_t chunk_bytes);

/* CRC32C of each block_bytes-sized block of nbytes bytes at buf (device,
 * 16-byte aligned); out (device) receives ceil(nbytes / block_bytes) values,
 * the last block being partial.  block_bytes must be a multiple of 4096 in
 * [4096, 1 << 24].  This is the digest that the memory manager of Sec. IV.A
 * would compare to skip unchanged transfers.  Returns FT_OK, FT_EINVAL or
 * FT_ECUDA. */
int ft_digest(const void *buf, uint64_t nbytes, uint32_t block_bytes,
              uint32_t *out, ft_stream stream);

/* ---- batched form: many tasks in one persistent, graph-captured launch ---- */

/* Tuning of the batched kernels.  A batch is voted by one persistent kernel
 * per (element kind, R) group; the fields apply to every group, and zeros
 * leave the choice to the autotuner when the plan is created.
 *   tile_blocks  4 KiB blocks per work tile (1..64); 0 = autotuned.
 *   ctas_per_sm  cap on resident CTAs per SM (1..8); 0 = as many as fit.  A
 *                voter CTA fills an SM's shared memory with its CRC tables,
 *                so one CTA per SM is what fits, and it is not searched.
 *   warps        warps per CTA: 8, 12 or 16; 0 = chosen per group.
 *   l2_prefetch  1 = no prefetch, 2 = each warp prefetches its tile's next
 *                block into L2; 0 = chosen per group.  When warps or
 *                l2_prefetch is set, every group takes that shape (warps 0
 *                then meaning 16, l2_prefetch 0 no prefetch).
 *   kernels      1 = the whole batch as one persistent kernel whose warps take
 *                the batch's tiles in turn whatever their element kind and R
 *                (16 warps, no prefetch; warps must then be 0 or 16 and
 *                l2_prefetch not 2); 2 = one kernel per group, the groups as
 *                parallel branches of the graph; 0 = the faster of the two as
 *                timed by the autotuner (one per group when warps or
 *                l2_prefetch rule out the one-kernel shape).
 * ft_plan_tune reports the tile size, the kernels choice, and a warps /
 * l2_prefetch value only when every group has it (0 when the groups differ;
 * ft_plan_groups gives each group's). */
typedef struct ft_tune {
    int32_t tile_blocks;
    int32_t ctas_per_sm;
    int32_t warps;
    int32_t l2_prefetch;
    int32_t kernels;
} ft_tune;

/* One (element kind, R) group of a plan and the launch shape it runs with. */
typedef struct ft_plan_group {
    int32_t  dtype;        /* FT_F32, FT_F64, FT_U8, or for bit-compared integers of
                              4 / 8 bytes FT_I32 / FT_I64 (the unsigned ones share them) */
    int32_t  R;
    int32_t  tasks;        /* tasks in the group */
    int32_t  warps;        /* warps per CTA of its kernel */
    int32_t  l2_prefetch;  /* 1 if a warp prefetches its tile's next block into L2 */
    int32_t  tile_blocks;  /* 4 KiB blocks per work tile */
    uint64_t tiles;        /* work tiles of the group */
} ft_plan_group;

typedef struct ft_plan ft_plan;   /* library-owned */

/* Build a plan for ntasks votes (each described as for ft_vote; every task
 * has its own dtype, R, tolerances and outputs; element indices in the
 * statistics are local to the task).  The plan copies the descriptors to a
 * device task table, autotunes what `tune` leaves open (NULL: everything) by
 * timing replays of the graph it will capture on the plan's own buffers,
 * which it overwrites: first the tile size, then each group's warps per CTA
 * and L2 prefetch in turn; the result is kept per batch signature for later
 * plans of the process.  It then captures one CUDA graph: the statistics
 * reset followed by the groups' persistent kernels as parallel branches, or
 * by the one kernel for the whole batch (ft_tune.kernels).
 * The caller keeps every buffer alive and in place until ft_plan_destroy.
 * Returns FT_OK, FT_EINVAL, FT_ENOMEM or FT_ECUDA. */
int ft_plan_create(ft_plan **plan, const ft_vote_desc *tasks, int32_t ntasks,
                   const ft_tune *tune);

/* Replay the plan's graph on `stream`: every task of the plan is voted. */
int ft_vote_batched(ft_plan *plan, ft_stream stream);

/* Launch the plan's kernels without the graph (same work: the statistics
 * reset, then the group kernels one after another on `stream`, or the one
 * kernel for the whole batch). */
int ft_vote_batched_nograph(ft_plan *plan, ft_stream stream);

/* Vote n tasks with one ft_vote each (one launch per task, in order, on
 * `stream`): the unbatched form that the batched plan is measured against. */
int ft_vote_many(const ft_vote_desc *descs, int32_t n, ft_stream stream);

/* The tuning the plan uses. */
int ft_plan_tune(const ft_plan *plan, ft_tune *out);

/* The plan's groups in launch order: out receives min(max, count) entries and
 * *n the count.  Returns FT_OK or FT_EINVAL. */
int ft_plan_groups(const ft_plan *plan, ft_plan_group *out, int32_t max, int32_t *n);

/* Free the plan.  Its replays must have completed (synchronize the streams
 * they were launched on first). */
int ft_plan_destroy(ft_plan *plan);

/* ---- batched vote without any allocation ---- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: code running inside a framework whose pool
 * owns all device memory, latency-critical loops where cudaMalloc / cudaFree
 * would synchronise the device, plug-ins that must not change the process's
 * allocation pattern.  It votes `ntasks` tasks (descriptors as for ft_vote,
 * read during the call) like ft_vote_batched, but keeps its scratch (task
 * table, per-task first tile, tile counters) in a fixed array of device
 * memory inside the library (about 580 KiB, held on every GPU that loads the
 * library until the process exits) and builds the batch in fixed host
 * buffers: the call allocates nothing, neither with cudaMalloc nor on the
 * host.  The caller still owns every input and output buffer.
 *   ntasks       0 .. FT_NOALLOC_MAX_TASKS; more is rejected with FT_EINVAL.
 *   tile_blocks  4 KiB blocks per work tile, 1 .. 64; 0 = automatic: 8,
 *                halved while the batch would make fewer tiles than the
 *                kernel has warps in one wave, down to 1.
 * The first call on a device looks up the array's device address (with that
 * device current).  The batch is copied to the array from a static host area
 * that every call refills, so a call on a stream that is being captured into
 * a graph is refused with FT_EINVAL (a replay would copy whatever batch the
 * area holds by then).  All calls share the array and it keeps the last
 * call's contents (counters and statistics are reset at the start of each
 * call): calls whose work overlaps on the GPU race on it, so order them on one
 * stream or synchronise between them.  Host threads are serialised while a
 * call builds its batch.
 * Returns FT_OK, FT_EINVAL or FT_ECUDA. */
#define FT_NOALLOC_MAX_TASKS 4096
int ft_vote_batched_noalloc(const ft_vote_desc *tasks, int32_t ntasks, int32_t tile_blocks,
                            ft_stream stream);

/* ---- serving form: continuous batching of vote requests ---- */

typedef struct ft_server ft_server;   /* library-owned */

typedef struct ft_server_config {
    uint64_t mem_budget_bytes;  /* admission budget: sum over admitted, not yet
                                   collected requests of (R+1) * n * sizeof(dtype) */
    int32_t  max_slots;         /* most requests packed into one batch (1..65536); the
                                   requests waiting are spread evenly over the free streams,
                                   so a batch packs several only when they outnumber them */
    int32_t  streams;           /* batches in flight at once (1..8)               */
    int32_t  tile_blocks;       /* batched-kernel tile, 1..64; 0 = automatic per batch:
                                   8, halved while the batch would make fewer tiles
                                   than its share of one wave of the kernel's warps
                                   (the wave divided by `streams`), down to 1 */
    int32_t  max_inflight;      /* most admitted, not yet collected requests (0 = 65536) */
    uint64_t max_batch_bytes;   /* a batch takes waiting requests (oldest first) while their
                                   (R+1)*n*sizeof(dtype) bytes stay within this, and at least
                                   one (0 = no limit): bounds how long a small request waits
                                   for the large ones packed with it */
    int32_t  reserved_sms;      /* with two or more streams, SMs that no batch's kernels fill,
                                   so that a batch arriving behind a large one finds SMs free:
                                   0 = 32, -1 = none, else 1 .. SM count - 1 */
    int32_t  idle_spin_us;      /* how long the worker thread keeps polling (one CPU core busy)
                                   after its last batch before it sleeps until the next request;
                                   a request that finds it asleep waits for a thread wake-up
                                   (tens of microseconds): 0 = 2000, -1 = do not poll */
    int32_t  size_ratio;        /* while another slot is free, a batch takes a waiting request only
                                   if its bytes are within this factor of the batch's first
                                   request's (a much smaller one would wait for the large one it
                                   is packed with); on the last free slot everything waiting is
                                   packed: 0 = 8, -1 = no limit, else 2 or more */
    int32_t  resident;          /* 0 = batches (above).  1 = resident mode (no batches, no
                                   launch per request): one persistent kernel on every SM takes
                                   each request from a host-mapped mailbox and votes it in
                                   tiles, the request with the fewest tiles left first;
                                   max_slots, streams, tile_blocks, max_batch_bytes,
                                   reserved_sms and size_ratio are not used.  2 = shared: the
                                   batches as with 0, and each request whose output has fewer
                                   4 KiB blocks than the resident kernel has voting warps goes
                                   to a resident kernel on the reserved_sms SMs that the batches
                                   leave free (32 when reserved_sms is 0 or -1) */
} ft_server_config;

typedef struct ft_result {
    int32_t  status;            /* FT_OK or the FT_ECUDA of the batch            */
    int32_t  R;
    uint64_t n;
    ft_stats stats;             /* copy of the request's statistics              */
    double   submit_us;         /* host clock (monotonic, microseconds) at submit */
    double   done_us;           /* host clock when the server saw the batch complete */
    double   launch_us;         /* host clock when the request's batch began to launch */
    double   launched_us;       /* host clock when its launch calls had returned */
} ft_result;

/* Start a server: one host thread that packs admitted requests into batches
 * and launches them on `streams` CUDA streams of the current device (each
 * with up to three auxiliary streams, on which a batch's further element-type
 * / R groups run in parallel).  With two or more streams no batch's kernels
 * occupy more than all but cfg->reserved_sms SMs, so that a batch is not held
 * behind all of a large one.  A batch votes its requests smallest first; in
 * a batch of at most 16 requests without caller statistics pointers, a lone
 * request and each one of 64 MiB or more ((R+1) * n * sizeof(dtype)) runs as
 * a single vote (the ft_vote kernels) beside the others' batched kernels.  A
 * request without a caller statistics pointer completes as soon as its own
 * tiles are voted: the kernel writes its statistics and a completion flag to
 * host-mapped memory (requests with caller pointers complete with their whole
 * batch).  The thread polls for new requests and completions without holding
 * the server's lock, and keeps polling for cfg->idle_spin_us after its last
 * batch before it sleeps.  Creation loads every kernel the server can launch
 * (a few tens of milliseconds the first time in a process), so that no
 * request pays CUDA's lazy loading of a kernel at its first launch.
 *
 * With cfg->resident = 1 there are no batches: the thread hands each request
 * to one of 32 device slots through a host-mapped mailbox, and one persistent
 * voter kernel (one CTA per SM, launched when a request arrives and nothing
 * is running) admits it and votes it in tiles, the request with the fewest
 * tiles left first, so a small request is not held behind a large one.  Each
 * request completes on its own (statistics and flag to host-mapped memory;
 * to desc->stats too when given).  The kernel leaves once nothing has arrived
 * for cfg->idle_spin_us (2 ms by default) and every request on it is done;
 * while requests keep arriving it holds every SM, so other kernels of the
 * process (and a second resident server on the same GPU) wait for it to
 * leave.  Requests beyond the 32 slots wait on the host.  With
 * cfg->resident = 2 the same kernel runs on the reserved SMs only and takes
 * the small requests (fewer 4 KiB blocks of output than its 511 voting warps
 * with the default 32 SMs), with no launch per request, while the larger ones
 * are batched and launched as with 0.
 * Returns FT_OK, FT_EINVAL, FT_ENOMEM or FT_ECUDA. */
int ft_server_create(ft_server **srv, const ft_server_config *cfg);

/* Admit one request (the replicas must already hold the duplicated results).
 * The server keeps the descriptor; the caller keeps every buffer alive and
 * unchanged until ft_poll has returned FT_OK for the ticket.  desc->stats may
 * be NULL: the server then keeps the statistics itself and returns them in
 * the ft_result only.  Returns FT_OK with *ticket set, FT_EAGAIN when the
 * request does not fit the free budget or the in-flight limit right now
 * (nothing is kept; retry later), or FT_EINVAL. */
int ft_submit(ft_server *srv, const ft_vote_desc *desc, uint64_t *ticket);

/* Wait up to timeout_us microseconds (0 = do not wait, < 0 = wait without a
 * limit) for a request.  FT_OK: done, *res filled, ticket retired and its
 * budget released.  FT_ETIMEDOUT: not done within the limit (the request
 * stays in flight; poll again).  FT_ENOTFOUND: unknown ticket. */
int ft_poll(ft_server *srv, uint64_t ticket, int64_t timeout_us, ft_result *res);

/* Bulk forms for clients with many requests in flight: one call and one
 * acquisition of the server's lock for a run of requests.
 *
 * ft_submit_many submits descs[0..n) in order, each as ft_submit would, and
 * stops at the first request that does not fit the free budget or the
 * in-flight limit right now.  descs is a host array of n pointers; tickets
 * (n entries) receives the ticket of each accepted request, and *accepted
 * their number, a prefix of the array (0..n).  Returns FT_OK (the requests
 * after the accepted prefix were refused for now: retry them later), or
 * FT_EINVAL when the first request not accepted is invalid (*accepted is its
 * index) or for bad arguments.
 *
 * ft_poll_many waits up to timeout_us (as ft_poll) for tickets[0], then
 * retires the longest prefix of tickets[0..n) whose requests are done,
 * filling results[i] (n entries, or NULL) for each, and sets *ndone to its
 * length.  Returns FT_OK (including *ndone == 0 after a wait of 0), or
 * FT_ETIMEDOUT when tickets[0] is not done, or FT_ENOTFOUND when a ticket of
 * the prefix is unknown (*ndone counts the requests retired before it), or
 * FT_EINVAL. */
int ft_submit_many(ft_server *srv, const ft_vote_desc *const *descs, int32_t n, uint64_t *tickets,
                   int32_t *accepted);
int ft_poll_many(ft_server *srv, const uint64_t *tickets, int32_t n, int64_t timeout_us, ft_result *results,
                 int32_t *ndone);

/* Hold back (paused != 0) or release the launching of admitted requests.
 * While paused, requests are admitted and queued on the host but no batch
 * starts, so ft_poll on them times out: the host-side way to exercise the
 * bounded wait without stalling anything on the GPU.  Returns FT_OK. */
int ft_server_pause(ft_server *srv, int32_t paused);

/* Stop the server after the batches in flight complete; requests not yet
 * launched and uncollected tickets are dropped.  No other thread may use the
 * server during or after this call.  Returns FT_OK. */
int ft_server_destroy(ft_server *srv);

/* Counters of a server since its creation. */
typedef struct ft_server_stats {
    uint64_t batches;                /* batches launched                                 */
    uint64_t requests;               /* requests launched in them                        */
    uint64_t completed;              /* requests whose batch has completed               */
    int32_t  max_batches_in_flight;  /* most batches on the device at the same time      */
    int32_t  inflight_requests;      /* admitted, not yet collected                      */
    uint64_t inflight_bytes;         /* their share of the budget                        */
    double   launch_host_us;         /* worker time spent laying out and launching batches */
    double   batch_span_us;          /* summed launch -> completion time of the batches    */
    double   queue_us;               /* summed submit -> taken into a batch time of the requests */
} ft_server_stats;
int ft_server_info(ft_server *srv, ft_server_stats *out);

/* The monotonic host clock (microseconds) of ft_result.submit_us / done_us. */
double ft_clock_us(void);

/* ---- value types of buffers, and task duplication (Sec. IV.D, IV.E) ---- */

/* The delta the paper chose for single precision after observing CPU/GPU
 * results differ by 0.001 % to 0.1 % (Sec. IV.D), as a relative tolerance. */
#define FT_PAPER_F32_REL_TOL 1e-3

/* Register a device area (bytes, a multiple of the element size) with its
 * value type and compare tolerances, as the paper's dls_register_data(ptr,
 * size, type, mode) tells its runtime how to compare a buffer (Sec. IV.E).
 * Areas may not overlap.  Returns FT_OK or FT_EINVAL. */
int ft_register_data(const void *ptr, uint64_t bytes, int32_t dtype, double abs_tol, double rel_tol);
int ft_unregister_data(const void *ptr);   /* FT_OK or FT_ENOTFOUND */

/* Type, tolerances and bytes from ptr to the end of the registered area that
 * contains ptr (any output pointer may be NULL).  FT_OK or FT_ENOTFOUND. */
int ft_registered_type(const void *ptr, int32_t *dtype, double *abs_tol, double *rel_tol,
                       uint64_t *bytes);

/* ft_vote into `out`, a registered area: element type, tolerances and n come
 * from its registration (n = bytes from out to the area's end / element size).
 * replicas: host array of R device pointers.  FT_ENOTFOUND if out is not in a
 * registered area. */
int ft_vote_registered(const void *const *replicas, int32_t R, void *out, uint32_t *block_crc,
                       ft_stats *stats, ft_stream stream);

/* A duplicated task: computes replica `replica` of the task's result into
 * `out` (device memory), on the GPU on `stream` or on the CPU followed by a
 * copy; returns FT_OK or any nonzero code to abort. */
typedef int (*ft_task_fn)(void *user, int32_t replica, void *out, ft_stream stream);

/* Task duplication followed by the vote (Sec. IV.D): calls task(user, r,
 * vote->replicas[r], stream) for r = 0..R-1, then ft_vote(vote, stream).  The
 * task may use a different kernel or processing unit for each replica (the
 * paper's HetDMR mode).  Returns the first nonzero task code, or ft_vote's. */
int ft_dmr_run(ft_task_fn task, void *user, const ft_vote_desc *vote, ft_stream stream);

/* ---- digest-driven checkpoint of a device buffer (Sec. IV.A, IV.C) ---- */

/* The paper's memory manager transfers data only when necessary and keeps a
 * backup copy so that a faulty run can be rolled back.  A checkpoint context
 * keeps the per-4-KiB CRC32C digests of the last checkpoint of one device
 * buffer of nbytes bytes and moves only the blocks whose digest changed.  A
 * change that leaves a block's CRC32C unchanged is not seen (a random change
 * escapes with probability 2^-32; changes of a few bits never do).
 * The context owns device memory for the digests and a block list and a
 * staging area of stage_bytes (0 = 64 MiB), plus as much pinned host memory. */
typedef struct ft_ckpt ft_ckpt;   /* library-owned */
int ft_ckpt_create(ft_ckpt **ckpt, uint64_t nbytes, uint64_t stage_bytes);

/* Bring host_copy (host memory, nbytes) up to date with dev_buf (device,
 * 16-byte aligned): the first call copies every block, later calls only the
 * blocks whose digest changed since the previous sync.  When more than an
 * eighth of the blocks of a buffer of 64 MiB or more changed, the whole buffer
 * is copied at once (faster than moving the blocks one by one).  Synchronous
 * (returns when host_copy is updated).  *blocks_copied (may be NULL) = blocks
 * moved.  host_copy in pinned memory makes the copies direct DMA. */
int ft_ckpt_sync(ft_ckpt *ckpt, const void *dev_buf, void *host_copy, ft_stream stream,
                 uint64_t *blocks_copied);

/* Roll dev_buf back to the checkpoint held in host_copy: uploads only the
 * blocks whose current device digest differs from the checkpoint's (all
 * blocks if no sync happened yet, or the whole buffer at once under the same
 * rule as ft_ckpt_sync).  Synchronous.  *blocks_copied = blocks moved. */
int ft_ckpt_restore(ft_ckpt *ckpt, void *dev_buf, const void *host_copy, ft_stream stream,
                    uint64_t *blocks_copied);

/* Forget the checkpoint's digests (the host copy was changed behind the
 * context's back): the next sync or restore moves every block. */
int ft_ckpt_forget(ft_ckpt *ckpt);

/* Free the context (sync and restore are synchronous, so nothing is in flight). */
int ft_ckpt_destroy(ft_ckpt *ckpt);

/* ---- memory areas with a host and a device sibling (Sec. IV.A) ---- */

/* The paper's memory manager keeps siblings of each registered area in the
 * memories of the processing units, tags each with the version of the data it
 * holds (a write access increases it by one), transfers data to a requesting
 * unit only when its sibling is older than the newest one, and, in the
 * fault-tolerant mode, makes sure that the version a kernel is about to
 * overwrite still exists in another memory so that a faulty run can be rolled
 * back.  An ft_area does this for one host and one device sibling; transfers
 * move only the 4 KiB blocks whose CRC32C differs (see ft_ckpt).  Requests are
 * synchronous.  An area is used by one thread at a time. */
#define FT_MEM_HOST     0
#define FT_MEM_DEVICE   1
#define FT_ACCESS_READ  1
#define FT_ACCESS_WRITE 2
typedef struct ft_area ft_area;   /* library-owned */

/* Register host_ptr (host memory, bytes long, caller-owned) as an area whose
 * host sibling holds version 1; allocates the device sibling.  Returns FT_OK,
 * FT_EINVAL, FT_ENOMEM or FT_ECUDA. */
int ft_area_create(ft_area **area, void *host_ptr, uint64_t bytes);

/* Access to the sibling in `memory` (FT_MEM_HOST / FT_MEM_DEVICE) with
 * `access` (FT_ACCESS_READ and/or FT_ACCESS_WRITE).  The sibling is first
 * brought to the newest version if it is older or invalid.  For a write, the
 * current version is first made to exist in the other memory too, and the
 * sibling's version then increases by one (the caller writes it next).
 * *ptr receives the sibling's address; *blocks_moved (may be NULL) the 4 KiB
 * blocks transferred.  FT_EINVAL if both siblings were invalidated. */
int ft_area_request(ft_area *area, int32_t memory, int32_t access, void **ptr, ft_stream stream,
                    uint64_t *blocks_moved);

/* A fault during a kernel that wrote the sibling in `memory` left it in an
 * unknown state: drop it; the other sibling still holds the previous version. */
int ft_area_invalidate(ft_area *area, int32_t memory);

/* Version held by each sibling (0 = none / invalid). */
int ft_area_versions(const ft_area *area, uint64_t *host_version, uint64_t *device_version);

int ft_area_destroy(ft_area *area);

/* ---- fault-aware rating of processing units (Sec. IV.B) ---- */

/* One kernel x processing-unit combination: its fault-free runtime (any time
 * unit) and how many of its runs were valid.  Host memory, caller-owned. */
typedef struct ft_unit_rating {
    double   runtime;
    uint64_t valid_runs;
    uint64_t total_runs;
} ft_unit_rating;

/* Observed fault probability p = (total - valid) / total (0 with no runs; the
 * paper prints v/t, read here as the share of faulty runs, which its own
 * example p = 0.75 -> four times the runtime requires). */
double ft_fault_probability(uint64_t valid_runs, uint64_t total_runs);

/* Fault-aware runtime F = runtime / (1 - p) (Sec. IV.B): the runtime stretched
 * by the expected number of attempts until a run is correct; +INFINITY when
 * every run so far was faulty (p = 1); NaN if valid_runs > total_runs. */
double ft_fault_aware_runtime(double runtime, uint64_t valid_runs, uint64_t total_runs);

/* Fold one vote into the ratings: replica r was produced by unit
 * unit_of_replica[r]; that run counts as valid iff stats->mismatch[r] == 0.
 * stats is a HOST copy of the vote's ft_stats.  Returns FT_OK or FT_EINVAL. */
int ft_rating_record(ft_unit_rating *units, int32_t nunits, const int32_t *unit_of_replica,
                     int32_t R, const ft_stats *stats);

/* Units in order of increasing F (ties keep index order) into order[0..count).
 * Units whose F is infinite are left out except in check rounds (round a
 * multiple of check_interval > 0), where they come first so that they run:
 * the paper uses a unit that always failed only at predefined check intervals,
 * to see whether it is still malfunctioning (Sec. IV.B).
 * The first entry is the light-weight mode's choice (Sec. IV.C), the first two
 * the DMR pair (Sec. IV.D).  Returns FT_OK or FT_EINVAL. */
int ft_rating_rank(const ft_unit_rating *units, int32_t nunits, uint64_t round,
                   uint64_t check_interval, int32_t *order, int32_t *count);

/* ---- misc ---- */
const char *ft_strerror(int code);
int         ft_last_cuda_error(void);     /* cudaError_t of the last FT_ECUDA in this thread */
uint64_t    ft_launch_count(void);        /* kernels this library has launched (all threads) */
const char *ft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FTVOTE_H */
