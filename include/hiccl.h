/*
 * hiccl.h -- C ABI of the GB300 hierarchical collective engine.
 *
 * A collective is composed from multicast, reduction and fence primitives
 * (HiCCL, arXiv 2408.05962, Sec. 3, Listing 1), factorized for a stated
 * hierarchy into per-level point-to-point copy and sum-reduce steps with
 * striping and pipelining (Sec. 4), and executed by one persistent CUDA
 * kernel per start (Sec. 5.2).  The P ranks are virtual: each rank is a set
 * of disjoint buffers in one GPU's memory, so every step is a copy or a
 * reduce between device buffers; per-level byte volumes are counted, not
 * measured on links.
 *
 * Conventions for every function below:
 *   - A status is returned; nothing aborts or throws (host memory running
 *     out inside a call is HICCL_ERR_NOMEM).  On failure the communicator's
 *     state is unchanged and hiccl_last_error() holds a message.
 *   - "device pointer" means a pointer into memory of the current CUDA
 *     device (cudaMalloc / PyTorch allocations); host pointers there are a
 *     caller error the library cannot detect before the kernel runs.
 *   - Counts are in elements of the communicator's dtype.
 *   - A communicator is not thread-safe; calls on one communicator must be
 *     serialized by the caller.  Different communicators are independent.
 */
#ifndef HICCL_H
#define HICCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hiccl_comm *hiccl_comm_t;

/* Payload element types.  F32 and I32 reductions are exact functions of the
 * hierarchy (see hiccl_add_reduction); BF16 and FP8E4M3 are reduced with FP32
 * accumulation. */
typedef enum {
  HICCL_F32 = 0,
  HICCL_I32 = 1,
  HICCL_BF16 = 2,
  HICCL_FP8E4M3 = 3
} hiccl_dtype_t;

/* Reduction operator (Sec. 3.1: "sum, max, logical or, etc.").
 *   SUM: see hiccl_add_reduction (all payloads).
 *   MAX / MIN: F32 IEEE maxNum / minNum (a NaN operand yields the other),
 *              I32, BF16 (exact: the result is one of the inputs); not FP8.
 *   LOR: I32 only; 1 where some contribution is nonzero, else 0.
 * A reduction with a single leaf is a copy: the operator is omitted (Sec. 3.1). */
typedef enum { HICCL_SUM = 0, HICCL_MAX = 1, HICCL_MIN = 2, HICCL_LOR = 3 } hiccl_op_t;

typedef enum {
  HICCL_OK = 0,
  HICCL_ERR_INVALID = 1,     /* bad argument, rank, hierarchy, stripe or pipeline */
  HICCL_ERR_STATE = 2,       /* call not allowed in the communicator's state      */
  HICCL_ERR_RACE = 3,        /* primitives of one epoch overlap (Sec. 3.2)         */
  HICCL_ERR_NOMEM = 4,       /* host or device allocation failed                   */
  HICCL_ERR_CUDA = 5,        /* a CUDA runtime call failed                         */
  HICCL_ERR_TIMEOUT = 6,     /* a dependency wait in the executor ran out          */
  HICCL_ERR_UNSUPPORTED = 7, /* valid request this build does not implement        */
  HICCL_ERR_TOO_LARGE = 8    /* request exceeds a fixed-size limit of the library  */
} hiccl_status_t;

/* ---- composition (Sec. 3, Listing 1) ---------------------------------------- */

/* Create a communicator over `nranks` (>= 1) virtual ranks whose payload is
 * `dtype`.  *out receives the handle (NULL on failure).  The handle owns all
 * library memory; release it with hiccl_destroy. */
hiccl_status_t hiccl_create(int nranks, hiccl_dtype_t dtype, hiccl_comm_t *out);

/* Register M(root, leaves, count) (Sec. 3.1): after execution every leaf j's
 * range recv[j][0, count) holds the root's send[root][0, count).
 *   send, recv : arrays of nranks device pointers, one per virtual rank, as
 *                each rank would pass its own buffer in the paper's SPMD API.
 *                Only send[root] and recv[j] for j in leaves are read; other
 *                entries may be NULL.  A root that is also a leaf with
 *                recv[root] == send[root] is in place (nothing to copy).
 *   leaves     : nleaves distinct ranks in [0, nranks); nleaves == 0 registers
 *                nothing (leaves may then be NULL).
 * The caller keeps every buffer valid and unmoved until hiccl_destroy.
 * Only allowed before hiccl_init / hiccl_plan (HICCL_ERR_STATE otherwise). */
hiccl_status_t hiccl_add_multicast(hiccl_comm_t comm, const void *const *send,
                                   void *const *recv, size_t count, int root,
                                   const int *leaves, int nleaves);

/* Register R(leaves, root, count, op) (Sec. 3.1): after execution the root's
 * range recv[root][0, count) holds the sum over the leaves i of
 * send[i][0, count).  Only send[i] for i in leaves and recv[root] are read;
 * leaves holds nleaves >= 1 distinct ranks.
 * Sum order (fixed, independent of root, stripe and pipeline): a rank
 * contributes its values; a group of the hierarchy contributes the left fold
 * of its non-empty subgroups' contributions in ascending subgroup order, in
 * the payload's arithmetic (F32: IEEE round-to-nearest-even adds, no fused
 * multiply-add; I32: wrapping adds; BF16/FP8: FP32 adds, rounded to the
 * payload at each hierarchy level).  Ownership and state as for multicast. */
hiccl_status_t hiccl_add_reduction(hiccl_comm_t comm, const void *const *send,
                                   void *const *recv, size_t count,
                                   const int *leaves, int nleaves, int root,
                                   hiccl_op_t op);

/* Register a fence (Sec. 3.3): primitives added after it depend on the
 * earlier ones whose buffer ranges they overlap (read-after-write,
 * write-after-read, write-after-write).  It is not a barrier. */
hiccl_status_t hiccl_add_fence(hiccl_comm_t comm);

/* Standard collectives of Table 2 (Sec. 3.2-3.3), registered natively as the
 * primitives the paper composes them from. */
typedef enum {
  HICCL_BROADCAST = 0,       /* M(root, U, dp)                          send dp, recv dp */
  HICCL_REDUCE = 1,          /* R(U, root, dp)                          send dp, recv dp */
  HICCL_ALLGATHER = 2,       /* sum_i M(i, U, d)                        send d,  recv dp */
  HICCL_REDUCESCATTER = 3,   /* sum_j R(U, j, d)                        send dp, recv d  */
  HICCL_ALLREDUCE = 4,       /* Listing 2: RS, fence, in-place AG       send dp, recv dp */
  HICCL_SCATTER = 5,         /* sum_j R(root, j, d)                     send dp, recv d  */
  HICCL_GATHER = 6,          /* sum_i M(i, root, d)                     send d,  recv dp */
  HICCL_ALLTOALL = 7,        /* sum_i sum_j M(i, j, d)                  send dp, recv dp */
  HICCL_ALLREDUCE_SINGLE = 8 /* sum_j R(U, j, dp) (single step)         send dp, recv dp */
} hiccl_collective_t;

/* Register collective `kind` over chunk length d (elements; d*P is the largest
 * per-rank buffer, Sec. 3.2) for per-rank buffers send[r], recv[r] (arrays of
 * nranks device pointers laid out as in the table above).  The reductions of
 * REDUCE, REDUCESCATTER, ALLREDUCE and ALLREDUCE_SINGLE combine with `op`
 * (other kinds ignore it).  Same ownership, state and error rules as
 * hiccl_add_multicast / hiccl_add_reduction. */
hiccl_status_t hiccl_add_collective(hiccl_comm_t comm, hiccl_collective_t kind, size_t d,
                                    const void *const *send, void *const *recv, int root,
                                    hiccl_op_t op);

/* ---- optimization (Sec. 4) -------------------------------------------------- */

/* Factorize the registered program, check the plan (hiccl_validate) and
 * upload it to the current device (Sec. 4, Sec. 5.2 "memoizing").
 *   hierarchy : nlevels (>= 1) factors >= 1, top level first, whose product
 *               is nranks; ranks of a level-l group are contiguous (Sec. 4.2).
 *   stripe    : s in [1, nranks], branches per primitive (Sec. 4.3).
 *   pipeline  : m >= 1, channels per branch (Sec. 4.5).
 * Errors: HICCL_ERR_INVALID (arguments), HICCL_ERR_RACE (overlapping
 * primitives within an epoch), HICCL_ERR_NOMEM / HICCL_ERR_CUDA (device
 * memory).  Allocates the step table, dependency counters and relay buffers
 * on the current device; they are freed by hiccl_destroy. */
hiccl_status_t hiccl_init(hiccl_comm_t comm, const int *hierarchy, int nlevels,
                          int stripe, int pipeline);

/* Host-only variant of hiccl_init: factorize and validate without touching
 * any GPU, so that the plan queries below work on a machine without one.
 * Pointers are only compared, never dereferenced.  hiccl_init may follow:
 * with the same hierarchy, stripe and pipeline it uploads this plan without
 * factorizing again (a caller can plan on one thread, check the plan's
 * device footprint with hiccl_plan_info, and upload it later). */
hiccl_status_t hiccl_plan(hiccl_comm_t comm, const int *hierarchy, int nlevels,
                          int stripe, int pipeline);

/* ---- execution (Sec. 5.2) --------------------------------------------------- */

/* Enqueue one execution of the collective on `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream) and return without waiting (the
 * paper's non-blocking start).  HICCL_ERR_STATE before hiccl_init or while a
 * previous start has not been waited on.  Stream order is kept: the launch
 * may become resident while the previous kernel of the stream drains
 * (programmatic dependent launch) but touches no memory before that kernel
 * has completed.  Under CUDA-graph capture only the launch is recorded; each
 * replay is a complete execution, and replays may be interleaved with other
 * starts of the communicator as long as its CTAS_PER_SM and THREADS options
 * are those it had at capture. */
hiccl_status_t hiccl_start(hiccl_comm_t comm, void *cuda_stream);

/* Block until the last start has finished and its buffers may be reused
 * (the paper's blocking wait).  Returns HICCL_ERR_TIMEOUT if a dependency
 * wait inside the executor exceeded its limit (the outputs are then
 * undefined; the communicator is reset and may be started again), and
 * HICCL_ERR_CUDA on a CUDA error. */
hiccl_status_t hiccl_wait(hiccl_comm_t comm);

/* ---- autotuning ------------------------------------------------------------------- */

typedef struct {
  int stripe;                     /* chosen s                                    */
  int pipeline;                   /* chosen m                                    */
  int order;                      /* HICCL_OPT_ORDER value                       */
  int threads;                    /* HICCL_OPT_THREADS value                     */
  unsigned long long item_bytes;  /* HICCL_OPT_ITEM_BYTES value                  */
  float us;                       /* median time of one start, microseconds      */
  int trials;                     /* configurations timed                        */
} hiccl_tune_t;

/* Pick the fastest configuration of an initialized communicator by timing it
 * on `cuda_stream` (each candidate: re-plan, upload, one warm-up and three
 * timed runs, median of CUDA-event times): executor knobs (work order, item
 * size) always; with (flags & 1) first the stripe s (its current value, 1,
 * and the bottom hierarchy factor) and pipeline depth m (1, 2, 4, 8), the
 * paper's optimization parameters (Sec. 4.1), with the executor defaults;
 * with a ring (HICCL_OPT_RING > 1) only stripes up to the node size.  None of
 * these changes a result bit; the ring, which does, is not tuned.
 * The communicator ends up initialized with the best configuration, which
 * *best receives (may be NULL).  The trials execute the collective: receive
 * buffers are overwritten.  Blocking. */
hiccl_status_t hiccl_autotune(hiccl_comm_t comm, void *cuda_stream, int flags, hiccl_tune_t *best);

/* ---- batched execution ---------------------------------------------------------- */

/* One communicator whose program is the union of the programs of `n` planned
 * communicators (hiccl_plan or hiccl_init), executed by one persistent launch
 * per hiccl_start: their steps share one ticket order, interleaved by
 * dependency depth so that the short early levels of one collective overlap
 * the bulk of another.  The members keep their own state; the group copies
 * their plans, allocates its own table, counters and relay buffers on the
 * current device, and references the members' user buffers (which must stay
 * valid).  Start, wait, hbm_bytes, plan_info, trace and destroy apply;
 * hiccl_level_bytes does not (query the members).  FP8 members cannot be
 * grouped with other payloads (HICCL_ERR_UNSUPPORTED).
 *
 * hiccl_start of any communicator may be recorded in a CUDA graph: under
 * stream capture it records only the executor launch (no state change), each
 * replay is a complete execution (the dependency counters re-arm on the
 * device), and the caller synchronizes replays on its stream. */
hiccl_status_t hiccl_group(const hiccl_comm_t *comms, int n, hiccl_comm_t *out);

/* The host half of hiccl_group: the same combined, checked table, left
 * planned (not uploaded, nothing allocated on a device) for inspection
 * (hiccl_plan_info, hiccl_get_step, hiccl_debug_image); it cannot be
 * started.  Same arguments and errors as hiccl_group. */
hiccl_status_t hiccl_group_plan(const hiccl_comm_t *comms, int n, hiccl_comm_t *out);

/* ---- accounting -------------------------------------------------------------- */

/* Bytes that cross each hierarchy level per execution (Sec. 4.1 and Fig. 1:
 * the factorization exists to cut the volume on the upper, slower levels;
 * Table 3 gives the per-node top-level volume of each collective): for every
 * copy destination and every reduce input on another rank, the step's bytes
 * are added to the level at which the two ranks first fall into different
 * subgroups.  per_level receives nlevels values (top level first); nlevels
 * must equal the hierarchy's.  Valid after hiccl_init or hiccl_plan;
 * HICCL_ERR_INVALID for a NULL array or a wrong nlevels, HICCL_ERR_STATE
 * before planning, HICCL_ERR_UNSUPPORTED for a group (query its members). */
hiccl_status_t hiccl_level_bytes(hiccl_comm_t comm, unsigned long long *per_level,
                                 int nlevels);

/* Device-memory bytes one execution reads and writes by the schedule's
 * definition: a copy reads its bytes once and writes them once per
 * destination; an f-input reduce reads f times its bytes and writes them once.
 * Sec. 6.2 defines throughput as the buffer bytes d*p over time; this call
 * gives, for the same execution, the bytes the factorized schedule moves
 * through device memory (relay buffers and every destination included),
 * the numerator of a bandwidth compared with the HBM roofline.  Either
 * output may be NULL.  Valid after hiccl_init or hiccl_plan; HICCL_ERR_STATE
 * before planning. */
hiccl_status_t hiccl_hbm_bytes(hiccl_comm_t comm, unsigned long long *read,
                               unsigned long long *write);

typedef struct {
  unsigned long long steps;          /* copy + reduce steps                      */
  unsigned long long copy_steps;
  unsigned long long reduce_steps;
  unsigned long long items;          /* executor work items per start            */
  unsigned long long edges;          /* dependency edges                         */
  unsigned long long stages;         /* longest dependency chain (steps)         */
  unsigned long long scratch_bytes;  /* relay buffers on the device              */
  unsigned long long table_bytes;    /* step table + counters on the device      */
  unsigned long long slots;          /* pipeline time slots of the work order    */
  unsigned long long runs;           /* contiguous data ranges the items move     */
} hiccl_plan_info_t;

/* Summary of the factorized plan.  Valid after hiccl_init or hiccl_plan. */
hiccl_status_t hiccl_plan_info(hiccl_comm_t comm, hiccl_plan_info_t *out);

/* One step of the plan, for inspection and host-side checking.
 *   kind: 0 copy, 1 reduce.  level: hierarchy level crossed, -1 local.
 *   op: the reduce's hiccl_op_t (0 for copies).
 *   src_addr/dst_addr: device addresses, or byte offsets into the relay
 *   arena where the matching *_scratch flag is 1.  preds: indices of the
 *   steps this one depends on.  Arrays must hold nsrc, ndst and npreds
 *   entries (query with NULL arrays first; counts are always written). */
typedef struct {
  int kind;
  int level;
  int nsrc;
  int ndst;
  int npreds;
  int prim;
  int branch;
  int channel;
  int op;
  int reserved;
  unsigned long long nbytes;
  unsigned long long slot;
} hiccl_step_desc_t;

hiccl_status_t hiccl_get_step(hiccl_comm_t comm, unsigned long long index,
                              hiccl_step_desc_t *desc,
                              unsigned long long *src_addr, int *src_scratch,
                              int *src_rank, unsigned long long *dst_addr,
                              int *dst_scratch, int *dst_rank,
                              unsigned long long *preds);

/* ---- tuning and diagnostics -------------------------------------------------- */

typedef enum {
  HICCL_OPT_TIMEOUT_NS = 0,   /* dependency-wait limit inside the executor (default 1e9)  */
  HICCL_OPT_CTAS_PER_SM = 1,  /* executor CTAs per SM, capped by occupancy (default 2)    */
  HICCL_OPT_ITEM_BYTES = 2,   /* largest work item, bytes of step data (default 49152; 65536 for FP8) */
  HICCL_OPT_ORDER = 3,        /* work order: 0 pipeline slots, 1 stage depth (default)    */
  HICCL_OPT_THREADS = 4,      /* threads per executor CTA: 128, 256 (default), 512       */
  HICCL_OPT_TRACE = 5,        /* 1: record per-item timestamps (hiccl_get_trace); default 0 */
  HICCL_OPT_SLOT_ITEMS = 6,   /* items a pipeline slot is spread over (0, default: grid)  */
  HICCL_OPT_RING = 7          /* ring(n) of Sec. 4.4: n nodes chained (default 1, tree)    */
} hiccl_option_t;

/* Set an option.  TIMEOUT_NS, CTAS_PER_SM and THREADS apply to the next start
 * (a start whose grid differs from the previous start's begins from zeroed
 * dependency counters; a CUDA graph that recorded a start before such a
 * change must be captured again);
 * ITEM_BYTES, ORDER, SLOT_ITEMS and RING must be set before hiccl_init /
 * hiccl_plan, TRACE before hiccl_init.  The steps of one pipeline slot of S
 * bytes are cut into work items of `cap` bytes, cap = S / D rounded up to a
 * multiple of 4096 and kept within [4096, ITEM_BYTES] (an item closes at the
 * first segment boundary at or past cap, so it holds less than cap + 4096
 * bytes): with SLOT_ITEMS = 0 (default) D is the executor's grid (its CTAs
 * on the device current at planning; 304 without one) for S under 12 MiB,
 * so that a short slot runs as one round of items over every CTA, and 768
 * for larger slots; SLOT_ITEMS = k > 0 sets D = k for every slot.
 * RING = n (Sec. 4.4, hybrid ring+tree): the n nodes of P/n ranks, which must
 * be the groups of one hierarchy level (n = f_0 * ... * f_{l-1}; checked at
 * planning, HICCL_ERR_INVALID otherwise), are chained starting at the root's
 * node and in ascending node order, cyclically, skipping nodes without
 * leaves; the tree factorizes inside each node.  A multicast hops node to
 * node; a reduction folds along the chain backwards: the last node's tree
 * fold is sent to the previous node, whose entry rank folds its own
 * subgroups' partials followed by the incoming partial, and so on back to the
 * root's node -- so with n > 1 the floating-point sum order depends on the
 * root's node.  The stripe may not exceed P/n when n > 1. */
hiccl_status_t hiccl_set_option(hiccl_comm_t comm, hiccl_option_t opt, long long value);

/* Executor trace of the last start (HICCL_OPT_TRACE set before hiccl_init).
 * For every work item, in ticket order, 6 values: the %globaltimer time (ns)
 * its staging began, the time its predecessors were satisfied and it was
 * handed to the data warps, the time its data movement ended, the time its
 * successors were released, the SM that ran it, and the index of its first
 * step (hiccl_get_step).  `out` receives min(capacity, 6 * items) values;
 * *written gets that count.  Call after
 * hiccl_wait.  HICCL_ERR_STATE if tracing was not enabled. */
hiccl_status_t hiccl_get_trace(hiccl_comm_t comm, unsigned long long *out, size_t capacity, size_t *written);

/* Check a planned table before it reaches the GPU (hiccl_init and
 * hiccl_group also run this check): the table order is topological (so the
 * dependency graph is acyclic) and the successor lists mirror it; every
 * user-buffer operand lies in its primitive's registered ranges and every
 * relay operand in the relay arena; the work-item entries of each step tile
 * its segments exactly once; no item mixes pipeline slots or exceeds 64
 * entries; the runs of an item cover its entries.  HICCL_ERR_INVALID with the
 * first violation in hiccl_last_error; HICCL_ERR_STATE without a plan. */
hiccl_status_t hiccl_validate(hiccl_comm_t comm);

/* Inspection: the executor's table image of a planned communicator, built on
 * the host exactly as hiccl_init uploads it but with relay operands as
 * offsets into the relay arena (relay base 0).  `recs` receives the
 * work-item records (16-byte aligned, `*recs_bytes` in all) and `items` the
 * 32-byte item descriptors in ticket order (`*nitems` of them); a record
 * holds, at 16-byte aligned offsets: nent entries {step, meta, pointer
 * offset, dependency count} (u32 each); nrun + 1 prefix sums of the runs'
 * segment counts (u32); nrun runs {entry u32, pad u32, byte offset u64,
 * bytes u64}; nptr inline operand pointers (u64); the completion section
 * (u32): per entry its step's completion target, nent + 1 successor-list
 * offsets, then the successors (absent when the item's descriptor says
 * 0xffffffff).  With NULL buffers (or too small capacities, in bytes) only
 * the sizes are returned.  HICCL_ERR_STATE without a plan. */
hiccl_status_t hiccl_debug_image(hiccl_comm_t comm, void *recs, size_t recs_capacity, size_t *recs_bytes,
                                 void *items, size_t items_capacity, size_t *nitems);

/* Host-side fault injection for tests of hiccl_validate: corrupt the host
 * copy of a planned (hiccl_plan, not uploaded) table.  what = 0: make a step
 * depend on a later step (a cycle); 1: move a user-buffer operand out of its
 * primitive's buffers; 2: drop the last entry's segments.  Nothing of it
 * reaches the GPU: hiccl_init on the corrupted communicator is refused. */
hiccl_status_t hiccl_debug_corrupt(hiccl_comm_t comm, int what);

/* Fault injection for tests: add `extra` (0 restores) phantom dependencies to
 * step `index` in the uploaded table, so that the executor's bounded wait for
 * it runs out and hiccl_wait reports HICCL_ERR_TIMEOUT.  Host-side only: it
 * changes one counter target; it never makes the GPU fault. */
hiccl_status_t hiccl_debug_withhold(hiccl_comm_t comm, unsigned long long index, int extra);

/* ---- execution without device allocation ------------------------------------- */

/* Size of the fixed device array hiccl_run_static works in. */
#define HICCL_STATIC_ARENA_BYTES (16ull << 20)

/* Run a planned communicator once, allocating nothing: for callers that
 * cannot call cudaMalloc themselves (code running under a caller-owned
 * memory pool or budget, or inside an allocator callback, where a library
 * allocation would fail or break accounting).  The paper has no counterpart:
 * HiCCL's staging buffers are its own allocations.
 *   comm   : planned with hiccl_plan (or hiccl_init); its registered send and
 *            recv buffers are the inputs and outputs, owned by the caller.
 *   stream : cudaStream_t to run on (NULL: legacy default stream).
 * The step table, dependency counters and relay buffers are placed in one
 * file-scope device array of HICCL_STATIC_ARENA_BYTES that every GPU loading
 * this library holds until the process exits; no cudaMalloc, cudaFree or
 * other allocating routine is called.  The first call on a device, with that
 * device current, looks the array's address up (cudaGetSymbolAddress, once
 * per device and process, safe from several host threads); make that first
 * call before any stream capture.  A cudaDeviceReset of the device
 * invalidates the address: do not call this again in that process after
 * one.  The call uploads the plan,
 * zeroes the counters (the array keeps the previous call's contents), runs
 * the executor and blocks until the stream reaches the end of the run.
 * Every call, from any communicator, uses the same array: calls that overlap
 * on the GPU (other host threads, other streams) race and must be serialized
 * by the caller.  Returns HICCL_ERR_TOO_LARGE, before any CUDA call, when
 * the plan needs more than HICCL_STATIC_ARENA_BYTES; HICCL_ERR_STATE without a
 * plan; HICCL_ERR_TIMEOUT if a wait of the executor ran out; HICCL_ERR_CUDA on
 * a CUDA error or any other executor error (as hiccl_wait decodes them).  It
 * does not set the hiccl_last_error message. */
hiccl_status_t hiccl_run_static(hiccl_comm_t comm, void *cuda_stream);

/* Message of the last failed call on `comm` ("" if none); a static string
 * for comm == NULL.  Valid until the next call on comm. */
const char *hiccl_last_error(hiccl_comm_t comm);

/* Free everything the communicator owns (after waiting for a pending start).
 * NULL is ignored. */
void hiccl_destroy(hiccl_comm_t comm);

#ifdef __cplusplus
}
#endif

#endif /* HICCL_H */
