/*
 * dagexec.h -- C ABI of the fine-grained DAG executor for one GB300 (sm_103a).
 *
 * The library runs an application DAG G = <(K,B),(E_I,E_O,E)> (paper §3,
 * "Problem Formulation": kernels K, buffers B = B_I u B_O, buffer->kernel
 * edges E_I, kernel->buffer edges E_O, buffer->buffer edges E) of
 * data-parallel kernels -- GEMM with fused bias/activation, row softmax and
 * elementwise nodes -- with fine-grained concurrency: one persistent kernel
 * pulls output tiles of all nodes from a device work queue and waits only on
 * the producer tiles whose region it reads (tile-granularity dependency
 * counters in HBM), so independent branches and the ready rows of dependent
 * nodes overlap.  This is the sub-kernel, work-item-level interleaving of
 * concurrent kernels that the paper names as its future work (§7,
 * Conclusion); the coarse-grained alternative (§1: each kernel finished,
 * with its copies, before its successors start) is kept as a baseline entry
 * point (dag_submit_coarse).
 *
 * Conventions (all entry points):
 *  - Plain C types only; a CUDA stream is passed as `void*` (a cudaStream_t,
 *    NULL = the legacy default stream).
 *  - The library owns all device memory: every buffer, the work queue, the
 *    dependency counters and the trace.  The caller owns host pointers.
 *  - Every function returns a dag_status; DAG_OK is 0.  On failure the
 *    thread-local message of dag_last_error() says why.  No exception and no
 *    abort crosses the ABI.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 *  - After a device error (DAG_EDEVICE, DAG_ETIMEOUT from the device) the
 *    handle is poisoned: every later call but dag_destroy returns the error.
 */
#ifndef DAGEXEC_H
#define DAGEXEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DAG_OK = 0,
  DAG_EINVAL = 1,       /* bad argument, id out of range, edge list disagrees with the buffers */
  DAG_ECYCLE = 2,       /* the kernel graph has a cycle (no valid schedule, Def. 5) */
  DAG_ESHAPE = 3,       /* operand shapes disagree, or a view does not fit its parent */
  DAG_EDTYPE = 4,       /* unsupported dtype combination (e.g. GEMM with mixed A/B dtypes) */
  DAG_EMULTIWRITER = 5, /* a buffer element written by two kernels, or a kernel writing what it reads */
  DAG_ENOMEM = 6,       /* device or host allocation failed */
  DAG_EBUSY = 7,        /* a submit is still in flight on this handle */
  DAG_ETIMEOUT = 8,     /* a device wait or dag_wait ran past its limit */
  DAG_EDEVICE = 9,      /* a CUDA call failed */
  DAG_EUNSUPPORTED = 10 /* shape/alignment the kernels do not handle */
} dag_status;

typedef enum { DAG_F32 = 0, DAG_BF16 = 1 } dag_dtype;

/* Kernel kinds (paper §5 transformer head: GEMM, softmax; §2: vadd) */
typedef enum { DAG_OP_GEMM = 0, DAG_OP_ADD = 1, DAG_OP_SOFTMAX = 2, DAG_OP_UNARY = 3 } dag_op;
typedef enum { DAG_ACT_NONE = 0, DAG_ACT_RELU = 1, DAG_ACT_GELU = 2 } dag_act;

/* buffer roles */
#define DAG_BUF_INPUT 1u    /* contents come from the caller (an isolated write, §3) */
#define DAG_BUF_OUTPUT 2u   /* read back by the caller (an isolated read, §3) */
#define DAG_BUF_RESIDENT 4u /* with INPUT: uploaded once and kept (weights); no per-submit upload */

/*
 * A buffer b in B: a row-major rows x cols matrix.  The library picks the
 * row pitch (a multiple of 16 elements).  view_of >= 0 makes this buffer a
 * column slice [col_offset, col_offset+cols) of buffer view_of (same rows and
 * dtype): a concat written in place by several kernels (§5, heads
 * concatenated).  component: unused for buffers (keep 0).
 */
typedef struct {
  int32_t rows, cols;
  int32_t dtype;      /* dag_dtype */
  uint32_t flags;     /* DAG_BUF_* */
  int32_t view_of;    /* -1, or parent buffer id (the parent must not be a view) */
  int32_t col_offset; /* first parent column of the slice */
} dag_buffer_desc;

/*
 * A kernel k in K.  Inputs a, b, bias and output out are buffer ids; their
 * roles define E_I (buffer -> kernel) and E_O (kernel -> buffer).
 *   GEMM     out = act(scale * A.B + bias)  A: (batch*M) x K; B: (batch*K) x N,
 *            or (batch*N) x K with trans_b = 1; bias: 1 x N or -1;
 *            out: (batch*M) x N.  A and B share one dtype; bf16 runs
 *            tensor-core tiles with f32 accumulation, f32 runs as set by
 *            dag_options.f32_gemm (dag_f32_gemm).
 *   ADD      out = act(A + B), same shapes.
 *   SOFTMAX  out[i,:] = softmax(scale * A[i,:]) (max-subtracted).
 *   UNARY    out = act(A).
 * component: task component id (paper §3, T in the partition of K); used by
 *   dag_analyze for FRONT/END/IN and intra/inter edge classification and by
 *   dag_submit_cq; dag_submit runs all components in one persistent launch.
 */
typedef struct {
  int32_t op;  /* dag_op */
  int32_t a, b, bias, out;
  int32_t trans_b;
  int32_t act; /* dag_act */
  float scale;
  int32_t batch;
  int32_t component;
} dag_node_desc;

/* An edge in the paper's form k_i,b_r -> k_j,b_s (§4.A): kernel src_node
 * writes buffer src_buf, which kernel dst_node reads as dst_buf.  On one GPU
 * the buffers of an intra edge are one object, so src_buf == dst_buf, or
 * dst_buf is a view overlapping src_buf.  Edges are optional (they are implied
 * by the buffer ids); when given, each must be implied (else DAG_EINVAL). */
typedef struct {
  int32_t src_node, src_buf, dst_node, dst_buf;
} dag_edge;

/* ready-queue ordering policies (paper §5: priority queue F ordered by the
 * bottom-level rank; HEFT's rank from profiled times) */
typedef enum {
  DAG_SCHED_RANK_MODEL = 0,  /* bottom-level rank from a roofline time model */
  DAG_SCHED_RANK_GIVEN = 1,  /* bottom-level rank from node_cost_us (measured profile or learned model) */
  DAG_SCHED_FIFO = 2         /* tiles in topological node order, no ranking */
} dag_sched;

typedef struct {
  uint64_t timeout_ns;        /* limit of every device spin-wait; 0 = 2 s */
  int32_t trace;              /* record a per-tile trace (tickets, times, SM) */
  int32_t max_ctas;           /* persistent grid size; 0 = one CTA per SM */
  int32_t scheduler;          /* dag_sched */
  int32_t tile_override;      /* 0 = automatic; else forces every bf16 GEMM to BN = tile_override (64/128/256),
                                 and every f32 GEMM that can take the wide tensor-core form to that width
                                 (128/256; 64 = the 128 x 64 form) */
  const float *node_cost_us;  /* per-node time estimates for DAG_SCHED_RANK_GIVEN (n_nodes entries) */
  int32_t debug_never_ready;  /* test hook: >0 makes that many tiles wait on a counter nothing releases,
                                 so the device wait runs out and reports DAG_ETIMEOUT */
  int32_t use_graph;          /* 1: dag_submit replays the persistent launch from a captured CUDA graph */
  int32_t autotune;           /* 1: dag_create times candidate plans (tile widths x queue orders) on the
                                 device with zeroed buffers and keeps the fastest (see dag_plan_info) */
  int32_t f32_gemm;           /* dag_f32_gemm: how f32 GEMMs run */
  int32_t split_k;            /* 0: split the K loop of bf16 GEMMs whose depth level leaves most SMs idle
                                 (up to 4 partials, summed in a fixed order); 1: never split */
  int32_t fuse;               /* dag_fuse: elementwise kernels run inside the epilogue of the tensor-core
                                 GEMM whose output they read, when that output has no other reader, is no
                                 view and no DAG input or output (up to 2 in a chain per GEMM; each step is
                                 rounded to its buffer's dtype exactly as if stored: bit-identical results) */
  int32_t keep_layout;        /* 0: a resident bf16/f32 input read only as the B operand of GEMMs with
                                 trans_b = 0 (all with one shape) is kept transposed (N x K per batch) on
                                 the device, made from its given layout at upload, so the tensor cores read
                                 it K-major; 1: every buffer keeps the caller's layout */
  int32_t rank_form;          /* dag_rank_form: the priority the ranked queue orders ready tiles by */
  int32_t merge;              /* 0: sibling GEMMs -- one task component, one A (trans_b = 0, batch 1), one
                                 K, activation and scale, each narrower than 256 columns, with resident
                                 weights (and biases) only they read and private intermediate outputs --
                                 run as one GEMM over their summed width: their weights, biases and
                                 outputs are laid out as column slices of parent buffers (see
                                 dag_merge_get; bit-identical results).  1: every GEMM keeps its own
                                 tiles.  keep_layout = 1 implies 1. */
} dag_options;

/* Ready-tile priority of the ranked schedulers (dag_options.rank_form).
 * DAG_RANK_UPWARD (default): the bottom-level (upward) rank of the tile's
 * kernel -- its cost plus the longest cost path to a sink -- as the paper's
 * priority queue F orders task components (§5) and HEFT ranks kernels.
 * DAG_RANK_CRITICAL_PATH: upward rank plus downward rank (the longest cost
 * path from a root to the kernel), so every kernel of the longest path has
 * the same, highest priority (the critical-path priority of CPOP, published
 * beside HEFT); a long chain of short kernels then keeps its place ahead of
 * wide independent work all along, where the upward rank lets it fall
 * behind once its remaining length drops below the wide work's cost. */
typedef enum { DAG_RANK_UPWARD = 0, DAG_RANK_CRITICAL_PATH = 1 } dag_rank_form;

/* Epilogue fusion (dag_options.fuse).  DAG_FUSE_NONE (default): every kernel
 * runs its own tiles.  DAG_FUSE_ACT: activation kernels run in the epilogue
 * of their GEMM.  DAG_FUSE_ALL: adds as well; the epilogue then waits for the
 * add's other operand and reads it row by row through L2.  A plan with fused
 * kernels runs a second build of the executor kernel that holds the fused
 * epilogue code; its higher register pressure slows every other tile of the
 * launch, which is why fusion is off unless asked for. */
typedef enum { DAG_FUSE_NONE = 0, DAG_FUSE_ACT = 1, DAG_FUSE_ALL = 2 } dag_fuse;

/* f32 GEMM arithmetic.  DAG_F32_GEMM_TENSOR (default): on the tensor cores
 * with the 3 x TF32 split (each operand x = hi + lo, hi = tf32(x),
 * lo = tf32(x - hi); A.B ~= Ahi.Bhi + Ahi.Blo + Alo.Bhi with f32
 * accumulation; about 2^-21 relative error per product), for every f32 GEMM
 * whose operand views start on 16-byte boundaries: 128 x 128 or 128 x 256
 * tiles when B is read K-major (trans_b, or a weight kept transposed) and N
 * exceeds 64 -- except in a DAG level too small for 128-column tiles with a
 * K loop too short to split (K < 1024), where twice as many 128 x 64 tiles
 * fill more SMs -- else 128 x 64 tiles; the others, and every f32 GEMM under
 * DAG_F32_GEMM_SIMT, run as f32 FFMA on the SM cores.
 * DAG_F32_GEMM_TENSOR_NARROW keeps every tensor-core f32 GEMM on 128 x 64
 * tiles, DAG_F32_GEMM_TENSOR_WIDE puts every one that can on 128 x 128 / 256
 * tiles (for comparisons). */
typedef enum {
  DAG_F32_GEMM_TENSOR = 0,
  DAG_F32_GEMM_SIMT = 1,
  DAG_F32_GEMM_TENSOR_NARROW = 2,
  DAG_F32_GEMM_TENSOR_WIDE = 3
} dag_f32_gemm;

typedef struct dag_handle dag_handle;

/*
 * dag_create: build the paper's DAG G = <(K,B),(E_I,E_O,E)> (§3, Problem
 * Formulation) from the node, buffer and optional edge lists (edges in the
 * k_i,b_r -> k_j,b_s form of §4.A, Design Frontend); validate it (acyclic,
 * as a valid schedule requires a topological dispatch order, Def. 5; one
 * writer per element; shapes and dtypes); tile every kernel; build the tile
 * dependency counters (the precedence set E_Q of the command-queue structure,
 * Def. 4 and its rules i-iii, taken from kernels down to output tiles); order
 * the tiles (a linear extension of the tile DAG ranked by the bottom-level
 * rank of §5, the priority of the task queue F in Alg. 1); and allocate all
 * device memory.  opts may be NULL.  *out receives the handle; free it with
 * dag_destroy.  Needs a CUDA device.
 * Errors: DAG_EINVAL (bad id, count or edge not implied by the buffers),
 * DAG_ECYCLE, DAG_ESHAPE, DAG_EDTYPE, DAG_EMULTIWRITER, DAG_EUNSUPPORTED,
 * DAG_ENOMEM (device allocation), DAG_EDEVICE; *out is untouched on error.
 */
dag_status dag_create(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                      const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts,
                      dag_handle **out);

/*
 * dag_batch_create: many DAGs in one plan and one persistent launch (a batch
 * is a DAG whose connected components are the items; their tiles share one
 * work queue, so small and large DAGs fill the GPU together).  Buffer ids of
 * item i in the returned handle are offset by the buffer counts of items
 * 0..i-1; node ids likewise by their node counts.  Everything else is as for
 * dag_create (opts applies to the whole batch).  The paper's DAG G of §3 may
 * already consist of several independent task components (the H heads of
 * §5's Experiment 1 are one DAG); a batch is such a G built from separate
 * descriptions.
 */
typedef struct {
  const dag_node_desc *nodes;
  int32_t n_nodes;
  const dag_buffer_desc *buffers;
  int32_t n_buffers;
} dag_batch_item;

dag_status dag_batch_create(const dag_batch_item *items, int n_items, const dag_options *opts, dag_handle **out);

/*
 * dag_set_input: give the host data of input buffer `buf` (rows x cols,
 * dense, its dtype: f32 or bf16 bit patterns): the source of the isolated
 * write (b_m, k) of §3 (an E_I edge with no producer), which Alg. 1's enq
 * enqueues before the kernel's ndrange command.  The pointer is recorded, not
 * copied: it must stay valid and unchanged until the next dag_wait returns.
 * The copy runs at the next dag_submit on an upload stream (a copy engine)
 * that overlaps compute; tiles reading the buffer wait on its ready flag.
 * Pinned memory (dag_host_alloc) makes the copy asynchronous.
 */
dag_status dag_set_input(dag_handle *h, int buf, const void *host_ptr);

/* dag_set_output: host destination (rows x cols, dense) that every following
 * dag_submit fills after the kernel (device->host on a copy stream): the
 * isolated read (k, b_n) of §3 (an E_O edge with no consumer), enqueued after
 * the kernel's ndrange command (§3, the enq rules; Alg. 1); NULL cancels.  Same lifetime rule as dag_set_input.  DAG_EINVAL for a weight
 * kept transposed on the device (dag_options.keep_layout). */
dag_status dag_set_output(dag_handle *h, int buf, void *host_ptr);

/*
 * dag_submit: enqueue one execution of a valid schedule (Def. 5): pending
 * uploads on the upload streams (each followed by its ready flag), one
 * persistent executor launch on `stream`, and registered readbacks.  This is
 * the device-side form of Alg. 1's dispatch loop (schedule / setup_cq /
 * dispatch, with the callbacks cb replaced by dependency counters in device
 * memory), at the granularity of output tiles instead of kernels: the
 * sub-kernel interleaving named as future work in §7.  Asynchronous; returns
 * after enqueue.  Errors: DAG_EBUSY if the previous submit was not waited
 * for; DAG_EDEVICE if a copy or the launch could not be enqueued; the error
 * of a poisoned handle.
 */
dag_status dag_submit(dag_handle *h, void *stream);

/* dag_submit_coarse: the coarse-grained baseline (§2, one command queue: each
 * kernel's write, ndrange and read commands finish before the next kernel's;
 * §5's default configuration): uploads on `stream`, then one launch per kernel
 * in topological order on `stream` (the same tile code, a grid of that
 * kernel's tiles, no cross-kernel overlap), then readbacks.
 * A GEMM with fused elementwise kernels launches in the place of the last of
 * them (DAG_FUSE_NONE gives one launch per kernel throughout). */
dag_status dag_submit_coarse(dag_handle *h, void *stream);

/*
 * dag_submit_cq: the paper's own fine-grained form (§4.B, Alg. 1; the
 * clustering scheme of §5) on CUDA streams, as a second, host-driven executor
 * over the same tiles:
 *   schedule: ready task components (every kernel of FRONT(T) has all its
 *     predecessors finished) wait in a priority queue F ordered by the largest
 *     bottom-level rank of their FRONT kernels (or by id with fifo = 1); the
 *     GPU is the only device, so one component at a time holds it;
 *   setup_cq: the kernels of T, starting from FRONT(T) and each once all its
 *     predecessors in T are processed, go round-robin to n_queues CUDA streams
 *     (the command queues Q): the uploads of its isolated inputs, then its
 *     launch (a grid of the kernel's tiles, as in dag_submit_coarse), then the
 *     readback of its output if registered; a predecessor on another stream
 *     is waited on through its event (the set E_Q); a GEMM with fused
 *     elementwise kernels launches in the turn of the last of them, and the
 *     turns before it launch nothing (their events still order successors);
 *   callbacks: after each kernel of END(T), a host function (the paper's cb)
 *     marks it finished; when all of END(T) have, T is finished, its ready
 *     successor components enter F and the device is returned.
 * Synchronous: returns when every kernel and readback has completed.
 * Components: DAG_TC_GIVEN uses dag_node_desc.component (the partition must
 * leave the component graph acyclic, else DAG_ECYCLE); DAG_TC_WHOLE puts the
 * DAG in one component; DAG_TC_PER_KERNEL makes every kernel a component
 * (the coarse-grained policies of §5, Experiments 2-3: one callback per
 * kernel).  Timings come from CUDA events on the streams; node_start_us /
 * node_end_us, if not NULL, receive each kernel's [start, end) from the first
 * dispatch (n_nodes entries each, caller-owned).
 */
typedef enum { DAG_TC_GIVEN = 0, DAG_TC_WHOLE = 1, DAG_TC_PER_KERNEL = 2 } dag_tc;

typedef struct {
  int32_t n_queues;       /* command queues (streams) per dispatched component, 1..32 */
  int32_t components;     /* dag_tc */
  int32_t fifo;           /* 1: F ordered by component id instead of rank */
  int32_t pad;
  uint64_t timeout_ns;    /* limit on waiting for any callback; 0 = 10 s; DAG_ETIMEOUT poisons the handle */
  float *node_start_us;   /* optional [n_nodes] */
  float *node_end_us;     /* optional [n_nodes] */
  int32_t *node_queue;    /* optional [n_nodes]: the queue setup_cq sent each kernel to (its component's
                             kernels round-robin over n_queues in dispatch order, Alg. 1) */
} dag_cq_options;

typedef struct {
  double device_us;       /* first dispatch -> last kernel end, CUDA events */
  double host_us;         /* the schedule loop's wall time, first dispatch -> last callback handled */
  double gap_us;          /* summed device idle between one component's last kernel end and the
                             next component's first kernel start (the callback round trip) */
  int32_t n_components;
  int32_t n_callbacks;
} dag_cq_result;

dag_status dag_submit_cq(dag_handle *h, const dag_cq_options *opts, dag_cq_result *result);

/* dag_wait: block until the last submit finished or timeout_ns passed
 * (DAG_ETIMEOUT, the submit stays in flight): the host side of Alg. 1's
 * sleep_till_cb_update, which waits until every kernel of G has finished.
 * Then reads the device error word: DAG_ETIMEOUT if a device wait ran out
 * (the handle is poisoned), DAG_EDEVICE on a CUDA error. */
dag_status dag_wait(dag_handle *h, uint64_t timeout_ns);

/* dag_poll: non-blocking dag_wait (Alg. 1's sleep_till_cb_update of §4.B
 * asked once instead of waited on): DAG_EBUSY while the last submit (with its
 * readbacks) is still running, else what dag_wait would return. */
dag_status dag_poll(dag_handle *h);

/* dag_get_output: synchronous device->host copy of buffer `buf` (rows x cols,
 * dense, the caller's layout even for a weight kept transposed on the
 * device) into host_ptr; call after dag_wait.  The on-demand form of the
 * isolated read (k, b_n) of §3.  host_ptr is caller-owned and must hold
 * rows x cols elements.  Errors: DAG_EINVAL (bad id or NULL pointer),
 * DAG_EBUSY (a submit not yet waited for), DAG_EDEVICE. */
dag_status dag_get_output(dag_handle *h, int buf, void *host_ptr);

/* dag_device_ptr: device address of buffer `buf` (borrowed, valid until
 * dag_destroy) and its row pitch in elements; NULL on a bad id and for a
 * weight kept transposed on the device (dag_options.keep_layout).  The
 * device-side buffer b of §3's B, for callers that chain their own kernels;
 * the paper's OpenCL buffers have no such accessor. */
const void *dag_device_ptr(dag_handle *h, int buf, int64_t *ld_elems);

/* dag_destroy: wait for outstanding work (bounded), free everything the
 * handle owns (device buffers, plan, streams, events); the handle is invalid
 * afterwards.  The paper has no counterpart beyond releasing the OpenCL
 * objects of §4.B; NULL is accepted (DAG_OK). */
dag_status dag_destroy(dag_handle *h);

/* dag_last_error: message of the last failure on this thread ("" if none).
 * Library plumbing with no counterpart in the paper. */
const char *dag_last_error(void);

/* dag_set_device: make CUDA device `ordinal` current for the calling host
 * thread inside the library (the library links its own CUDA runtime, so a
 * device chosen through another runtime instance does not carry over).
 * Handles created afterwards on this thread live on that device.  The paper's
 * device set A (§4.B) has one GPU here; this picks which. */
dag_status dag_set_device(int ordinal);

/* pinned host memory for asynchronous uploads/readbacks: the host side of the
 * isolated writes and reads of §3 (dag_set_input / dag_set_output), so that
 * they run on the copy engines beside the launch.  NULL on failure
 * (dag_last_error says why);
 * dag_host_free(NULL) is a no-op. */
void *dag_host_alloc(size_t bytes);
void dag_host_free(void *p);

/*
 * dag_run_noalloc: run a DAG on caller-owned device buffers without
 * allocating any device memory.  The paper has no counterpart; this exists
 * for callers that cannot call cudaMalloc (a process whose device memory is
 * fully reserved by its own pool, code running inside an allocator or an
 * error path, embedders whose allocator owns every device byte).
 *   buffer_ptrs[i], row_pitch[i]: device address and row pitch (elements)
 *     of every root buffer i (ignored for views, which live inside their
 *     parent).  Pitches must be >= cols and a multiple of 16 bytes; pointers
 *     16-byte aligned.  Inputs must already hold their data; outputs and
 *     intermediates are written in place.  No two root buffers may share an
 *     element of device memory (an output placed on an input, say): the
 *     planner treats roots as distinct objects, so overlapping roots are
 *     rejected with DAG_EINVAL before any device work.
 *   The executor's own working state (tile queue, dependency counters, node
 *   parameters, TMA descriptors, control block) lives in a fixed 1 MiB device
 *   array that every GPU loading this library holds until process exit.  A
 *   DAG whose plan does not fit is rejected with DAG_ENOMEM before any device
 *   work (roughly 15k tiles).
 *   The call is synchronous: it enqueues on `stream`, waits for it, and
 *   returns DAG_OK, DAG_ETIMEOUT (a device wait ran out) or an error.
 *   The first call on each device looks up the array's device address with
 *   that device current; make that first call before any stream capture.
 *   Every call shares the one array and clears the parts that must start at
 *   zero; calls that overlap on the GPU (from several host threads or
 *   streams) race on it, so callers must serialise them.
 *   opts may be NULL; tracing and the debug hook are ignored here.
 */
dag_status dag_run_noalloc(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers, int n_buffers,
                           void *const *buffer_ptrs, const int64_t *row_pitch, const dag_options *opts,
                           void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous admission of inference DAGs                           */
/* ------------------------------------------------------------------------ */
/*
 * A model is an inference DAG at a fixed batch size: its RESIDENT inputs are
 * weights (host data given here, uploaded once per slot and kept on the
 * device), its other inputs are the per-request activations, its OUTPUT
 * buffers are read back per request.  A slot is one planned instance of a
 * model with its own device buffers and stream.  Requests are admitted in
 * arrival order as soon as their model has an idle slot, or a new slot fits
 * in the free device memory (less hbm_reserve_bytes) under max_slots; an
 * admitted request launches immediately, so requests arriving while others
 * run overlap them on the device.  node_cost_us (may be NULL) gives the
 * per-kernel costs that rank each slot's queue (learned or measured).
 * No counterpart in the paper, which runs one DAG at a time: each request is
 * one persistent launch of its slot's plan (dag_submit, a valid schedule in
 * the sense of Def. 5, ordered by §5's bottom-level ranks).
 */
typedef struct {
  const dag_node_desc *nodes;
  int32_t n_nodes;
  const dag_buffer_desc *buffers;
  int32_t n_buffers;
  const void *const *weights;   /* [n_buffers]: host data of every RESIDENT input, NULL elsewhere */
  const float *node_cost_us;    /* [n_nodes] or NULL */
} dag_model_desc;

typedef struct {
  int32_t model;
  int32_t status;               /* dag_status of the request */
  double t_arrive_s, t_launch_s, t_done_s;  /* steady clock, seconds */
} dag_request_info;

typedef struct dag_server dag_server;
dag_status dag_server_create(const dag_model_desc *models, int n_models, int max_slots, size_t hbm_reserve_bytes,
                             const dag_options *opts, dag_server **out);
/* default request inputs/outputs of a model (streamed inputs and OUTPUT
 * buffers in buffer order), used when dag_server_submit gets NULL */
dag_status dag_server_set_io(dag_server *s, int model, const void *const *inputs, void *const *outputs);
/* create up to n_slots idle slots of a model now (planning and weight upload
 * ahead of the first requests) */
dag_status dag_server_warm(dag_server *s, int model, int n_slots);
/* queue a request (thread-safe); host buffers stay valid until it completes */
dag_status dag_server_submit(dag_server *s, int model, const void *const *inputs, void *const *outputs,
                             uint64_t *ticket);
/* complete finished requests, admit and launch waiting ones; returns the
 * number completed */
int dag_server_progress(dag_server *s);
/* drive progress until the request completes; fills info; releases the ticket */
dag_status dag_server_wait(dag_server *s, uint64_t ticket, uint64_t timeout_ns, dag_request_info *info);
/* open-loop run: n requests of the given models arriving as a Poisson process
 * of rate_hz (seeded SplitMix64 exponential gaps); latency_us[i] = completion
 * (readback done) minus scheduled arrival */
dag_status dag_server_simulate(dag_server *s, const int32_t *model_seq, int n, double rate_hz, uint64_t seed,
                               double *latency_us, double *wall_s, int *max_in_flight);
int dag_server_slots(dag_server *s);
dag_status dag_server_destroy(dag_server *s);

/* ------------------------------------------------------------------------ */
/* Learned cost model                                                        */
/* ------------------------------------------------------------------------ */
/*
 * A 3-layer perceptron x (in_dim) -> ReLU(64) -> ReLU(64) -> 1 that predicts
 * the (log) execution time of a kernel's tiles from its features; the
 * predictions become per-kernel costs (dag_options.node_cost_us with
 * DAG_SCHED_RANK_GIVEN), i.e. the bottom-level ranks that order the ready
 * queue (paper §5: priority queue F ordered by bottom-level rank; HEFT's
 * profiled kernel times).  Forward pass, mean-squared-error backward pass and
 * Adam run as CUDA kernels; arrays below are host arrays (copied in and out).
 * Parameters are one packed f32 array: W1 [in_dim][64], b1 [64], W2 [64][64],
 * b2 [64], W3 [64], b3 [1]; they start at zero, set them with
 * dag_mlp_set_params before training.  in_dim is 1..32.
 */
typedef struct dag_mlp dag_mlp;
dag_status dag_mlp_create(int in_dim, dag_mlp **out);
int dag_mlp_param_count(const dag_mlp *m);
dag_status dag_mlp_set_params(dag_mlp *m, const float *params, int n);
dag_status dag_mlp_get_params(dag_mlp *m, float *params, int n);
/* loss = mean over the n samples of (f(x_i) - y_i)^2; grad = d loss / d params
 * (X: n x in_dim row-major, y: n).  Deterministic: the per-64-sample chunks
 * are summed in index order. */
dag_status dag_mlp_loss_grad(dag_mlp *m, const float *X, const float *y, int n, float *loss, float *grad);
/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on
 * consecutive minibatches of `batch` samples, cycling through the samples in
 * the order given. */
dag_status dag_mlp_train(dag_mlp *m, const float *X, const float *y, int n, int steps, int batch, float lr);
dag_status dag_mlp_predict(dag_mlp *m, const float *X, int n, float *out);
dag_status dag_mlp_destroy(dag_mlp *m);

/* ------------------------------------------------------------------------ */
/* Inspection                                                                */
/* ------------------------------------------------------------------------ */

/* Host-only analysis (no device needed), following §3 Defs. 1-3 and the
 * classification of buffer edges and copies that follows them.  Per kernel:
 * the bit set cls[k] (1 = FRONT(T), 2 = END(T), 4 = IN(T)) of its task
 * component T.  Per E_I / E_O pair: isolated vs dependent copy.  Per
 * producer->consumer buffer edge: intra vs inter.  Arrays are caller-owned,
 * sized as documented; counts are returned. */
typedef struct {
  int32_t node, buf;
  int32_t is_write;    /* 1: (b,k) in E_I (a write to the device); 0: (k,b) in E_O (a read back) */
  int32_t isolated;    /* 1: isolated copy; 0: dependent copy */
} dag_copy_class;

typedef struct {
  int32_t src_node, src_buf, dst_node, dst_buf;
  int32_t inter;       /* 1: endpoints in different task components */
} dag_edge_class;

typedef struct {
  int32_t n_nodes;
  int32_t *cls;                /* [n_nodes] FRONT|END|IN bits */
  int32_t *topo;               /* [n_nodes] Kahn order, smallest id first */
  dag_copy_class *copies;      /* [cap_copies] */
  int32_t cap_copies, n_copies;
  dag_edge_class *edge_cls;    /* [cap_edges] */
  int32_t cap_edges, n_edge_cls;
} dag_analysis;

dag_status dag_analyze(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                       const dag_buffer_desc *buffers, int n_buffers, dag_analysis *out);

/* One executed tile: output region of one kernel, with the tickets it drew
 * from one global counter after acquiring its inputs (start) and after
 * writing its output, before releasing it (end), %globaltimer times (ns) of
 * the claim of its queue position, the end of its waits, the start of its
 * epilogue / SIMT work and its release, and the SM it ran on.  A GEMM whose
 * K loop is split (split != 0) has S tiles per output region, split =
 * (s << 8) | S: partials s < S-1 write partial sums to scratch, and partial
 * S-1 waits for them, adds them in order and writes the region.  A GEMM tile
 * with fused elementwise kernels (dag_fusion_get) carries the GEMM's id and
 * region and writes the last fused kernel's output there; like a finishing
 * partial, its start ticket is drawn after the waits of its epilogue. */
typedef struct {
  int32_t node, r0, r1, c0, c1;   /* region of the kernel's output buffer */
  uint32_t start_ticket, end_ticket;
  uint32_t smid;
  int32_t split, pad;
  uint64_t t_claim_ns, t_start_ns, t_work_ns, t_end_ns;
} dag_trace_record;

/* dag_trace_get: records of the last submit in queue order (needs
 * opts.trace; call after dag_wait); *n = number of tiles.  The data of the
 * paper's Gantt charts (§2, §5) at tile granularity; the tickets let a checker
 * confirm that the run was a valid schedule (Def. 5). */
dag_status dag_trace_get(dag_handle *h, dag_trace_record *out, int cap, int *n);

/* dag_trace_stamps: per tile (queue order of the last submit), ten
 * %globaltimer stamps (ns): claim, dependencies satisfied, last operand load
 * issued, first MMA, last MMA committed, workers start, accumulator ready,
 * body done (the first worker warp's part: its stores issued, or completed
 * where they are TMA stores), fence and barrier done, release done (0 where
 * a phase does not apply).  out holds 10 * cap values.  Diagnostic; needs
 * opts.trace.  The phases inside each bar of the paper's Gantt charts (§2,
 * §5), per tile. */
dag_status dag_trace_stamps(dag_handle *h, uint64_t *out, int cap, int *n);

/* dag_trace_launch: the window of the last persistent launch traced (needs
 * dag_options.trace): enter_exit[0] = the earliest CTA entry, enter_exit[1] =
 * the latest CTA exit, on the %globaltimer clock (ns) of dag_trace_stamps, so
 * that the executor's own start-up and tear-down show beside the tiles' phases
 * (the launch's part of the paper's Gantt charts, §2 and §5).  DAG_EINVAL if
 * tracing is off or the last submit was not a persistent launch. */
dag_status dag_trace_launch(dag_handle *h, uint64_t *enter_exit);

/* Static plan facts (no counterpart in the paper; critical_path_us is the
 * largest bottom-level rank of §5 under the roofline time model). */
typedef struct {
  int32_t n_tiles, n_counters, n_waits, grid;
  int32_t smem_bytes;
  double flops, bytes;           /* algorithmic totals (2MNK per GEMM; each operand read once + output written once) */
  double critical_path_us;       /* sum over the critical path of max(flops/peak, bytes/bw) under the peaks given to dag_set_peaks */
  double work_bound_us;          /* max(critical path, total flops/peak, total bytes/bw) */
  int32_t tile_override, scheduler;  /* the plan's tile policy and queue order (the autotuner's choice) */
  double tuned_us;               /* autotune: measured makespan of the chosen plan (0 if not tuned) */
  double buffer_bytes;           /* device memory of the handle's buffers (every buffer at its row pitch, a
                                    weight kept transposed in its N x K form); 0 for caller-owned buffers */
} dag_plan_info;

dag_status dag_plan_get(dag_handle *h, dag_plan_info *out);

/* Sibling GEMMs merged by the planner (dag_options.merge): per kernel v,
 * leader[v] = the kernel whose tiles compute it (itself for that kernel; -1
 * if v keeps its own tiles) and col_offset[v] = its first column in the
 * merged GEMM's output (0 if not merged).  The merged kernel's tiles (its id
 * in dag_tiles_get and the trace) cover the summed width.  cap entries at
 * most; *n = kernel count.  The parent buffers are internal: the buffer
 * calls reject their ids with DAG_EINVAL, as any id the caller did not
 * describe.  dag_merge_host: the same without a device.  Not
 * in the paper: a planning step below its kernels, which still run in a
 * topological order of G (Def. 5). */
dag_status dag_merge_get(dag_handle *h, int32_t *leader, int32_t *col_offset, int cap, int *n);
dag_status dag_merge_host(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers, int n_buffers,
                          const dag_options *opts, int32_t *leader, int32_t *col_offset);

/* Per-kernel costs (us) the plan's ranks were computed from: the roofline
 * time model's, or node_cost_us as given; n = kernel count.  These are the
 * kernel times behind §5's bottom-level ranks (HEFT's profiled times). */
dag_status dag_node_costs_get(dag_handle *h, float *out, int cap, int *n);

/* Per-tile static description in queue order: {node, r0, r1, c0, c1,
 * cfg | split << 16} (cfg: the tile shape code; split as in dag_trace_record).
 * A tile is this library's unit of fine-grained dispatch: the role the work
 * groups of concurrently dispatched kernels play in §2. */
dag_status dag_tiles_get(dag_handle *h, int32_t *out6, int cap, int *n);

/* Epilogue fusion of the plan (see dag_options.fuse): out[v] = the GEMM
 * kernel whose tiles compute kernel v, or -1 when v runs its own tiles;
 * n = kernel count.  A fused kernel's buffer between the GEMM and it is never
 * written; the GEMM's tiles write the last fused kernel's output, and their
 * trace records carry the GEMM's id.  Not in the paper: the fused kernels
 * still finish in a topological order of G (Def. 5), their tiles with the
 * GEMM's. */
dag_status dag_fusion_get(dag_handle *h, int32_t *out, int cap, int *n);

/* Host-only: the fusion dag_create would choose (as dag_fusion_get), n_nodes
 * entries in out. */
dag_status dag_fusion_host(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                           const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts, int32_t *out);

/* Host-only planning, no device needed: the tiles in queue order (as
 * dag_tiles_get) that dag_create would build for a GPU with n_sm SMs running
 * one executor CTA per SM.  info may be NULL.  The queue is a topological
 * order of the tile graph, the tile-level form of Def. 5's dispatch order. */
dag_status dag_plan_host(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                         const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts, int n_sm,
                         int32_t *out6, int cap, int *n_tiles, dag_plan_info *info);

/* Peaks used by the roofline estimates and the time model (TFLOP/s, GB/s),
 * the time model behind §5's bottom-level ranks when no measured or learned
 * kernel times are given. */
void dag_set_peaks(double bf16_tflops, double f32_tflops, double hbm_gbs);

#ifdef __cplusplus
}
#endif
#endif /* DAGEXEC_H */
