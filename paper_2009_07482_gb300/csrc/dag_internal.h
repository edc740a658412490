// dag_internal.h -- plan structures shared by the host planner and the
// device executor of libdagexec (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dagexec.h"

namespace dagx {

// Tile kinds.  A tile is a rectangle of one kernel's output buffer.
enum TileOp : int32_t {
  T_GEMM_BF16 = 0,  // tcgen05 (TMEM accumulator), TMA-fed, 128 x BN
  T_GEMM_F32 = 1,   // exact-f32 SIMT FFMA, BM x BN
  T_ADD = 2,        // 128-bit elementwise add (+ activation)
  T_UNARY = 3,      // 128-bit elementwise activation
  T_SOFTMAX = 4,    // warp-per-row softmax over whole rows
  T_GEMM_TF32 = 5,  // f32 GEMM on the tensor cores, 3 x TF32 split, 128 x 64
  T_GEMM_TF32W = 6  // the same, 128 x BN (BN = cfg: 128 or 256), B K-major, K blocks of 16
};

// f32 SIMT GEMM tile shapes (cfg field of a T_GEMM_F32 tile)
enum F32Cfg : int32_t { F32_64x64 = 0, F32_128x64 = 1, F32_128x128 = 2 };

// CTA layout: warp 0 = scheduler + TMA producer, warp 1 = MMA issuer,
// warp 2 = releaser (publishes finished tiles to the dependency counters),
// warp 3 idle, warps 4-11 = 256 worker threads (GEMM epilogues, the operand
// split of f32 tensor-core tiles, and every SIMT tile).
constexpr int kThreads = 384;
constexpr int kWorkerBase = 128;    // first worker thread
constexpr int kWorkers = 256;       // worker threads
constexpr int kBM = 128;            // bf16 GEMM tile rows (MMA M)
constexpr int kBK = 64;             // bf16 K per stage (one 128-byte swizzle row)
constexpr int kStages = 4;          // TMA -> MMA pipeline depth
constexpr int kBKF = 32;            // f32 K per stage (one 128-byte swizzle row)
constexpr int kTf32BN = 64;         // f32 tensor-core tile width (128 x 64 form)
constexpr int kBKW = 16;            // f32 K per stage of the wide form (64-byte swizzle rows)
constexpr int kWideP = 8;           // stages per TMEM partial sum of the wide form (128 of K)
constexpr int kParts = 4;           // TMEM partial slots of an f32 tensor-core tile (4 x 64 columns)
constexpr int kMaxBN = 256;
constexpr int kStageA = kBM * kBK * 2;        // 16 KiB
constexpr int kStageB = kMaxBN * kBK * 2;     // 32 KiB
constexpr int kAccCols = 256;                 // one 128 x 256 f32 accumulator
constexpr int kTmemCols = 2 * kAccCols;       // double-buffered accumulators
constexpr int kSlots = 2;                     // scheduler -> MMA / workers tile ring
constexpr int kRelSlots = 4;                  // workers -> releaser ring of finished tiles
constexpr int kWorkerScratch = 32 * 1024;     // per-CTA worker scratch: epilogue staging / f32 tiles
constexpr int kEpiRows = 32;                  // epilogue store box: 32 rows x 128 bytes per warp
constexpr int kMaxPost = 2;                   // elementwise kernels fused into one GEMM epilogue

struct TileDesc {
  int32_t node;   // kernel id
  int32_t op;     // TileOp
  int32_t r0, r1; // rows of the output buffer (row-stacked batches: within one batch)
  int32_t c0, c1; // columns of the output buffer (view coordinates)
  int32_t cfg;    // bf16: BN; f32: F32Cfg; others: 0
  int32_t wait_begin, wait_count;  // into ExecParams::waits
  int32_t rel_begin, rel_count;    // into ExecParams::rels
  int32_t split;  // split K: (s << 8) | S for partial s of S (the last one finishes the tile); 0 = whole K
};
static_assert(sizeof(TileDesc) == 48, "TileDesc layout");
__host__ __device__ inline int split_count(const TileDesc &t) { return t.split & 0xFF; }
__host__ __device__ inline int split_index(const TileDesc &t) { return t.split >> 8; }
// a partial of a split tile that is not the last: it stores raw f32 partial sums
__host__ __device__ inline bool split_partial(const TileDesc &t) { return t.split && split_index(t) < split_count(t) - 1; }

// A dependency: counter[idx] must reach base(epoch) + target.  With
// kWaitFlag set, idx is an input-buffer ready flag that must equal epoch+1.
struct Wait {
  uint32_t idx;
  uint32_t target;
};
constexpr uint32_t kWaitFlag = 0x80000000u;
// With kWaitLate set, idx is a counter the workers wait on before the tile's
// epilogue rather than the scheduler before its loads (a split-K tile's
// finishing partial waits so for the other partials, and a GEMM tile with
// fused elementwise kernels for their other operands).
constexpr uint32_t kWaitLate = 0x40000000u;

// An elementwise kernel fused into a GEMM epilogue: out = act(v + X) for an
// add (X its other operand, same rows and columns as the GEMM output), or
// act(v) for an activation; v is the previous step's value rounded to the
// dtype that step's kernel stores.
struct PostOp {
  const void *X;    // add: the other operand (view-adjusted); activation: null
  int64_t ldx;      // X row pitch (elements)
  int32_t x_dt;     // 0 = f32, 1 = bf16
  int32_t act;      // dag_act
  int32_t out_dt;   // dtype this kernel's output is stored in
  int32_t xvec;     // X rows start on 16-byte boundaries
};

struct NodeParams {
  const void *A, *B, *bias;
  void *C;
  int64_t lda, ldb, ldc;   // row pitches in elements
  int32_t M, N, K, batch;  // per-batch GEMM dims (M = rows for elementwise/softmax, N = cols)
  int32_t trans_b, act;
  float scale;
  int32_t a_dt, b_dt, c_dt, bias_dt;  // 0 = f32, 1 = bf16
  int32_t tmap_a, tmap_b;             // tensor-map indices (bf16 GEMM), else -1
  int32_t vec;                        // 16-byte vector paths are aligned
  int32_t tmap_c;                     // output tensor map for the TMA-store epilogue, else -1
  float *scratch;                     // split K: partial sums, (S-1) blocks of 128 x BN f32 per output tile
  int32_t n_post;                     // elementwise kernels fused into the epilogue (C, ldc, c_dt and
                                      // tmap_c then describe the last one's output)
  int32_t o_dt;                       // dtype of the GEMM's own output (rounding point before post[0])
  PostOp post[kMaxPost];
};

struct Ctrl {
  uint32_t head;        // next queue position (persistent mode)
  uint32_t exit_count;  // CTAs that left the loop
  uint32_t epoch;       // completed persistent launches
  uint32_t ticket;      // trace ticket counter
  uint32_t err_code;    // 0, or a DevErr
  uint32_t err_tile;
  uint32_t abort;       // set on error: every CTA leaves its waits
  uint32_t pad;
  uint64_t t_enter;     // tracing: earliest CTA entry of the launch (%globaltimer ns)
  uint64_t t_exit;      // tracing: latest CTA exit
};

enum DevErr : uint32_t { E_NONE = 0, E_DEP_TIMEOUT = 1, E_PIPE_TIMEOUT = 2, E_BAD_TILE = 3 };

// Per-tile phase stamps (%globaltimer, ns), recorded when tracing is on.
enum Stamp : int {
  S_CLAIM = 0,     // scheduler claimed the queue position
  S_READY = 1,     // scheduler: dependencies satisfied
  S_LOADED = 2,    // scheduler: last TMA load of the tile issued (bf16 GEMM)
  S_MMA0 = 3,      // MMA warp: accumulator free, first MMA issued
  S_MMA1 = 4,      // MMA warp: last MMA issued and committed
  S_WORK = 5,      // workers picked the tile up
  S_ACC = 6,       // workers: accumulator complete observed (bf16 GEMM)
  S_BODY = 7,      // workers: all output stores issued
  S_SYNC = 8,      // workers: proxy fence + barrier done
  S_END = 9,       // release done
  kNumStamps = 10
};

struct TraceRec {
  uint32_t start_ticket, end_ticket, smid, tile;
  uint64_t stamp[kNumStamps];
};

struct ExecParams {
  const TileDesc *tiles;
  int32_t n_tiles;
  int32_t mode;        // 0 = persistent queue, 1 = coarse (one tile per CTA, no waits)
  int32_t tile_begin;  // coarse: first tile of this launch
  int32_t trace_on;
  int32_t fused;       // some GEMM epilogue runs fused elementwise kernels (selects the kernel variant)
  int32_t pad_;
  const Wait *waits;
  const uint32_t *rels;
  const NodeParams *nodes;
  const CUtensorMap *tmaps;
  uint32_t *counters;
  uint32_t *flags;
  Ctrl *ctrl;
  TraceRec *trace;
  uint64_t timeout_ns;
};

// launchers (exec_kernel.cu)
int exec_smem_bytes();
cudaError_t exec_prepare();  // sets the kernel's shared-memory attribute (once per process)
cudaError_t launch_persistent(const ExecParams &p, int grid, cudaStream_t s);
cudaError_t launch_coarse(const ExecParams &p, int tile_begin, int n, cudaStream_t s);
// dst (batch blocks of N x K, row pitch ldd) = per-block transpose of src
// (batch blocks of K x N, row pitch lds); elem_bytes 2 or 4 (layout.cu)
cudaError_t launch_transpose(const void *src, int64_t lds, void *dst, int64_t ldd, int batch, int K, int N,
                             int elem_bytes, cudaStream_t st);
int max_coresident_ctas_per_sm();

// Plan a DAG over caller-owned device buffers and serialise every device-side
// plan array (tensor maps, queue, waits, releases, node parameters, zeroed
// counters, flags and control block) into `blob`, laid out for a device
// region starting at `region` of `capacity` bytes; fills the kernel
// parameters that point into that region.  DAG_ENOMEM if it does not fit.
dag_status plan_into_region(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers, int n_buffers,
                            void *const *ptrs, const int64_t *lds, const dag_options *opts, char *region,
                            size_t capacity, std::vector<char> &blob, ExecParams &xp, int &grid);
// set the thread-local message returned by dag_last_error
dag_status report_error(dag_status s, const char *msg);

}  // namespace dagx
