// exec_kernel.cu -- the persistent DAG executor kernel (fine-grained path) and
// its per-kernel launch form (coarse-grained baseline).
//
// Fine-grained mode: each CTA loops { claim the next queue position with one
// atomic; wait (acquire, bounded) until the dependency counters of that tile
// reach their targets; run the tile; release (increment) the counters of the
// row blocks it wrote }.  The queue order is a linear extension of the tile
// dependency graph, so any tile a CTA waits on was claimed earlier by a CTA
// that is running and never waits on a later tile: the loop cannot deadlock
// for any grid size, and the deadline bounds every wait regardless.  This
// replaces the paper's host-side callback chain (Alg. 1: setup_cq, cb) with
// device counters, at the granularity of output tiles rather than kernels.
#include <climits>

#include "dag_internal.h"
#include "ptx.cuh"
#include "tiles.cuh"

namespace dagx {

constexpr int kSmemStages = kStages * (kStageA + kStageB);
constexpr int kSmemBytes = kSmemStages + 256 + 1024;  // stages + control block + alignment slack

__device__ __forceinline__ void record_error(const ExecParams &p, uint32_t code, int tile) {
  if (atomicCAS(&p.ctrl->err_code, 0u, code) == 0u) p.ctrl->err_tile = (uint32_t)tile;
  atomicExch(&p.ctrl->abort, 1u);
  __threadfence();
}

// Wait until every dependency of tile t is satisfied in this epoch.
__device__ __forceinline__ bool wait_deps(const ExecParams &p, const TileDesc &t, uint32_t epoch) {
  const uint64_t deadline = globaltimer() + p.timeout_ns;
  for (int i = 0; i < t.wait_count; ++i) {
    const Wait w = p.waits[t.wait_begin + i];
    uint32_t spins = 0;
    if (w.idx & kWaitFlag) {
      const uint32_t *f = p.flags + (w.idx & ~kWaitFlag);
      while ((int32_t)(ld_acquire(f) - (epoch + 1u)) < 0) {
        if ((++spins & 63u) == 0 && (globaltimer() > deadline || ld_relaxed(&p.ctrl->abort))) return false;
        __nanosleep(64);
      }
    } else {
      const uint32_t *c = p.counters + w.idx;
      const uint32_t base = epoch * w.target;
      while (ld_acquire(c) - base < w.target) {
        if ((++spins & 63u) == 0 && (globaltimer() > deadline || ld_relaxed(&p.ctrl->abort))) return false;
        __nanosleep(32);
      }
    }
  }
  return true;
}

__global__ void __launch_bounds__(kThreads, 1) dag_exec_kernel(const __grid_constant__ ExecParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  SmemCtl *ctl = reinterpret_cast<SmemCtl *>(smem + kSmemStages);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->accum, 1);
    mbar_fence_init();
    ctl->fail = 0;
  }
  if (warp == 0) {
    tmem_alloc(&ctl->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  PipeState ps = {0u, 0u, 0u, 0u, 0u};
  const uint32_t epoch = (p.mode == 0) ? ld_relaxed(&p.ctrl->epoch) : 0u;
  int iter = 0;

  for (;;) {
    if (tid == 0) {
      int t = INT_MAX;
      if (p.mode == 0) {
        if (!ld_relaxed(&p.ctrl->abort)) t = (int)atomicAdd(&p.ctrl->head, 1u);
      } else if (iter == 0) {
        t = p.tile_begin + (int)blockIdx.x;
      }
      if (t < p.n_tiles) {
        if (p.mode == 0) {
          if (!wait_deps(p, p.tiles[t], epoch)) {
            if (!ld_relaxed(&p.ctrl->abort)) record_error(p, E_DEP_TIMEOUT, t);
            t = INT_MAX;
          }
          fence_proxy_async_global();  // our TMA reads follow the acquired generic writes
        }
        if (t != INT_MAX && p.trace_on) {
          ctl->start_ticket = atomicAdd(&p.ctrl->ticket, 1u);
          ctl->t_start = globaltimer();
        }
      } else {
        t = INT_MAX;
      }
      ctl->tile = t;
    }
    __syncthreads();
    const int t = ctl->tile;
    if (t >= p.n_tiles || ctl->fail) break;
    ++iter;
    const TileDesc td = p.tiles[t];
    const NodeParams &np = p.nodes[td.node];
    const uint64_t deadline = globaltimer() + p.timeout_ns;
    switch (td.op) {
      case T_GEMM_BF16:
        if (!tile_gemm_bf16(p, td, np, smem, ctl, ps, deadline) && tid == 0) record_error(p, E_PIPE_TIMEOUT, t);
        break;
      case T_GEMM_F32:
        if (td.cfg == F32_128x128) tile_gemm_f32<128, 128>(td, np, reinterpret_cast<float *>(smem));
        else if (td.cfg == F32_128x64) tile_gemm_f32<128, 64>(td, np, reinterpret_cast<float *>(smem));
        else tile_gemm_f32<64, 64>(td, np, reinterpret_cast<float *>(smem));
        break;
      case T_ADD: tile_eltwise(td, np, true); break;
      case T_UNARY: tile_eltwise(td, np, false); break;
      case T_SOFTMAX: tile_softmax(td, np); break;
      default:
        if (tid == 0) record_error(p, E_BAD_TILE, t);
        break;
    }
    fence_proxy_async_global();  // make this tile's generic stores visible to later TMA readers
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      if (p.trace_on) {
        TraceRec r;
        r.start_ticket = ctl->start_ticket;
        r.end_ticket = atomicAdd(&p.ctrl->ticket, 1u);  // drawn before the release
        r.smid = smid();
        r.tile = (uint32_t)t;
        r.t_start = ctl->t_start;
        r.t_end = globaltimer();
        p.trace[t] = r;
      }
      if (p.mode == 0)
        for (int i = 0; i < td.rel_count; ++i) red_release_add(&p.counters[p.rels[td.rel_begin + i]], 1u);
    }
  }

  // teardown: free TMEM; the last CTA of a persistent launch rewinds the queue
  // and advances the epoch that the counter targets are measured from.
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(ctl->tmem_base, kTmemCols);
  }
  if (tid == 0 && p.mode == 0) {
    __threadfence();
    const uint32_t n = atomicAdd(&p.ctrl->exit_count, 1u);
    if (n == gridDim.x - 1) {
      p.ctrl->head = 0;
      p.ctrl->exit_count = 0;
      __threadfence();
      atomicAdd(&p.ctrl->epoch, 1u);
    }
  }
}

int exec_smem_bytes() { return kSmemBytes; }

cudaError_t exec_prepare() {
  return cudaFuncSetAttribute(dag_exec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

int max_coresident_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dag_exec_kernel, kThreads, kSmemBytes) != cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_persistent(const ExecParams &p, int grid, cudaStream_t s) {
  ExecParams q = p;
  q.mode = 0;
  q.tile_begin = 0;
  dag_exec_kernel<<<grid, kThreads, kSmemBytes, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const ExecParams &p, int tile_begin, int n, cudaStream_t s) {
  ExecParams q = p;
  q.mode = 1;
  q.tile_begin = tile_begin;
  dag_exec_kernel<<<n, kThreads, kSmemBytes, s>>>(q);
  return cudaGetLastError();
}

}  // namespace dagx
