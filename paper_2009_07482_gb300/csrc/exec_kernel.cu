// exec_kernel.cu -- the persistent DAG executor kernel (fine-grained path) and
// its per-kernel launch form (coarse-grained baseline).
//
// Fine-grained mode: the CTAs pull output tiles of all kernels from one work
// queue.  Inside a CTA three roles run concurrently, connected by mbarrier
// rings in shared memory:
//   scheduler (warp 0, lane 0): claim the next queue position with one
//     atomic, wait (acquire, bounded) until the dependency counters of that
//     tile reach their targets, publish it in the tile ring, and for a bf16
//     GEMM tile stream its operands into the stage ring with TMA;
//   MMA (warp 1, lane 0): for each bf16 GEMM tile, tcgen05.mma over the stage
//     ring into one of two TMEM accumulators;
//   workers (warps 4-11): GEMM epilogues (TMEM -> global) and every SIMT tile
//     (f32 GEMM, softmax, elementwise); after a tile they release (increment)
//     the counters of the row blocks it wrote.
// So the next tile's dependency wait and operand loads overlap the current
// tile's MMAs and epilogue.  The queue order is a linear extension of the
// tile dependency graph and each CTA handles its tiles in claim order, so the
// smallest unfinished queue position is always runnable: no deadlock for any
// grid size, and every wait has a deadline regardless.  This replaces the
// paper's host-side callback chain (Alg. 1: setup_cq, cb) with device
// counters, at the granularity of output tiles rather than kernels.
#include <climits>

#include "dag_internal.h"
#include "ptx.cuh"
#include "tiles.cuh"

namespace dagx {

constexpr int kSmemStages = kStages * (kStageA + kStageB);
constexpr int kSmemCtl = (int)((sizeof(SmemCtl) + 255) / 256 * 256);
constexpr int kSmemBytes = kSmemStages + kWorkerScratch + kSmemCtl + 1024;  // + alignment slack
static_assert(kSmemBytes <= 232448, "shared memory budget");

// worker-side broadcast values (written by the worker leader)
struct WorkerShared {
  int32_t tile;
  int32_t ok;
  uint32_t late_ticket;  // a tile with waits before its epilogue: start ticket drawn after them
};

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
    if (w.idx & kWaitLate) continue;  // taken by the workers before the epilogue
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

// The late waits of tile t (worker leader, before the epilogue).
__device__ __forceinline__ bool wait_late(const ExecParams &p, const TileDesc &t, uint32_t epoch) {
  const uint64_t deadline = globaltimer() + p.timeout_ns;
  for (int i = 0; i < t.wait_count; ++i) {
    const Wait w = p.waits[t.wait_begin + i];
    if (!(w.idx & kWaitLate)) continue;
    const uint32_t *c = p.counters + (w.idx & ~kWaitLate);
    const uint32_t base = epoch * w.target;
    uint32_t spins = 0;
    while (ld_acquire(c) - base < w.target) {
      if ((++spins & 63u) == 0 && (globaltimer() > deadline || ld_relaxed(&p.ctrl->abort))) return false;
      __nanosleep(32);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// scheduler + TMA producer (one thread)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void run_scheduler(const ExecParams &p, uint8_t *smem, SmemCtl *ctl, uint32_t epoch) {
  Ring slot = {0u, 0u}, st = {0u, 0u};
  for (int iter = 0;; ++iter) {
    int t = -1;
    if (!ctl->fail) {
      if (p.mode == 0) {
        if (!ld_relaxed(&p.ctrl->abort)) {
          t = (int)atomicAdd(&p.ctrl->head, 1u);
          if (t >= p.n_tiles) t = -1;
        }
      } else if (iter == 0) {
        t = p.tile_begin + (int)blockIdx.x;
      }
    }
    TileDesc td;
    uint64_t tc = 0, ts = 0;
    uint32_t tk = 0;
    if (t >= 0) {
      td = p.tiles[t];
      if (p.trace_on) tc = globaltimer();
      if (p.trace_on) p.trace[t].stamp[S_CLAIM] = tc;
      if (p.mode == 0) {
        if (!wait_deps(p, td, epoch)) {
          if (!ld_relaxed(&p.ctrl->abort)) record_error(p, E_DEP_TIMEOUT, t);
          ctl->fail = 1;
          t = -1;
        } else {
          fence_proxy_async_global();  // our TMA reads follow the acquired generic writes
        }
      }
      if (t >= 0 && p.trace_on) {
        tk = atomicAdd(&p.ctrl->ticket, 1u);
        ts = globaltimer();
        p.trace[t].stamp[S_READY] = ts;
      }
    }
    // publish in the tile ring (the slot must have been consumed by MMA and workers)
    if (!mbar_wait(&ctl->slot_empty[slot.idx], slot.phase ^ 1u, globaltimer() + 2 * p.timeout_ns + 1000000000ull)) {
      record_error(p, E_PIPE_TIMEOUT, t);
      ctl->fail = 1;
      return;
    }
    TileSlot &s = ctl->slot[slot.idx];
    s.t = t;
    s.start_ticket = tk;
    s.t_claim = tc;
    s.t_start = ts;
    mbar_arrive(&ctl->slot_full[slot.idx]);
    slot.next(kSlots);
    if (t < 0) return;
    if (td.op == T_GEMM_BF16 || td.op == T_GEMM_TF32 || td.op == T_GEMM_TF32W) {
      const uint64_t dl = globaltimer() + p.timeout_ns;
      const bool ok = td.op == T_GEMM_BF16   ? gemm_produce(p, td, p.nodes[td.node], smem, ctl, st, dl)
                      : td.op == T_GEMM_TF32 ? tf32_produce(p, td, p.nodes[td.node], smem, ctl, st, dl)
                                             : tf32w_produce(p, td, p.nodes[td.node], smem, ctl, st, dl);
      if (!ok) {
        record_error(p, E_PIPE_TIMEOUT, t);
        ctl->fail = 1;
      }
      if (p.trace_on) p.trace[t].stamp[S_LOADED] = globaltimer();
    }
  }
}

// ---------------------------------------------------------------------------
// MMA issuer (one thread)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void run_mma(const ExecParams &p, uint8_t *smem, SmemCtl *ctl) {
  Ring slot = {0u, 0u}, st = {0u, 0u};
  uint32_t accb = 0, ph[2] = {0u, 0u};
  uint32_t split_par = 0;  // bit s: parity of the next split[s] phase
  uint32_t pq = 0;         // f32 K-block partials issued
  const uint64_t slot_limit = 2 * p.timeout_ns + 1000000000ull;
  for (;;) {
    if (!mbar_wait(&ctl->slot_full[slot.idx], slot.phase, globaltimer() + slot_limit)) {
      ctl->fail = 1;
      return;
    }
    const int t = ctl->slot[slot.idx].t;
    mbar_arrive(&ctl->slot_empty[slot.idx]);
    slot.next(kSlots);
    if (t < 0) return;
    const TileDesc td = p.tiles[t];
    if (td.op != T_GEMM_BF16 && td.op != T_GEMM_TF32 && td.op != T_GEMM_TF32W) continue;
    // a wide f32 tile of 256 columns holds both accumulator buffers
    const bool both = td.op == T_GEMM_TF32W && td.cfg == 256;
    const uint64_t dl = globaltimer() + p.timeout_ns;
    if (!mbar_wait(&ctl->acc_empty[accb], ph[accb] ^ 1u, dl)) { ctl->fail = 1; return; }
    ph[accb] ^= 1u;
    if (both) {
      if (!mbar_wait(&ctl->acc_empty[accb ^ 1u], ph[accb ^ 1u] ^ 1u, dl)) { ctl->fail = 1; return; }
      ph[accb ^ 1u] ^= 1u;
    }
    tc_fence_after();
    if (p.trace_on) p.trace[t].stamp[S_MMA0] = globaltimer();
    const uint32_t acc = ctl->tmem_base + accb * kAccCols;
    bool ok;
    if (td.op == T_GEMM_BF16) {
      ok = gemm_mma(td, p.nodes[td.node], smem, ctl, st, acc, dl);
    } else if (td.op == T_GEMM_TF32) {
      ok = tf32_mma(p.nodes[td.node], smem, ctl, st, split_par, pq, acc, dl);
    } else {
      uint32_t tS, tX;
      tf32w_cols(td, ctl->tmem_base, accb, tS, tX);
      ok = tf32w_mma(td, p.nodes[td.node], smem, ctl, st, split_par, pq, tS, tX, dl);
    }
    if (!ok) {
      ctl->fail = 1;
      return;
    }
    if (td.op == T_GEMM_BF16) mma_commit(&ctl->acc_full[accb]);  // f32 tiles signal per partial
    if (p.trace_on) p.trace[t].stamp[S_MMA1] = globaltimer();
    if (!both) accb ^= 1u;  // a tile holding both buffers leaves the next tile where it started
  }
}

// ---------------------------------------------------------------------------
// releaser (warp 2, lane 0): publishes each finished tile -- one gpu-scope
// release fence, then a relaxed increment of every counter the tile
// releases -- while the workers already run the next tile.  The workers'
// writes are ordered before the hand-over by their barrier and the ring's
// mbarrier (release / acquire at CTA scope), and the fence is cumulative.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void run_releaser(const ExecParams &p, SmemCtl *ctl) {
  Ring r = {0u, 0u};
  const uint64_t slot_limit = 2 * p.timeout_ns + 1000000000ull;
  for (;;) {
    if (!mbar_wait(&ctl->rel_full[r.idx], r.phase, globaltimer() + slot_limit)) {
      ctl->fail = 1;
      return;
    }
    const RelSlot s = ctl->rel[r.idx];
    mbar_arrive(&ctl->rel_empty[r.idx]);
    r.next(kRelSlots);
    if (s.t < 0) return;
    const TileDesc &td = p.tiles[s.t];
    if (p.trace_on) {
      TraceRec &tr = p.trace[s.t];
      tr.start_ticket = s.start_ticket;
      tr.end_ticket = atomicAdd(&p.ctrl->ticket, 1u);  // drawn before the release (the fence orders it)
      tr.smid = smid();
      tr.tile = (uint32_t)s.t;
      tr.stamp[S_WORK] = s.t_work;
    }
    fence_acq_rel_gpu();
    if (p.mode == 0)
      for (int i = 0; i < td.rel_count; ++i) red_relaxed_add(&p.counters[p.rels[td.rel_begin + i]], 1u);
    if (p.trace_on) p.trace[s.t].stamp[S_END] = globaltimer();
  }
}

// ---------------------------------------------------------------------------
// workers (256 threads); every decision is taken by the leader and broadcast
// through shared memory, so all workers reach the same named barriers
// ---------------------------------------------------------------------------
template <bool kFused>
__device__ __forceinline__ void run_workers(const ExecParams &p, uint8_t *smem, SmemCtl *ctl, WorkerShared *ws) {
  const int wt = threadIdx.x - kWorkerBase;
  const uint32_t epoch = p.mode == 0 ? ld_relaxed(&p.ctrl->epoch) : 0u;
  Ring slot = {0u, 0u};
  uint32_t accb = 0, ph[2] = {0u, 0u};
  Tf32State fs = {{0u, 0u}, 0u, 0u};  // the workers split f32 stages and add up their partials
  float *fsm = reinterpret_cast<float *>(smem + kSmemStages);
  const uint64_t slot_limit = 2 * p.timeout_ns + 1000000000ull;
  Ring rel = {0u, 0u};
  // hand a finished tile (or -1: no more) to the releaser (worker leader only)
  auto hand_over = [&](int t, uint32_t start_ticket, uint64_t t_work) -> bool {
    if (!mbar_wait(&ctl->rel_empty[rel.idx], rel.phase ^ 1u, globaltimer() + slot_limit)) return false;
    ctl->rel[rel.idx] = RelSlot{t, start_ticket, t_work};
    mbar_arrive(&ctl->rel_full[rel.idx]);
    rel.next(kRelSlots);
    return true;
  };
  for (;;) {
    if (wt == 0) {
      const bool ok = mbar_wait(&ctl->slot_full[slot.idx], slot.phase, globaltimer() + slot_limit);
      ws->tile = ok ? ctl->slot[slot.idx].t : -2;
      ws->ok = 1;
    }
    worker_sync();
    const int t = ws->tile;
    if (t < 0) {
      if (wt == 0) {
        if (t == -2) ctl->fail = 1;
        hand_over(-1, 0u, 0ull);
      }
      return;
    }
    const TileSlot sl = ctl->slot[slot.idx];
    const uint64_t t_work = (p.trace_on && wt == 0) ? globaltimer() : 0;
    const TileDesc td = p.tiles[t];
    const NodeParams &np = p.nodes[td.node];
    // waits taken before the epilogue: a split tile's finishing partial (the
    // other partials' sums) and a tile with fused adds (their other operands);
    // its start ticket is drawn after them
    // (the plain variant keeps the split-only form, so its code is unchanged)
    const bool late = kFused ? p.mode == 0 &&
                                   (td.op == T_GEMM_BF16 || td.op == T_GEMM_TF32 || td.op == T_GEMM_TF32W) &&
                                   !split_partial(td) && (td.split || np.n_post)
                             : td.split && !split_partial(td) && p.mode == 0;
    const bool both = td.op == T_GEMM_TF32W && td.cfg == 256;  // holds both accumulator buffers
    bool ok = true;
    switch (td.op) {
      case T_GEMM_BF16:
      case T_GEMM_TF32:
      case T_GEMM_TF32W: {
        stage_bias(td, np, ctl);
        uint32_t acc = ctl->tmem_base + accb * kAccCols;
        if (td.op == T_GEMM_TF32W) {
          uint32_t tX;
          tf32w_cols(td, ctl->tmem_base, accb, acc, tX);
          const bool mine = tf32w_worker_loop(td, np, smem, ctl, fs, acc, tX, globaltimer() + p.timeout_ns);
          if (!mine) ws->ok = 0;  // any warp that timed out fails the tile
          worker_sync();
          if (late) {  // split K: the other partials' sums; fused adds: their operands
            if (wt == 0 && ws->ok) {
              if (!wait_late(p, td, epoch)) ws->ok = 0;
              else if (p.trace_on) ws->late_ticket = atomicAdd(&p.ctrl->ticket, 1u);
            }
            worker_sync();
          }
          if (p.trace_on && wt == 0) p.trace[t].stamp[S_ACC] = globaltimer();
        } else if (td.op == T_GEMM_TF32) {
          const bool mine = tf32_worker_loop(np, smem, ctl, fs, acc, globaltimer() + p.timeout_ns);
          if (!mine) ws->ok = 0;  // any warp that timed out fails the tile
          worker_sync();
          if (kFused && late) {
            if (wt == 0 && ws->ok) {
              if (!wait_late(p, td, epoch)) ws->ok = 0;
              else if (p.trace_on) ws->late_ticket = atomicAdd(&p.ctrl->ticket, 1u);
            }
            worker_sync();
          }
          if (p.trace_on && wt == 0) p.trace[t].stamp[S_ACC] = globaltimer();
        } else {
          int kb0, kb1;
          gemm_krange(td, np, kb0, kb1);
          for (int kb = kb0; kb < kb1; ++kb) {  // the MMA issuer consumes these stages
            fs.st.next(kStages);
            if (fs.st.idx == 0) ++fs.pass;
          }
          if (wt == 0) {
            bool w = mbar_wait(&ctl->acc_full[accb], ph[accb], globaltimer() + p.timeout_ns);
            if (w && late) {
              w = wait_late(p, td, epoch);
              if (w && p.trace_on) ws->late_ticket = atomicAdd(&p.ctrl->ticket, 1u);
            }
            ws->ok = w ? 1 : 0;
            if (p.trace_on) p.trace[t].stamp[S_ACC] = globaltimer();
          }
          worker_sync();
          ph[accb] ^= 1u;
        }
        ok = ws->ok != 0;
        if (ok) {
          tc_fence_after();
          if (kFused && np.n_post) gemm_epilogue<true>(p, td, np, ctl, acc, smem + kSmemStages);
          else gemm_epilogue<false>(p, td, np, ctl, acc, smem + kSmemStages);
        }
        tc_fence_before();
        break;
      }
      case T_GEMM_F32:
        if (td.cfg == F32_128x128) tile_gemm_f32<128, 128>(td, np, fsm);
        else if (td.cfg == F32_128x64) tile_gemm_f32<128, 64>(td, np, fsm);
        else tile_gemm_f32<64, 64>(td, np, fsm);
        break;
      case T_ADD: tile_eltwise(td, np, true); break;
      case T_UNARY: tile_eltwise(td, np, false); break;
      case T_SOFTMAX: tile_softmax(td, np); break;
      default: ok = false; break;
    }
    if (p.trace_on && wt == 0) p.trace[t].stamp[S_BODY] = globaltimer();
    fence_proxy_async_global();  // this tile's generic stores, before any later TMA read of them
    worker_sync();
    if (wt == 0) {
      if (p.trace_on) p.trace[t].stamp[S_SYNC] = globaltimer();
      const bool tc = td.op == T_GEMM_BF16 || td.op == T_GEMM_TF32 || td.op == T_GEMM_TF32W;
      if (tc) mbar_arrive(&ctl->acc_empty[accb]);
      if (both) mbar_arrive(&ctl->acc_empty[accb ^ 1u]);
      if (!ok) {
        record_error(p, tc ? E_PIPE_TIMEOUT : E_BAD_TILE, t);
        ctl->fail = 1;
      } else if (!hand_over(t, late ? ws->late_ticket : sl.start_ticket, t_work)) {  // the releaser publishes it
        record_error(p, E_PIPE_TIMEOUT, t);
        ctl->fail = 1;
      }
      mbar_arrive(&ctl->slot_empty[slot.idx]);
    }
    if ((td.op == T_GEMM_BF16 || td.op == T_GEMM_TF32 || td.op == T_GEMM_TF32W) && !both) accb ^= 1u;
    slot.next(kSlots);
  }
}

// kFused: some GEMM of the plan runs fused elementwise kernels in its
// epilogue; the plain variant is compiled without that code, so that its
// register allocation does not pay for it.
template <bool kFused>
__global__ void __launch_bounds__(kThreads, 1) dag_exec_kernel(const __grid_constant__ ExecParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  SmemCtl *ctl = reinterpret_cast<SmemCtl *>(smem + kSmemStages + kWorkerScratch);
  __shared__ WorkerShared ws;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0 && p.trace_on) atomicMin(reinterpret_cast<unsigned long long *>(&p.ctrl->t_enter), globaltimer());

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
      mbar_init(&ctl->split[s], kWorkers / 32);  // one arrival per worker warp
      ctl->issued[s] = 0;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->acc_full[b], 1);
      mbar_init(&ctl->acc_empty[b], 1);
    }
    for (int q = 0; q < kParts; ++q) {
      mbar_init(&ctl->pfull[q], 1);
      mbar_init(&ctl->pempty[q], kWorkers / 32);
    }
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&ctl->slot_full[s], 1);
      mbar_init(&ctl->slot_empty[s], 2);  // MMA warp + worker leader
    }
    for (int s = 0; s < kRelSlots; ++s) {
      mbar_init(&ctl->rel_full[s], 1);
      mbar_init(&ctl->rel_empty[s], 1);
    }
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

  if (warp == 0) {
    if (lane == 0) run_scheduler(p, smem, ctl, p.mode == 0 ? ld_relaxed(&p.ctrl->epoch) : 0u);
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) run_mma(p, smem, ctl);
    __syncwarp();
  } else if (warp == 2) {
    if (lane == 0) run_releaser(p, ctl);
    __syncwarp();
  } else if (warp >= kWorkerBase / 32) {
    run_workers<kFused>(p, smem, ctl, &ws);
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
  if (tid == 0 && p.trace_on) atomicMax(reinterpret_cast<unsigned long long *>(&p.ctrl->t_exit), globaltimer());
}

int exec_smem_bytes() { return kSmemBytes; }

cudaError_t exec_prepare() {
  const cudaError_t e = cudaFuncSetAttribute(dag_exec_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemBytes);
  return e ? e : cudaFuncSetAttribute(dag_exec_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

int max_coresident_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dag_exec_kernel<false>, kThreads, kSmemBytes) != cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_persistent(const ExecParams &p, int grid, cudaStream_t s) {
  ExecParams q = p;
  q.mode = 0;
  q.tile_begin = 0;
  if (q.fused) dag_exec_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(q);
  else dag_exec_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const ExecParams &p, int tile_begin, int n, cudaStream_t s) {
  ExecParams q = p;
  q.mode = 1;
  q.tile_begin = tile_begin;
  if (q.fused) dag_exec_kernel<true><<<n, kThreads, kSmemBytes, s>>>(q);
  else dag_exec_kernel<false><<<n, kThreads, kSmemBytes, s>>>(q);
  return cudaGetLastError();
}

}  // namespace dagx
