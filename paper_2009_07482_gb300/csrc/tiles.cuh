// tiles.cuh -- the tile kinds the executor runs.  GEMM main loops are split
// between the producer and MMA warps; every other piece of work (GEMM
// epilogues, f32 SIMT GEMMs, softmax, elementwise) runs on the 256 worker
// threads, which synchronise among themselves with a named barrier.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "dag_internal.h"
#include "ptx.cuh"

namespace dagx {

// ---------------------------------------------------------------------------
// scalar helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__device__ __forceinline__ uint16_t f32_to_bf16(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float load_elem(const void *base, int dt, int64_t i) {
  return dt == 0 ? __ldcg(static_cast<const float *>(base) + i)
                 : bf16_to_f32(__ldcg(static_cast<const unsigned short *>(base) + i));
}

__device__ __forceinline__ void store_elem(void *base, int dt, int64_t i, float v) {
  if (dt == 0) static_cast<float *>(base)[i] = v;
  else static_cast<uint16_t *>(base)[i] = f32_to_bf16(v);
}

// activation: none, ReLU, GELU (exact erf form)
__device__ __forceinline__ float activate(int act, float x) {
  if (act == 1) return x < 0.f ? 0.f : x;
  if (act == 2) return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
  return x;
}

// barrier among the 256 worker threads only (id 1; id 0 is __syncthreads)
__device__ __forceinline__ void worker_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory"); }

// ---------------------------------------------------------------------------
// Shared control block of one CTA (lives after the pipeline stages)
// ---------------------------------------------------------------------------
struct TileSlot {
  int32_t t;             // queue position, or -1 = no more tiles
  uint32_t start_ticket;
  uint64_t t_claim, t_start;
};

struct RelSlot {
  int32_t t;             // finished queue position, or -1 = no more tiles
  uint32_t start_ticket;
  uint64_t t_work;
};

struct SmemCtl {
  uint64_t full[kStages];      // TMA -> MMA: stage filled
  uint64_t empty[kStages];     // MMA -> TMA: stage consumed
  uint64_t split[kStages];     // workers -> MMA: f32 stage split into tf32 halves
  uint32_t issued[kStages];    // producer: uses of stage s whose loads were issued
  uint64_t pfull[kParts];      // MMA -> workers: f32 K-block partial p in TMEM
  uint64_t pempty[kParts];     // workers (8 warps) -> MMA: partial p added up
  uint64_t acc_full[2];        // MMA -> workers: accumulator b complete
  uint64_t acc_empty[2];       // workers -> MMA: accumulator b drained
  uint64_t slot_full[kSlots];  // scheduler -> MMA, workers: slot published
  uint64_t slot_empty[kSlots]; // MMA + workers -> scheduler: slot consumed
  TileSlot slot[kSlots];
  uint64_t rel_full[kRelSlots];   // workers -> releaser: tile finished
  uint64_t rel_empty[kRelSlots];  // releaser -> workers: slot free
  RelSlot rel[kRelSlots];
  uint32_t tmem_base;
  int32_t fail;                // CTA-local failure flag
  float bias[kMaxBN];          // bias slice of the GEMM tile in the epilogue
};

// A position in a ring of mbarrier-guarded buffers.
struct Ring {
  uint32_t idx, phase;
  __device__ __forceinline__ void next(uint32_t n) {
    if (++idx == n) { idx = 0; phase ^= 1u; }
  }
};

// The splitters skip the stages of bf16 tiles without waiting on them, so
// for an f32 stage a parity wait alone could match an older phase of full[s].
// They first wait until the producer has issued that use of the stage (then
// every earlier phase of full[s] has completed, and the next one cannot
// complete before they split this one), then wait on its parity.
__device__ __forceinline__ void stage_issued(SmemCtl *ctl, uint32_t s) {
  volatile uint32_t *c = &ctl->issued[s];
  *c = *c + 1u;
}
__device__ __forceinline__ bool stage_wait_use(SmemCtl *ctl, uint32_t s, uint32_t use, uint64_t deadline) {
  const volatile uint32_t *c = &ctl->issued[s];
  uint32_t n = 0;
  while ((int32_t)(*c - (use + 1u)) < 0) {
    if ((++n & 255u) == 0 && globaltimer() > deadline) return false;
  }
  return mbar_wait(&ctl->full[s], use & 1u, deadline);
}

// ---------------------------------------------------------------------------
// bf16 GEMM tile, 128 x BN on the tensor cores (tcgen05, f32 accumulator in
// TMEM).  Producer side (scheduler warp, lane 0): all K blocks of the tile
// into the stage ring.  A: box {64 (K), 128 (M)}; B K-major (trans_b):
// box {64 (K), BN}; B MN-major: BN/64 boxes {64 (N), 64 (K)}.  All with the
// 128-byte swizzle.
// ---------------------------------------------------------------------------
// K blocks [kb0, kb1) of a bf16 GEMM tile (a split tile's share of the K loop)
__device__ __forceinline__ void gemm_krange(const TileDesc &t, const NodeParams &np, int &kb0, int &kb1) {
  const int kiters = (np.K + kBK - 1) / kBK;
  if (!t.split) { kb0 = 0; kb1 = kiters; return; }
  const int S = split_count(t), s = split_index(t);
  const int per = (kiters + S - 1) / S;
  kb0 = min(kiters, s * per);
  kb1 = min(kiters, kb0 + per);
}

__device__ __forceinline__ bool gemm_produce(const ExecParams &p, const TileDesc &t, const NodeParams &np,
                                             uint8_t *smem, SmemCtl *ctl, Ring &st, uint64_t deadline) {
  const int BN = t.cfg, M = np.M;
  const int bt = t.r0 / M, m0 = t.r0 - bt * M, n0 = t.c0;
  int kb0, kiters;
  gemm_krange(t, np, kb0, kiters);
  const CUtensorMap *ta = p.tmaps + np.tmap_a;
  const CUtensorMap *tb = p.tmaps + np.tmap_b;
  const int trans_b = np.trans_b;
  const uint32_t bytes = (uint32_t)(kStageA + BN * kBK * 2);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  for (int kb = kb0; kb < kiters; ++kb) {
    if (!mbar_wait(&ctl->empty[st.idx], st.phase ^ 1u, deadline)) return false;
    uint64_t *bar = &ctl->full[st.idx];
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_3d(sA + st.idx * kStageA, ta, bar, kb * kBK, m0, bt);
    uint8_t *dB = sB + st.idx * kStageB;
    if (trans_b) {
      tma_load_3d(dB, tb, bar, kb * kBK, n0, bt);
    } else {
      for (int j = 0; j < BN / 64; ++j) tma_load_3d(dB + j * (64 * kBK * 2), tb, bar, n0 + j * 64, kb * kBK, bt);
    }
    stage_issued(ctl, st.idx);
    st.next(kStages);
  }
  return true;
}

// MMA side (MMA warp, lane 0): accumulate the tile into the TMEM columns at
// tmem_d, then the caller commits to acc_full[b].
__device__ __forceinline__ bool gemm_mma(const TileDesc &t, const NodeParams &np, uint8_t *smem, SmemCtl *ctl,
                                         Ring &st, uint32_t tmem_d, uint64_t deadline) {
  const int BN = t.cfg;
  int kb0, kiters;
  gemm_krange(t, np, kb0, kiters);
  const int trans_b = np.trans_b;
  const uint32_t idesc = idesc_bf16((uint32_t)BN, trans_b ? 0u : 1u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  for (int kb = kb0; kb < kiters; ++kb) {
    if (!mbar_wait(&ctl->full[st.idx], st.phase, deadline)) return false;
    tc_fence_after();
    const uint32_t a0 = smem_u32(sA + st.idx * kStageA);
    const uint32_t b0 = smem_u32(sB + st.idx * kStageB);
    // K-major, 128-byte swizzle: a K step of 16 bf16 is 32 bytes along the row.
    // B MN-major: 16 K rows of 128 bytes = 2048 bytes per step, 64-column
    // chunks 8 KiB apart (leading offset), 8-row groups 1 KiB apart (stride offset).
    // The descriptors are built once per stage and stepped in their start
    // address field (16-byte units; shared addresses stay below 2^18 bytes,
    // so the 14-bit field never carries).
    const uint64_t ad0 = smem_desc_sw128(a0, 16, 1024);
    const uint64_t bd0 = trans_b ? smem_desc_sw128(b0, 16, 1024) : smem_desc_sw128(b0, 64 * kBK * 2, 1024);
    const uint64_t bstep = trans_b ? 32 >> 4 : 2048 >> 4;
#pragma unroll
    for (int kk = 0; kk < kBK / 16; ++kk)
      mma_bf16(tmem_d, ad0 + (uint64_t)(kk * (32 >> 4)), bd0 + (uint64_t)kk * bstep, idesc,
               (kb != kb0 || kk != 0) ? 1u : 0u);
    mma_commit(&ctl->empty[st.idx]);
    st.next(kStages);
  }
  return true;
}

// ---------------------------------------------------------------------------
// f32 GEMM tile, 128 x 64, on the tensor cores with the 3 x TF32 split: each
// operand x = hi + lo, and A.B ~= Ahi.Bhi + Ahi.Blo + Alo.Bhi accumulated in
// f32 in TMEM.  The tensor cores read a 32-bit operand as tf32 by dropping
// its low 13 bits, so hi is x itself as stored (read as trunc(x)) and
// lo = x - trunc(x), exact in f32 and read with its top 11 significant bits:
// the dropped Alo.Blo and the truncation of lo are ~2^-21 relative per
// product.  One stage holds one K block of 32 (128-byte rows):
//   A area (16 KiB): A, K-major, as loaded (Ahi)
//   B area: [0, 8K) B, K-major (an MN-major B is transposed in place; Bhi),
//           [8K, 16K) Blo, [16K, 32K) Alo
// The producer loads raw f32 with TMA; each worker warp splits its share of
// the stage (an MN-major box is transposed by one warp) and arrives on
// split[s] (8 arrivals); the MMA issuer then runs three tf32 MMAs per K step
// of 8.
// ---------------------------------------------------------------------------
constexpr int kTf32BBytes = kTf32BN * kBKF * 4;  // 8 KiB
constexpr int kTf32Blo = kTf32BBytes;            // offsets in the B area
constexpr int kTf32Alo = 2 * kTf32BBytes;
static_assert(kTf32Alo + kStageA <= kStageB, "tf32 stage layout");

__device__ __forceinline__ bool tf32_produce(const ExecParams &p, const TileDesc &t, const NodeParams &np,
                                             uint8_t *smem, SmemCtl *ctl, Ring &st, uint64_t deadline) {
  const int M = np.M;
  const int bt = t.r0 / M, m0 = t.r0 - bt * M, n0 = t.c0;
  const int kiters = (np.K + kBKF - 1) / kBKF;
  const CUtensorMap *ta = p.tmaps + np.tmap_a;
  const CUtensorMap *tb = p.tmaps + np.tmap_b;
  const int trans_b = np.trans_b;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  for (int kb = 0; kb < kiters; ++kb) {
    if (!mbar_wait(&ctl->empty[st.idx], st.phase ^ 1u, deadline)) return false;
    uint64_t *bar = &ctl->full[st.idx];
    mbar_arrive_expect_tx(bar, (uint32_t)(kStageA + kTf32BBytes));
    tma_load_3d(sA + st.idx * kStageA, ta, bar, kb * kBKF, m0, bt);
    uint8_t *dB = sB + st.idx * kStageB;
    if (trans_b) {
      tma_load_3d(dB, tb, bar, kb * kBKF, n0, bt);  // box {32 (K), 64 (N)}
    } else {
      // box {32 (N), 32 (K)}: 4 KiB per 32 columns
      for (int j = 0; j < kTf32BN / 32; ++j) tma_load_3d(dB + j * 4096, tb, bar, n0 + j * 32, kb * kBKF, bt);
    }
    stage_issued(ctl, st.idx);
    st.next(kStages);
  }
  return true;
}

// lo of an f32 bit pattern: x minus its truncation to tf32 (exact)
__device__ __forceinline__ uint32_t tf32_lo(uint32_t u) {
  return __float_as_uint(__uint_as_float(u) - __uint_as_float(u & 0xFFFFE000u));
}
__device__ __forceinline__ uint4 tf32_lo4(uint4 x) {
  return make_uint4(tf32_lo(x.x), tf32_lo(x.y), tf32_lo(x.z), tf32_lo(x.w));
}

// One worker warp's share of splitting a filled stage (wid = worker warp
// 0..7).  A and a K-major B: lo of each 16-byte chunk at the same layout
// offset.  An MN-major B: box j (columns 32j..32j+31 as 32 K rows of 128
// bytes, chunk c of row k at (c ^ (k % 8))) is transposed in place by worker
// warp j alone -- the 4 (K) x 4 (N) blocks of one box only overwrite one
// another -- into K-major rows 32j..32j+31 (row n, chunk k/4 at
// ((k/4) ^ (n % 8))), with its lo alongside.
__device__ __forceinline__ void tf32_split_warp(uint8_t *a, uint8_t *b, int trans_b, int wid, int lane) {
  constexpr int kAw = kStageA / 16 / 8;        // 128 chunks of A per warp
  uint4 *A4 = reinterpret_cast<uint4 *>(a) + wid * kAw;
  uint4 *Alo = reinterpret_cast<uint4 *>(b + kTf32Alo) + wid * kAw;
  uint4 xa[kAw / 32];
#pragma unroll
  for (int j = 0; j < kAw / 32; ++j) xa[j] = A4[lane + 32 * j];
#pragma unroll
  for (int j = 0; j < kAw / 32; ++j) Alo[lane + 32 * j] = tf32_lo4(xa[j]);
  uint4 *B4 = reinterpret_cast<uint4 *>(b);
  uint4 *Blo = reinterpret_cast<uint4 *>(b + kTf32Blo);
  if (trans_b) {
    constexpr int kBw = kTf32BBytes / 16 / 8;  // 64 chunks of B per warp
#pragma unroll
    for (int j = 0; j < kBw / 32; ++j) {
      const int i = wid * kBw + lane + 32 * j;
      Blo[i] = tf32_lo4(B4[i]);
    }
    return;
  }
  if (wid >= kTf32BN / 32) return;
  // box `wid`: 64 blocks (8 K quads x 8 N quads), two per lane
  uint4 v[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int t = lane + 32 * u, kq = t & 7, c = t >> 3;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = 4 * kq + r;
      v[u][r] = B4[(wid * 4096 + k * 128 + ((c ^ (k & 7)) << 4)) >> 4];
    }
  }
  __syncwarp();  // the whole box is read before any of it is overwritten
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int t = lane + 32 * u, kq = t & 7, c = t >> 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = 32 * wid + 4 * c + q;
      uint4 col;
      col.x = q == 0 ? v[u][0].x : q == 1 ? v[u][0].y : q == 2 ? v[u][0].z : v[u][0].w;
      col.y = q == 0 ? v[u][1].x : q == 1 ? v[u][1].y : q == 2 ? v[u][1].z : v[u][1].w;
      col.z = q == 0 ? v[u][2].x : q == 1 ? v[u][2].y : q == 2 ? v[u][2].z : v[u][2].w;
      col.w = q == 0 ? v[u][3].x : q == 1 ? v[u][3].y : q == 2 ? v[u][3].z : v[u][3].w;
      const int o = (n * 128 + ((kq ^ (n & 7)) << 4)) >> 4;
      B4[o] = col;
      Blo[o] = tf32_lo4(col);
    }
  }
}

// MMA side of an f32 tile: three tf32 MMAs per K step of 8 (32 bytes).  The
// tensor cores' f32 accumulation is not round-to-nearest, and its error
// grows with the number of MMAs summed into one accumulator; so each K block
// goes into a fresh 64-column partial (a ring of kParts in the tile's TMEM
// accumulator), and the workers add the partials in f32 registers.  Partial
// q of the CTA's stream of f32 K blocks is slot q % kParts, parity
// (q / kParts) & 1.
__device__ __forceinline__ bool tf32_mma(const NodeParams &np, uint8_t *smem, SmemCtl *ctl, Ring &st,
                                         uint32_t &split_par, uint32_t &pq, uint32_t tmem_acc, uint64_t deadline) {
  const int kiters = (np.K + kBKF - 1) / kBKF;
  constexpr uint32_t idesc = idesc_tf32((uint32_t)kTf32BN);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  for (int kb = 0; kb < kiters; ++kb) {
    if (!mbar_wait(&ctl->split[st.idx], (split_par >> st.idx) & 1u, deadline)) return false;
    split_par ^= 1u << st.idx;
    const uint32_t ps = pq % kParts;
    if (!mbar_wait(&ctl->pempty[ps], ((pq / kParts) & 1u) ^ 1u, deadline)) return false;
    const uint32_t tmem_d = tmem_acc + ps * kTf32BN;
    tc_fence_after();
    const uint32_t ahi = smem_u32(sA + st.idx * kStageA);
    const uint32_t bhi = smem_u32(sB + st.idx * kStageB);
    const uint32_t blo = bhi + kTf32Blo, alo = bhi + kTf32Alo;
    const uint64_t dah0 = smem_desc_sw128(ahi, 16, 1024), dal0 = smem_desc_sw128(alo, 16, 1024);
    const uint64_t dbh0 = smem_desc_sw128(bhi, 16, 1024), dbl0 = smem_desc_sw128(blo, 16, 1024);
#pragma unroll
    for (int kk = 0; kk < kBKF / 8; ++kk) {
      // a K step of 8 is 32 bytes: 2 in the descriptors' 16-byte address field
      const uint64_t o = (uint64_t)(kk * 2);
      const uint64_t dah = dah0 + o, dal = dal0 + o, dbh = dbh0 + o, dbl = dbl0 + o;
      // the small products first, then the large one
      mma_tf32(tmem_d, dal, dbh, idesc, kk != 0 ? 1u : 0u);
      mma_tf32(tmem_d, dah, dbl, idesc, 1u);
      mma_tf32(tmem_d, dah, dbh, idesc, 1u);
    }
    mma_commit(&ctl->empty[st.idx]);
    mma_commit(&ctl->pfull[ps]);
    ++pq;
    st.next(kStages);
  }
  return true;
}

// Worker side of an f32 tile: each worker warp, on its own, for each K
// block splits its share of the stage (then arrives on split[s]; the MMA
// issuer needs all 8) and adds up the partial of the K block kLag earlier
// (its TMEM lane quadrant, columns half*32 .. +32 of the 64); at the end the
// sum goes to columns 0..63 of the accumulator for the epilogue.  Waits are
// taken by lane 0 and shared within the warp.  false if a wait ran out.
constexpr int kLag = 2;
static_assert(kLag < kParts, "the MMA issuer runs up to kParts partials ahead");

struct Tf32State {
  Ring st;          // position in the stage ring
  uint32_t pass;    // completed passes over the stage ring
  uint32_t pq;      // f32 K-block partials added up
};

__device__ __forceinline__ bool tf32_worker_loop(const NodeParams &np, uint8_t *smem, SmemCtl *ctl, Tf32State &fs,
                                                 uint32_t tmem_acc, uint64_t deadline) {
  const int wid = (threadIdx.x - kWorkerBase) >> 5, lane = threadIdx.x & 31;
  const int half = wid >> 2;
  const uint32_t lanes = (uint32_t)((threadIdx.x >> 5 & 3) * 32) << 16;
  const int kiters = (np.K + kBKF - 1) / kBKF;
  const int trans_b = np.trans_b;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  float sum[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) sum[i] = 0.0f;
  bool ok = true;
  for (int kb = 0; kb < kiters + kLag; ++kb) {
    if (kb < kiters) {
      if (ok) {
        int w = 0;
        if (lane == 0) w = stage_wait_use(ctl, fs.st.idx, fs.pass, deadline) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      }
      if (ok) {
        tf32_split_warp(sA + fs.st.idx * kStageA, sB + fs.st.idx * kStageB, trans_b, wid, lane);
        fence_proxy_async_shared();  // generic writes -> visible to the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->split[fs.st.idx]);
      }
      fs.st.next(kStages);
      if (fs.st.idx == 0) ++fs.pass;
    }
    if (kb >= kLag) {
      const uint32_t ps = fs.pq % kParts;
      if (ok) {
        int w = 0;
        if (lane == 0) w = mbar_wait(&ctl->pfull[ps], (fs.pq / kParts) & 1u, deadline) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      }
      if (ok) {
        tc_fence_after();
        float v[32];
        tmem_ld32(tmem_acc + lanes + ps * kTf32BN + half * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) sum[i] += v[i];
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->pempty[ps]);
      ++fs.pq;
    }
  }
  if (ok) {
    tmem_st32(tmem_acc + lanes + half * 32, sum);
    tc_fence_before();
  }
  return ok;
}

// ---------------------------------------------------------------------------
// f32 GEMM tile on the tensor cores, wide form: 128 x BN (BN = 128 or 256),
// B K-major, the same 3 x TF32 split.  A stage holds one K block of 16
// (64-byte rows, 64-byte swizzle):
//   A area: Ahi [0, 8K), Alo [8K, 16K)
//   B area: Bhi [0, BN * 64), Blo [BN * 64, 2 * BN * 64)
// so the split is elementwise at equal offsets (no layout work), and each
// stage is 2 K steps x 3 MMAs of 128 x BN x 8.  Per K block the stage's
// shared-memory traffic (TMA write, split read and write, MMA operand reads)
// is 6 x (8K + BN * 64) bytes for 2 x 128 x BN x 16 x 3 tf32 flops: four times
// the work per byte of the 128 x 64 form at BN = 256.
// The tensor cores' f32 accumulation is not round-to-nearest and its error
// grows with the number of MMAs summed into one accumulator, so the tile's K
// loop is cut into partials of kWideP stages (128 of K): partial 0 goes
// straight into the sum S, every later one into X, which the workers add
// into S (f32, round to nearest) before the MMA issuer may start the next
// partial there.  S and X: BN = 128 -> the tile's accumulator buffer (S its
// columns 0..127, X 128..255); BN = 256 -> S the tile's buffer, X the other
// one (such a tile holds both accumulator buffers).
// ---------------------------------------------------------------------------
constexpr int kWideLag = kStages - 1;  // stages the splitters run ahead of a partial's end
static_assert(kBM * kBKW * 4 * 2 <= kStageA && 256 * kBKW * 4 * 2 <= kStageB, "wide tf32 stage layout");

// K blocks [kb0, kb1) of a wide f32 tile (a split tile's share of the K loop)
__device__ __forceinline__ void tf32w_krange(const TileDesc &t, const NodeParams &np, int &kb0, int &kb1) {
  const int kiters = (np.K + kBKW - 1) / kBKW;
  if (!t.split) { kb0 = 0; kb1 = kiters; return; }
  const int S = split_count(t), s = split_index(t);
  const int per = (kiters + S - 1) / S;
  kb0 = min(kiters, s * per);
  kb1 = min(kiters, kb0 + per);
}

// two TMEM column ranges of a wide tile: the sum S and the partial X
__device__ __forceinline__ void tf32w_cols(const TileDesc &t, uint32_t tmem_base, uint32_t accb, uint32_t &tS,
                                           uint32_t &tX) {
  tS = tmem_base + accb * kAccCols;
  tX = t.cfg == 256 ? tmem_base + (accb ^ 1u) * kAccCols : tS + 128u;
}

__device__ __forceinline__ bool tf32w_produce(const ExecParams &p, const TileDesc &t, const NodeParams &np,
                                              uint8_t *smem, SmemCtl *ctl, Ring &st, uint64_t deadline) {
  const int BN = t.cfg, M = np.M;
  const int bt = t.r0 / M, m0 = t.r0 - bt * M, n0 = t.c0;
  int kb0, kb1;
  tf32w_krange(t, np, kb0, kb1);
  const CUtensorMap *ta = p.tmaps + np.tmap_a;
  const CUtensorMap *tb = p.tmaps + np.tmap_b;
  const uint32_t bytes = (uint32_t)((kBM + BN) * kBKW * 4);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  for (int kb = kb0; kb < kb1; ++kb) {
    if (!mbar_wait(&ctl->empty[st.idx], st.phase ^ 1u, deadline)) return false;
    uint64_t *bar = &ctl->full[st.idx];
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_3d(sA + st.idx * kStageA, ta, bar, kb * kBKW, m0, bt);   // box {16 (K), 128 (M)}
    tma_load_3d(sB + st.idx * kStageB, tb, bar, kb * kBKW, n0, bt);   // box {16 (K), BN (N)}
    stage_issued(ctl, st.idx);
    st.next(kStages);
  }
  return true;
}

// MMA side of a wide f32 tile.  Partial q of the CTA's stream of f32
// partials (shared with the 128 x 64 form) signals pfull[q % kParts]; the
// workers arrive on pempty[q % kParts] once it is added up.
__device__ __forceinline__ bool tf32w_mma(const TileDesc &t, const NodeParams &np, uint8_t *smem, SmemCtl *ctl,
                                          Ring &st, uint32_t &split_par, uint32_t &pq, uint32_t tS, uint32_t tX,
                                          uint64_t deadline) {
  const int BN = t.cfg;
  int kb0, kb1;
  tf32w_krange(t, np, kb0, kb1);
  const uint32_t idesc = idesc_tf32((uint32_t)BN);
  const uint32_t blo_off = (uint32_t)BN * kBKW * 4;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  uint32_t dst = tS;
  for (int kb = kb0; kb < kb1; ++kb) {
    const int j = kb - kb0;
    if (j % kWideP == 0) {  // a new partial
      const int part = j / kWideP;
      const uint32_t ps = pq % kParts;
      // its barrier slot is free once partial pq - kParts was added up
      if (!mbar_wait(&ctl->pempty[ps], ((pq / kParts) & 1u) ^ 1u, deadline)) return false;
      if (part >= 2) {  // X holds partial pq - 1 until the workers have added it into S
        const uint32_t q1 = pq - 1u;
        if (!mbar_wait(&ctl->pempty[q1 % kParts], (q1 / kParts) & 1u, deadline)) return false;
      }
      dst = part == 0 ? tS : tX;
    }
    if (!mbar_wait(&ctl->split[st.idx], (split_par >> st.idx) & 1u, deadline)) return false;
    split_par ^= 1u << st.idx;
    tc_fence_after();
    const uint32_t ahi = smem_u32(sA + st.idx * kStageA), alo = ahi + kBM * kBKW * 4;
    const uint32_t bhi = smem_u32(sB + st.idx * kStageB), blo = bhi + blo_off;
    const uint64_t dah0 = smem_desc_sw64(ahi), dal0 = smem_desc_sw64(alo);
    const uint64_t dbh0 = smem_desc_sw64(bhi), dbl0 = smem_desc_sw64(blo);
#pragma unroll
    for (int kk = 0; kk < kBKW / 8; ++kk) {
      // a K step of 8 is 32 bytes: 2 in the descriptors' 16-byte address field
      const uint64_t o = (uint64_t)(kk * 2);
      const uint64_t dah = dah0 + o, dal = dal0 + o, dbh = dbh0 + o, dbl = dbl0 + o;
      // the small products first, then the large one
      mma_tf32(dst, dal, dbh, idesc, (j % kWideP != 0 || kk != 0) ? 1u : 0u);
      mma_tf32(dst, dah, dbl, idesc, 1u);
      mma_tf32(dst, dah, dbh, idesc, 1u);
    }
    mma_commit(&ctl->empty[st.idx]);
    if ((j + 1) % kWideP == 0 || kb + 1 == kb1) {
      mma_commit(&ctl->pfull[pq % kParts]);
      ++pq;
    }
    st.next(kStages);
  }
  return true;
}

// Worker side of a wide f32 tile: each worker warp splits its eighth of every
// stage (Ahi -> Alo, Bhi -> Blo at equal offsets) and arrives on split[s];
// kWideLag stages after a partial's last stage it waits for the partial and,
// from the second on, adds X into S over its lane quadrant and half of the
// columns.  false if a wait ran out.
__device__ __forceinline__ bool tf32w_worker_loop(const TileDesc &t, const NodeParams &np, uint8_t *smem,
                                                  SmemCtl *ctl, Tf32State &fs, uint32_t tS, uint32_t tX,
                                                  uint64_t deadline) {
  const int wid = (threadIdx.x - kWorkerBase) >> 5, lane = threadIdx.x & 31;
  const int BN = t.cfg;
  const int half = wid >> 2;
  const uint32_t lanes = (uint32_t)((threadIdx.x >> 5 & 3) * 32) << 16;
  int kb0, kb1;
  tf32w_krange(t, np, kb0, kb1);
  const int n = kb1 - kb0;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  const int a_chunks = kBM * kBKW * 4 / 16 / 8;   // 64 16-byte chunks of Ahi per warp
  const int b_chunks = BN * kBKW * 4 / 16 / 8;    // 64 or 128 of Bhi
  bool ok = true;
  int part = 0;
  for (int j = 0; j < n + kWideLag; ++j) {
    if (j < n) {
      if (ok) {
        int w = 0;
        if (lane == 0) w = stage_wait_use(ctl, fs.st.idx, fs.pass, deadline) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      }
      if (ok) {
        uint4 *A4 = reinterpret_cast<uint4 *>(sA + fs.st.idx * kStageA) + wid * a_chunks;
        uint4 *B4 = reinterpret_cast<uint4 *>(sB + fs.st.idx * kStageB) + wid * b_chunks;
        uint4 xa[2], xb[4];
#pragma unroll
        for (int u = 0; u < 2; ++u) xa[u] = A4[lane + 32 * u];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < b_chunks / 32) xb[u] = B4[lane + 32 * u];
        uint4 *Alo = A4 + kBM * kBKW * 4 / 16;        // Alo sits 8 KiB after Ahi
        uint4 *Blo = B4 + BN * kBKW * 4 / 16;         // Blo sits BN * 64 bytes after Bhi
#pragma unroll
        for (int u = 0; u < 2; ++u) Alo[lane + 32 * u] = tf32_lo4(xa[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < b_chunks / 32) Blo[lane + 32 * u] = tf32_lo4(xb[u]);
        fence_proxy_async_shared();  // generic writes -> visible to the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->split[fs.st.idx]);
      }
      fs.st.next(kStages);
      if (fs.st.idx == 0) ++fs.pass;
    }
    // the next partial to add up ends at stage e_next; it is added up as soon
    // as the MMA issuer has finished it (checked after every split), and at
    // the latest kWideLag stages after its end
    const int e_next = min(n, (part + 1) * kWideP) - 1;
    bool due = part * kWideP < n && j >= e_next + kWideLag;
    if (!due && part * kWideP < n && j >= e_next && ok) {
      int r = 0;
      if (lane == 0) r = mbar_try_wait(&ctl->pfull[fs.pq % kParts], (fs.pq / kParts) & 1u) ? 1 : 0;
      due = __shfl_sync(0xffffffffu, r, 0) != 0;
    }
    if (due) {
      const uint32_t ps = fs.pq % kParts;
      if (ok) {
        int w = 0;
        if (lane == 0) w = mbar_wait(&ctl->pfull[ps], (fs.pq / kParts) & 1u, deadline) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      }
      if (ok && part > 0) {
        tc_fence_after();
        for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
          float x[32], y[32];
          tmem_ld32x2(tX + lanes + (uint32_t)c, x, tS + lanes + (uint32_t)c, y);
#pragma unroll
          for (int i = 0; i < 32; ++i) y[i] += x[i];
          tmem_st32(tS + lanes + (uint32_t)c, y);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->pempty[ps]);
      ++fs.pq;
      ++part;
    }
  }
  if (ok) tc_fence_after();
  return ok;
}

// Elementwise kernels fused into a GEMM epilogue, on 32 consecutive values of
// one output row (row grow, columns col..col+31): each step first rounds the
// value to the dtype of the buffer the previous kernel would have stored,
// then applies act(v + X) (an add; X read through L2, written by other SMs in
// this launch) or act(v) -- the arithmetic of the elementwise tile itself.
__device__ __forceinline__ float round_dt(int dt, float x) { return dt == 1 ? bf16_to_f32(f32_to_bf16(x)) : x; }

__device__ __forceinline__ void load_row32(const PostOp &q, int64_t grow, bool row_ok, int col, int N,
                                           float (&x)[32]) {
  if (row_ok && q.xvec && col + 32 <= N) {
    if (q.x_dt == 1) {
      const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const uint16_t *>(q.X) + grow * q.ldx + col);
      uint4 w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] = __ldcg(src + k);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t ww[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          x[8 * k + 2 * i] = __uint_as_float(ww[i] << 16);
          x[8 * k + 2 * i + 1] = __uint_as_float(ww[i] & 0xFFFF0000u);
        }
      }
    } else {
      const float4 *src = reinterpret_cast<const float4 *>(static_cast<const float *>(q.X) + grow * q.ldx + col);
      float4 w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = __ldcg(src + k);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        x[4 * k] = w[k].x; x[4 * k + 1] = w[k].y; x[4 * k + 2] = w[k].z; x[4 * k + 3] = w[k].w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      x[i] = (row_ok && col + i < N) ? load_elem(q.X, q.x_dt, grow * q.ldx + col + i) : 0.f;
  }
}

__device__ __forceinline__ void post_ops(const NodeParams &np, float (&v)[32], int64_t grow, bool row_ok, int col,
                                         int N) {
  int dt = np.o_dt;
  for (int j = 0; j < np.n_post; ++j) {
    const PostOp &q = np.post[j];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = round_dt(dt, v[i]);
    if (q.X) {
      float x[32];
      load_row32(q, grow, row_ok, col, N, x);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = activate(q.act, v[i] + x[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = activate(q.act, v[i]);
    }
    dt = q.out_dt;
  }
}

// Epilogue (workers): TMEM accumulator -> scale, bias, activation, cast ->
// global.  Worker warp w reads TMEM lanes 32*(w%4).. and the columns of half
// (w-4)/4 of the tile; each thread owns one output row.  With an output
// tensor map, the two warps of a quadrant take alternate 128-byte column
// chunks of their 32 rows and write each through a
// 128-byte-swizzled shared staging block (one TMA store per chunk, clipped at
// the buffer's edges); otherwise it stores directly.  Fused elementwise
// kernels (npg.n_post) run on the values before the cast; C is then the last
// one's output (kPost; the executor is built with and without that code).
template <bool kPost>
__device__ __forceinline__ void gemm_epilogue(const ExecParams &p, const TileDesc &t, const NodeParams &npg,
                                              const SmemCtl *ctl, uint32_t tmem_acc, uint8_t *scratch) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int BN = t.cfg;
  const int M = npg.M, N = npg.N;
  const int act = npg.act, c_dt = npg.c_dt, vec = npg.vec, tmap_c = npg.tmap_c;
  const float scale = npg.scale;
  void *const Cp = npg.C;
  const int64_t ldc = npg.ldc;
  const int bt = t.r0 / M, m0 = t.r0 - bt * M, n0 = t.c0;
  const int quad = warp & 3;
  const int wid = (threadIdx.x - kWorkerBase) >> 5;
  const int half = wid >> 2;
  const int cw = BN / 2;
  const uint32_t trow = tmem_acc + ((uint32_t)(quad * 32) << 16);
  // split K: this tile's scratch blocks (128 x BN f32 each, row-major)
  const int S = split_count(t), sidx = split_index(t);
  const float *parts = nullptr;
  if (S) {
    const int mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN;
    const int64_t local = ((int64_t)bt * mt + m0 / kBM) * nt + n0 / BN;
    parts = npg.scratch + local * (S - 1) * (int64_t)(kBM * BN);
  }
  const int trow_local = quad * 32 + lane;  // this thread's row in the tile
  if (S && sidx < S - 1) {
    // a partial: raw f32 sums to its scratch block
    float *dst = const_cast<float *>(parts) + (int64_t)sidx * (kBM * BN) + (int64_t)trow_local * BN;
    for (int c = half * cw; c < (half + 1) * cw; c += 32) {
      float v[32];
      tmem_ld32(trow + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4 *>(dst + c + 4 * j) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
    return;
  }
  // the finishing partial adds the others' sums, in partial order, before its own
  auto add_parts = [&](float (&v)[32], int c) {
    if (!S) return;
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    for (int q = 0; q < S - 1; ++q) {
      const float4 *src = reinterpret_cast<const float4 *>(parts + (int64_t)q * (kBM * BN) + (int64_t)trow_local * BN + c);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 x = __ldcg(src + j);
        acc[4 * j] += x.x; acc[4 * j + 1] += x.y; acc[4 * j + 2] += x.z; acc[4 * j + 3] += x.w;
      }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = acc[i] + v[i];
  };
  if (tmap_c >= 0) {
    const CUtensorMap *mc = p.tmaps + tmap_c;
    uint8_t *stg = scratch + wid * (kEpiRows * 128);          // 4 KiB, 1024-aligned
    uint8_t *myrow = stg + lane * 128;
    const int step = c_dt == 1 ? 64 : 32;                       // columns per 128-byte row chunk
    // the two warps of a TMEM lane quadrant take alternate whole chunks
    // (a 64-column tile has a single bf16 chunk: the second warp idles)
    for (int c = half * step; c < BN; c += 2 * step) {
      for (int sub = 0; sub < step; sub += 32) {
        float v[32];
        tmem_ld32(trow + (uint32_t)(c + sub), v);
        add_parts(v, c + sub);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = activate(act, fmaf(v[i], scale, ctl->bias[c + sub + i]));
        if constexpr (kPost) {
          const int row = m0 + trow_local;
          post_ops(npg, v, (int64_t)bt * M + row, row < M, n0 + c + sub, N);
        }
        if (sub == 0) {
          // only now wait for the previous chunk's store to leave the staging
          // block: its read overlapped this chunk's TMEM load and arithmetic
          if (lane == 0) bulk_wait_read();
          __syncwarp();
        }
        // 16-byte chunk j of this row goes to position j ^ (row % 8) (128-byte swizzle)
        if (c_dt == 1) {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = (sub >> 3) + jj;  // sub = 0 -> chunks 0..3, sub = 32 -> chunks 4..7
            uint4 q;
            q.x = (uint32_t)f32_to_bf16(v[8 * jj + 0]) | ((uint32_t)f32_to_bf16(v[8 * jj + 1]) << 16);
            q.y = (uint32_t)f32_to_bf16(v[8 * jj + 2]) | ((uint32_t)f32_to_bf16(v[8 * jj + 3]) << 16);
            q.z = (uint32_t)f32_to_bf16(v[8 * jj + 4]) | ((uint32_t)f32_to_bf16(v[8 * jj + 5]) << 16);
            q.w = (uint32_t)f32_to_bf16(v[8 * jj + 6]) | ((uint32_t)f32_to_bf16(v[8 * jj + 7]) << 16);
            *reinterpret_cast<uint4 *>(myrow + ((j ^ (lane & 7)) << 4)) = q;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint4 q = make_uint4(__float_as_uint(v[4 * j]), __float_as_uint(v[4 * j + 1]),
                                       __float_as_uint(v[4 * j + 2]), __float_as_uint(v[4 * j + 3]));
            *reinterpret_cast<uint4 *>(myrow + ((j ^ (lane & 7)) << 4)) = q;
          }
        }
      }
      fence_proxy_async_shared();       // generic shared writes -> visible to the TMA engine
      __syncwarp();
      if (lane == 0 && n0 + c < N) {
        tma_store_3d(mc, stg, n0 + c, m0 + quad * 32, bt);
        bulk_commit();
      }
    }
    if (lane == 0) {
      bulk_wait_all();                  // stores complete before the tile is released
      fence_proxy_async_global();
    }
    __syncwarp();
    return;
  }
  const int row = m0 + quad * 32 + lane;
  const bool row_ok = row < M;
  const int64_t grow = (int64_t)bt * M + row;
  for (int c = half * cw; c < (half + 1) * cw; c += 32) {
    float v[32];
    tmem_ld32(trow + (uint32_t)c, v);
    add_parts(v, c);
    const int col = n0 + c;
    if (col >= N || !row_ok) continue;
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = activate(act, fmaf(v[i], scale, ctl->bias[c + i]));
    if constexpr (kPost) post_ops(npg, v, grow, true, col, N);
    if (vec && col + 32 <= N) {
      if (c_dt == 1) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(Cp) + grow * ldc + col);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t w[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            w[i] = (uint32_t)f32_to_bf16(v[8 * q + 2 * i]) | ((uint32_t)f32_to_bf16(v[8 * q + 2 * i + 1]) << 16);
          dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else {
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(Cp) + grow * ldc + col);
#pragma unroll
        for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    } else {
      for (int i = 0; i < 32 && col + i < N; ++i) store_elem(Cp, c_dt, grow * ldc + col + i, v[i]);
    }
  }
}

// stage the bias slice [n0, n0+BN) of a GEMM tile in shared memory (workers)
__device__ __forceinline__ void stage_bias(const TileDesc &t, const NodeParams &np, SmemCtl *ctl) {
  const int wt = threadIdx.x - kWorkerBase;
  const void *const bias = np.bias;
  const int N = np.N, bdt = np.bias_dt;
  for (int i = wt; i < t.cfg; i += kWorkers) {
    const int n = t.c0 + i;
    ctl->bias[i] = (bias && n < N) ? load_elem(bias, bdt, n) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// f32 GEMM tile, exact f32 (SIMT FFMA), BM x BN on the 256 workers as 16 x 16
// threads, double-buffered shared memory with register prefetch of the next
// K slice (BK = 16, or 8 for 128 x 128 to fit the worker scratch).  Each
// thread owns a (BM/16) x (BN/16) block split into 4-wide groups 64 apart, so
// shared reads are conflict-free.
// ---------------------------------------------------------------------------
template <int BM, int BN>
__host__ __device__ constexpr int f32_bk() { return (BM == 128 && BN == 128) ? 8 : 16; }
template <int BM, int BN>
__host__ __device__ constexpr int f32_smem() { return 2 * f32_bk<BM, BN>() * ((BM + 4) + (BN + 4)) * 4; }
static_assert(f32_smem<128, 128>() <= kWorkerScratch && f32_smem<128, 64>() <= kWorkerScratch &&
                  f32_smem<64, 64>() <= kWorkerScratch,
              "f32 tile scratch");

template <int BM, int BN>
__device__ __forceinline__ void tile_gemm_f32(const TileDesc &t, const NodeParams &npg, float *smem) {
  constexpr int BK = f32_bk<BM, BN>();
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LDA_S = BM + 4, LDB_S = BN + 4;
  float *As = smem;                      // [2][BK][LDA_S]
  float *Bs = smem + 2 * BK * LDA_S;     // [2][BK][LDB_S]
  const int tid = threadIdx.x - kWorkerBase;
  const int ty = tid >> 4, tx = tid & 15;
  const int M = npg.M, N = npg.N, K = npg.K;
  const int trans_b = npg.trans_b, act = npg.act, c_dt = npg.c_dt, bias_dt = npg.bias_dt, vec = npg.vec;
  const int64_t lda = npg.lda, ldb = npg.ldb, ldc = npg.ldc;
  const float scale = npg.scale;
  const void *const bias = npg.bias;
  void *const Cp = npg.C;
  const int bt = t.r0 / M;
  const int m0 = t.r0 - bt * M, n0 = t.c0;
  const float *A = static_cast<const float *>(npg.A) + (int64_t)bt * M * lda;
  const float *B = static_cast<const float *>(npg.B) + (int64_t)bt * (trans_b ? (int64_t)N * ldb : (int64_t)K * ldb);

  // loader mapping: each thread moves EA (EB) consecutive elements of one row
  constexpr int EA = BM * BK / kWorkers;      // 4 or 8
  constexpr int EB = BN * BK / kWorkers;      // 4 or 8
  float ra[EA], rb[EB];

  auto load_run = [&](float *dst, const float *src, int n, auto en_tag) {
    constexpr int EN = decltype(en_tag)::value;  // 4 or 8: whole float4s
    if (vec && n >= EN) {
#pragma unroll
      for (int q = 0; q < EN / 4; ++q) {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(src) + q);
        dst[4 * q] = v.x; dst[4 * q + 1] = v.y; dst[4 * q + 2] = v.z; dst[4 * q + 3] = v.w;
      }
      return;
    }
#pragma unroll
    for (int i = 0; i < EN; ++i) dst[i] = i < n ? __ldcg(src + i) : 0.f;
  };
  using TagA = std::integral_constant<int, EA>;
  using TagB = std::integral_constant<int, EB>;

  auto load_a = [&](int k0) {
    const int r = tid / (BK / EA), kq = (tid % (BK / EA)) * EA;
    const int gm = m0 + r, gk = k0 + kq;
    if (gm < M) load_run(ra, A + (int64_t)gm * lda + gk, K - gk, TagA{});
    else {
#pragma unroll
      for (int i = 0; i < EA; ++i) ra[i] = 0.f;
    }
  };
  auto store_a = [&](int buf) {
    const int r = tid / (BK / EA), kq = (tid % (BK / EA)) * EA;
#pragma unroll
    for (int i = 0; i < EA; ++i) As[(buf * BK + kq + i) * LDA_S + r] = ra[i];
  };
  auto load_b = [&](int k0) {
    if (trans_b) {  // B stored N x K
      const int c = tid / (BK / EB), kq = (tid % (BK / EB)) * EB;
      const int gn = n0 + c, gk = k0 + kq;
      if (gn < N) load_run(rb, B + (int64_t)gn * ldb + gk, K - gk, TagB{});
      else {
#pragma unroll
        for (int i = 0; i < EB; ++i) rb[i] = 0.f;
      }
    } else {        // B stored K x N
      const int kr = tid / (BN / EB), cq = (tid % (BN / EB)) * EB;
      const int gk = k0 + kr, gn = n0 + cq;
      if (gk < K) load_run(rb, B + (int64_t)gk * ldb + gn, N - gn, TagB{});
      else {
#pragma unroll
        for (int i = 0; i < EB; ++i) rb[i] = 0.f;
      }
    }
  };
  auto store_b = [&](int buf) {
    if (trans_b) {
      const int c = tid / (BK / EB), kq = (tid % (BK / EB)) * EB;
#pragma unroll
      for (int i = 0; i < EB; ++i) Bs[(buf * BK + kq + i) * LDB_S + c] = rb[i];
    } else {
      const int kr = tid / (BN / EB), cq = (tid % (BN / EB)) * EB;
#pragma unroll
      for (int i = 0; i < EB; ++i) Bs[(buf * BK + kr) * LDB_S + cq + i] = rb[i];
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const int nk = (K + BK - 1) / BK;
  load_a(0);
  load_b(0);
  store_a(0);
  store_b(0);
  worker_sync();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      load_a((kt + 1) * BK);
      load_b((kt + 1) * BK);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[TM], b[TN];
#pragma unroll
      for (int g = 0; g < TM / 4; ++g) {
        const float4 v = *reinterpret_cast<const float4 *>(&As[(cur * BK + k) * LDA_S + g * 64 + ty * 4]);
        a[g * 4 + 0] = v.x; a[g * 4 + 1] = v.y; a[g * 4 + 2] = v.z; a[g * 4 + 3] = v.w;
      }
#pragma unroll
      for (int g = 0; g < TN / 4; ++g) {
        const float4 v = *reinterpret_cast<const float4 *>(&Bs[(cur * BK + k) * LDB_S + g * 64 + tx * 4]);
        b[g * 4 + 0] = v.x; b[g * 4 + 1] = v.y; b[g * 4 + 2] = v.z; b[g * 4 + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store_a(cur ^ 1);
      store_b(cur ^ 1);
    }
    worker_sync();
  }

  // epilogue
  float bv[TN];
#pragma unroll
  for (int g = 0; g < TN / 4; ++g)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + g * 64 + tx * 4 + j;
      bv[g * 4 + j] = (bias && n < N) ? load_elem(bias, bias_dt, n) : 0.f;
    }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + (i / 4) * 64 + ty * 4 + (i % 4);
    if (m >= M) continue;
    const int64_t grow = (int64_t)bt * M + m;
#pragma unroll
    for (int g = 0; g < TN / 4; ++g) {
      const int n = n0 + g * 64 + tx * 4;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = activate(act, fmaf(acc[i][g * 4 + j], scale, bv[g * 4 + j]));
      if (vec && n + 4 <= N && c_dt == 0) {
        *reinterpret_cast<float4 *>(static_cast<float *>(Cp) + grow * ldc + n) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        for (int j = 0; j < 4 && n + j < N; ++j) store_elem(Cp, c_dt, grow * ldc + n + j, v[j]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Row softmax over whole rows [r0, r1): one warp per row, two rows per warp
// in flight; max and sum by warp shuffles; rows of up to 32 * V columns stay
// in registers (one read of the input), longer rows are streamed three times.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int V>
__device__ __forceinline__ void softmax_rows_reg(const NodeParams &np, int r0, int r1, int stride) {
  const int lane = threadIdx.x & 31;
  const int N = np.N;
  const float s = np.scale;
  const void *const A = np.A;
  void *const C = np.C;
  const int a_dt = np.a_dt, c_dt = np.c_dt;
  const int64_t lda = np.lda, ldc = np.ldc;
  for (int r = r0; r < r1; r += 2 * stride) {
    const int rr[2] = {r, r + stride};
    float x[2][V];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const int j = lane + 32 * i;
        x[q][i] = (rr[q] < r1 && j < N) ? s * load_elem(A, a_dt, (int64_t)rr[q] * lda + j) : -INFINITY;
      }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (rr[q] >= r1) continue;
      float m = -INFINITY;
#pragma unroll
      for (int i = 0; i < V; ++i) m = fmaxf(m, x[q][i]);
      m = warp_max(m);
      float sum = 0.f;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        x[q][i] = (lane + 32 * i < N) ? expf(x[q][i] - m) : 0.f;
        sum += x[q][i];
      }
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const int j = lane + 32 * i;
        if (j < N) store_elem(C, c_dt, (int64_t)rr[q] * ldc + j, x[q][i] * inv);
      }
    }
  }
}

// Rows of up to 256 elements with 16-byte aligned rows: lane l holds
// elements 4l..4l+3 and 128+4l..128+4l+3 of a row (vector loads and stores).
// Each warp keeps R rows in registers and prefetches its next R rows while
// it reduces, exponentiates and stores the current ones, so about
// 2 x R x 1 KiB per warp are in flight (the tile is memory-latency bound);
// the R rows' max and sum reductions are interleaved.
__device__ __forceinline__ void store4(void *base, int dt, int64_t i, const float (&v)[4]) {
  if (dt == 0) {
    *reinterpret_cast<float4 *>(static_cast<float *>(base) + i) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    const uint32_t a = (uint32_t)f32_to_bf16(v[0]) | ((uint32_t)f32_to_bf16(v[1]) << 16);
    const uint32_t b = (uint32_t)f32_to_bf16(v[2]) | ((uint32_t)f32_to_bf16(v[3]) << 16);
    *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(base) + i) = make_uint2(a, b);
  }
}

template <int R, int ADT>
__device__ __forceinline__ void softmax_rows_vec256(const NodeParams &np, int r0, int r1, int stride) {
  const int lane = threadIdx.x & 31;
  const int N = np.N;
  const float s = np.scale;
  void *const C = np.C;
  const int c_dt = np.c_dt;
  const int64_t lda = np.lda, ldc = np.ldc;
  // the two 4-element groups of this lane; a group is either wholly inside
  // the row or wholly outside (N is a multiple of 4)
  const int j0 = 4 * lane, j1 = 128 + 4 * lane;
  const bool g0 = j0 < N, g1 = j1 < N;
  // raw loaded bits stay untouched until the rows are computed, so the loads
  // of the next rows remain in flight meanwhile
  uint4 x[R][2], y[R][2];
  auto load_rows = [&](int rb, uint4 (&z)[R][2]) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = rb + q * stride;
      z[q][0] = z[q][1] = make_uint4(0u, 0u, 0u, 0u);
      if (r < r1) {
        if (ADT == 0) {
          const float *row = static_cast<const float *>(np.A) + (int64_t)r * lda;
          if (g0) z[q][0] = __ldcg(reinterpret_cast<const uint4 *>(row + j0));
          if (g1) z[q][1] = __ldcg(reinterpret_cast<const uint4 *>(row + j1));
        } else {
          const uint16_t *row = static_cast<const uint16_t *>(np.A) + (int64_t)r * lda;
          if (g0) { const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(row + j0)); z[q][0].x = a.x; z[q][0].y = a.y; }
          if (g1) { const uint2 a = __ldcg(reinterpret_cast<const uint2 *>(row + j1)); z[q][1].x = a.x; z[q][1].y = a.y; }
        }
      }
    }
  };
  auto value = [&](const uint4 &z, int e) -> float {
    if (ADT == 0) return __uint_as_float(e == 0 ? z.x : e == 1 ? z.y : e == 2 ? z.z : z.w);
    const uint32_t w = e < 2 ? z.x : z.y;
    return __uint_as_float((e & 1) ? (w & 0xFFFF0000u) : (w << 16));
  };
  load_rows(r0, x);
  for (int rb = r0; rb < r1; rb += R * stride) {
    const int nb = rb + R * stride;
    if (nb < r1) load_rows(nb, y);  // prefetch the next rows
    // all R rows at once: their reductions are independent shuffle chains
    float v[R][8], m[R], sum[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      m[q] = -INFINITY;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[q][e] = g0 ? s * value(x[q][0], e) : -INFINITY;
        v[q][4 + e] = g1 ? s * value(x[q][1], e) : -INFINITY;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) m[q] = fmaxf(m[q], v[q][i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < R; ++q) m[q] = fmaxf(m[q], __shfl_xor_sync(0xffffffffu, m[q], off));
#pragma unroll
    for (int q = 0; q < R; ++q) {
      sum[q] = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v[q][i] = ((i < 4 && g0) || (i >= 4 && g1)) ? __expf(v[q][i] - m[q]) : 0.f;
        sum[q] += v[q][i];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < R; ++q) sum[q] += __shfl_xor_sync(0xffffffffu, sum[q], off);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = rb + q * stride;
      if (r >= r1) continue;
      const float inv = 1.f / sum[q];
      float o0[4], o1[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        o0[e] = v[q][e] * inv;
        o1[e] = v[q][4 + e] * inv;
      }
      if (g0) store4(C, c_dt, (int64_t)r * ldc + j0, o0);
      if (g1) store4(C, c_dt, (int64_t)r * ldc + j1, o1);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      x[q][0] = y[q][0];
      x[q][1] = y[q][1];
    }
  }
}

// Rows of 257..2048 elements (N a multiple of 4, 16-byte aligned rows): lane
// l holds the 4-element groups l, l + 32, ..., l + 32 (G - 1) of each of R
// rows in registers -- one read of the input and one write of the output per
// row, with the loads of the R rows issued before any arithmetic (4 G R
// values per lane, 64 at most; more rows in flight made the executor kernel
// spill registers) -- max and sum by interleaved shuffle reductions, __expf
// as in the 256-element path.
template <int G, int R, int ADT>
__device__ __forceinline__ void softmax_rows_wide(const NodeParams &np, int r0, int r1, int stride) {
  const int lane = threadIdx.x & 31;
  const int N = np.N;
  const float s = np.scale;
  void *const C = np.C;
  const int c_dt = np.c_dt;
  const int64_t lda = np.lda, ldc = np.ldc;
  for (int rb = r0; rb < r1; rb += R * stride) {
    float v[R][G][4];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = rb + q * stride;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int j = 4 * (lane + 32 * i);
        const bool ok = r < r1 && j < N;
        if (ADT == 0) {
          const float4 a = ok ? __ldcg(reinterpret_cast<const float4 *>(static_cast<const float *>(np.A) +
                                                                       (int64_t)r * lda + j))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
          v[q][i][0] = a.x; v[q][i][1] = a.y; v[q][i][2] = a.z; v[q][i][3] = a.w;
        } else {
          const uint2 a = ok ? __ldcg(reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(np.A) +
                                                                     (int64_t)r * lda + j))
                             : make_uint2(0u, 0u);
          v[q][i][0] = __uint_as_float(a.x << 16); v[q][i][1] = __uint_as_float(a.x & 0xFFFF0000u);
          v[q][i][2] = __uint_as_float(a.y << 16); v[q][i][3] = __uint_as_float(a.y & 0xFFFF0000u);
        }
      }
    }
    float m[R], sum[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      m[q] = -INFINITY;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const bool ok = 4 * (lane + 32 * i) < N;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          v[q][i][e] = s * v[q][i][e];
          if (ok) m[q] = fmaxf(m[q], v[q][i][e]);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < R; ++q) m[q] = fmaxf(m[q], __shfl_xor_sync(0xffffffffu, m[q], off));
#pragma unroll
    for (int q = 0; q < R; ++q) {
      sum[q] = 0.f;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const bool ok = 4 * (lane + 32 * i) < N;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          v[q][i][e] = ok ? __expf(v[q][i][e] - m[q]) : 0.f;
          sum[q] += v[q][i][e];
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < R; ++q) sum[q] += __shfl_xor_sync(0xffffffffu, sum[q], off);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = rb + q * stride;
      if (r >= r1) continue;
      const float inv = 1.f / sum[q];
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int j = 4 * (lane + 32 * i);
        if (j >= N) continue;
        const float o[4] = {v[q][i][0] * inv, v[q][i][1] * inv, v[q][i][2] * inv, v[q][i][3] * inv};
        store4(C, c_dt, (int64_t)r * ldc + j, o);
      }
    }
  }
}

__device__ __noinline__ void tile_softmax(const TileDesc &t, const NodeParams &np) {
  const int wid = (threadIdx.x - kWorkerBase) >> 5, lane = threadIdx.x & 31;
  constexpr int nw = kWorkers / 32;
  const int N = np.N;
  if (N <= 256 && np.vec && (N & 3) == 0) {
    if (np.a_dt == 0) softmax_rows_vec256<4, 0>(np, t.r0 + wid, t.r1, nw);
    else softmax_rows_vec256<4, 1>(np, t.r0 + wid, t.r1, nw);
  } else if (N <= 2048 && np.vec && (N & 3) == 0) {
    if (N <= 512) {
      if (np.a_dt == 0) softmax_rows_wide<4, 2, 0>(np, t.r0 + wid, t.r1, nw);
      else softmax_rows_wide<4, 2, 1>(np, t.r0 + wid, t.r1, nw);
    } else if (N <= 1024) {
      if (np.a_dt == 0) softmax_rows_wide<8, 1, 0>(np, t.r0 + wid, t.r1, nw);
      else softmax_rows_wide<8, 1, 1>(np, t.r0 + wid, t.r1, nw);
    } else {
      if (np.a_dt == 0) softmax_rows_wide<16, 1, 0>(np, t.r0 + wid, t.r1, nw);
      else softmax_rows_wide<16, 1, 1>(np, t.r0 + wid, t.r1, nw);
    }
  } else if (N <= 256) {
    softmax_rows_reg<8>(np, t.r0 + wid, t.r1, nw);
  } else if (N <= 1024) {
    softmax_rows_reg<32>(np, t.r0 + wid, t.r1, nw);
  } else {
    const float s = np.scale;
    const void *const A = np.A;
    void *const C = np.C;
    const int a_dt = np.a_dt, c_dt = np.c_dt;
    const int64_t lda = np.lda, ldc = np.ldc;
    for (int r = t.r0 + wid; r < t.r1; r += nw) {
      const int64_t ia = (int64_t)r * lda, ic = (int64_t)r * ldc;
      float m = -INFINITY;
      for (int j = lane; j < N; j += 32) m = fmaxf(m, s * load_elem(A, a_dt, ia + j));
      m = warp_max(m);
      float sum = 0.f;
      for (int j = lane; j < N; j += 32) sum += expf(s * load_elem(A, a_dt, ia + j) - m);
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
      for (int j = lane; j < N; j += 32) store_elem(C, c_dt, ic + j, expf(s * load_elem(A, a_dt, ia + j) - m) * inv);
    }
  }
}

// ---------------------------------------------------------------------------
// Elementwise add / activation over rows [r0, r1) x cols [c0, c1): eight
// consecutive elements per step, 128-bit loads and stores when the rows are
// 16-byte aligned, four steps per thread in flight.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load8(const void *base, int dt, int64_t i, float (&v)[8]) {
  if (dt == 0) {
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + i));
    const float4 b = __ldcg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + i) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(static_cast<const uint16_t *>(base) + i));
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);
      v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  }
}
__device__ __forceinline__ void store8(void *base, int dt, int64_t i, const float (&v)[8]) {
  if (dt == 0) {
    float4 *d = reinterpret_cast<float4 *>(static_cast<float *>(base) + i);
    d[0] = make_float4(v[0], v[1], v[2], v[3]);
    d[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = (uint32_t)f32_to_bf16(v[2 * k]) | ((uint32_t)f32_to_bf16(v[2 * k + 1]) << 16);
    *reinterpret_cast<uint4 *>(static_cast<uint16_t *>(base) + i) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Fast path: A, B and C of one dtype, 16-byte aligned rows, whole 8-element
// groups.  Raw 16-byte loads of U groups per thread (both operands) are all
// issued before any is used -- about 64 registers of data in flight per
// thread, 64 KiB per SM -- and converted only when added.
template <int DT, int U>
__device__ __forceinline__ void eltwise_raw(const TileDesc &t, const NodeParams &np, bool add) {
  constexpr int W = DT == 0 ? 2 : 1;  // 16-byte words per 8-element group
  const int wt = threadIdx.x - kWorkerBase;
  const int width = t.c1 - t.c0;
  const int groups = width / 8;
  const int total = (t.r1 - t.r0) * groups;
  const int act = np.act;
  const char *A = static_cast<const char *>(np.A);
  const char *B = static_cast<const char *>(np.B);
  char *C = static_cast<char *>(np.C);
  constexpr int es = DT == 0 ? 4 : 2;
  for (int base = wt; base < total; base += U * kWorkers) {
    uint4 a[U][W], b[U][W];
    int64_t oc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int g = base + u * kWorkers;
      const int gg = g < total ? g : 0;
      const int r = t.r0 + gg / groups, c = t.c0 + (gg % groups) * 8;
      oc[u] = g < total ? ((int64_t)r * np.ldc + c) * es : -1;
      const uint4 *pa = reinterpret_cast<const uint4 *>(A + ((int64_t)r * np.lda + c) * es);
      const uint4 *pb = reinterpret_cast<const uint4 *>(B + ((int64_t)r * np.ldb + c) * es);
#pragma unroll
      for (int q = 0; q < W; ++q) {
        a[u][q] = g < total ? __ldcg(pa + q) : make_uint4(0u, 0u, 0u, 0u);
        b[u][q] = (add && g < total) ? __ldcg(pb + q) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (oc[u] < 0) continue;
      uint4 o[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const uint32_t aw[4] = {a[u][q].x, a[u][q].y, a[u][q].z, a[u][q].w};
        const uint32_t bw[4] = {b[u][q].x, b[u][q].y, b[u][q].z, b[u][q].w};
        uint32_t ow[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (DT == 0) {
            const float x = __uint_as_float(aw[k]) + (add ? __uint_as_float(bw[k]) : 0.f);
            ow[k] = __float_as_uint(activate(act, x));
          } else {
            const float x0 = __uint_as_float(aw[k] << 16) + (add ? __uint_as_float(bw[k] << 16) : 0.f);
            const float x1 = __uint_as_float(aw[k] & 0xFFFF0000u) + (add ? __uint_as_float(bw[k] & 0xFFFF0000u) : 0.f);
            ow[k] = (uint32_t)f32_to_bf16(activate(act, x0)) | ((uint32_t)f32_to_bf16(activate(act, x1)) << 16);
          }
        }
        o[q] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
      }
      uint4 *pc = reinterpret_cast<uint4 *>(C + oc[u]);
#pragma unroll
      for (int q = 0; q < W; ++q) pc[q] = o[q];
    }
  }
}

__device__ __forceinline__ void tile_eltwise(const TileDesc &t, const NodeParams &npg, bool add) {
  if (npg.vec && ((t.c1 - t.c0) & 7) == 0 && npg.a_dt == npg.c_dt && (!add || npg.b_dt == npg.c_dt)) {
    if (npg.c_dt == 1) eltwise_raw<1, 8>(t, npg, add);
    else eltwise_raw<0, 4>(t, npg, add);
    return;
  }
  const void *const A = npg.A;
  const void *const B = npg.B;
  void *const C = npg.C;
  const int64_t lda = npg.lda, ldb = npg.ldb, ldc = npg.ldc;
  const int a_dt = npg.a_dt, b_dt = npg.b_dt, c_dt = npg.c_dt, act = npg.act, vec = npg.vec;
  const int wt = threadIdx.x - kWorkerBase;
  const int width = t.c1 - t.c0;
  const int groups = (width + 7) / 8;  // 8-element groups per row
  const int total = (t.r1 - t.r0) * groups;
  constexpr int U = 4;
  for (int base = wt; base < total; base += U * kWorkers) {
    float a[U][8], b[U][8];
    int64_t ic[U];
    int cc[U];
    bool whole[U], live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int g = base + u * kWorkers;
      live[u] = g < total;
      const int r = t.r0 + (live[u] ? g / groups : 0);
      const int c = t.c0 + (live[u] ? (g % groups) * 8 : 0);
      cc[u] = c;
      whole[u] = live[u] && vec && c + 8 <= t.c1;
      ic[u] = (int64_t)r * ldc + c;
      const int64_t ia = (int64_t)r * lda + c, ib = (int64_t)r * ldb + c;
      if (whole[u]) {
        load8(A, a_dt, ia, a[u]);
        if (add) load8(B, b_dt, ib, b[u]);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          a[u][k] = (live[u] && c + k < t.c1) ? load_elem(A, a_dt, ia + k) : 0.f;
          b[u][k] = (add && live[u] && c + k < t.c1) ? load_elem(B, b_dt, ib + k) : 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!live[u]) continue;
      float o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = activate(act, add ? a[u][k] + b[u][k] : a[u][k]);
      if (whole[u]) {
        store8(C, c_dt, ic[u], o);
      } else {
        for (int k = 0; k < 8 && cc[u] + k < t.c1; ++k) store_elem(C, c_dt, ic[u] + k, o[k]);
      }
    }
  }
}

}  // namespace dagx
