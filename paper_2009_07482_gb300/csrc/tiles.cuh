// tiles.cuh -- the tile kinds the executor runs.  Each function computes one
// rectangle of one kernel's output with all 256 threads of the CTA.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

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

// ---------------------------------------------------------------------------
// Shared control block of one CTA (lives after the pipeline stages)
// ---------------------------------------------------------------------------
struct SmemCtl {
  uint64_t full[kStages];   // TMA -> MMA: stage filled
  uint64_t empty[kStages];  // MMA -> TMA: stage consumed
  uint64_t accum;           // MMA -> epilogue: accumulator complete
  uint32_t tmem_base;
  int32_t tile;             // tile index broadcast by thread 0
  int32_t fail;             // CTA-local failure flag
  uint32_t start_ticket;
  uint64_t t_start;
};

// Pipeline phase state, persistent across tiles.  Thread 0 owns the producer
// fields, thread 32 the MMA fields; every thread tracks the accumulator parity.
struct PipeState {
  uint32_t pstage, pphase, mstage, mphase, aphase;
};

// ---------------------------------------------------------------------------
// bf16 GEMM tile, 128 x BN, tcgen05 with the accumulator in TMEM
//   thread 0  : TMA producer (A box 64x128, B boxes) into a kStages ring
//   thread 32 : MMA issuer (4 x K=16 per stage), commits to the empty barriers
//   all warps : epilogue, TMEM -> registers -> scale/bias/act/cast -> global
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tile_gemm_bf16(const ExecParams &p, const TileDesc &t, const NodeParams &np,
                                               uint8_t *smem, SmemCtl *ctl, PipeState &ps,
                                               uint64_t deadline) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int BN = t.cfg;
  const int M = np.M, N = np.N;
  const int bt = t.r0 / M;
  const int m0 = t.r0 - bt * M;
  const int n0 = t.c0;
  const int kiters = (np.K + kBK - 1) / kBK;
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kStageA;
  bool ok = true;

  if (tid == 0) {
    const CUtensorMap *ta = p.tmaps + np.tmap_a;
    const CUtensorMap *tb = p.tmaps + np.tmap_b;
    const uint32_t bytes = (uint32_t)(kStageA + BN * kBK * 2);
    for (int kb = 0; kb < kiters; ++kb) {
      if (!mbar_wait(&ctl->empty[ps.pstage], ps.pphase ^ 1u, deadline)) { ok = false; break; }
      uint64_t *bar = &ctl->full[ps.pstage];
      mbar_arrive_expect_tx(bar, bytes);
      tma_load_3d(sA + ps.pstage * kStageA, ta, bar, kb * kBK, m0, bt);
      uint8_t *dB = sB + ps.pstage * kStageB;
      if (np.trans_b) {
        tma_load_3d(dB, tb, bar, kb * kBK, n0, bt);                // box {64 (K), BN}
      } else {
        for (int j = 0; j < BN / 64; ++j)                          // boxes {64 (N), 64 (K)}
          tma_load_3d(dB + j * (64 * kBK * 2), tb, bar, n0 + j * 64, kb * kBK, bt);
      }
      if (++ps.pstage == kStages) { ps.pstage = 0; ps.pphase ^= 1u; }
    }
  } else if (tid == 32) {
    const uint32_t idesc = idesc_bf16((uint32_t)BN, np.trans_b ? 0u : 1u);
    const uint32_t tmem = ctl->tmem_base;
    for (int kb = 0; kb < kiters; ++kb) {
      if (!mbar_wait(&ctl->full[ps.mstage], ps.mphase, deadline)) { ok = false; break; }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + ps.mstage * kStageA);
      const uint32_t b0 = smem_u32(sB + ps.mstage * kStageB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K-major, 128-byte swizzle: a K step of 16 bf16 is 32 bytes along the row
        const uint64_t ad = smem_desc_sw128(a0 + kk * 32, 16, 1024);
        // B K-major: same; B MN-major: 16 K rows of 128 bytes = 2048 bytes per step,
        // 64-column chunks 8 KiB apart (leading offset), 8-row groups 1 KiB apart (stride offset)
        const uint64_t bd = np.trans_b ? smem_desc_sw128(b0 + kk * 32, 16, 1024)
                                       : smem_desc_sw128(b0 + kk * 2048, 64 * kBK * 2, 1024);
        mma_bf16(tmem, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&ctl->empty[ps.mstage]);
      if (++ps.mstage == kStages) { ps.mstage = 0; ps.mphase ^= 1u; }
    }
    if (ok) mma_commit(&ctl->accum);
  }
  if (!ok) ctl->fail = 1;

  // ---- epilogue ----
  const bool acc_ok = mbar_wait(&ctl->accum, ps.aphase, deadline);
  ps.aphase ^= 1u;
  if (!acc_ok) {
    ctl->fail = 1;
    return false;
  }
  tc_fence_after();
  const int quad = warp & 3;            // TMEM lanes 32*quad .. 32*quad+31
  const int half = warp >> 2;           // column half
  const int row = m0 + quad * 32 + lane;
  const bool row_ok = row < M;
  const int64_t grow = (int64_t)bt * M + row;
  const int cw = BN / 2;
  const float scale = np.scale;
  for (int c = half * cw; c < (half + 1) * cw; c += 16) {
    float v[16];
    tmem_ld16(ctl->tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
    const int col = n0 + c;
    if (!row_ok || col >= N) continue;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float x = v[i] * scale;
      if (np.bias && col + i < N) x += load_elem(np.bias, np.bias_dt, col + i);
      v[i] = activate(np.act, x);
    }
    if (np.vec && col + 16 <= N) {
      if (np.c_dt == 1) {
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = (uint32_t)f32_to_bf16(v[2 * i]) | ((uint32_t)f32_to_bf16(v[2 * i + 1]) << 16);
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(np.C) + grow * np.ldc + col);
        dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
        dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else {
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(np.C) + grow * np.ldc + col);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      }
    } else {
      for (int i = 0; i < 16 && col + i < N; ++i) store_elem(np.C, np.c_dt, grow * np.ldc + col + i, v[i]);
    }
  }
  tc_fence_before();
  return true;
}

// ---------------------------------------------------------------------------
// f32 GEMM tile, exact f32 (SIMT FFMA), BM x BN with 16 x 16 threads, BK = 16,
// double-buffered shared memory.  Each thread owns a (BM/16) x (BN/16) block
// split into 4-wide groups 64 apart, so shared reads are conflict-free.
// ---------------------------------------------------------------------------
template <int BM, int BN>
__device__ __forceinline__ void tile_gemm_f32(const TileDesc &t, const NodeParams &np, float *smem) {
  constexpr int BK = 16;
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LDA_S = BM + 4, LDB_S = BN + 4;
  float *As = smem;                      // [2][BK][LDA_S]
  float *Bs = smem + 2 * BK * LDA_S;     // [2][BK][LDB_S]
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int M = np.M, N = np.N, K = np.K;
  const int bt = t.r0 / M;
  const int m0 = t.r0 - bt * M, n0 = t.c0;
  const float *A = static_cast<const float *>(np.A) + (int64_t)bt * M * np.lda;
  const float *B = static_cast<const float *>(np.B) +
                   (int64_t)bt * (np.trans_b ? (int64_t)N * np.ldb : (int64_t)K * np.ldb);

  // loader mapping: A tile BM x BK -> EA elements per thread along k
  constexpr int EA = BM * BK / kThreads;      // 4 or 8
  constexpr int EB = BN * BK / kThreads;      // 4 or 8
  float ra[EA], rb[EB];

  auto load_a = [&](int k0) {
    const int r = tid / (BK / EA), kq = (tid % (BK / EA)) * EA;
    const int gm = m0 + r, gk = k0 + kq;
#pragma unroll
    for (int i = 0; i < EA; ++i)
      ra[i] = (gm < M && gk + i < K) ? __ldcg(A + (int64_t)gm * np.lda + gk + i) : 0.f;
  };
  auto store_a = [&](int buf) {
    const int r = tid / (BK / EA), kq = (tid % (BK / EA)) * EA;
#pragma unroll
    for (int i = 0; i < EA; ++i) As[(buf * BK + kq + i) * LDA_S + r] = ra[i];
  };
  auto load_b = [&](int k0) {
    if (np.trans_b) {  // B stored N x K
      const int c = tid / (BK / EB), kq = (tid % (BK / EB)) * EB;
      const int gn = n0 + c, gk = k0 + kq;
#pragma unroll
      for (int i = 0; i < EB; ++i)
        rb[i] = (gn < N && gk + i < K) ? __ldcg(B + (int64_t)gn * np.ldb + gk + i) : 0.f;
    } else {           // B stored K x N
      const int kr = tid / (BN / EB), cq = (tid % (BN / EB)) * EB;
      const int gk = k0 + kr, gn = n0 + cq;
#pragma unroll
      for (int i = 0; i < EB; ++i)
        rb[i] = (gk < K && gn + i < N) ? __ldcg(B + (int64_t)gk * np.ldb + gn + i) : 0.f;
    }
  };
  auto store_b = [&](int buf) {
    if (np.trans_b) {
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
  __syncthreads();
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
    __syncthreads();
  }

  // epilogue
  const float scale = np.scale;
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
      for (int j = 0; j < 4; ++j) {
        float x = acc[i][g * 4 + j] * scale;
        if (np.bias && n + j < N) x += load_elem(np.bias, np.bias_dt, n + j);
        v[j] = activate(np.act, x);
      }
      if (np.vec && n + 4 <= N && np.c_dt == 0) {
        *reinterpret_cast<float4 *>(static_cast<float *>(np.C) + grow * np.ldc + n) =
            make_float4(v[0], v[1], v[2], v[3]);
      } else {
        for (int j = 0; j < 4 && n + j < N; ++j) store_elem(np.C, np.c_dt, grow * np.ldc + n + j, v[j]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Row softmax over whole rows [r0, r1): one warp per row, max and sum by warp
// shuffles; rows of up to 1024 columns stay in registers (one read of the
// input), longer rows are streamed three times.
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

__device__ __forceinline__ void tile_softmax(const TileDesc &t, const NodeParams &np) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = np.N;
  const float s = np.scale;
  for (int r = t.r0 + warp; r < t.r1; r += kThreads / 32) {
    const int64_t ia = (int64_t)r * np.lda, ic = (int64_t)r * np.ldc;
    if (N <= 1024) {
      float x[32];
      float m = -INFINITY;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = lane + 32 * i;
        x[i] = j < N ? s * load_elem(np.A, np.a_dt, ia + j) : -INFINITY;
        m = fmaxf(m, x[i]);
      }
      m = warp_max(m);
      float sum = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = lane + 32 * i;
        x[i] = j < N ? expf(x[i] - m) : 0.f;
        sum += x[i];
      }
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = lane + 32 * i;
        if (j < N) store_elem(np.C, np.c_dt, ic + j, x[i] * inv);
      }
    } else {
      float m = -INFINITY;
      for (int j = lane; j < N; j += 32) m = fmaxf(m, s * load_elem(np.A, np.a_dt, ia + j));
      m = warp_max(m);
      float sum = 0.f;
      for (int j = lane; j < N; j += 32) sum += expf(s * load_elem(np.A, np.a_dt, ia + j) - m);
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
      for (int j = lane; j < N; j += 32)
        store_elem(np.C, np.c_dt, ic + j, expf(s * load_elem(np.A, np.a_dt, ia + j) - m) * inv);
    }
  }
}

// ---------------------------------------------------------------------------
// Elementwise add / activation over rows [r0, r1) x cols [c0, c1): eight
// consecutive elements per thread step, 128-bit loads and stores when the
// rows are 16-byte aligned.
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

__device__ __forceinline__ void tile_eltwise(const TileDesc &t, const NodeParams &np, bool add) {
  const int width = t.c1 - t.c0;
  const int groups = (width + 7) / 8;                // 8-element groups per row
  const int64_t total = (int64_t)(t.r1 - t.r0) * groups;
  for (int64_t g = threadIdx.x; g < total; g += kThreads) {
    const int r = t.r0 + (int)(g / groups);
    const int c = t.c0 + (int)(g % groups) * 8;
    const int64_t ia = (int64_t)r * np.lda + c, ib = (int64_t)r * np.ldb + c, ic = (int64_t)r * np.ldc + c;
    float a[8], b[8];
    if (np.vec && c + 8 <= t.c1) {
      load8(np.A, np.a_dt, ia, a);
      if (add) load8(np.B, np.b_dt, ib, b);
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = activate(np.act, add ? a[k] + b[k] : a[k]);
      store8(np.C, np.c_dt, ic, a);
    } else {
      for (int k = 0; k < 8 && c + k < t.c1; ++k) {
        float x = load_elem(np.A, np.a_dt, ia + k);
        if (add) x += load_elem(np.B, np.b_dt, ib + k);
        store_elem(np.C, np.c_dt, ic + k, activate(np.act, x));
      }
    }
  }
}

}  // namespace dagx
