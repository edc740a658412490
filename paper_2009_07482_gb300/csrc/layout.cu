// layout.cu -- device-side layout change of resident GEMM weights.
//
// A GEMM's B operand stored K x N (row-major, N contiguous) reaches the
// tensor cores as MN-major shared-memory tiles: several 128-byte-wide TMA
// boxes per stage.  Stored N x K (K contiguous), the same stage is one box,
// and the bf16 K loop on a fully loaded GPU streams measurably faster.  A
// weight that is uploaded once and read only as the B operand of GEMMs is
// therefore kept transposed on the device: it is copied in its given layout
// into a staging area and transposed here, per batch block.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dag_internal.h"

namespace dagx {
namespace {

// dst (batch blocks of N x K, row pitch ldd) = per-block transpose of src
// (batch blocks of K x N, row pitch lds); 32 x 32 tiles through shared memory
template <typename T>
__global__ void __launch_bounds__(256) transpose_blocks(const T *__restrict__ src, int64_t lds, T *__restrict__ dst,
                                                        int64_t ldd, int K, int N) {
  __shared__ T tile[32][33];
  const int64_t b = blockIdx.z;
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const T *s = src + b * K * lds;
  T *d = dst + b * N * ldd;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int k = k0 + i, n = n0 + threadIdx.x;
    if (k < K && n < N) tile[i][threadIdx.x] = s[(int64_t)k * lds + n];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int n = n0 + i, k = k0 + threadIdx.x;
    if (n < N && k < K) d[(int64_t)n * ldd + k] = tile[threadIdx.x][i];
  }
}

}  // namespace

cudaError_t launch_transpose(const void *src, int64_t lds, void *dst, int64_t ldd, int batch, int K, int N,
                             int elem_bytes, cudaStream_t st) {
  if (batch <= 0 || K <= 0 || N <= 0) return cudaSuccess;
  if ((K + 31) / 32 > 65535 || batch > 65535) return cudaErrorInvalidValue;
  const dim3 grid((N + 31) / 32, (K + 31) / 32, batch), block(32, 8);
  if (elem_bytes == 2)
    transpose_blocks<uint16_t><<<grid, block, 0, st>>>(static_cast<const uint16_t *>(src), lds,
                                                       static_cast<uint16_t *>(dst), ldd, K, N);
  else
    transpose_blocks<uint32_t><<<grid, block, 0, st>>>(static_cast<const uint32_t *>(src), lds,
                                                       static_cast<uint32_t *>(dst), ldd, K, N);
  return cudaGetLastError();
}

}  // namespace dagx
