// costmodel.cu -- the learned cost model: a 3-layer perceptron
//   x (in_dim) -> relu(x W1 + b1) (H) -> relu(. W2 + b2) (H) -> . W3 + b3 (1)
// with its forward pass, mean-squared-error backward pass and Adam update as
// CUDA kernels.  It predicts the log of a tile's execution time from node
// features; the planner turns predictions into bottom-level ranks that order
// the ready queue (the paper's priority queue F ordered by bottom-level rank,
// §5, with the per-kernel times HEFT takes from profiling).
//
// Parameters live in one packed f32 array: W1 [in][H], b1 [H], W2 [H][H],
// b2 [H], W3 [H], b3 [1] (row-major, x W convention).  A gradient is
// computed in chunks of 64 samples, one CTA per chunk, each writing its
// partial sums; a second kernel adds the chunks in index order, so results do
// not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "dag_internal.h"
#include "dagexec.h"

namespace {

constexpr int kH = 64;        // hidden width
constexpr int kMaxIn = 32;    // largest input width
constexpr int kChunk = 64;    // samples per CTA
constexpr int kT = 256;       // threads per CTA

struct Layout {
  int in;
  int w1, b1, w2, b2, w3, b3, total;
};

__host__ __device__ inline Layout layout(int in) {
  Layout L;
  L.in = in;
  L.w1 = 0;
  L.b1 = L.w1 + in * kH;
  L.w2 = L.b1 + kH;
  L.b2 = L.w2 + kH * kH;
  L.w3 = L.b2 + kH;
  L.b3 = L.w3 + kH;
  L.total = L.b3 + 1;
  return L;
}

// Forward (and optionally backward) over one chunk of samples in shared
// memory.  grad == nullptr: write predictions only.
__global__ void __launch_bounds__(kT) mlp_chunk_kernel(const float *__restrict__ P, int in, const float *__restrict__ X,
                                                     const float *__restrict__ y, int n, float inv_n,
                                                     float *__restrict__ pred, float *__restrict__ part_grad,
                                                     float *__restrict__ part_loss) {
  const Layout L = layout(in);
  extern __shared__ float sm[];
  float *W1 = sm;                                  // [kMaxIn * kH]
  float *b1 = W1 + kMaxIn * kH;                    // [kH]
  float *W2 = b1 + kH;                             // [kH * kH]
  float *b2 = W2 + kH * kH;                        // [kH]
  float *W3 = b2 + kH;                             // [kH]
  float(*xs)[kMaxIn] = reinterpret_cast<float(*)[kMaxIn]>(W3 + kH);       // [kChunk][kMaxIn]
  float(*z1)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(&xs[kChunk][0]);  // [kChunk][kH+1]
  float(*z2)[kH + 1] = z1 + kChunk;
  float(*d2)[kH + 1] = z2 + kChunk;
  float *dout = &d2[kChunk][0];                    // [kChunk]
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * kChunk;
  const int cn = min(kChunk, n - s0);
  for (int i = tid; i < in * kH; i += kT) W1[i] = P[L.w1 + i];
  for (int i = tid; i < kH * kH; i += kT) W2[i] = P[L.w2 + i];
  for (int i = tid; i < kH; i += kT) { b1[i] = P[L.b1 + i]; b2[i] = P[L.b2 + i]; W3[i] = P[L.w3 + i]; }
  for (int i = tid; i < kChunk * in; i += kT) {
    const int r = i / in, c = i % in;
    xs[r][c] = r < cn ? X[(int64_t)(s0 + r) * in + c] : 0.f;
  }
  __syncthreads();
  // z1 = x W1 + b1 ; kept pre-activation for the ReLU mask
  for (int i = tid; i < kChunk * kH; i += kT) {
    const int r = i / kH, j = i % kH;
    float a = b1[j];
    for (int k = 0; k < in; ++k) a = fmaf(xs[r][k], W1[k * kH + j], a);
    z1[r][j] = a;
  }
  __syncthreads();
  for (int i = tid; i < kChunk * kH; i += kT) {
    const int r = i / kH, j = i % kH;
    float a = b2[j];
    for (int k = 0; k < kH; ++k) a = fmaf(fmaxf(z1[r][k], 0.f), W2[k * kH + j], a);
    z2[r][j] = a;
  }
  __syncthreads();
  const float b3 = P[L.b3];
  if (tid < kChunk) {
    float a = b3;
    for (int k = 0; k < kH; ++k) a = fmaf(fmaxf(z2[tid][k], 0.f), W3[k], a);
    if (pred && tid < cn) pred[s0 + tid] = a;
    const float e = (y && tid < cn) ? a - y[s0 + tid] : 0.f;
    dout[tid] = 2.f * e * inv_n;                 // d(mean squared error)/d out
    if (part_loss) d2[tid][kH] = e * e;          // scratch column for the loss
  }
  __syncthreads();
  if (!part_grad) return;
  float *g = part_grad + (int64_t)blockIdx.x * L.total;
  if (tid == 0) {
    float l = 0.f, db3 = 0.f;
    for (int r = 0; r < kChunk; ++r) { l += d2[r][kH]; db3 += dout[r]; }
    part_loss[blockIdx.x] = l;
    g[L.b3] = db3;
  }
  // dW3 = relu(z2)^T dout ; dz2 = dout W3^T * (z2 > 0)
  if (tid < kH) {
    float a = 0.f;
    for (int r = 0; r < kChunk; ++r) a = fmaf(fmaxf(z2[r][tid], 0.f), dout[r], a);
    g[L.w3 + tid] = a;
  }
  __syncthreads();
  for (int i = tid; i < kChunk * kH; i += kT) {
    const int r = i / kH, j = i % kH;
    d2[r][j] = z2[r][j] > 0.f ? dout[r] * W3[j] : 0.f;
  }
  __syncthreads();
  // dW2 = relu(z1)^T dz2 ; db2 = column sums of dz2
  for (int i = tid; i < kH * kH; i += kT) {
    const int k = i / kH, j = i % kH;
    float a = 0.f;
    for (int r = 0; r < kChunk; ++r) a = fmaf(fmaxf(z1[r][k], 0.f), d2[r][j], a);
    g[L.w2 + i] = a;
  }
  if (tid < kH) {
    float a = 0.f;
    for (int r = 0; r < kChunk; ++r) a += d2[r][tid];
    g[L.b2 + tid] = a;
  }
  __syncthreads();
  // dz1 = (dz2 W2^T) * (z1 > 0), written over z2 (no longer needed)
  for (int i = tid; i < kChunk * kH; i += kT) {
    const int r = i / kH, k = i % kH;
    float a = 0.f;
    for (int j = 0; j < kH; ++j) a = fmaf(d2[r][j], W2[k * kH + j], a);
    z2[r][k] = z1[r][k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // dW1 = x^T dz1 ; db1 = column sums of dz1
  for (int i = tid; i < in * kH; i += kT) {
    const int k = i / kH, j = i % kH;
    float a = 0.f;
    for (int r = 0; r < kChunk; ++r) a = fmaf(xs[r][k], z2[r][j], a);
    g[L.w1 + i] = a;
  }
  if (tid < kH) {
    float a = 0.f;
    for (int r = 0; r < kChunk; ++r) a += z2[r][tid];
    g[L.b1 + tid] = a;
  }
}

// grad[p] = sum over chunks c = 0..C-1 of part[c][p], in that order
__global__ void reduce_chunks(const float *__restrict__ part, int C, int P, float *__restrict__ grad,
                              const float *__restrict__ part_loss, float *__restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) {
    float a = 0.f;
    for (int c = 0; c < C; ++c) a += part[(int64_t)c * P + p];
    grad[p] = a;
  }
  if (p == 0 && loss) {
    float a = 0.f;
    for (int c = 0; c < C; ++c) a += part_loss[c];
    *loss = a;
  }
}

// Adam (Kingma & Ba 2015) with bias correction; t = 1, 2, ...
__global__ void adam_step(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

constexpr int kSmem = (kMaxIn * kH + kH + kH * kH + kH + kH + kChunk * kMaxIn + 3 * kChunk * (kH + 1) + kChunk) *
                      (int)sizeof(float);

}  // namespace

struct dag_mlp {
  int in = 0;
  Layout L{};
  float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *part = nullptr, *part_loss = nullptr;
  float *loss = nullptr;
  int part_cap = 0;  // chunks the partial buffers hold
  long adam_t = 0;
  cudaStream_t st = nullptr;
};

static dag_status ensure_parts(dag_mlp *m, int chunks) {
  if (chunks <= m->part_cap) return DAG_OK;
  if (m->part) cudaFree(m->part);
  if (m->part_loss) cudaFree(m->part_loss);
  m->part = m->part_loss = nullptr;
  if (cudaMalloc(&m->part, (size_t)chunks * m->L.total * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->part_loss, (size_t)chunks * sizeof(float)) != cudaSuccess)
    return dagx::report_error(DAG_ENOMEM, "cost model: partial-gradient buffers");
  m->part_cap = chunks;
  return DAG_OK;
}

extern "C" dag_status dag_mlp_create(int in_dim, dag_mlp **out) {
  if (!out || in_dim < 1 || in_dim > kMaxIn)
    return dagx::report_error(DAG_EINVAL, "dag_mlp_create: input width must be 1..32");
  if (cudaFuncSetAttribute(mlp_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_mlp_create: shared memory attribute");
  dag_mlp *m = new dag_mlp();
  m->in = in_dim;
  m->L = layout(in_dim);
  const size_t bytes = (size_t)m->L.total * sizeof(float);
  if (cudaMalloc(&m->params, bytes) != cudaSuccess || cudaMalloc(&m->m, bytes) != cudaSuccess ||
      cudaMalloc(&m->v, bytes) != cudaSuccess || cudaMalloc(&m->grad, bytes) != cudaSuccess ||
      cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete m;
    return dagx::report_error(DAG_ENOMEM, "dag_mlp_create: device allocation");
  }
  cudaMemset(m->params, 0, bytes);
  cudaMemset(m->m, 0, bytes);
  cudaMemset(m->v, 0, bytes);
  *out = m;
  return DAG_OK;
}

extern "C" int dag_mlp_param_count(const dag_mlp *m) { return m ? m->L.total : 0; }

extern "C" dag_status dag_mlp_set_params(dag_mlp *m, const float *params, int n) {
  if (!m || !params || n != m->L.total) return dagx::report_error(DAG_EINVAL, "dag_mlp_set_params: size");
  if (cudaMemcpy(m->params, params, (size_t)n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_mlp_set_params: copy");
  cudaMemset(m->m, 0, (size_t)n * sizeof(float));
  cudaMemset(m->v, 0, (size_t)n * sizeof(float));
  m->adam_t = 0;
  return DAG_OK;
}

extern "C" dag_status dag_mlp_get_params(dag_mlp *m, float *params, int n) {
  if (!m || !params || n != m->L.total) return dagx::report_error(DAG_EINVAL, "dag_mlp_get_params: size");
  if (cudaMemcpy(params, m->params, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_mlp_get_params: copy");
  return DAG_OK;
}

// Full-batch loss and gradient on device arrays (X: n x in, y: n).
static dag_status loss_grad_dev(dag_mlp *m, const float *dX, const float *dy, int n) {
  const int chunks = (n + kChunk - 1) / kChunk;
  dag_status s = ensure_parts(m, chunks);
  if (s) return s;
  mlp_chunk_kernel<<<chunks, kT, kSmem, m->st>>>(m->params, m->in, dX, dy, n, 1.f / (float)n, nullptr, m->part,
                                                 m->part_loss);
  reduce_chunks<<<(m->L.total + 255) / 256, 256, 0, m->st>>>(m->part, chunks, m->L.total, m->grad, m->part_loss,
                                                               m->loss);
  if (cudaGetLastError() != cudaSuccess) return dagx::report_error(DAG_EDEVICE, "cost model: launch");
  return DAG_OK;
}

static dag_status upload(const float *h, size_t n, float **d) {
  if (cudaMalloc(d, std::max<size_t>(1, n) * sizeof(float)) != cudaSuccess)
    return dagx::report_error(DAG_ENOMEM, "cost model: sample buffers");
  if (n && cudaMemcpy(*d, h, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "cost model: sample copy");
  return DAG_OK;
}

extern "C" dag_status dag_mlp_loss_grad(dag_mlp *m, const float *X, const float *y, int n, float *loss,
                                        float *grad) {
  if (!m || !X || !y || n < 1) return dagx::report_error(DAG_EINVAL, "dag_mlp_loss_grad: arguments");
  float *dX = nullptr, *dy = nullptr;
  dag_status s = upload(X, (size_t)n * m->in, &dX);
  if (!s) s = upload(y, (size_t)n, &dy);
  if (!s) s = loss_grad_dev(m, dX, dy, n);
  if (!s && cudaStreamSynchronize(m->st) != cudaSuccess) s = dagx::report_error(DAG_EDEVICE, "cost model: run");
  if (!s && grad) cudaMemcpy(grad, m->grad, (size_t)m->L.total * sizeof(float), cudaMemcpyDeviceToHost);
  if (!s && loss) {
    cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost);
    *loss /= (float)n;
  }
  cudaFree(dX);
  cudaFree(dy);
  return s;
}

extern "C" dag_status dag_mlp_train(dag_mlp *m, const float *X, const float *y, int n, int steps, int batch,
                                    float lr) {
  if (!m || !X || !y || n < 1 || steps < 0 || batch < 1) return dagx::report_error(DAG_EINVAL, "dag_mlp_train: arguments");
  batch = std::min(batch, n);
  float *dX = nullptr, *dy = nullptr;
  dag_status s = upload(X, (size_t)n * m->in, &dX);
  if (!s) s = upload(y, (size_t)n, &dy);
  // minibatches are consecutive windows of the sample order the caller gives
  for (int t = 0; t < steps && !s; ++t) {
    const int start = (int)(((long)t * batch) % n);
    const int cnt = std::min(batch, n - start);
    s = loss_grad_dev(m, dX + (size_t)start * m->in, dy + start, cnt);
    if (s) break;
    m->adam_t++;
    const float c1 = 1.f - powf(0.9f, (float)m->adam_t), c2 = 1.f - powf(0.999f, (float)m->adam_t);
    adam_step<<<(m->L.total + 255) / 256, 256, 0, m->st>>>(m->params, m->grad, m->m, m->v, m->L.total, lr, 0.9f,
                                                           0.999f, 1e-8f, c1, c2);
  }
  if (!s && cudaStreamSynchronize(m->st) != cudaSuccess) s = dagx::report_error(DAG_EDEVICE, "cost model: training");
  cudaFree(dX);
  cudaFree(dy);
  return s;
}

extern "C" dag_status dag_mlp_predict(dag_mlp *m, const float *X, int n, float *out) {
  if (!m || !X || !out || n < 1) return dagx::report_error(DAG_EINVAL, "dag_mlp_predict: arguments");
  float *dX = nullptr, *dp = nullptr;
  dag_status s = upload(X, (size_t)n * m->in, &dX);
  if (!s && cudaMalloc(&dp, (size_t)n * sizeof(float)) != cudaSuccess) s = dagx::report_error(DAG_ENOMEM, "predict");
  if (!s) {
    mlp_chunk_kernel<<<(n + kChunk - 1) / kChunk, kT, kSmem, m->st>>>(m->params, m->in, dX, nullptr, n, 1.f, dp,
                                                                     nullptr, nullptr);
    if (cudaStreamSynchronize(m->st) != cudaSuccess) s = dagx::report_error(DAG_EDEVICE, "predict: run");
  }
  if (!s) cudaMemcpy(out, dp, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(dX);
  cudaFree(dp);
  return s;
}

extern "C" dag_status dag_mlp_destroy(dag_mlp *m) {
  if (!m) return DAG_OK;
  cudaFree(m->params);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->grad);
  cudaFree(m->loss);
  if (m->part) cudaFree(m->part);
  if (m->part_loss) cudaFree(m->part_loss);
  if (m->st) cudaStreamDestroy(m->st);
  delete m;
  return DAG_OK;
}
