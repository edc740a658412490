// noalloc.cu -- dag_run_noalloc: run a DAG without allocating device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a device memory
// pool is locked down or exhausted by design (a serving process that
// reserved all of HBM up front), code inside allocator hooks or error
// handlers, and embedders whose own allocator owns every device byte.  For
// them this entry point takes every buffer as caller-owned device memory and
// keeps the executor's own working state -- the tile queue, dependency
// counters, node parameters, TMA descriptors and control block -- in one
// fixed array below, which every GPU that loads this library holds from
// module load until process exit.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "dag_internal.h"
#include "dagexec.h"

namespace {

// Fixed working area of dag_run_noalloc on each device: 1 MiB.
constexpr size_t kNoAllocBytes = size_t(1) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
char *g_scratch[kMaxDevices] = {};

// Root buffers are distinct objects to the planner (one writer per element,
// dependency counters per buffer), so caller memory of two roots must not
// share an element.  Each root covers rows of `cols` elements `pitch` apart;
// two roots overlap when some row segment of one meets a row segment of the
// other.  Checked before any device work (and with no device call).
dag_status check_disjoint_roots(const dag_buffer_desc *b, int n, void *const *ptrs, const int64_t *lds) {
  struct Span {
    uint64_t p, end, pitch, width, rows;
    int id;
  };
  std::vector<Span> sp;
  for (int i = 0; i < n; ++i) {
    if (b[i].view_of >= 0 || !ptrs[i] || lds[i] <= 0 || b[i].rows <= 0 || b[i].cols <= 0) continue;
    const uint64_t es = b[i].dtype == DAG_BF16 ? 2 : 4;
    const uint64_t p = (uint64_t)(uintptr_t)ptrs[i], pitch = (uint64_t)lds[i] * es, w = (uint64_t)b[i].cols * es;
    sp.push_back(Span{p, p + (uint64_t)(b[i].rows - 1) * pitch + w, pitch, w, (uint64_t)b[i].rows, i});
  }
  std::sort(sp.begin(), sp.end(), [](const Span &x, const Span &y) { return x.p < y.p; });
  for (size_t a = 0; a < sp.size(); ++a)
    for (size_t c = a + 1; c < sp.size() && sp[c].p < sp[a].end; ++c) {
      const Span &x = sp[a], &y = sp[c];
      bool meet = true;
      if (x.pitch == y.pitch && x.width <= x.pitch && y.width <= y.pitch) {
        // row i of x starts at x.p + i L, row j of y at y.p + j L; with
        // t = (y.p - x.p) + (j - i) L they meet iff -y.width < t < x.width,
        // which only k = j - i = floor(-d / L) or that + 1 can satisfy
        const int64_t L = (int64_t)x.pitch, d = (int64_t)(y.p - x.p);
        const int64_t k0 = -((d + L - 1) / L);
        meet = false;
        for (int64_t k = k0; k <= k0 + 1 && !meet; ++k) {
          if (k < -((int64_t)x.rows - 1) || k > (int64_t)y.rows - 1) continue;
          const int64_t t = d + k * L;
          meet = t > -(int64_t)y.width && t < (int64_t)x.width;
        }
      }
      if (meet) {
        char msg[128];
        snprintf(msg, sizeof msg, "dag_run_noalloc: root buffers %d and %d overlap in device memory",
                 std::min(x.id, y.id), std::max(x.id, y.id));
        return dagx::report_error(DAG_EINVAL, msg);
      }
    }
  return DAG_OK;
}

}  // namespace

extern "C" dag_status dag_run_noalloc(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers,
                                      int n_buffers, void *const *buffer_ptrs, const int64_t *row_pitch,
                                      const dag_options *opts, void *stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n_buffers > 0 && (!buffers || !buffer_ptrs || !row_pitch))
    return dagx::report_error(DAG_EINVAL, "dag_run_noalloc: null buffer, pointer or pitch array");
  if (dag_status s = check_disjoint_roots(buffers, n_buffers, buffer_ptrs, row_pitch)) return s;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: no usable current CUDA device");
  char *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: cudaGetSymbolAddress of the fixed scratch failed");
      g_scratch[dev] = static_cast<char *>(p);
    }
    scratch = g_scratch[dev];
  }
  std::vector<char> blob;
  dagx::ExecParams xp;
  int grid = 0;
  dag_status s = dagx::plan_into_region(nodes, n_nodes, buffers, n_buffers, buffer_ptrs, row_pitch, opts, scratch,
                                        kNoAllocBytes, blob, xp, grid);
  if (s) return s;
  if (xp.n_tiles == 0) return DAG_OK;
  // The copy also clears the counters, flags and control block left by the
  // previous call: they are zero in the blob.
  if (cudaMemcpyAsync(scratch, blob.data(), blob.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      dagx::launch_persistent(xp, grid, stream) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: copy or launch failed");
  if (cudaStreamSynchronize(stream) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: device error during the run");
  dagx::Ctrl c;
  if (cudaMemcpy(&c, xp.ctrl, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess)
    return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: reading the device error word failed");
  if (c.err_code == dagx::E_DEP_TIMEOUT || c.err_code == dagx::E_PIPE_TIMEOUT)
    return dagx::report_error(DAG_ETIMEOUT, "dag_run_noalloc: a device wait ran past its limit");
  if (c.err_code) return dagx::report_error(DAG_EDEVICE, "dag_run_noalloc: device error");
  return DAG_OK;
}
