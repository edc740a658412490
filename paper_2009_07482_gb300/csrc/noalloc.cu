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

}  // namespace

extern "C" dag_status dag_run_noalloc(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers,
                                      int n_buffers, void *const *buffer_ptrs, const int64_t *row_pitch,
                                      const dag_options *opts, void *stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
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
