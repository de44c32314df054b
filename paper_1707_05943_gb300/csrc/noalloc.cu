// noalloc.cu -- fdtd_march_noalloc: the FP64 march for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// a host framework that owns all device memory through its own pool and bans
// other allocations, or a plugin loaded into such a process, which may use
// only the buffers the host hands it.  Those callers can still pass their own
// input and output buffers, but not the march's scratch: the ring of D+2 rows,
// the boundary tables, the norm partials and the barrier words.  The call
// synchronises its stream before it returns (to report device-side errors),
// so it is a plain blocking call, not something to record into a graph.
//
// Here that scratch is one file-scope __device__ array of kScratchBytes.  The
// CUDA runtime places it when the module is loaded, so every GPU that loads
// this library holds it until the process exits.  Host code cannot use the
// array's name as a device address (it names a host-side shadow); the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on it.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "fdtd_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_scratch on the current device (set-up on first use)
fdtd_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return FDTD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) return FDTD_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return FDTD_OK;
}

}  // namespace

extern "C" {

size_t fdtd_noalloc_max_bytes(void) { return kScratchBytes; }

fdtd_status fdtd_march_noalloc(const fdtd_params* p, void* cuda_stream, void* row_out, double* norms_out) {
  if (!p || !row_out || !norms_out) return FDTD_ERR_INVALID_ARG;
  if (p->struct_size != sizeof(fdtd_params)) return FDTD_ERR_INVALID_ARG;
  if (p->precision != FDTD_F64) return FDTD_ERR_UNSUPPORTED;
  // no snapshots: nothing would read them, and they would only take scratch
  fdtd_params q = *p;
  q.tstep = -1;
  q.max_probes = 0;
  fdtd_plan_s plan;
  plan.record_errors = false;
  size_t need = 0;
  fdtd_status st = fdtd_plan_fill(&plan, &q, 1, cuda_stream, &need);
  if (st != FDTD_OK) return st;
  if (need > kScratchBytes) return FDTD_ERR_WORKSPACE;  // larger than the built-in scratch
  void* scratch = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FDTD_ERR_CUDA;
  st = scratch_address(dev, &scratch);
  if (st != FDTD_OK) return st;
  cudaStream_t s = plan.stream;
  // bind, build the boundary (which zeroes the ring, norms and barrier words
  // left by the previous call), march every row
  st = fdtd_bind_workspace(&plan, scratch, kScratchBytes);
  if (st == FDTD_OK) st = fdtd_set_boundary(&plan, FDTD_BOUNDARY_ANALYTIC, nullptr, 0);
  if (st == FDTD_OK) st = fdtd_march(&plan, q.nt);
  if (st != FDTD_OK) {
    // work queued before the failure may still be running on the shared array:
    // let it finish, so that a caller who retries at once does not overlap it
    cudaStreamSynchronize(s);
    return st;
  }
  // outputs: the last row and the per-row norms, copied device to device
  const char* ws = static_cast<const char*>(scratch);
  const size_t row_bytes = plan.elem * (size_t)q.nx;
  const char* last = ws + plan.off_ring + plan.elem * (size_t)((plan.rows_done - 1) % plan.R) * plan.stride;
  cudaError_t e = cudaMemcpyAsync(row_out, last, row_bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(norms_out, ws + plan.off_norms, sizeof(double) * (size_t)q.nt, cudaMemcpyDeviceToDevice, s);
  cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return FDTD_ERR_CUDA;
  fdtd::SyncWords sw;
  e = cudaMemcpy(&sw, ws + plan.off_sync, sizeof sw, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return FDTD_ERR_CUDA;
  if (sw.status != 0) return (fdtd_status)sw.status;
  return FDTD_OK;
}

}  // extern "C"
