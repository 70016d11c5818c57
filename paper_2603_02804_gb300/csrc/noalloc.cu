// Fixed device scratch for qf_train_step_noalloc.
//
// Callers that cannot allocate device memory (no cudaMalloc, no caching
// allocator) still need somewhere to keep the state buffers, checkpoints and
// gradient partials of a training step. This file reserves one fixed block
// for them: a file-scope __device__ array that the driver places in device
// memory when the library's device code is loaded on a GPU, and that stays
// there until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "qfuse.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QF_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

namespace qf {

// Device address of the scratch on the current device. In host code the
// array's name only stands for the device symbol, so the address is looked up
// with cudaGetSymbolAddress while that device is current. The lookup runs on
// every call made outside a stream capture: after a cudaDeviceReset the
// module is loaded again and the old address is no longer valid. A call made
// during a capture may not trigger a module load, so it uses the address that
// the last uncaptured call on this device cached, and fails without one.
cudaError_t noalloc_scratch(cudaStream_t st, void** ptr, size_t* bytes) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  } else if (!g_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *ptr = g_addr[dev];
  *bytes = QF_NOALLOC_MAX_BYTES;
  return cudaSuccess;
}

}  // namespace qf
