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
// array's name only stands for the device symbol, so the address has to be
// looked up once per device, with that device current.
cudaError_t noalloc_scratch(void** ptr, size_t* bytes) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *ptr = g_addr[dev];
  *bytes = QF_NOALLOC_MAX_BYTES;
  return cudaSuccess;
}

}  // namespace qf
