// psq_compute_noalloc: psq_compute on a fixed-size device scratch array that lives in this
// file, for callers that cannot allocate device memory themselves (see include/psq.h).
#include <mutex>

#include "psq_internal.h"

namespace {

// File-scope device scratch.  Every device that loads this library holds it until the process
// exits.  In host code the symbol is only a host-side stand-in: its device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static __device__ __align__(256) unsigned char g_scratch[PSQ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

psq_status psq::noalloc_scratch(void** ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return psq::set_error(PSQ_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return psq::set_error(PSQ_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
    if (e != cudaSuccess) {
      g_addr[dev] = nullptr;
      return psq::set_error(PSQ_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  *ptr = g_addr[dev];
  return PSQ_OK;
}

extern "C" psq_status psq_compute_noalloc(psq_job* job, unsigned mask, double* d_out[5], void* stream) {
  if (!job) return psq::set_error(PSQ_ERR_ARG, "job is NULL");
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return psq::set_error(PSQ_ERR_CUDA, cudaGetErrorString(e));
  // the scratch address is per device: the job's device must be the current one
  if (dev != psq::job_device(job)) return psq::set_error(PSQ_ERR_ARG, "the current device is not the job's device");
  void* ptr = nullptr;
  const psq_status st = psq::noalloc_scratch(&ptr);
  if (st != PSQ_OK) return st;
  return psq::compute_on(job, mask, ptr, PSQ_NOALLOC_SCRATCH_BYTES, d_out, stream, true);
}
