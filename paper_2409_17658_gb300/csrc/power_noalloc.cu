// power_noalloc.cu -- rd_power_until_periodic_noalloc: the period search for
// callers that cannot allocate device memory themselves.
//
// The scratch is one file-scope array in this translation unit's own module,
// so it is only reserved on a device once this module is loaded there, and it
// is then held until the process exits.  Host code never passes the array's
// name to a kernel (in host code that name is a host-side stand-in, not a
// device address); it resolves the device address once per device with
// cudaGetSymbolAddress and passes that.
#include <mutex>

#include "rd_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, resolved on first use per device.
rd_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    rd::set_cuda_error(e);
    return RD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_dev[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      rd::set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      return RD_ERR_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return RD_OK;
}

}  // namespace

extern "C" rd_status rd_power_until_periodic_noalloc(const int16_t* A_dev, int64_t N, int64_t lda, int kmax,
                                                     int64_t* gamma_host, int32_t* k_out, int32_t* p_out,
                                                     int64_t* q_out, cudaStream_t s) {
  if (!A_dev || !gamma_host || !k_out || !p_out || !q_out) return RD_ERR_ARG;
  if (N < 1 || lda < N || lda % 8 != 0 || kmax < 1 || kmax > (1 << 20)) return RD_ERR_ARG;
  if (!rd::aligned16(A_dev)) return RD_ERR_ARG;
  size_t need = 0;
  if (rd_power_work_bytes(N, lda, kmax, 2, &need) != RD_OK) return RD_ERR_ARG;
  if (need > (size_t)RD_NOALLOC_SCRATCH_BYTES) return RD_ERR_NOMEM;  // beyond the static maximum
  void* scratch = nullptr;
  const rd_status rc = scratch_address(&scratch);
  if (rc != RD_OK) return rc;
  return rd::power_search(A_dev, N, lda, kmax, scratch, (size_t)RD_NOALLOC_SCRATCH_BYTES, rd::dense_power_product,
                          nullptr, gamma_host, k_out, p_out, q_out, s, false, false);
}
