// host_io.cu -- the (min,+) product for operands that live in host memory.
//
// rd_minplus_gemm_host stages A and B into the caller's device buffer, runs the
// same product as rd_minplus_gemm, and copies C back, all enqueued on one stream.
// A caller that alternates two streams and two staging buffers overlaps the
// copies of one product with the arithmetic of the other.
#include <cuda_runtime.h>

#include "rd_internal.cuh"

namespace rd {
namespace {

struct HostLayout {
  int64_t ldk, ldn;  // device leading dimensions of A (K columns) and of B, C (N columns)
  size_t a_off, b_off, c_off, bytes;
};

bool host_layout(int64_t M, int64_t N, int64_t K, HostLayout* L) {
  if (M < 0 || N < 0 || K < 0) return false;
  if (M > ((int64_t)1 << 31) || N > ((int64_t)1 << 31) || K > ((int64_t)1 << 31)) return false;
  L->ldk = (K + 7) / 8 * 8;
  L->ldn = (N + 7) / 8 * 8;
  L->a_off = 0;
  L->b_off = round_up((size_t)M * (size_t)L->ldk * 2, 256);
  L->c_off = L->b_off + round_up((size_t)K * (size_t)L->ldn * 2, 256);
  L->bytes = L->c_off + round_up((size_t)M * (size_t)L->ldn * 2, 256);
  return true;
}

}  // namespace
}  // namespace rd

using namespace rd;

extern "C" rd_status rd_minplus_gemm_host_work_bytes(int64_t M, int64_t N, int64_t K, size_t* bytes) {
  HostLayout L;
  if (!bytes || !host_layout(M, N, K, &L)) return RD_ERR_ARG;
  *bytes = L.bytes;
  return RD_OK;
}

extern "C" rd_status rd_minplus_gemm_host(const int16_t* A_host, int64_t lda, const int16_t* B_host, int64_t ldb,
                                          int16_t* C_host, int64_t ldc, int64_t M, int64_t N, int64_t K,
                                          void* work_dev, size_t work_bytes, int32_t* min_out, cudaStream_t s) {
  HostLayout L;
  if (!host_layout(M, N, K, &L)) return RD_ERR_ARG;
  if (M > 0 && N > 0) {
    if (!C_host || ldc < N) return RD_ERR_ARG;
    if (K > 0 && (!A_host || !B_host || lda < K || ldb < N)) return RD_ERR_ARG;
    if (!work_dev || (reinterpret_cast<uintptr_t>(work_dev) & 255u) != 0) return RD_ERR_ARG;
    if (work_bytes < L.bytes) return RD_ERR_NOMEM;
  }
  if (M == 0 || N == 0) return rd_minplus_gemm(nullptr, 8, nullptr, 8, nullptr, 8, M, N, K, min_out, s);
  char* w = static_cast<char*>(work_dev);
  int16_t* A = reinterpret_cast<int16_t*>(w + L.a_off);
  int16_t* B = reinterpret_cast<int16_t*>(w + L.b_off);
  int16_t* C = reinterpret_cast<int16_t*>(w + L.c_off);
  cudaError_t e = cudaSuccess;
  if (K > 0) {
    e = cudaMemcpy2DAsync(A, (size_t)L.ldk * 2, A_host, (size_t)lda * 2, (size_t)K * 2, (size_t)M,
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(B, (size_t)L.ldn * 2, B_host, (size_t)ldb * 2, (size_t)N * 2, (size_t)K,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return RD_ERR_CUDA;
    }
  }
  const rd_status st = rd_minplus_gemm(A, L.ldk, B, L.ldn, C, L.ldn, M, N, K, min_out, s);
  if (st != RD_OK) return st;
  e = cudaMemcpy2DAsync(C_host, (size_t)ldc * 2, C, (size_t)L.ldn * 2, (size_t)N * 2, (size_t)M,
                        cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return RD_ERR_CUDA;
  }
  return RD_OK;
}
