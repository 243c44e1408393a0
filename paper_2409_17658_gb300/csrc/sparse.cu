// sparse.cu -- the dense x sparse power step: C = A (x) B with A sparse.
//
// A(G) is very sparse (at m = 9, 0.55 % of entries are finite, 121 arcs per
// row on average) while its powers are dense.  Since A^k (x) A = A (x) A^k, a
// power step can be computed as R = A (x) P_k: row i of R is the entrywise
// minimum, over the arcs i -> t, of (A[i][t] + row t of P_k).  That is
// N * nnz(A) add-mins instead of N^3.
//
// Block-sparse form of A: the rows are grouped in blocks of R consecutive rows.
// For each block, the entries are the columns t where any of its R rows has a
// finite A[i][t] (sorted); each entry is one record of W(R) 32-bit words:
// {t, w_0, .., w_{R-1}, padding}, w_r = A[b R + r][t] duplicated into both
// halfwords, RD_INF where row b R + r has no arc to t.  The product kernel loads
// row t of B once per entry and applies it to all R rows, so B is read
// nnz/(reuse) times instead of nnz times; RD_INF weights cannot lower a minimum
// (INF + b >= INF >= acc), so the kernel needs no branch per row.  Consecutive
// words share many successors (R = 4 reads B 1.8x less often, R = 8 2.6x), at
// the price of R - popcount wasted DPX operations per entry.
//
// The product is bound by the SM's load path (L1/LSU), so the kernel keeps it
// for B: a CTA stages chunks of records in shared memory with coalesced loads,
// and each thread owns 16 columns (two 16-byte loads per B row), which halves
// the per-entry bookkeeping per byte of B.
#include "rd_internal.cuh"
#include "sparse_tile.cuh"

namespace rd {
namespace {

// One warp per block of R rows: number of columns where some row of the block is finite.
template <int R>
__global__ void sparse_count_kernel(const int16_t* __restrict__ A, int64_t lda, int64_t M, int64_t K, int64_t nb,
                                    int64_t* __restrict__ cnt) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;
  int64_t total = 0;
  for (int64_t c0 = 0; c0 < K; c0 += 256) {
    const int64_t col = c0 + lane * 8;
    uint32_t any = 0;
    if (col < K) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t row = b * R + r;
        if (row < M) any |= finite_mask(*reinterpret_cast<const uint4*>(A + row * lda + col));
      }
      if (col + 8 > K) any &= (1u << (K - col)) - 1u;
    }
    total += __popc(any);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xFFFFFFFFu, total, o);
  if (lane == 0) cnt[b] = total;
}

// In-place exclusive scan of v[0..n) by one CTA; v[n] receives the total.
__global__ void exclusive_scan_kernel(int64_t* v, int64_t n) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = (i < n) ? v[i] : 0;
    int64_t y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) y += t;
    }
    if (lane == 31) warp_sums[warp] = y;
    __syncthreads();
    if (warp == 0) {
      int64_t ws = (lane < nwarps) ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xFFFFFFFFu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < nwarps) warp_sums[lane] = ws;
    }
    __syncthreads();
    const int64_t incl = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + y;
    if (i < n) v[i] = incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) v[n] = carry;
}

// One warp per block: the sorted columns and their R-vectors of duplicated weights, as records.
template <int R>
__global__ void sparse_build_kernel(const int16_t* __restrict__ A, int64_t lda, int64_t M, int64_t K, int64_t nb,
                                    const int64_t* __restrict__ start, uint32_t* __restrict__ rec) {
  constexpr int W = record_words(R);
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;
  int64_t pos = start[b];
  const uint4 inf4 = make_uint4(kInf2, kInf2, kInf2, kInf2);
  for (int64_t c0 = 0; c0 < K; c0 += 256) {
    const int64_t col = c0 + lane * 8;
    uint4 v[R];
    uint32_t any = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = b * R + r;
      v[r] = (col < K && row < M) ? *reinterpret_cast<const uint4*>(A + row * lda + col) : inf4;
      any |= finite_mask(v[r]);
    }
    if (col >= K) any = 0;
    else if (col + 8 > K) any &= (1u << (K - col)) - 1u;
    const int cnt = __popc(any);
    int excl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xFFFFFFFFu, excl, o);
      if (lane >= o) excl += t;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, excl, 31);
    excl -= cnt;
    int64_t p = pos + excl;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if ((any >> e) & 1u) {
        uint32_t* out = rec + p * W;
        out[0] = (uint32_t)(col + e);
#pragma unroll
        for (int r = 0; r < R; ++r) out[1 + r] = half_of(v[r], e) * 0x00010001u;
#pragma unroll
        for (int q = 1 + R; q < W; ++q) out[q] = 0u;
        ++p;
      }
    }
    pos += total;
  }
}

template <int R, bool RING>
__global__ void __launch_bounds__(128) sparse_minplus_kernel(SparseArgs a) {
  const int16_t* B = a.B;
  int16_t* C = a.C;
  if (RING) {
    if (*(volatile const int32_t*)&a.st->done) return;
    const int k = *(volatile const int32_t*)&a.st->k;
    B = a.ring + (int64_t)(k % a.slots) * a.slot_elems;
    C = a.ring + (int64_t)((k + 1) % a.slots) * a.slot_elems;
  }
  sparse_tile_body<R>(a, B, C, blockIdx.x, blockIdx.y);
}

template <int R, bool RING>
__global__ void __launch_bounds__(kTmaThreads) sparse_tma_kernel(SparseArgs a, int32_t* err_plain, uint32_t wait_limit,
                                                                  int stop_at) {
  const int16_t* B = a.B;
  int16_t* C = a.C;
  int32_t* err = err_plain;
  if (RING) {
    if (*(volatile const int32_t*)&a.st->done) return;
    const int k = *(volatile const int32_t*)&a.st->k;
    B = a.ring + (int64_t)(k % a.slots) * a.slot_elems;
    C = a.ring + (int64_t)((k + 1) % a.slots) * a.slot_elems;
    err = &a.st->err;
  }
  if (*(volatile const int32_t*)err & kErrTimeout) return;  // an earlier CTA gave up: the launch is void
  sparse_tma_tile_body<R>(a, B, C, blockIdx.x, blockIdx.y, err, wait_limit, stop_at);
}

template <bool RING>
cudaError_t launch_sparse_tma(int R, const SparseArgs& a, int32_t* err, cudaStream_t s, uint32_t wait_limit = kWaitLimit,
                              int stop_at = -1) {
  const int64_t nb = (a.M + R - 1) / R;
  const int64_t gy = (a.Ncols + kSlabCols - 1) / kSlabCols;
  if (nb <= 0 || gy <= 0) return cudaSuccess;
  if (nb > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nb, (unsigned)gy);
  switch (R) {
    case 1: sparse_tma_kernel<1, RING><<<grid, kTmaThreads, kTmaSmemBytes, s>>>(a, err, wait_limit, stop_at); break;
    case 2: sparse_tma_kernel<2, RING><<<grid, kTmaThreads, kTmaSmemBytes, s>>>(a, err, wait_limit, stop_at); break;
    case 4: sparse_tma_kernel<4, RING><<<grid, kTmaThreads, kTmaSmemBytes, s>>>(a, err, wait_limit, stop_at); break;
    case 8: sparse_tma_kernel<8, RING><<<grid, kTmaThreads, kTmaSmemBytes, s>>>(a, err, wait_limit, stop_at); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool RING>
cudaError_t launch_sparse(int R, const SparseArgs& a, cudaStream_t s) {
  const int64_t nb = (a.M + R - 1) / R;
  // 128 threads x 16 columns: measured best on GB300 at m = 9 and m = 10 (32, 64 and 256 are
  // slower) -- a wider CTA spreads each staged entry record over more columns
  const int threads = 128;
  const int64_t gy = (a.Ncols + threads * 16 - 1) / (threads * 16);
  if (nb <= 0 || gy <= 0) return cudaSuccess;
  if (nb > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nb, (unsigned)gy);
  switch (R) {
    case 1: sparse_minplus_kernel<1, RING><<<grid, threads, 0, s>>>(a); break;
    case 2: sparse_minplus_kernel<2, RING><<<grid, threads, 0, s>>>(a); break;
    case 4: sparse_minplus_kernel<4, RING><<<grid, threads, 0, s>>>(a); break;
    case 8: sparse_minplus_kernel<8, RING><<<grid, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

struct SparsePlan {
  int R;
  const int64_t* start;
  const uint32_t* rec;
};

cudaError_t sparse_power_product(const Run& r, const void* ctx, cudaStream_t s) {
  const SparsePlan* pl = static_cast<const SparsePlan*>(ctx);
  SparseArgs a{};
  a.M = r.N;
  a.start = pl->start;
  a.rec = pl->rec;
  a.ldb = r.ld;
  a.ldc = r.ld;
  a.Ncols = r.N;
  a.min_out = &r.st->mu;
  a.diag_out = &r.st->dmin;
  a.st = r.st;
  a.ring = r.ring;
  a.slot_elems = r.slot_elems;
  a.slots = r.slots;
  return launch_sparse<true>(pl->R, a, s);
}

bool valid_r(int R) { return R == 1 || R == 2 || R == 4 || R == 8; }

rd_status cuda_fail(cudaError_t e) {
  set_cuda_error(e);
  return RD_ERR_CUDA;
}

}  // namespace
}  // namespace rd

using namespace rd;

extern "C" rd_status rd_sparse_count(const int16_t* A, int64_t lda, int64_t M, int64_t K, int R,
                                     int64_t* block_start_dev, int64_t* entries_host, cudaStream_t s) {
  if (!A || !block_start_dev || !entries_host || M < 1 || K < 1 || !valid_r(R)) return RD_ERR_ARG;
  if (lda < K || lda % 8 != 0 || !aligned16(A)) return RD_ERR_ARG;
  const int64_t nb = (M + R - 1) / R;
  const int warps_per_cta = 8;
  const int64_t ctas = (nb + warps_per_cta - 1) / warps_per_cta;
  if (ctas > 0x7FFFFFFF) return RD_ERR_ARG;
  switch (R) {
    case 1: sparse_count_kernel<1><<<(unsigned)ctas, 32 * warps_per_cta, 0, s>>>(A, lda, M, K, nb, block_start_dev); break;
    case 2: sparse_count_kernel<2><<<(unsigned)ctas, 32 * warps_per_cta, 0, s>>>(A, lda, M, K, nb, block_start_dev); break;
    case 4: sparse_count_kernel<4><<<(unsigned)ctas, 32 * warps_per_cta, 0, s>>>(A, lda, M, K, nb, block_start_dev); break;
    default: sparse_count_kernel<8><<<(unsigned)ctas, 32 * warps_per_cta, 0, s>>>(A, lda, M, K, nb, block_start_dev); break;
  }
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(block_start_dev, nb);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(entries_host, block_start_dev + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  return RD_OK;
}

extern "C" int rd_sparse_record_words(int R) { return valid_r(R) ? record_words(R) : 0; }

extern "C" rd_status rd_sparse_build(const int16_t* A, int64_t lda, int64_t M, int64_t K, int R,
                                     const int64_t* block_start_dev, uint32_t* records_dev, cudaStream_t s) {
  if (!A || !block_start_dev || !records_dev || M < 1 || K < 1 || !valid_r(R)) return RD_ERR_ARG;
  if (lda < K || lda % 8 != 0 || !aligned16(A) || !aligned16(records_dev) || K > 0xFFFFFFFFll) return RD_ERR_ARG;
  const int64_t nb = (M + R - 1) / R;
  const int warps_per_cta = 8;
  const int64_t ctas = (nb + warps_per_cta - 1) / warps_per_cta;
  if (ctas > 0x7FFFFFFF) return RD_ERR_ARG;
  const unsigned g = (unsigned)ctas, t = 32 * warps_per_cta;
  switch (R) {
    case 1: sparse_build_kernel<1><<<g, t, 0, s>>>(A, lda, M, K, nb, block_start_dev, records_dev); break;
    case 2: sparse_build_kernel<2><<<g, t, 0, s>>>(A, lda, M, K, nb, block_start_dev, records_dev); break;
    case 4: sparse_build_kernel<4><<<g, t, 0, s>>>(A, lda, M, K, nb, block_start_dev, records_dev); break;
    default: sparse_build_kernel<8><<<g, t, 0, s>>>(A, lda, M, K, nb, block_start_dev, records_dev); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  return RD_OK;
}

extern "C" rd_status rd_sparse_minplus(int R, int64_t M, const int64_t* block_start, const uint32_t* records,
                                       const int16_t* B, int64_t ldb, int64_t N, int16_t* C, int64_t ldc,
                                       int32_t* min_out, cudaStream_t s) {
  if (!valid_r(R) || M < 0 || N < 0) return RD_ERR_ARG;
  if (M > 0 && N > 0) {
    if (!block_start || !records || !B || !C) return RD_ERR_ARG;
    if (!aligned16(B) || !aligned16(C) || !aligned16(records) || ldb < N || ldb % 8 != 0 || ldc < N ||
        ldc % 8 != 0)
      return RD_ERR_ARG;
  }
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (M == 0 || N == 0) return RD_OK;
  SparseArgs a{};
  a.M = M;
  a.start = block_start;
  a.rec = records;
  a.B = B;
  a.ldb = ldb;
  a.C = C;
  a.ldc = ldc;
  a.Ncols = N;
  a.min_out = min_out;
  e = launch_sparse<false>(R, a, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return RD_OK;
}

extern "C" rd_status rd_sparse_minplus_tma_bounded(int R, int64_t M, const int64_t* block_start,
                                                   const uint32_t* records, const int16_t* B, int64_t ldb, int64_t N,
                                                   int16_t* C, int64_t ldc, int32_t* min_out, int32_t* err_dev,
                                                   uint32_t wait_limit, int32_t stop_at, cudaStream_t s) {
  if (!valid_r(R) || M < 0 || N < 0 || !err_dev) return RD_ERR_ARG;
  if (wait_limit < 1 || stop_at < -1) return RD_ERR_ARG;
  if (M > 0 && N > 0) {
    if (!block_start || !records || !B || !C) return RD_ERR_ARG;
    if (!aligned16(B) || !aligned16(C) || !aligned16(records) || ldb < N || ldb % 8 != 0 || ldc < N ||
        ldc % 8 != 0)
      return RD_ERR_ARG;
  }
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (M == 0 || N == 0) return RD_OK;
  SparseArgs a{};
  a.M = M;
  a.start = block_start;
  a.rec = records;
  a.B = B;
  a.ldb = ldb;
  a.C = C;
  a.ldc = ldc;
  a.Ncols = N;
  a.min_out = min_out;
  e = launch_sparse_tma<false>(R, a, err_dev, s, wait_limit, stop_at);
  if (e != cudaSuccess) return cuda_fail(e);
  return RD_OK;
}

extern "C" rd_status rd_sparse_minplus_tma(int R, int64_t M, const int64_t* block_start, const uint32_t* records,
                                           const int16_t* B, int64_t ldb, int64_t N, int16_t* C, int64_t ldc,
                                           int32_t* min_out, int32_t* err_dev, cudaStream_t s) {
  return rd_sparse_minplus_tma_bounded(R, M, block_start, records, B, ldb, N, C, ldc, min_out, err_dev, kWaitLimit, -1,
                                       s);
}

extern "C" rd_status rd_power_until_periodic_sparse(const int16_t* A_dev, int64_t N, int64_t lda, int R,
                                                    const int64_t* block_start, const uint32_t* records, int kmax,
                                                    void* work_dev, size_t work_bytes, int64_t* gamma_host,
                                                    int32_t* k_out, int32_t* p_out, int64_t* q_out, cudaStream_t s) {
  if (!A_dev || !block_start || !records || !work_dev || !gamma_host || !k_out || !p_out || !q_out) return RD_ERR_ARG;
  if (N < 1 || lda < N || lda % 8 != 0 || kmax < 1 || kmax > (1 << 20) || !valid_r(R)) return RD_ERR_ARG;
  if (!aligned16(A_dev) || !aligned16(records) || (reinterpret_cast<uintptr_t>(work_dev) & 255u) != 0)
    return RD_ERR_ARG;
  const SparsePlan plan{R, block_start, records};
  return power_search(A_dev, N, lda, kmax, work_dev, work_bytes, sparse_power_product, &plan, gamma_host, k_out,
                      p_out, q_out, s);
}

// ---------------------------------------------------------------- autotuner for R

extern "C" rd_status rd_sparse_tune(const int16_t* A, int64_t lda, int64_t N, void* scratch_dev, size_t scratch_bytes,
                                    int* best_R, float* ms_per_R, cudaStream_t s) {
  if (!A || !scratch_dev || !best_R || N < 1 || lda < N || lda % 8 != 0 || !aligned16(A)) return RD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(scratch_dev) & 255u) != 0) return RD_ERR_ARG;
  const size_t out_bytes = round_up((size_t)N * (size_t)lda * 2, 256);
  if (scratch_bytes < out_bytes + 4096) return RD_ERR_NOMEM;
  char* base = static_cast<char*>(scratch_dev);
  int16_t* C = reinterpret_cast<int16_t*>(base);
  char* plan_base = base + out_bytes;
  const size_t plan_room = scratch_bytes - out_bytes;
  const int cands[4] = {1, 2, 4, 8};
  float best_ms = -1.f;
  int best = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e);
  rd_status rc = RD_OK;
  for (int ci = 0; ci < 4 && rc == RD_OK; ++ci) {
    const int R = cands[ci];
    if (ms_per_R) ms_per_R[ci] = -1.f;
    const int64_t nb = (N + R - 1) / R;
    const size_t start_bytes = round_up((size_t)(nb + 1) * 8, 256);
    if (start_bytes > plan_room) continue;
    int64_t* start = reinterpret_cast<int64_t*>(plan_base);
    int64_t entries = 0;
    rc = rd_sparse_count(A, lda, N, N, R, start, &entries, s);
    if (rc != RD_OK) break;
    const size_t rec_bytes = round_up((size_t)entries * 4 * record_words(R), 256);
    if (start_bytes + rec_bytes > plan_room) continue;  // this candidate does not fit: skipped
    uint32_t* rec = reinterpret_cast<uint32_t*>(plan_base + start_bytes);
    rc = rd_sparse_build(A, lda, N, N, R, start, rec, s);
    if (rc != RD_OK) break;
    // A (x) A moves the same bytes and does the same DPX work as A (x) P_k.
    rc = rd_sparse_minplus(R, N, start, rec, A, lda, N, C, lda, nullptr, s);  // warm-up
    if (rc != RD_OK) break;
    e = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      rc = rd_sparse_minplus(R, N, start, rec, A, lda, N, C, lda, nullptr, s);
      if (rc != RD_OK) break;
    }
    if (rc != RD_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    ms /= 3.f;
    if (ms_per_R) ms_per_R[ci] = ms;
    if (best == 0 || ms < best_ms) {
      best = R;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RD_OK) return rc;
  if (best == 0) return RD_ERR_NOMEM;
  *best_R = best;
  rd_tune_entry_t t{};
  t.mode = RD_TUNE_SPARSE_R;
  t.key = rd_tune_bucket(N);
  t.p[0] = best;
  t.ms = best_ms;
  tune_put(t);  // a full table keeps its entries; the caller still has *best_R
  return RD_OK;
}
