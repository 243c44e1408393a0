// power.cu -- Algorithm 2 of Sec. 4.B on the device: successive normalised powers
// of A, gamma = min diag (Corollary 6), and the first repeat P_j = P_i, which is
// the relation A^j = q (x) A^i of Lemma 2 / Prop. 7.
//
// Each power step k -> k+1 is four launches on one stream, all of which take
// their operands from a device-resident state, so the same launch sequence is
// valid for every step (no host round trip between steps):
//   1. minplus_gemm (ring mode): R = P_k (x) A, with atomicMin of min R and of
//      min diag R into the state;
//   2. normalise_hash: P_{k+1} = R - mu on finite entries (mu = min R, kept in
//      the int64 offset o_{k+1} = o_k + mu), range check, and an
//      order-independent 64-bit hash of P_{k+1};
//   3. finalize (one warp): offsets, gamma_{k+1} = o_k + min diag R, hash
//      table, list of earlier powers with the same hash;
//   4. compare_resolve: exact comparison of P_{k+1} with each candidate, and
//      (last CTA to arrive) the decision: stop, or advance k.
// Kernels check state->done first and return at once after the stop, so the
// host may enqueue several steps before it looks at the state.
#include <mutex>
#include <vector>

#include "power_dev.cuh"
#include "rd_internal.cuh"

namespace rd {
namespace {

// __global__ wrappers of the bodies in power_dev.cuh (one run per launch).
__global__ void init_state_kernel(PowerState* st, int kmax, int slots) { init_state_body(st, kmax, slots); }

__global__ void reduce_min_diag_kernel(const int16_t* __restrict__ X, int64_t N, int64_t ld, PowerState* st) {
  reduce_min_diag_body(X, N, ld, st);
}

template <bool COPY>
__global__ void normalise_hash_kernel(const int16_t* __restrict__ src, PowerState* st, int16_t* ring,
                                      int64_t slot_elems, int slots, int64_t N, int64_t ld) {
  normalise_hash_body<COPY>(src, st, ring, slot_elems, slots, N, ld);
}

__global__ void finalize_kernel(PowerState* st) { finalize_body(st); }

__global__ void compare_resolve_kernel(PowerState* st, int16_t* ring, int64_t slot_elems, int slots, int64_t N,
                                       int64_t ld) {
  compare_resolve_body(st, ring, slot_elems, slots, N, ld);
}

int reduction_grid() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;
}

cudaError_t enqueue_first(const Run& r, int kmax, cudaStream_t s) {
  init_state_kernel<<<1, 256, 0, s>>>(r.st, kmax, r.slots);
  reduce_min_diag_kernel<<<r.grid, kRedThreads, 0, s>>>(r.A, r.N, r.ld, r.st);
  normalise_hash_kernel<true><<<r.grid, kRedThreads, 0, s>>>(r.A, r.st, r.ring, r.slot_elems, r.slots, r.N, r.ld);
  finalize_kernel<<<1, 32, 0, s>>>(r.st);
  compare_resolve_kernel<<<r.grid, kRedThreads, 0, s>>>(r.st, r.ring, r.slot_elems, r.slots, r.N, r.ld);
  return cudaGetLastError();
}

// One power step: the product (dense or sparse), then normalise/hash, finalize, compare.
cudaError_t enqueue_step(const Run& r, ProductFn product, const void* ctx, cudaStream_t s) {
  cudaError_t e = product(r, ctx, s);
  if (e != cudaSuccess) return e;
  normalise_hash_kernel<false><<<r.grid, kRedThreads, 0, s>>>(nullptr, r.st, r.ring, r.slot_elems, r.slots, r.N,
                                                               r.ld);
  finalize_kernel<<<1, 32, 0, s>>>(r.st);
  compare_resolve_kernel<<<r.grid, kRedThreads, 0, s>>>(r.st, r.ring, r.slot_elems, r.slots, r.N, r.ld);
  return cudaGetLastError();
}

rd_status fail(cudaError_t e) {
  set_cuda_error(e);
  return RD_ERR_CUDA;
}

}  // namespace

// R = P_k (x) A with the DPX GEMM in ring mode.
cudaError_t dense_power_product(const Run& r, const void*, cudaStream_t s) {
  GemmParams p{};
  p.lda = r.ld;
  p.B = r.A;
  p.ldb = r.ld;
  p.ldc = r.ld;
  p.M = r.N;
  p.N = r.N;
  p.K = r.N;
  p.min_out = &r.st->mu;
  p.diag_out = &r.st->dmin;
  p.st = r.st;
  p.ring = r.ring;
  p.slot_elems = r.slot_elems;
  p.slots = r.slots;
  return launch_minplus_gemm(p, true, s);
}

// Algorithm 2 on a validated work area: state header, then the ring of powers.
// No host heap use: the gamma table is copied straight into gamma_host.
rd_status power_search(const int16_t* A_dev, int64_t N, int64_t lda, int kmax, void* work_dev, size_t work_bytes,
                       ProductFn product, const void* ctx, int64_t* gamma_host, int32_t* k_out, int32_t* p_out,
                       int64_t* q_out, cudaStream_t s) {
  const size_t sb = state_bytes(kmax), pb = slot_bytes(N, lda);
  if (work_bytes < sb + 2 * pb) return RD_ERR_NOMEM;
  const size_t slots64 = (work_bytes - sb) / pb;
  Run r{};
  r.st = reinterpret_cast<PowerState*>(work_dev);
  r.ring = reinterpret_cast<int16_t*>(reinterpret_cast<char*>(work_dev) + sb);
  r.slot_elems = (int64_t)(pb / 2);
  r.slots = (int)(slots64 > (size_t)kmax + 1 ? (size_t)kmax + 1 : slots64);
  r.N = N;
  r.ld = lda;
  r.A = A_dev;
  r.grid = reduction_grid();
  cudaError_t e = enqueue_first(r, kmax, s);
  if (e != cudaSuccess) return fail(e);
  // Steps per host check: large products are long enough that one check per
  // step costs nothing; small ones are batched (surplus steps exit at once).
  const int chunk = (N >= 2048) ? 1 : (N >= 512 ? 4 : 16);
  int enqueued = 1;
  PowerState h{};
  for (;;) {
    e = cudaMemcpyAsync(&h, r.st, sizeof(PowerState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    if (h.done || enqueued >= kmax) break;
    const int n = (kmax - enqueued < chunk) ? (kmax - enqueued) : chunk;
    for (int i = 0; i < n; ++i) {
      e = enqueue_step(r, product, ctx, s);
      if (e != cudaSuccess) return fail(e);
    }
    enqueued += n;
  }
  const int last = (h.done == 1) ? h.found_j : h.k;
  e = cudaMemcpyAsync(gamma_host, reinterpret_cast<char*>(work_dev) + kStateHeader + 8 * (size_t)(kmax + 1),
                      8 * (size_t)(kmax + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  for (int k = 0; k <= kmax; ++k)
    if (k < 1 || k > last) gamma_host[k] = RD_GAMMA_UNSET;
  if (h.done == 1) {
    *k_out = h.found_i;
    *p_out = h.found_j - h.found_i;
    *q_out = h.found_q;
    return RD_OK;
  }
  *k_out = 0;
  *p_out = 0;
  *q_out = 0;
  if (h.done == 3) return status_from_err(h.err);
  return RD_NOT_FOUND;
}

}  // namespace rd

using namespace rd;

extern "C" rd_status rd_power_work_bytes(int64_t N, int64_t ld, int kmax, int slots, size_t* bytes) {
  if (N < 1 || ld < N || ld % 8 != 0 || kmax < 1 || slots < 2 || !bytes) return RD_ERR_ARG;
  *bytes = state_bytes(kmax) + (size_t)slots * slot_bytes(N, ld);
  return RD_OK;
}

extern "C" rd_status rd_power_slot(int64_t N, int64_t ld, int kmax, size_t work_bytes, int k, size_t* byte_offset) {
  if (N < 1 || ld < N || ld % 8 != 0 || kmax < 1 || k < 1 || k > kmax || !byte_offset) return RD_ERR_ARG;
  const size_t sb = state_bytes(kmax), pb = slot_bytes(N, ld);
  if (work_bytes < sb + 2 * pb) return RD_ERR_ARG;
  size_t slots = (work_bytes - sb) / pb;
  if (slots > (size_t)kmax + 1) slots = (size_t)kmax + 1;
  *byte_offset = sb + (size_t)(k % slots) * pb;
  return RD_OK;
}

extern "C" rd_status rd_power_until_periodic(const int16_t* A_dev, int64_t N, int64_t lda, int kmax, void* work_dev,
                                             size_t work_bytes, int64_t* gamma_host, int32_t* k_out, int32_t* p_out,
                                             int64_t* q_out, cudaStream_t s) {
  if (!A_dev || !work_dev || !gamma_host || !k_out || !p_out || !q_out) return RD_ERR_ARG;
  if (N < 1 || lda < N || lda % 8 != 0 || kmax < 1 || kmax > (1 << 20)) return RD_ERR_ARG;
  if (!aligned16(A_dev) || (reinterpret_cast<uintptr_t>(work_dev) & 255u) != 0) return RD_ERR_ARG;
  return power_search(A_dev, N, lda, kmax, work_dev, work_bytes, dense_power_product, nullptr, gamma_host, k_out,
                      p_out, q_out, s);
}

// ---------------------------------------------------------------- rd_gamma_R: per-process cache

namespace {
struct Cached {
  bool valid = false;
  bool found = false;
  int k = 0, p = 0, j = 0;
  int64_t q = 0;
  std::vector<int64_t> gamma;
};
std::mutex g_cache_mu;
Cached g_cache[RD_MAX_M + 1];
constexpr int kGammaKmax = 256;

rd_status finish_cached(rd_status rc, const std::vector<int64_t>& g, int32_t k, int32_t p, int64_t q, Cached* out) {
  if (rc != RD_OK && rc != RD_NOT_FOUND) return rc;
  out->valid = true;
  out->found = (rc == RD_OK);
  out->k = k;
  out->p = p;
  out->q = q;
  out->j = out->found ? k + p : kGammaKmax;
  out->gamma = g;
  return RD_OK;
}

rd_status compute_cached(int m, Cached* out) {
  int64_t N = 0, ld = 0;
  if (rd_state_count(m, &N) != RD_OK) return RD_ERR_ARG;
  rd_padded_dim(N, &ld);
  const int slots = (N <= 8192) ? 16 : 8;
  size_t wbytes = 0;
  rd_power_work_bytes(N, ld, kGammaKmax, slots, &wbytes);
  int16_t* A = nullptr;
  void* work = nullptr;
  cudaStream_t s = nullptr;
  rd_status rc = RD_OK;
  std::vector<int64_t> g((size_t)kGammaKmax + 1);
  int32_t k = 0, p = 0;
  int64_t q = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&A, (size_t)N * (size_t)ld * 2);
  if (e == cudaSuccess) e = cudaMalloc(&work, wbytes);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
  }
  if (rc == RD_OK) rc = rd_build_transfer(m, A, ld, s);
  const int split_j = rd_split_default_j(m);
  if (rc == RD_OK && split_j > 0) {
    // the row-split step: A(G) (x) P_k from the row rules, in two passes
    size_t pbytes = 0;
    void* plan = nullptr;
    int16_t* X = nullptr;
    rd_split_info_t info{};
    rc = rd_split_plan_bytes(m, split_j, &pbytes);
    if (rc == RD_OK) e = cudaMalloc(&plan, pbytes);
    if (rc == RD_OK && e == cudaSuccess) rc = rd_split_plan(m, split_j, plan, pbytes, &info, s);
    if (rc == RD_OK && e == cudaSuccess) e = cudaMalloc(&X, (size_t)info.x_rows * (size_t)ld * 2);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
    }
    if (rc == RD_OK)
      rc = rd_power_until_periodic_split(A, ld, &info, plan, X, ld, kGammaKmax, work, wbytes, g.data(), &k, &p, &q, s);
    if (s) cudaStreamSynchronize(s);
    if (plan) cudaFree(plan);
    if (X) cudaFree(X);
    if (A) cudaFree(A);
    if (work) cudaFree(work);
    if (s) cudaStreamDestroy(s);
    return finish_cached(rc, g, k, p, q, out);
  }
  // m = 1: the dense x sparse step (A(G) is sparse, its powers are dense)
  int kR = 2;
  if (rc == RD_OK && N >= 1024) {  // small matrices: any R is a few microseconds
    int best = 0;
    const size_t sb = state_bytes(kGammaKmax);
    rc = rd_sparse_tune(A, ld, N, static_cast<char*>(work) + sb, wbytes - sb, &best, nullptr, s);
    if (rc == RD_OK) kR = best;
  }
  const int64_t nb = (N + kR - 1) / kR;
  int64_t* start = nullptr;
  uint32_t* rec = nullptr;
  int64_t entries = 0;
  if (rc == RD_OK) {
    e = cudaMalloc(&start, (size_t)(nb + 1) * sizeof(int64_t));
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
    }
  }
  if (rc == RD_OK) rc = rd_sparse_count(A, ld, N, N, kR, start, &entries, s);
  if (rc == RD_OK) {
    e = cudaMalloc(&rec, (size_t)(entries > 0 ? entries : 1) * 4 * rd_sparse_record_words(kR));
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
    }
  }
  if (rc == RD_OK) rc = rd_sparse_build(A, ld, N, N, kR, start, rec, s);
  if (rc == RD_OK)
    rc = rd_power_until_periodic_sparse(A, N, ld, kR, start, rec, kGammaKmax, work, wbytes, g.data(), &k, &p, &q, s);
  if (s) cudaStreamSynchronize(s);
  if (start) cudaFree(start);
  if (rec) cudaFree(rec);
  if (A) cudaFree(A);
  if (work) cudaFree(work);
  if (s) cudaStreamDestroy(s);
  return finish_cached(rc, g, k, p, q, out);
}
}  // namespace

extern "C" rd_status rd_gamma_R(int m, int64_t n, int64_t* out) {
  if (m < 1 || m > RD_MAX_M || n < 3 || !out) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  Cached& c = g_cache[m];
  if (!c.valid) {
    const rd_status rc = compute_cached(m, &c);
    if (rc != RD_OK) return rc;
  }
  if (n <= c.j) {
    *out = c.gamma[(size_t)n];
    return RD_OK;
  }
  if (!c.found) return RD_NOT_FOUND;
  const int64_t t = (n - c.k) / c.p;
  *out = c.gamma[(size_t)(c.k + (n - c.k) % c.p)] + c.q * t;
  return RD_OK;
}
