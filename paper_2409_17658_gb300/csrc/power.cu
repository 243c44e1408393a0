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

#include "rd_internal.cuh"

namespace rd {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // splitmix64 finaliser (Steele, Lea and Flood, 2014)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Hash of one entry at (i, j) with value v; the matrix hash is the wrapping sum
// over all entries, so it does not depend on the order of the reduction.
__device__ __forceinline__ unsigned long long entry_hash(int64_t i, int64_t j, uint32_t v) {
  return mix64(((unsigned long long)i << 32) ^ ((unsigned long long)j << 15) ^ (unsigned long long)v);
}

template <typename T>
__device__ __forceinline__ T block_reduce_min(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T r = sh[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = min(r, sh[w]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long block_reduce_sum(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

__global__ void init_state_kernel(PowerState* st, int kmax, int slots) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->k = 0;
    st->done = 0;
    st->err = 0;
    st->kmax = kmax;
    st->mu = kInf;
    st->dmin = kInf;
    st->blocks_done = 0;
    st->ncand = 0;
    for (int c = 0; c < kMaxCand; ++c) {
      st->cand[c] = 0;
      st->mismatch[c] = 0;
    }
    st->found_i = 0;
    st->found_j = 0;
    st->found_q = 0;
    st->hacc = 0;
    st->range_bad = 0;
    st->slots = slots;
  }
  int64_t* off = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(st) + kStateHeader);
  int64_t* gam = off + (kmax + 1);
  unsigned long long* h = reinterpret_cast<unsigned long long*>(gam + (kmax + 1));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= kmax; i += gridDim.x * blockDim.x) {
    off[i] = 0;
    gam[i] = RD_GAMMA_UNSET;
    h[i] = 0;
  }
}

// min over the N x N matrix and over its diagonal (the k = 1 step has no product epilogue).
__global__ void reduce_min_diag_kernel(const int16_t* __restrict__ X, int64_t N, int64_t ld, PowerState* st) {
  __shared__ int32_t sh[kRedThreads / 32];
  const int64_t chunks_per_row = (N + 7) / 8, total = N * chunks_per_row;
  int32_t lm = kInf, ld_min = kInf;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = c / chunks_per_row, j0 = (c % chunks_per_row) * 8;
    const uint4 v = *reinterpret_cast<const uint4*>(X + i * ld + j0);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (j0 + e >= N) break;
      const int32_t x = (int32_t)(int16_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
      lm = min(lm, x);
      if (j0 + e == i) ld_min = min(ld_min, x);
    }
  }
  lm = block_reduce_min(lm, sh);
  ld_min = block_reduce_min(ld_min, sh);
  if (threadIdx.x == 0) {
    if (lm < kInf) atomicMin(&st->mu, lm);
    if (ld_min < kInf) atomicMin(&st->dmin, ld_min);
  }
}

// P_{k+1} = R - mu on finite entries (in place, or copied from `src` for k + 1 = 1), its hash,
// and the range check that keeps int16 exact.
template <bool COPY>
__global__ void normalise_hash_kernel(const int16_t* __restrict__ src, PowerState* st, int16_t* ring,
                                      int64_t slot_elems, int slots, int64_t N, int64_t ld) {
  __shared__ unsigned long long shh[kRedThreads / 32];
  if (*(volatile const int32_t*)&st->done) return;
  const int kn = *(volatile const int32_t*)&st->k + 1;
  int16_t* dst = ring + (int64_t)(kn % slots) * slot_elems;
  const int16_t* s = COPY ? src : dst;
  const int32_t mu_raw = *(volatile const int32_t*)&st->mu;
  const int32_t mu = (mu_raw >= kInf) ? 0 : mu_raw;
  const int64_t chunks_per_row = (N + 7) / 8, total = N * chunks_per_row;
  unsigned long long h = 0;
  int bad = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = c / chunks_per_row, j0 = (c % chunks_per_row) * 8;
    const uint4 v = *reinterpret_cast<const uint4*>(s + i * ld + j0);
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (j0 + e >= N) break;
      const int sh = 16 * (e & 1);
      int32_t x = (int32_t)(int16_t)((w[e >> 1] >> sh) & 0xFFFF);
      if (COPY) bad |= (x != kInf) && (x < 0 || x > kMaxFinite);  // the operand contract
      if (x != kInf) {
        x -= mu;
        bad |= (x < 0 || x > kMaxFinite);
      }
      w[e >> 1] = (w[e >> 1] & ~(0xFFFFu << sh)) | ((uint32_t)(x & 0xFFFF) << sh);
      h += entry_hash(i, j0 + e, (uint32_t)(x & 0xFFFF));
    }
    *reinterpret_cast<uint4*>(dst + i * ld + j0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  h = block_reduce_sum(h, shh);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    atomicAdd(&st->hacc, h);
    if (bad) atomicOr(&st->range_bad, 1);
  }
}

// One warp: bookkeeping of power kn = k + 1 and the list of hash matches.
__global__ void finalize_kernel(PowerState* st) {
  if (*(volatile const int32_t*)&st->done) return;
  const int kn = st->k + 1;
  int64_t* off = st_offset(st);
  int64_t* gam = st_gamma(st);
  unsigned long long* hs = st_hash(st);
  const unsigned long long hk = st->hacc;
  if (threadIdx.x == 0) {
    const int32_t mu = (st->mu >= kInf) ? 0 : st->mu;
    off[kn] = off[kn - 1] + mu;
    gam[kn] = (st->dmin >= kInf) ? RD_GAMMA_INF : off[kn - 1] + st->dmin;
    hs[kn] = hk;
    if (st->range_bad) {
      st->err |= 1;
      st->done = 3;
    }
  }
  __syncwarp();
  if (st->range_bad) return;
  for (int i = 1 + (int)threadIdx.x; i < kn; i += 32) {
    if (hs[i] != hk) continue;
    if (kn - i >= st->slots) {
      atomicOr(&st->err, 2);  // the matching power has left the ring: cannot verify
      continue;
    }
    const int slot = atomicAdd(&st->ncand, 1);
    if (slot < kMaxCand) st->cand[slot] = i;
    else atomicOr(&st->err, 4);
  }
  __syncwarp();
  if (threadIdx.x == 0 && st->err) st->done = 3;
}

// Exact comparison of P_kn with every candidate; the last CTA decides and advances k.
__global__ void compare_resolve_kernel(PowerState* st, int16_t* ring, int64_t slot_elems, int slots, int64_t N,
                                       int64_t ld) {
  __shared__ int last;
  if (*(volatile const int32_t*)&st->done) return;
  const int kn = *(volatile const int32_t*)&st->k + 1;
  const int ncand = min(*(volatile const int32_t*)&st->ncand, kMaxCand);
  const int16_t* pk = ring + (int64_t)(kn % slots) * slot_elems;
  const int64_t chunks_per_row = (N + 7) / 8, total = N * chunks_per_row;
  for (int c = 0; c < ncand; ++c) {
    const int16_t* pi = ring + (int64_t)(st->cand[c] % slots) * slot_elems;
    int diff = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total && !diff;
         t += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = t / chunks_per_row, j0 = (t % chunks_per_row) * 8;
      const uint4 a = *reinterpret_cast<const uint4*>(pk + i * ld + j0);
      const uint4 b = *reinterpret_cast<const uint4*>(pi + i * ld + j0);
      const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
      const int64_t rem = N - j0;
      const int valid = rem < 8 ? (int)rem : 8;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t x = wa[q] ^ wb[q];
        const uint32_t lo = (2 * q < valid) ? (x & 0xFFFFu) : 0u;
        const uint32_t hi = (2 * q + 1 < valid) ? (x >> 16) : 0u;
        diff |= (lo | hi) != 0;
      }
    }
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(&st->mismatch[c], 1);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  int found = -1;
  for (int c = 0; c < ncand; ++c) {
    const int i = st->cand[c];
    if (!(*(volatile int32_t*)&st->mismatch[c]) && (found < 0 || i < found)) found = i;
  }
  int64_t* off = st_offset(st);
  if (found >= 1) {
    st->found_i = found;
    st->found_j = kn;
    st->found_q = off[kn] - off[found];
    st->done = 1;
  } else if (kn >= st->kmax) {
    st->done = 2;
  }
  st->k = kn;
  st->mu = kInf;
  st->dmin = kInf;
  st->hacc = 0;
  st->ncand = 0;
  st->range_bad = 0;
  for (int c = 0; c < kMaxCand; ++c) st->mismatch[c] = 0;
  st->blocks_done = 0;
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
  if (h.done == 3) return (h.err & 1) ? RD_ERR_RANGE : RD_ERR_NOMEM;
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
  // the dense x sparse step (A(G) is sparse, its powers are dense)
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
