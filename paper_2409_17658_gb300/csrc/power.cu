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

// One power step: the product, then normalise/hash (unless the product did it), finalize, compare.
cudaError_t enqueue_step(const Run& r, ProductFn product, const void* ctx, bool normalised, cudaStream_t s) {
  cudaError_t e = product(r, ctx, s);
  if (e != cudaSuccess) return e;
  if (!normalised)
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

// ---------------------------------------------------------------- small matrices: one CTA per search
//
// For N <= kSmallN the whole search runs in one CTA with A, the current power and the next raw product
// in shared memory (96 KB at N = 128): one launch and one host read per search instead of four
// launches per power.  The CTA leaves the work area exactly as the step kernels do -- state header,
// offsets, gamma, a hash per power, and each normalised power in its ring slot -- and follows the same
// rules: P_1 = A - min A, P_{k+1} = (P_k (x) A) - mu, gamma_k = o_{k-1} + the raw diagonal minimum,
// the operand contract and the range check, a hash match with a power that has left the ring is an
// error (kErrRing), more than kMaxCand matches is an error, and the smallest exactly equal earlier power
// ends the search.  The products are exact, so the result equals the large-matrix path's.
constexpr int64_t kSmallN = 128;
constexpr int kSmallThreads = 1024;

size_t small_smem(int64_t N, int kmax) {
  const size_t np = (size_t)((N + 7) / 8 * 8);
  return 3 * (size_t)N * np * 2 + 8 * (size_t)(kmax + 1);
}

__global__ void __launch_bounds__(kSmallThreads) small_search_kernel(const int16_t* __restrict__ A, int64_t N,
                                                                     int64_t lda, int kmax, PowerState* st,
                                                                     int16_t* ring, int64_t slot_elems, int slots) {
  extern __shared__ uint4 smq[];
  __shared__ int32_t red[32];
  __shared__ unsigned long long redh[32];
  const int n = (int)N, np = (int)((N + 7) / 8 * 8), cells = n * np, half = np / 2;
  int16_t* sA = reinterpret_cast<int16_t*>(smq);  // n x np, columns >= n are RD_INF
  int16_t* sP = sA + cells;                       // the current normalised power
  int16_t* sR = sP + cells;                       // the next raw product
  unsigned long long* shash = reinterpret_cast<unsigned long long*>(sR + cells);  // a hash per power

  init_state_body(st, kmax, slots);
  for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
    const int i = idx / np, j = idx % np;
    sA[idx] = (j < n) ? A[(int64_t)i * lda + j] : kInf;
  }
  __syncthreads();
  int64_t* off = st_offset(st);
  int64_t* gam = st_gamma(st);
  unsigned long long* hs = st_hash(st);

  for (int kn = 1; kn <= kmax; ++kn) {
    const int16_t* src = sA;
    if (kn > 1) {
      // raw product R = P_{kn-1} (x) A: two columns per DPX add-min, the P entry in both halves
      const uint32_t* a32 = reinterpret_cast<const uint32_t*>(sA);
      for (int q = threadIdx.x; q < n * half; q += blockDim.x) {
        const int i = q / half, jp = q % half;
        const int16_t* prow = sP + i * np;
        uint32_t acc = kInf2;
        for (int t = 0; t < n; ++t) acc = __viaddmin_s16x2((uint32_t)(uint16_t)prow[t] * 0x00010001u, a32[t * half + jp], acc);
        reinterpret_cast<uint32_t*>(sR)[q] = acc;
      }
      __syncthreads();
      src = sR;
    }
    // min and diagonal minimum of the raw matrix; on the first power also the operand contract
    int32_t lm = kInf, ldm = kInf;
    int bad = 0;
    for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
      const int i = idx / np, j = idx % np;
      if (j >= n) continue;
      const int32_t x = src[idx];
      if (kn == 1) bad |= (x != kInf) && (x < 0 || x > kMaxFinite);
      lm = min(lm, x);
      if (i == j) ldm = min(ldm, x);
    }
    lm = block_reduce_min(lm, red);
    ldm = block_reduce_min(ldm, red);
    const int32_t mu = (lm >= kInf) ? 0 : lm;
    // P_kn = raw - mu on finite entries, into shared memory and its ring slot, with its hash
    int16_t* slot = ring + (int64_t)(kn % slots) * slot_elems;
    unsigned long long h = 0;
    for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
      const int i = idx / np, j = idx % np;
      int32_t x = src[idx];
      if (j < n) {
        if (x != kInf) {
          x -= mu;
          bad |= (x < 0 || x > kMaxFinite);
        }
        slot[(int64_t)i * lda + j] = (int16_t)x;
        h += mix64(((unsigned long long)idx << 16) ^ (unsigned long long)(uint16_t)x);
      } else {
        x = kInf;
      }
      sP[idx] = (int16_t)x;
    }
    h = block_reduce_sum(h, redh);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
      off[kn] = off[kn - 1] + mu;
      gam[kn] = (ldm >= kInf) ? RD_GAMMA_INF : off[kn - 1] + ldm;
      hs[kn] = h;
      shash[kn] = h;
    }
    if (bad) {
      if (threadIdx.x == 0) {
        st->err |= kErrRange;
        st->done = 3;
        st->k = kn - 1;
      }
      return;
    }
    __syncthreads();  // the slot and shash entries are visible to the whole CTA
    // earlier powers with the same hash: one that has left the ring, or more than kMaxCand resident
    // ones, is an error; otherwise the smallest resident one equal entry by entry ends the search
    int err = 0, ncand = 0, found = -1;
    for (int i = 1; i < kn; ++i) {
      if (shash[i] != h) continue;
      if (kn - i >= slots)
        err |= kErrRing;
      else if (++ncand > kMaxCand)
        err |= kErrCandidates;
    }
    for (int i = 1; i < kn && found < 0 && !err; ++i) {
      if (shash[i] != h) continue;
      const int16_t* pi = ring + (int64_t)(i % slots) * slot_elems;
      int diff = 0;
      for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
        const int r = idx / np, c = idx % np;
        if (c < n) diff |= (pi[(int64_t)r * lda + c] != sP[idx]);
      }
      if (!__syncthreads_or(diff)) found = i;
    }
    if (err) {
      if (threadIdx.x == 0) {
        st->err |= err;
        st->done = 3;
        st->k = kn - 1;
      }
      return;
    }
    if (found >= 1) {
      if (threadIdx.x == 0) {
        st->found_i = found;
        st->found_j = kn;
        st->found_q = off[kn] - off[found];
        st->done = 1;
        st->k = kn;
      }
      return;
    }
    if (kn >= kmax) {
      if (threadIdx.x == 0) {
        st->done = 2;
        st->k = kn;
      }
      return;
    }
    __syncthreads();  // sP is read by the next product
  }
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

namespace {
// The host outputs of a finished search from its final state header and gamma array.
rd_status search_outputs(const PowerState& h, void* work_dev, int kmax, int64_t* gamma_host, int32_t* k_out,
                         int32_t* p_out, int64_t* q_out, cudaStream_t s) {
  const int last = (h.done == 1) ? h.found_j : h.k;
  cudaError_t e = cudaMemcpyAsync(gamma_host, reinterpret_cast<char*>(work_dev) + kStateHeader + 8 * (size_t)(kmax + 1),
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
}  // namespace

// Algorithm 2 on a validated work area: state header, then the ring of powers.
// No host heap use: the gamma table is copied straight into gamma_host.
namespace {
// Per host thread and device: two page-locked copies of the search state and their events, for the checks
// of power_search (made on first use; host memory, not device memory).
struct HostCheck {
  PowerState* st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool tried = false, ok = false;
};
constexpr int kCheckDevices = 16;
HostCheck* host_check() {
  thread_local HostCheck hc[kCheckDevices];
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCheckDevices) return nullptr;
  HostCheck& h = hc[dev];
  if (!h.tried) {
    h.tried = true;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h.st), 2 * sizeof(PowerState), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev[1], cudaEventDisableTiming);
    h.ok = e == cudaSuccess;
  }
  return h.ok ? &h : nullptr;
}
}  // namespace

rd_status power_search(const int16_t* A_dev, int64_t N, int64_t lda, int kmax, void* work_dev, size_t work_bytes,
                       ProductFn product, const void* ctx, int64_t* gamma_host, int32_t* k_out, int32_t* p_out,
                       int64_t* q_out, cudaStream_t s, bool normalised, bool lookahead) {
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
  cudaError_t e = cudaSuccess;
  PowerState h{};
  if (N <= kSmallN) {
    // one CTA runs the whole search (the product's operands A and P_k fit in shared memory)
    const size_t smem = small_smem(N, kmax);
    if (smem <= 200 * 1024) {
      e = cudaFuncSetAttribute(small_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        small_search_kernel<<<1, kSmallThreads, smem, s>>>(A_dev, N, lda, kmax, r.st, r.ring, r.slot_elems, r.slots);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, r.st, sizeof(PowerState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(e);
      return search_outputs(h, work_dev, kmax, gamma_host, k_out, p_out, q_out, s);
    }
  }
  e = enqueue_first(r, kmax, s);
  if (e != cudaSuccess) return fail(e);
  // Steps per host check: large products are long enough that one check per
  // step costs nothing; small ones are batched (surplus steps exit at once).
  // The row-split step (normalised) is about N / 100 times cheaper than the
  // dense one, so it batches up to larger N.
  const int chunk = normalised ? (N >= 16384 ? 1 : (N >= 4096 ? 4 : 8)) : (N >= 2048) ? 1 : (N >= 512 ? 4 : 16);
  int enqueued = 1, cur = 0;
  HostCheck* hcp = lookahead ? host_check() : nullptr;
  if (hcp == nullptr) {
    // one block at a time: the host reads the state after each block before enqueuing the next
    for (;;) {
      e = cudaMemcpyAsync(&h, r.st, sizeof(PowerState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(e);
      if (h.done || enqueued >= kmax) break;
      const int n = (kmax - enqueued < chunk) ? (kmax - enqueued) : chunk;
      for (int i = 0; i < n; ++i) {
        e = enqueue_step(r, product, ctx, normalised, s);
        if (e != cudaSuccess) return fail(e);
      }
      enqueued += n;
    }
    return search_outputs(h, work_dev, kmax, gamma_host, k_out, p_out, q_out, s);
  }
  // One block of steps stays queued ahead of the block the host is checking, so the GPU never waits for
  // the host: the state after each block is copied to pinned host memory and an event marks it; steps
  // enqueued after the relation was found exit at kernel entry.
  HostCheck& hc = *hcp;
  auto enqueue_block = [&](int slot) -> cudaError_t {
    const int n = (kmax - enqueued < chunk) ? (kmax - enqueued) : chunk;
    cudaError_t x = cudaSuccess;
    for (int i = 0; i < n && x == cudaSuccess; ++i) x = enqueue_step(r, product, ctx, normalised, s);
    enqueued += n;
    if (x == cudaSuccess) x = cudaMemcpyAsync(&hc.st[slot], r.st, sizeof(PowerState), cudaMemcpyDeviceToHost, s);
    if (x == cudaSuccess) x = cudaEventRecord(hc.ev[slot], s);
    return x;
  };
  e = enqueue_block(cur);  // the first power's state, with the first block of steps
  bool pending = e == cudaSuccess;
  while (e == cudaSuccess && pending) {
    const bool more = enqueued < kmax;
    if (more) e = enqueue_block(1 - cur);
    if (e == cudaSuccess) e = cudaEventSynchronize(hc.ev[cur]);
    if (e != cudaSuccess) break;
    h = hc.st[cur];
    if (h.done) break;
    pending = more;
    cur = 1 - cur;
  }
  if (e != cudaSuccess) return fail(e);
  return search_outputs(h, work_dev, kmax, gamma_host, k_out, p_out, q_out, s);
}

}  // namespace rd

using namespace rd;

extern "C" rd_status rd_power_work_bytes(int64_t N, int64_t ld, int kmax, int slots, size_t* bytes) {
  if (N < 1 || ld < N || ld % 8 != 0 || kmax < 1 || slots < 2 || !bytes) return RD_ERR_ARG;
  *bytes = state_bytes(kmax) + (size_t)slots * slot_bytes(N, ld);
  return RD_OK;
}

extern "C" rd_status rd_power_slot(int64_t N, int64_t ld, int kmax, size_t work_bytes, int k, size_t* byte_offset) {
  if (N < 1 || ld < N || ld % 8 != 0 || kmax < 1 || k < 0 || k > kmax || !byte_offset) return RD_ERR_ARG;
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
  const int split_j = rd_split_default_j(m);
  const size_t mat = (size_t)N * (size_t)ld * 2;
  // Low-memory form when A(G), 8 ring slots and the whole intermediate of the row split do not fit (m >= 11:
  // 73 GB per power): 3 ring slots with A(G) built in the first (it is read only for the first power), the
  // intermediate in 8192-column chunks, and a repeat whose earlier power has left the ring verified by
  // re-deriving that power (rd_power_until_periodic_split).
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const bool lowmem = split_j > 0 && N > 8192 && mat * 11 > free_b;
  const int slots = lowmem ? 3 : (N <= 8192) ? 16 : 8;
  size_t wbytes = 0;
  rd_power_work_bytes(N, ld, kGammaKmax, slots, &wbytes);
  int16_t* A = nullptr;
  int16_t* A_own = nullptr;
  void* work = nullptr;
  cudaStream_t s = nullptr;
  rd_status rc = RD_OK;
  std::vector<int64_t> g((size_t)kGammaKmax + 1);
  int32_t k = 0, p = 0;
  int64_t q = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess && !lowmem) e = cudaMalloc(&A_own, mat);
  if (e == cudaSuccess) e = cudaMalloc(&work, wbytes);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
  }
  A = A_own;
  if (rc == RD_OK && lowmem) {
    size_t off0 = 0;
    rc = rd_power_slot(N, ld, kGammaKmax, wbytes, 0, &off0);
    A = reinterpret_cast<int16_t*>(static_cast<char*>(work) + off0);
  }
  if (rc == RD_OK) rc = rd_build_transfer(m, A, ld, s);
  if (rc == RD_OK && N <= kSmallN) {
    // small matrices: the whole search in one CTA
    rc = rd_power_until_periodic(A, N, ld, kGammaKmax, work, wbytes, g.data(), &k, &p, &q, s);
    if (s) cudaStreamSynchronize(s);
    if (A_own) cudaFree(A_own);
    if (work) cudaFree(work);
    if (s) cudaStreamDestroy(s);
    return finish_cached(rc, g, k, p, q, out);
  }
  if (rc == RD_OK && split_j > 0) {
    // the row-split step: A(G) (x) P_k from the row rules, in two passes
    size_t pbytes = 0;
    void* plan = nullptr;
    int16_t* X = nullptr;
    rd_split_info_t info{};
    rc = rd_split_plan_bytes(m, split_j, &pbytes);
    if (rc == RD_OK) e = cudaMalloc(&plan, pbytes);
    if (rc == RD_OK && e == cudaSuccess) rc = rd_split_plan(m, split_j, plan, pbytes, &info, s);
    if (lowmem) info.chunk_cols = 8192;
    const int64_t ldx = lowmem ? info.chunk_cols : ld;
    if (rc == RD_OK && e == cudaSuccess) e = cudaMalloc(&X, (size_t)info.x_rows * (size_t)ldx * 2);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = (e == cudaErrorMemoryAllocation) ? RD_ERR_NOMEM : RD_ERR_CUDA;
    }
    if (rc == RD_OK)
      rc = rd_power_until_periodic_split(A, ld, &info, plan, X, ldx, kGammaKmax, work, wbytes, g.data(), &k, &p, &q, s);
    if (s) cudaStreamSynchronize(s);
    if (plan) cudaFree(plan);
    if (X) cudaFree(X);
    if (A_own) cudaFree(A_own);
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
  if (A_own) cudaFree(A_own);
  if (work) cudaFree(work);
  if (s) cudaStreamDestroy(s);
  return finish_cached(rc, g, k, p, q, out);
}
}  // namespace

extern "C" rd_status rd_gamma_R_clear(void) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  for (auto& c : g_cache) c = Cached{};
  return RD_OK;
}

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

// ---------------------------------------------------------------- relation records (checkpoint / resume)

bool rd::relation_ok(const rd_relation_t* rel, const int64_t* gamma) {
  if (!rel || !gamma) return false;
  const int m = rel->m;
  if (m < 1 || m > RD_MAX_M || rel->j < 1 || rel->j > RD_RELATION_MAX_J) return false;
  if (rel->found == 1) {
    if (rel->k < 1 || rel->p < 1 || (int64_t)rel->k + rel->p != rel->j) return false;
  } else if (rel->found != 0 || rel->k != 0 || rel->p != 0 || rel->q != 0) {
    return false;
  }
  // every label is >= 0, and the word of m a's follows itself with label 2m: 0 <= min diag A^n <= 2mn
  for (int64_t n = 1; n <= rel->j; ++n)
    if (gamma[n] < 0 || gamma[n] > 2 * (int64_t)m * n) return false;
  // min diag (q (x) A^k) = q + min diag A^k
  if (rel->found == 1 && gamma[rel->j] != gamma[rel->k] + rel->q) return false;
  return true;
}

namespace {
void fill_relation(int m, const Cached& c, rd_relation_t* rel) {
  *rel = rd_relation_t{};
  rel->m = m;
  rel->found = c.found ? 1 : 0;
  rel->k = c.found ? c.k : 0;
  rel->p = c.found ? c.p : 0;
  rel->q = c.found ? c.q : 0;
  rel->j = c.j;
}
}  // namespace

extern "C" rd_status rd_gamma_R_export(int m, rd_relation_t* rel, int64_t* gamma, int64_t cap) {
  if (m < 1 || m > RD_MAX_M || !rel) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  Cached& c = g_cache[m];
  if (!c.valid) {
    const rd_status rc = compute_cached(m, &c);
    if (rc != RD_OK) return rc;
  }
  fill_relation(m, c, rel);
  if (!gamma) return RD_OK;
  if (cap < (int64_t)c.j + 1) return RD_ERR_ARG;
  gamma[0] = RD_GAMMA_UNSET;
  for (int n = 1; n <= c.j; ++n) gamma[n] = c.gamma[(size_t)n];
  return RD_OK;
}

extern "C" rd_status rd_gamma_R_import(const rd_relation_t* rel, const int64_t* gamma) {
  if (!rd::relation_ok(rel, gamma)) return RD_ERR_ARG;
  Cached c;
  c.valid = true;
  c.found = rel->found == 1;
  c.k = rel->k;
  c.p = rel->p;
  c.q = rel->q;
  c.j = rel->j;
  c.gamma.assign(gamma, gamma + rel->j + 1);
  c.gamma[0] = RD_GAMMA_UNSET;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_cache[rel->m] = std::move(c);
  return RD_OK;
}
