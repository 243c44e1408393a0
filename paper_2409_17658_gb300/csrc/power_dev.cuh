// power_dev.cuh -- device bodies of the power-step kernels (normaliser / hash,
// finalize, exact compare), shared by the single-run and the multi-run launchers.
// The striding bodies split their rows into `parts` parts and work on part `part`
// (by default blockIdx.x of gridDim.x), so a multi-run kernel can give each run its
// own blockIdx.y, and the multi-run step kernel can run the parts as work items.
// Data another CTA may have written earlier in the same launch (the product, the
// normalised power, the search state) is read through L2 (__ldcg, volatile).
#pragma once

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

// Hash of the 16-byte chunk of row i starting at column j0 (8 entries, entries past
// the last column already replaced by RD_INF): the NH sum of UMAC (Black, Halevi,
// Krawczyk, Krovetz and Rogaway, 1999) over its four 32-bit words,
// (w0 + k0)(w1 + k1) + (w2 + k2)(w3 + k3) mod 2^64, with keys drawn from the chunk's
// position by multiplicative hashing.  The matrix hash is the wrapping sum over all
// chunks, so it does not depend on the order of the reduction; equal matrices hash
// equal, and the hash only pre-filters the exact compare.
__device__ __forceinline__ unsigned long long chunk_hash(int64_t i, int64_t j0, const uint32_t w[4]) {
  const uint32_t k0 = ((uint32_t)i * 0x9E3779B1u) ^ (((uint32_t)j0 >> 3) * 0x85EBCA77u);
  const uint32_t k1 = k0 * 0xC2B2AE3Du, k2 = k0 ^ 0x27D4EB2Fu, k3 = k2 * 0x165667B1u;
  return (unsigned long long)(w[0] + k0) * (unsigned long long)(w[1] + k1) +
         (unsigned long long)(w[2] + k2) * (unsigned long long)(w[3] + k3);
}

// Lanes e >= valid of a chunk: RD_INF (their contents are padding and must not matter).
__device__ __forceinline__ void mask_tail(uint32_t w[4], int valid) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (2 * q >= valid) w[q] = (w[q] & 0xFFFF0000u) | (uint32_t)kInf;
    if (2 * q + 1 >= valid) w[q] = (w[q] & 0x0000FFFFu) | ((uint32_t)kInf << 16);
  }
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

__device__ __forceinline__ void init_state_body(PowerState* st, int kmax, int slots) {
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
    for (int l = 0; l < 4; ++l) st->lvl_done[l] = 0;
    st->queue = 0;
    st->exited = 0;
    st->far_i = kFarNone;
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
// Blocks stride over rows, threads over the 16-byte chunks of a row.
__device__ __forceinline__ void reduce_min_diag_body(const int16_t* __restrict__ X, int64_t N, int64_t ld,
                                                     PowerState* st) {
  __shared__ int32_t sh[kRedThreads / 32];
  const int64_t cpr = (N + 7) / 8;
  int32_t lm = kInf, ld_min = kInf;
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
    const int16_t* row = X + i * ld;
    for (int64_t c = threadIdx.x; c < cpr; c += blockDim.x) {
      const int64_t j0 = c * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(row + j0);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (j0 + e >= N) break;
        const int32_t x = (int32_t)(int16_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
        lm = min(lm, x);
        if (j0 + e == i) ld_min = min(ld_min, x);
      }
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
// and the range check that keeps int16 exact.  Blocks stride over rows, threads over chunks.
template <bool COPY>
__device__ __forceinline__ void normalise_hash_body(const int16_t* __restrict__ src, PowerState* st, int16_t* ring,
                                                    int64_t slot_elems, int slots, int64_t N, int64_t ld,
                                                    int64_t part = -1, int64_t parts = -1) {
  __shared__ unsigned long long shh[kRedThreads / 32];
  const int64_t b0 = part < 0 ? (int64_t)blockIdx.x : part, nb = parts < 0 ? (int64_t)gridDim.x : parts;
  if (*(volatile const int32_t*)&st->done) return;
  const int kn = *(volatile const int32_t*)&st->k + 1;
  int16_t* dst = ring + (int64_t)(kn % slots) * slot_elems;
  const int16_t* s = COPY ? src : dst;
  const int32_t mu_raw = *(volatile const int32_t*)&st->mu;
  const int32_t mu = (mu_raw >= kInf) ? 0 : mu_raw;
  const int64_t cpr = (N + 7) / 8;
  unsigned long long h = 0;
  int bad = 0;
  for (int64_t i = b0; i < N; i += nb) {
    for (int64_t c = threadIdx.x; c < cpr; c += blockDim.x) {
      const int64_t j0 = c * 8;
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(s + i * ld + j0));
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
      const int64_t rem = N - j0;
      const int valid = rem < 8 ? (int)rem : 8;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (e >= valid) break;
        const int sh = 16 * (e & 1);
        int32_t x = (int32_t)(int16_t)((w[e >> 1] >> sh) & 0xFFFF);
        if (COPY) bad |= (x != kInf) && (x < 0 || x > kMaxFinite);  // the operand contract
        if (x != kInf) {
          x -= mu;
          bad |= (x < 0 || x > kMaxFinite);
        }
        w[e >> 1] = (w[e >> 1] & ~(0xFFFFu << sh)) | ((uint32_t)(x & 0xFFFF) << sh);
      }
      *reinterpret_cast<uint4*>(dst + i * ld + j0) = make_uint4(w[0], w[1], w[2], w[3]);
      if (valid < 8) mask_tail(w, valid);
      h += chunk_hash(i, j0, w);
    }
  }
  h = block_reduce_sum(h, shh);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    atomicAdd(&st->hacc, h);
    if (bad) atomicOr(&st->range_bad, 1);
  }
}

// One warp: bookkeeping of power kn = k + 1 and the list of hash matches.
__device__ __forceinline__ void finalize_body(PowerState* st) {
  volatile PowerState* vs = st;
  if (vs->done) return;
  const int kn = vs->k + 1;
  int64_t* off = st_offset(st);
  int64_t* gam = st_gamma(st);
  unsigned long long* hs = st_hash(st);
  const unsigned long long hk = vs->hacc;
  const int32_t bad_range = vs->range_bad;
  if (threadIdx.x == 0) {
    const int32_t mu_raw = vs->mu, dmin = vs->dmin;
    const int32_t mu = (mu_raw >= kInf) ? 0 : mu_raw;
    off[kn] = off[kn - 1] + mu;
    gam[kn] = (dmin >= kInf) ? RD_GAMMA_INF : off[kn - 1] + dmin;
    hs[kn] = hk;
    if (bad_range) {
      st->err |= kErrRange;
      st->done = 3;
    }
  }
  __syncwarp();
  if (bad_range) return;
  for (int i = 1 + (int)threadIdx.x; i < kn; i += 32) {
    if (hs[i] != hk) continue;
    if (kn - i >= st->slots) {
      atomicMin(&st->far_i, i);  // the matching power has left the ring: decided after the compare
      continue;
    }
    const int slot = atomicAdd(&st->ncand, 1);
    if (slot < kMaxCand) st->cand[slot] = i;
    else atomicOr(&st->err, kErrCandidates);
  }
  __syncwarp();
  if (threadIdx.x == 0 && st->err) st->done = 3;
}

// Exact comparison of P_kn with every candidate; the last CTA (of `parts`) decides and advances k.
__device__ __forceinline__ void compare_resolve_body(PowerState* st, int16_t* ring, int64_t slot_elems, int slots,
                                                     int64_t N, int64_t ld, int64_t part = -1, int64_t parts = -1) {
  __shared__ int last;
  const int64_t b0 = part < 0 ? (int64_t)blockIdx.x : part, nb = parts < 0 ? (int64_t)gridDim.x : parts;
  if (*(volatile const int32_t*)&st->done) return;
  const int kn = *(volatile const int32_t*)&st->k + 1;
  const int ncand = min(*(volatile const int32_t*)&st->ncand, kMaxCand);
  const int16_t* pk = ring + (int64_t)(kn % slots) * slot_elems;
  const int64_t cpr = (N + 7) / 8;
  for (int c = 0; c < ncand; ++c) {
    const int16_t* pi = ring + (int64_t)(*(volatile const int32_t*)&st->cand[c] % slots) * slot_elems;
    int diff = 0;
    for (int64_t i = b0; i < N && !diff; i += nb) {
      for (int64_t cc = threadIdx.x; cc < cpr; cc += blockDim.x) {
        const int64_t j0 = cc * 8;
        const uint4 a = __ldcg(reinterpret_cast<const uint4*>(pk + i * ld + j0));
        const uint4 b = __ldcg(reinterpret_cast<const uint4*>(pi + i * ld + j0));
        uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
        const int64_t rem = N - j0;
        if (rem < 8) {
          mask_tail(wa, (int)rem);
          mask_tail(wb, (int)rem);
        }
        diff |= (wa[0] != wb[0]) | (wa[1] != wb[1]) | (wa[2] != wb[2]) | (wa[3] != wb[3]);
      }
    }
    if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(&st->mismatch[c], 1);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&st->blocks_done, 1u) == (unsigned)(nb - 1));
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  int found = -1;
  for (int c = 0; c < ncand; ++c) {
    const int i = *(volatile const int32_t*)&st->cand[c];
    if (!(*(volatile int32_t*)&st->mismatch[c]) && (found < 0 || i < found)) found = i;
  }
  volatile int64_t* off = st_offset(st);
  const int32_t far = *(volatile int32_t*)&st->far_i;
  if (found >= 1) {
    st->found_i = found;
    st->found_j = kn;
    st->found_q = off[kn] - off[found];
    st->done = 1;
  } else if (far != kFarNone) {
    // no power in the ring equals P_kn, but one that has left it has the same hash: stop, and leave
    // the pair for a caller that can re-derive P_far
    st->found_i = far;
    st->found_j = kn;
    st->err |= kErrRing;
    st->done = 3;
  } else if (kn >= st->kmax) {
    st->done = 2;
  }
  st->far_i = kFarNone;
  st->k = kn;
  st->mu = kInf;
  st->dmin = kInf;
  st->hacc = 0;
  st->ncand = 0;
  st->range_bad = 0;
  for (int c = 0; c < kMaxCand; ++c) st->mismatch[c] = 0;
  st->blocks_done = 0;
}


}  // namespace
}  // namespace rd
