// sparse_tile.cuh -- the block-sparse (min,+) product tile, shared by the
// single-product launcher (sparse.cu) and the multi-run period search.
#pragma once

#include "rd_internal.cuh"

namespace rd {
namespace {

__device__ __forceinline__ uint32_t finite_mask(const uint4& v) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    m |= ((w[q] & 0xFFFFu) != (uint32_t)kInf ? 1u : 0u) << (2 * q);
    m |= ((w[q] >> 16) != (uint32_t)kInf ? 1u : 0u) << (2 * q + 1);
  }
  return m;
}

__device__ __forceinline__ uint32_t half_of(const uint4& v, int e) {
  const uint32_t w = (e >> 1) == 0 ? v.x : (e >> 1) == 1 ? v.y : (e >> 1) == 2 ? v.z : v.w;
  return (e & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// 32-bit words per entry record: {t, w_0..w_{R-1}} padded to a multiple of 16 bytes
// (records are moved by 16-byte bulk copies).
__host__ __device__ constexpr int record_words(int R) { return ((1 + R + 3) / 4) * 4; }

struct SparseArgs {
  int64_t M;  // rows of the sparse operand and of C
  const int64_t* start;
  const uint32_t* rec;  // entry records, record_words(R) words each
  const int16_t* B;     // dense right operand, rows indexed by the records' t
  int64_t ldb;
  int16_t* C;
  int64_t ldc;
  int64_t Ncols;
  int32_t* min_out;
  int32_t* diag_out;
  PowerState* st;  // ring mode: B = P_k, C = the slot of power k + 1
  int16_t* ring;
  int64_t slot_elems;
  int slots;
};

constexpr int kChunk = 128;  // entry records staged in shared memory at a time

// One CTA = one block b of R rows x a slab of 16 * blockDim.x columns of C = A (x) B.
// Thread t owns columns [base + 8t, base + 8t + 8) and [base + 8(T + t), base + 8(T + t) + 8),
// so each of its two loads per B row is part of one contiguous warp-wide sweep.
// srec: kChunk * record_words(R) words of shared memory for the staged entry records.
template <int R>
__device__ __forceinline__ void sparse_tile_body(const SparseArgs& a, const int16_t* __restrict__ B,
                                                 int16_t* __restrict__ C, const int64_t b, const int64_t slab,
                                                 uint32_t* __restrict__ srec) {
  constexpr int W = record_words(R);
  constexpr int U = (R >= 8) ? 2 : 4;  // entries whose B rows are in flight together
  const int T = blockDim.x;
  const int64_t base = slab * T * 16;
  const int64_t col[2] = {base + threadIdx.x * 8, base + (T + threadIdx.x) * 8};
  const bool ok0 = col[0] < a.Ncols, ok1 = col[1] < a.Ncols;
  const uint4 inf4 = make_uint4(kInf2, kInf2, kInf2, kInf2);
  uint32_t acc[R][8];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = kInf2;

  const int64_t e_begin = a.start[b], e_end = a.start[b + 1];
  for (int64_t c0 = e_begin; c0 < e_end; c0 += kChunk) {
    const int n_in = (e_end - c0 < kChunk) ? (int)(e_end - c0) : kChunk;
    __syncthreads();  // the previous chunk has been consumed
    for (int i = threadIdx.x; i < n_in * W; i += T) srec[i] = __ldg(a.rec + c0 * W + i);
    __syncthreads();
    int e = 0;
    for (; e + U <= n_in; e += U) {
      uint4 pv[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t t = srec[(e + u) * W];
        const int16_t* row = B + (int64_t)t * a.ldb;
        pv[u][0] = ok0 ? __ldg(reinterpret_cast<const uint4*>(row + col[0])) : inf4;
        pv[u][1] = ok1 ? __ldg(reinterpret_cast<const uint4*>(row + col[1])) : inf4;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t p8[8] = {pv[u][0].x, pv[u][0].y, pv[u][0].z, pv[u][0].w,
                                pv[u][1].x, pv[u][1].y, pv[u][1].z, pv[u][1].w};
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t w = srec[(e + u) * W + 1 + r];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = __viaddmin_s16x2(p8[c], w, acc[r][c]);
        }
      }
    }
    for (; e < n_in; ++e) {
      const uint32_t t = srec[e * W];
      const int16_t* row = B + (int64_t)t * a.ldb;
      const uint4 q0 = ok0 ? __ldg(reinterpret_cast<const uint4*>(row + col[0])) : inf4;
      const uint4 q1 = ok1 ? __ldg(reinterpret_cast<const uint4*>(row + col[1])) : inf4;
      const uint32_t p8[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t w = srec[e * W + 1 + r];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = __viaddmin_s16x2(p8[c], w, acc[r][c]);
      }
    }
  }

  int32_t lmin = kInf, ldiag = kInf;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t row = b * R + r;
    if (row >= a.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(h == 0 ? ok0 : ok1)) continue;
      const uint4 out = make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      const int64_t c = col[h];
      if (c + 8 <= a.Ncols) {
        *reinterpret_cast<uint4*>(C + row * a.ldc + c) = out;
      } else {
#pragma unroll
        for (int e2 = 0; e2 < 8; ++e2)
          if (c + e2 < a.Ncols) C[row * a.ldc + c + e2] = (int16_t)half_of(out, e2);
      }
#pragma unroll
      for (int e2 = 0; e2 < 8; ++e2) {
        if (c + e2 < a.Ncols) {
          const int32_t v = (int32_t)half_of(out, e2);
          lmin = min(lmin, v);
          if (c + e2 == row) ldiag = min(ldiag, v);
        }
      }
    }
  }
  if (a.min_out != nullptr || a.diag_out != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xFFFFFFFFu, lmin, o));
      ldiag = min(ldiag, __shfl_xor_sync(0xFFFFFFFFu, ldiag, o));
    }
    __shared__ int32_t red_m[8], red_d[8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red_m[warp] = lmin;
      red_d[warp] = ldiag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t bm = kInf, bd = kInf;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        bm = min(bm, red_m[w]);
        bd = min(bd, red_d[w]);
      }
      if (a.min_out != nullptr && bm < kInf) atomicMin(a.min_out, bm);
      if (a.diag_out != nullptr && bd < kInf) atomicMin(a.diag_out, bd);
    }
  }
}



template <int R>
__device__ __forceinline__ void sparse_tile_body(const SparseArgs& a, const int16_t* __restrict__ B,
                                                 int16_t* __restrict__ C, const int64_t b, const int64_t slab) {
  __shared__ __align__(16) uint32_t srec[kChunk * record_words(R)];
  sparse_tile_body<R>(a, B, C, b, slab, srec);
}

// ---------------------------------------------------------------- the same tile fed by bulk copies
//
// A producer warp streams, for each entry of the block, its record and the row segment
// B[t][slab] into a ring of kStages shared-memory stages with cp.async.bulk (one
// mbarrier per stage counts the bytes in); two consumer warps wait for a stage, apply
// it to their 16 columns and release it through a second mbarrier.  The loads of B no
// longer go through the SM's load/store path, and up to kStages row segments per CTA
// are in flight without holding registers.  Every wait is bounded: past the bound the
// kernel sets kErrTimeout in *err, stops, waits (bounded again) for the copies it has
// in flight, and returns, so a fault in the protocol cannot hang the GPU.  The bound
// (wait_limit) and a stop point for the producer (stop_at: it issues entries
// [0, stop_at) of each block and no more; -1 for none) are kernel arguments, so a
// test can make the consumers' wait run out with no copy in flight.

constexpr int kStages = 16;
constexpr int kTmaConsumers = 64;                  // two warps, 16 columns per thread
constexpr int kTmaThreads = kTmaConsumers + 32;    // plus one producer warp
constexpr int kSlabCols = kTmaConsumers * 16;      // 1024 columns per CTA
constexpr int kRecordSlot = 64;                    // bytes reserved for the record in a stage
constexpr int kStageBytes = kRecordSlot + kSlabCols * 2;
constexpr size_t kTmaSmemBytes = (size_t)kStages * kStageBytes + 2 * kStages * sizeof(uint64_t);
constexpr uint32_t kWaitLimit = 1u << 20;          // try_wait rounds before a wait gives up (default)

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// true once the phase of parity `parity` has completed; false after `limit` tries, or as
// soon as another CTA has reported a timeout in *err (checked every 1024 tries; err may be null),
// so that one failure ends the whole launch quickly
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const int32_t* err, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (err != nullptr && (it & 1023u) == 1023u && (*(volatile const int32_t*)err & kErrTimeout)) return false;
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int R>
__device__ __forceinline__ void sparse_tma_tile_body(const SparseArgs& a, const int16_t* __restrict__ B,
                                                     int16_t* __restrict__ C, const int64_t b, const int64_t slab,
                                                     int32_t* err, uint32_t wait_limit, int stop_at) {
  constexpr int W = record_words(R);
  constexpr uint32_t kRecBytes = W * 4;
  extern __shared__ __align__(128) unsigned char tsm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(tsm + (size_t)kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  __shared__ int issued_sh, consumed_sh[2], failed_sh;
  __shared__ int32_t red_m[3], red_d[3];
  const int tid = threadIdx.x;
  const int64_t e0 = a.start[b];
  const int n_e = (int)(a.start[b + 1] - e0);
  const int64_t col_base = slab * kSlabCols;
  const int64_t ncols_padded = (a.Ncols + 7) / 8 * 8;
  const int64_t row_cols = (ncols_padded - col_base < kSlabCols) ? (ncols_padded - col_base) : kSlabCols;
  const uint32_t row_bytes = (uint32_t)row_cols * 2;
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(saddr(&full[q]), 1);
      mbar_init(saddr(&empty[q]), 2);
    }
    issued_sh = 0;
    consumed_sh[0] = consumed_sh[1] = 0;
    failed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  uint32_t acc[R][8];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = kInf2;
  const int64_t col[2] = {col_base + (int64_t)tid * 8, col_base + kSlabCols / 2 + (int64_t)tid * 8};
  const bool ok0 = (tid < kTmaConsumers) && col[0] < a.Ncols;
  const bool ok1 = (tid < kTmaConsumers) && col[1] < a.Ncols;

  if (tid >= kTmaConsumers) {
    // producer warp: lanes fetch the next 32 entries' columns, lane 0 issues the copies
    const int lane = tid - kTmaConsumers;
    const int n_issue = (stop_at >= 0 && stop_at < n_e) ? stop_at : n_e;
    int issued = 0, fail = 0;
    for (int base = 0; base < n_issue && !fail; base += 32) {
      const int e = base + lane;
      const uint32_t t_lane = (e < n_e) ? __ldg(a.rec + (e0 + e) * W) : 0u;
      const int cnt = (n_issue - base < 32) ? (n_issue - base) : 32;
      for (int u = 0; u < cnt; ++u) {
        const uint32_t t = __shfl_sync(0xFFFFFFFFu, t_lane, u);
        int f = 0;
        if (lane == 0) {
          const int i = base + u, slot = i % kStages;
          if (i >= kStages &&
              !mbar_wait(saddr(&empty[slot]), (uint32_t)((i / kStages) & 1) ^ 1u, err, wait_limit)) {
            f = 1;
          } else {
            unsigned char* stg = tsm + (size_t)slot * kStageBytes;
            const uint32_t bar = saddr(&full[slot]);
            mbar_arrive_expect(bar, kRecBytes + row_bytes);
            bulk_copy_g2s(saddr(stg), a.rec + (e0 + i) * W, kRecBytes, bar);
            bulk_copy_g2s(saddr(stg + kRecordSlot), B + (int64_t)t * a.ldb + col_base, row_bytes, bar);
            issued = i + 1;
          }
        }
        fail = __shfl_sync(0xFFFFFFFFu, f, 0);
        if (fail) break;
      }
    }
    if (lane == 0) {
      issued_sh = issued;
      if (fail) {
        atomicOr(err, kErrTimeout);
        atomicOr(&failed_sh, 1);
      }
    }
  } else {
    // consumer warps
    const uint4 inf4 = make_uint4(kInf2, kInf2, kInf2, kInf2);
    int i = 0;
    for (; i < n_e; ++i) {
      const int slot = i % kStages;
      if (*(volatile int*)&failed_sh ||
          !mbar_wait(saddr(&full[slot]), (uint32_t)((i / kStages) & 1), err, wait_limit)) {
        atomicOr(err, kErrTimeout);
        atomicOr(&failed_sh, 1);
        break;
      }
      const unsigned char* stg = tsm + (size_t)slot * kStageBytes;
      const uint32_t* rec = reinterpret_cast<const uint32_t*>(stg);
      const uint4* row = reinterpret_cast<const uint4*>(stg + kRecordSlot);
      const uint4 q0 = ok0 ? row[tid] : inf4;
      const uint4 q1 = ok1 ? row[kTmaConsumers + tid] : inf4;
      const uint32_t p8[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t w = rec[1 + r];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = __viaddmin_s16x2(p8[c], w, acc[r][c]);
      }
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(saddr(&empty[slot]));
    }
    if ((tid & 31) == 0) consumed_sh[tid >> 5] = i;
  }
  __syncthreads();
  // after a failure: let every issued copy land before the CTA's shared memory is released
  if (tid == 0 && failed_sh) {
    const int done = consumed_sh[0] < consumed_sh[1] ? consumed_sh[0] : consumed_sh[1];
    for (int i = done; i < issued_sh; ++i)  // bounded by the default limit, not cut short by the error flag
      mbar_wait(saddr(&full[i % kStages]), (uint32_t)((i / kStages) & 1), nullptr, kWaitLimit);
  }

  int32_t lmin = kInf, ldiag = kInf;
  if (tid < kTmaConsumers && !failed_sh) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = b * R + r;
      if (row >= a.M) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!(h == 0 ? ok0 : ok1)) continue;
        const uint4 out = make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
        const int64_t c = col[h];
        if (c + 8 <= a.Ncols) {
          *reinterpret_cast<uint4*>(C + row * a.ldc + c) = out;
        } else {
#pragma unroll
          for (int e2 = 0; e2 < 8; ++e2)
            if (c + e2 < a.Ncols) C[row * a.ldc + c + e2] = (int16_t)half_of(out, e2);
        }
#pragma unroll
        for (int e2 = 0; e2 < 8; ++e2) {
          if (c + e2 < a.Ncols) {
            const int32_t v = (int32_t)half_of(out, e2);
            lmin = min(lmin, v);
            if (c + e2 == row) ldiag = min(ldiag, v);
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(0xFFFFFFFFu, lmin, o));
    ldiag = min(ldiag, __shfl_xor_sync(0xFFFFFFFFu, ldiag, o));
  }
  if ((tid & 31) == 0) {
    red_m[tid >> 5] = lmin;
    red_d[tid >> 5] = ldiag;
  }
  __syncthreads();
  if (tid == 0) {
    int32_t bm = kInf, bd = kInf;
    for (int w2 = 0; w2 < kTmaThreads / 32; ++w2) {
      bm = min(bm, red_m[w2]);
      bd = min(bd, red_d[w2]);
    }
    if (a.min_out != nullptr && bm < kInf) atomicMin(a.min_out, bm);
    if (a.diag_out != nullptr && bd < kInf) atomicMin(a.diag_out, bd);
  }
}

}  // namespace
}  // namespace rd
