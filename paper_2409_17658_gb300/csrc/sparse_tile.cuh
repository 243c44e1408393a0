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

// 32-bit words per entry record: {t, w_0..w_{R-1}} padded to 8 or 16-byte multiples.
__host__ __device__ constexpr int record_words(int R) { return R == 1 ? 2 : ((1 + R + 3) / 4) * 4; }

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
template <int R>
__device__ __forceinline__ void sparse_tile_body(const SparseArgs& a, const int16_t* __restrict__ B,
                                                 int16_t* __restrict__ C, const int64_t b, const int64_t slab) {
  constexpr int W = record_words(R);
  constexpr int U = (R >= 8) ? 2 : 4;  // entries whose B rows are in flight together
  __shared__ __align__(16) uint32_t srec[kChunk * W];
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
    __shared__ int32_t red_m[4], red_d[4];
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


}  // namespace
}  // namespace rd
