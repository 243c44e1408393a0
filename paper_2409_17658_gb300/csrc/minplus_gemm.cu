// minplus_gemm.cu -- C = A (x) B, C[i][j] = min_t (A[i][t] + B[t][j]) (Sec. 3),
// on int16 operands with the DPX fused add-min __viaddmin_s16x2.
//
// Design (sm_103a):
//  * Two output columns share one 32-bit register: acc = (C[i][j], C[i][j+1]).
//    One DPX instruction updates both with min(a + b, acc), where b holds
//    (B[t][j], B[t][j+1]) -- the natural packing of row-major B -- and a holds
//    A[i][t] in both halfwords.  The duplication of A is done once per tile when
//    it is staged into shared memory (A^T tile, one 32-bit word per element), so
//    the inner loop is only 128-bit shared loads and DPX instructions.
//  * On this part the DPX unit retires 64 lanes per clock per SM, half the issue
//    rate, so the shared-memory loads and the loop overhead fit in the other half
//    of the issue slots: the kernel is bound by the DPX pipe, not by memory.
//  * CTA tile 128 x 256 x 32, 256 threads, 8 x 16 outputs (64 packed registers)
//    per thread, two CTAs per SM.  B tiles are fetched with cp.async (16 B) into a
//    3-stage ring; A tiles go through registers (prefetched one tile ahead) so
//    they can be transposed and duplicated on the way into shared memory.
//  * CTAs are rasterised in groups of 16 row tiles, so the resident wave reuses
//    its operand panels from L2 (DRAM traffic is not the bound, but re-reads are
//    kept low).
//  * Ragged edges (M, N, K not multiples of the tile) are filled with RD_INF, the
//    neutral element of min, so no padding is required of the caller.
//  * No overflow: operands lie in [0, 0x1FFF] or are 0x3FFF, so every sum is at
//    most 0x7FFE; accumulators start at RD_INF and only decrease, so an entry
//    whose terms all involve RD_INF ends exactly at RD_INF.
#include <cooperative_groups.h>

#include "rd_internal.cuh"

namespace rd {
namespace {

constexpr int BM = 128, BN = 256, BK = 32, NT = 256;
constexpr int BSTAGES = 3;
constexpr int kGroupM = 16;  // row tiles per rasterisation group
constexpr int AS_WORDS = BK * BM;         // one A^T buffer, duplicated int16 -> 32-bit words
constexpr int BS_WORDS = BK * (BN / 2);   // one B stage, packed int16 pairs
constexpr size_t SMEM_BYTES = (size_t)(2 * AS_WORDS + BSTAGES * BS_WORDS) * 4;
// The narrow tile (BM x 128) for products with few output tiles: half the columns per thread, so twice
// the CTAs over the same product, and shared memory for three CTAs per SM.
constexpr int BN_NARROW = 128;
constexpr size_t smem_bytes(int bn) { return (size_t)(2 * AS_WORDS + BSTAGES * BK * (bn / 2)) * 4; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t pack2(int16_t lo, int16_t hi) {
  return (uint32_t)(uint16_t)lo | ((uint32_t)(uint16_t)hi << 16);
}

// One BM x BN output tile of C = A (x) B at (m0, n0), plus its contribution to the
// minimum (min_out) and the diagonal minimum (diag_out) when those are not null.  SPLIT: the tile
// of this CTA's K slice is left in shared memory ([BM][BN/2] packed words) for a cluster reduction.
template <bool SPLIT = false, int BNT = BN>
__device__ __forceinline__ void gemm_tile(const int16_t* __restrict__ Ag, const int16_t* __restrict__ Bg,
                                          int16_t* __restrict__ Cg, const int64_t M, const int64_t N,
                                          const int64_t K, const int64_t lda, const int64_t ldb, const int64_t ldc,
                                          const int64_t m0, const int64_t n0, int32_t* min_out, int32_t* diag_out,
                                          uint32_t* smem) {
  constexpr int BSW = BK * (BNT / 2);  // one B stage, in words
  constexpr int NBC = BNT / 64;        // 16-byte chunks of a B stage per thread
  constexpr int CPR = BNT / 8;         // 16-byte chunks per B row
  constexpr int NV = BNT / 32;         // accumulator words per row of a thread (BNT / 16 columns)
  constexpr int PARTS = BNT / 128;     // 128-column parts of a thread's columns
  uint32_t* As = smem;                 // [2][BK][BM]
  uint32_t* Bs = smem + 2 * AS_WORDS;  // [BSTAGES][BK][BNT/2]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int KT = (int)((K + BK - 1) / BK);

  // ---- staging helpers
  uint4 areg[2];
  // Interior tiles (all rows and columns inside C) over whole k-tiles take the unchecked
  // path: per-thread source pointers computed once, no per-chunk bounds arithmetic.
  const bool full_mn = (m0 + BM <= M) && (n0 + BNT <= N);
  const int kt_full = (int)(K / BK);
  const int16_t* a_src[2];
  const int16_t* b_src[NBC];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = tid + h * NT;
    a_src[h] = Ag + (m0 + (c >> 2)) * lda + (c & 3) * 8;
  }
#pragma unroll
  for (int h = 0; h < NBC; ++h) {
    const int c = tid + h * NT;
    b_src[h] = Bg + (int64_t)(c / CPR) * ldb + n0 + (c % CPR) * 8;
  }
  const int64_t b_step = (int64_t)BK * ldb;

  auto load_a_regs = [&](int kt) {
    if (full_mn && kt < kt_full) {
#pragma unroll
      for (int h = 0; h < 2; ++h) areg[h] = __ldg(reinterpret_cast<const uint4*>(a_src[h] + (int64_t)kt * BK));
      return;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * NT, row = c >> 2, kc = (c & 3) * 8;
      const int64_t gi = m0 + row, gk = (int64_t)kt * BK + kc;
      if (gi < M && gk + 8 <= K) {
        areg[h] = __ldg(reinterpret_cast<const uint4*>(Ag + gi * lda + gk));
      } else {
        int16_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (gi < M && gk + e < K) ? Ag[gi * lda + gk + e] : kInf;
        areg[h] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
      }
    }
  };
  auto store_a_smem = [&](int buf) {
    uint32_t* dst = As + buf * AS_WORDS;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * NT, row = c >> 2, kc = (c & 3) * 8;
      const uint32_t w[4] = {areg[h].x, areg[h].y, areg[h].z, areg[h].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dst[(kc + 2 * q) * BM + row] = __byte_perm(w[q], 0, 0x1010);      // low half in both halves
        dst[(kc + 2 * q + 1) * BM + row] = __byte_perm(w[q], 0, 0x3232);  // high half in both halves
      }
    }
  };
  auto load_b_stage = [&](int kt, int stage) {
    uint32_t* dst = Bs + stage * BSW;
    if (full_mn && kt < kt_full) {
#pragma unroll
      for (int h = 0; h < NBC; ++h) {
        const int c = tid + h * NT;
        cp_async16(dst + (c / CPR) * (BNT / 2) + (c % CPR) * 4, b_src[h] + (int64_t)kt * b_step);
      }
      return;
    }
#pragma unroll
    for (int h = 0; h < NBC; ++h) {
      const int c = tid + h * NT, kr = c / CPR, jc = (c % CPR) * 8;
      const int64_t gk = (int64_t)kt * BK + kr, gj = n0 + jc;
      uint32_t* d = dst + kr * (BNT / 2) + jc / 2;
      if (gk < K && gj + 8 <= N) {
        cp_async16(d, Bg + gk * ldb + gj);
      } else {
        int16_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (gk < K && gj + e < N) ? Bg[gk * ldb + gj + e] : kInf;
        *reinterpret_cast<uint4*>(d) =
            make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
      }
    }
  };

  uint32_t acc[8][NV];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[r][c] = kInf2;

  // ---- prologue
#pragma unroll
  for (int s = 0; s < BSTAGES - 1; ++s) {
    if (s < KT) load_b_stage(s, s);
    cp_async_commit();
  }
  if (KT > 0) {
    load_a_regs(0);
    store_a_smem(0);
  }
  if (KT > 1) load_a_regs(1);
  cp_async_wait<BSTAGES - 2>();
  __syncthreads();

  // ---- main loop
  for (int kt = 0; kt < KT; ++kt) {
    {
      const int nk = kt + BSTAGES - 1;
      if (nk < KT) load_b_stage(nk, nk % BSTAGES);
      cp_async_commit();
    }
    const uint32_t* a_s = As + (kt & 1) * AS_WORDS + ty * 8;
    const uint32_t* b_s = Bs + (kt % BSTAGES) * BSW + tx * 4;
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(a_s + kk * BM);
      const uint4 a1 = *reinterpret_cast<const uint4*>(a_s + kk * BM + 4);
      const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      uint32_t b[NV];
#pragma unroll
      for (int part = 0; part < PARTS; ++part) {
        const uint4 bp = *reinterpret_cast<const uint4*>(b_s + kk * (BNT / 2) + part * 64);
        b[part * 4] = bp.x;
        b[part * 4 + 1] = bp.y;
        b[part * 4 + 2] = bp.z;
        b[part * 4 + 3] = bp.w;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[r][c] = __viaddmin_s16x2(a[r], b[c], acc[r][c]);
    }
    if (kt + 1 < KT) {
      store_a_smem((kt + 1) & 1);
      if (kt + 2 < KT) load_a_regs(kt + 2);
    }
    cp_async_wait<BSTAGES - 2>();
    __syncthreads();
  }

  if (SPLIT) {
    cp_async_wait<0>();
    __syncthreads();  // no copy in flight and no warp still reading the staging buffers
    uint4* T = reinterpret_cast<uint4*>(smem);
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int part = 0; part < PARTS; ++part)
        T[(ty * 8 + r) * (BNT / 8) + part * 16 + tx] =
            make_uint4(acc[r][part * 4], acc[r][part * 4 + 1], acc[r][part * 4 + 2], acc[r][part * 4 + 3]);
    return;
  }

  // ---- epilogue: store, and reduce the minimum and the diagonal minimum
  uint32_t vmin = kInf2;
  int32_t dmin = kInf;
  const bool want_diag = (diag_out != nullptr) && (m0 < n0 + BNT) && (n0 < m0 + BM);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t gi = m0 + ty * 8 + r;
#pragma unroll
    for (int part = 0; part < PARTS; ++part) {
      const int64_t gj = n0 + part * 128 + tx * 8;
      const uint32_t* w = &acc[r][part * 4];
#pragma unroll
      for (int c = 0; c < 4; ++c) vmin = __vmins2(vmin, w[c]);
      if (gi < M) {
        if (gj + 8 <= N) {
          *reinterpret_cast<uint4*>(Cg + gi * ldc + gj) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (gj + e < N) Cg[gi * ldc + gj + e] = (int16_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
        }
        if (want_diag && gi < N) {
#pragma unroll
          for (int e = 0; e < 8; ++e)  // static indexes only, so acc stays in registers
            if (gi == gj + e) dmin = min(dmin, (int32_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF));
        }
      }
    }
  }
  if (min_out != nullptr || want_diag) {
    int32_t lm = min((int32_t)(vmin & 0xFFFF), (int32_t)(vmin >> 16));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lm = min(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
      dmin = min(dmin, __shfl_xor_sync(0xFFFFFFFFu, dmin, o));
    }
    __shared__ int32_t red_m[NT / 32], red_d[NT / 32];
    if ((tid & 31) == 0) {
      red_m[tid >> 5] = lm;
      red_d[tid >> 5] = dmin;
    }
    __syncthreads();
    if (tid == 0) {
      int32_t bm = kInf, bd = kInf;
      for (int w = 0; w < NT / 32; ++w) {
        bm = min(bm, red_m[w]);
        bd = min(bd, red_d[w]);
      }
      if (min_out != nullptr && bm < kInf) atomicMin(min_out, bm);
      if (want_diag && bd < kInf) atomicMin(diag_out, bd);
    }
  }
}

// Grouped rasterisation: consecutive tiles cover kGroupM row tiles x a run of column tiles, so a
// wave of resident CTAs shares its A panels and B panels in L2 instead of sweeping all of B.
__device__ __forceinline__ void grouped_tile(int64_t linear, int64_t gx, int64_t gy, int64_t* tile_m,
                                             int64_t* tile_n) {
  const int64_t per_group = (int64_t)kGroupM * gx;
  const int64_t first_m = (linear / per_group) * kGroupM;
  const int64_t group_rows = (gy - first_m < kGroupM) ? (gy - first_m) : kGroupM;
  const int64_t in_group = linear % per_group;
  *tile_m = first_m + in_group % group_rows;
  *tile_n = in_group / group_rows;
}

template <bool RING, int BNT = BN>
__global__ void __launch_bounds__(NT, BNT == BN ? 2 : 3) minplus_gemm_kernel(GemmParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int16_t* Ag = p.A;
  int16_t* Cg = p.C;
  if (RING) {
    const PowerState* st = p.st;
    if (*(volatile const int32_t*)&st->done) return;
    const int k = *(volatile const int32_t*)&st->k;
    Ag = p.ring + (int64_t)(k % p.slots) * p.slot_elems;
    Cg = p.ring + (int64_t)((k + 1) % p.slots) * p.slot_elems;
  }
  int64_t tm, tn;
  grouped_tile((int64_t)blockIdx.y * gridDim.x + blockIdx.x, gridDim.x, gridDim.y, &tm, &tn);
  gemm_tile<false, BNT>(Ag, p.B, Cg, p.M, p.N, p.K, p.lda, p.ldb, p.ldc, tm * BM, tn * BNT, p.min_out, p.diag_out,
                        smem);
}

// ---- split K for small products: a cluster of S CTAs per output tile, CTA r computing the tile over
// its K slice [r kslice, (r + 1) kslice); the S partial tiles, left in the CTAs' shared memory, meet in
// distributed shared memory, CTA r min-reducing rows [r BM/S, (r + 1) BM/S) of the tile and writing
// them (with the minimum).  Used when the output tiles alone would not fill one wave of the GPU.
template <int BNT>
__global__ void __launch_bounds__(NT, BNT == BN ? 2 : 3) minplus_gemm_splitk_kernel(GemmParams p, int64_t kslice) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) uint32_t smem[];
  const int rank = (int)cluster.block_rank(), S = (int)cluster.num_blocks();
  int64_t tm, tn;
  grouped_tile((int64_t)blockIdx.y * gridDim.x + blockIdx.x, gridDim.x, gridDim.y, &tm, &tn);
  const int64_t m0 = tm * BM, n0 = tn * BNT;
  const int64_t k0 = (int64_t)rank * kslice, k1 = (k0 + kslice < p.K) ? k0 + kslice : p.K;
  gemm_tile<true, BNT>(p.A + k0, p.B + k0 * p.ldb, nullptr, p.M, p.N, k1 - k0, p.lda, p.ldb, p.ldc, m0, n0, nullptr,
                       nullptr, smem);
  cluster.sync();  // every partial tile is in place
  const int rows = BM / S;
  uint32_t vmin = kInf2;
  int32_t emin = kInf;
  for (int v = threadIdx.x; v < rows * (BNT / 8); v += NT) {
    const int row = rank * rows + v / (BNT / 8), c8 = v % (BNT / 8);
    uint4 r = make_uint4(kInf2, kInf2, kInf2, kInf2);
    for (int q = 0; q < S; ++q) {
      const uint4 t = cluster.map_shared_rank(reinterpret_cast<uint4*>(smem), q)[row * (BNT / 8) + c8];
      r = make_uint4(__vmins2(r.x, t.x), __vmins2(r.y, t.y), __vmins2(r.z, t.z), __vmins2(r.w, t.w));
    }
    // the tile's word w covers columns 2w, 2w + 1: vector c8 = part * 16 + tx holds part * 128 + tx * 8 ..
    const int part = c8 / 16, tx = c8 % 16;
    const int64_t gi = m0 + row, gj = n0 + part * 128 + tx * 8;
    if (gi >= p.M || gj >= p.N) continue;
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    if (gj + 8 <= p.N) {
      *reinterpret_cast<uint4*>(p.C + gi * p.ldc + gj) = r;
      vmin = __vmins2(__vmins2(vmin, r.x), __vmins2(__vmins2(r.y, r.z), r.w));
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (gj + e < p.N) {
          const int32_t x = (int32_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
          p.C[gi * p.ldc + gj + e] = (int16_t)x;
          emin = min(emin, x);
        }
    }
  }
  if (p.min_out != nullptr) {
    int32_t lm = min(emin, min((int32_t)(vmin & 0xFFFF), (int32_t)(vmin >> 16)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = min(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
    __shared__ int32_t red_m[NT / 32];
    if ((threadIdx.x & 31) == 0) red_m[threadIdx.x >> 5] = lm;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t bm = kInf;
      for (int w2 = 0; w2 < NT / 32; ++w2) bm = min(bm, red_m[w2]);
      if (bm < kInf) atomicMin(p.min_out, bm);
    }
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// ---- stream-K for products with few output tiles.  The units of work are (output tile, k-tile) pairs,
// tile by tile in the grouped order; a grid of exactly the resident CTAs (two per SM) takes equal
// contiguous runs of them, so every SM does the same number of add-mins whatever the tile count.  A run
// covers whole tiles in its middle and may start and end partway through a tile.  A CTA computes each
// segment of its run into a partial tile in shared memory; a whole tile goes straight to C.  A partial
// tile goes to the CTA's slot of the workspace (slot 0 for the tile of its first unit, slot 1 for the
// tile of its last), then the CTA counts itself in on that tile; the CTA that arrives last takes the
// minimum of its own partial and the others' slots and writes C.  Min is exact and order-free, so the
// result is bit-identical to one CTA per tile.  Nothing waits on another CTA; the last CTA resets the
// tile's counter, so the workspace's counters are zero again when the launch ends.
// Unit arithmetic is 32-bit: the host takes this form only when U * gridDim.x < 2^32.
struct StreamK {
  uint32_t gx, gy;  // column and row tiles of C
  uint32_t KT;      // k-tiles per tile
  uint32_t U;       // units: gx * gy * KT
  uint4* part;      // [2 * gridDim.x][BM * BN / 8] partial tiles
  uint32_t* cnt;    // [gx * gy] CTAs arrived per tile; zero between launches
};

constexpr int kSkVec = BM * BN / 8;  // 16-byte vectors of one partial tile
constexpr int kSkBatch = 8;          // vectors a thread reduces at once (kSkVec is a multiple of NT * kSkBatch)
static_assert(kSkVec % (NT * kSkBatch) == 0, "the reduction's batches cover the tile exactly");
static_assert((size_t)kSkVec * 16 <= SMEM_BYTES, "a partial tile fits in the staging buffers");

__device__ __forceinline__ uint32_t sk_first_unit(uint32_t c, uint32_t U, uint32_t G) { return c * U / G; }
// the CTA whose run holds unit u: the largest c with sk_first_unit(c) <= u
__device__ __forceinline__ uint32_t sk_cta_of(uint32_t u, uint32_t U, uint32_t G) { return ((u + 1) * G - 1) / U; }

// Writes vector v of a 128 x 256 tile at (m0, n0) of C (the layout gemm_tile<true> leaves in shared
// memory: row v / 32, columns (v % 32 / 16) * 128 + (v % 16) * 8 ..), folding its entries into vmin/emin.
__device__ __forceinline__ void sk_store(const GemmParams& p, int64_t m0, int64_t n0, int v, const uint4& r,
                                         uint32_t& vmin, int32_t& emin) {
  const int row = v / (BN / 8), c8 = v % (BN / 8);
  const int64_t gi = m0 + row, gj = n0 + (c8 / 16) * 128 + (c8 % 16) * 8;
  if (gi >= p.M || gj >= p.N) return;
  if (gj + 8 <= p.N) {
    *reinterpret_cast<uint4*>(p.C + gi * p.ldc + gj) = r;
    vmin = __vmins2(__vmins2(vmin, r.x), __vmins2(__vmins2(r.y, r.z), r.w));
  } else {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (gj + e < p.N) {
        const int32_t x = (int32_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
        p.C[gi * p.ldc + gj + e] = (int16_t)x;
        emin = min(emin, x);
      }
  }
}

// The segment a CTA works on: its first unit and the tile's coordinates, derived from the CTA's run.
struct SkSeg {
  uint32_t t, ka, kb;
  int64_t m0, n0;
};
__device__ __forceinline__ SkSeg sk_segment(const StreamK& sk, uint32_t u, uint32_t u_end) {
  SkSeg g;
  g.t = u / sk.KT;
  g.ka = u - g.t * sk.KT;
  g.kb = (sk.KT - g.ka < u_end - u) ? sk.KT : g.ka + (u_end - u);
  // the grouped order of grouped_tile, in 32-bit arithmetic
  const uint32_t per_group = (uint32_t)kGroupM * sk.gx, first_m = g.t / per_group * kGroupM;
  const uint32_t group_rows = (sk.gy - first_m < (uint32_t)kGroupM) ? sk.gy - first_m : (uint32_t)kGroupM;
  const uint32_t in_group = g.t % per_group;
  g.m0 = (int64_t)(first_m + in_group % group_rows) * BM;
  g.n0 = (int64_t)(in_group / group_rows) * BN;
  return g;
}

// Folds a thread's minimum of the entries it wrote into min_out (one atomic per warp).
__device__ __forceinline__ void sk_min_out(int32_t* min_out, uint32_t vmin, int32_t emin) {
  int32_t lm = min(emin, min((int32_t)(vmin & 0xFFFF), (int32_t)(vmin >> 16)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lm = min(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
  if ((threadIdx.x & 31) == 0 && lm < kInf) atomicMin(min_out, lm);
}

__global__ void __launch_bounds__(NT, 2) minplus_gemm_streamk_kernel(GemmParams p, StreamK sk) {
  extern __shared__ __align__(16) uint32_t smem[];
  // the run's position lives in shared memory, so no register is held across the tile's main loop
  __shared__ uint32_t s_u;
  __shared__ int s_last;
  const uint4* T = reinterpret_cast<const uint4*>(smem);
  if (threadIdx.x == 0) s_u = sk_first_unit(blockIdx.x, sk.U, gridDim.x);
  __syncthreads();
  for (;;) {
    const uint32_t u = *(volatile uint32_t*)&s_u, u_end = sk_first_unit(blockIdx.x + 1, sk.U, gridDim.x);
    if (u >= u_end) break;
    {
      const SkSeg g = sk_segment(sk, u, u_end);
      const int64_t k0 = (int64_t)g.ka * BK, klen = (int64_t)(g.kb - g.ka) * BK;
      const int64_t kext = (p.K - k0 < klen) ? p.K - k0 : klen;
      gemm_tile<true, BN>(p.A + k0, p.B + k0 * p.ldb, nullptr, p.M, p.N, kext, p.lda, p.ldb, p.ldc, g.m0, g.n0,
                          nullptr, nullptr, smem);
    }
    __syncthreads();  // the partial tile is complete in shared memory
    const uint32_t G = gridDim.x, c = blockIdx.x;
    const uint32_t uu = *(volatile uint32_t*)&s_u;
    const SkSeg g = sk_segment(sk, uu, u_end);
    uint32_t vmin = kInf2;
    int32_t emin = kInf;
    if (g.ka == 0 && g.kb == sk.KT) {
      for (int v = threadIdx.x; v < kSkVec; v += NT) sk_store(p, g.m0, g.n0, v, T[v], vmin, emin);
    } else {
      const uint32_t cf = sk_cta_of(g.t * sk.KT, sk.U, G), cl = sk_cta_of((g.t + 1) * sk.KT - 1, sk.U, G);
      const uint32_t first_tile = sk_first_unit(c, sk.U, G) / sk.KT;
      uint4* mine = sk.part + (int64_t)(2 * c + (g.t == first_tile ? 0 : 1)) * kSkVec;
      for (int v = threadIdx.x; v < kSkVec; v += NT) __stcg(mine + v, T[v]);
      __threadfence();  // this CTA's partial is visible before it is counted
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(sk.cnt + g.t, 1u) == cl - cf);
      __syncthreads();
      if (s_last) {
        __threadfence();
        // kSkBatch vectors per thread at a time, each partial's kSkBatch loads in flight together
        for (int v0 = threadIdx.x; v0 < kSkVec; v0 += NT * kSkBatch) {
          uint4 r[kSkBatch];
#pragma unroll
          for (int i = 0; i < kSkBatch; ++i) r[i] = T[v0 + i * NT];
          for (uint32_t q = cf; q <= cl; ++q) {
            if (q == c) continue;
            const uint32_t slot = 2 * q + (g.t == sk_first_unit(q, sk.U, G) / sk.KT ? 0 : 1);
            const uint4* src = sk.part + (int64_t)slot * kSkVec + v0;
            uint4 o[kSkBatch];
#pragma unroll
            for (int i = 0; i < kSkBatch; ++i) o[i] = __ldcg(src + i * NT);
#pragma unroll
            for (int i = 0; i < kSkBatch; ++i)
              r[i] = make_uint4(__vmins2(r[i].x, o[i].x), __vmins2(r[i].y, o[i].y), __vmins2(r[i].z, o[i].z),
                                __vmins2(r[i].w, o[i].w));
          }
#pragma unroll
          for (int i = 0; i < kSkBatch; ++i) sk_store(p, g.m0, g.n0, v0 + i * NT, r[i], vmin, emin);
        }
        if (threadIdx.x == 0) sk.cnt[g.t] = 0u;  // every contributor has arrived: ready for the next launch
      }
    }
    if (p.min_out != nullptr) sk_min_out(p.min_out, vmin, emin);
    __syncthreads();  // the partial tile is read before the next segment's prologue overwrites it
    if (threadIdx.x == 0) s_u = uu + (g.kb - g.ka);
    __syncthreads();
  }
}

// ---- batched products: one persistent launch over the tiles of up to kMaxBatch products

constexpr int kMaxBatch = 128;

struct BatchProblem {
  const int16_t* A;
  const int16_t* B;
  int16_t* C;
  int64_t lda, ldb, ldc, M, N, K;
  int32_t* min_out;
  int64_t tiles_m, tiles_n;
};

struct BatchParams {
  int count;
  int64_t tile_start[kMaxBatch + 1];  // prefix sums of the tile counts, in schedule order
  BatchProblem p[kMaxBatch];
};

// CTA c takes tiles c, c + gridDim.x, ... of the concatenated tile list.  Problems are
// ordered by decreasing K (tile cost), so the round robin hands out the long tiles first.
__global__ void __launch_bounds__(NT, 2) minplus_gemm_batched_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int64_t total = bp.tile_start[bp.count];
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = bp.count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bp.tile_start[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const BatchProblem& q = bp.p[lo];
    int64_t tm, tn;
    grouped_tile(t - bp.tile_start[lo], q.tiles_n, q.tiles_m, &tm, &tn);
    __syncthreads();  // the previous tile's shared memory is no longer read
    gemm_tile(q.A, q.B, q.C, q.M, q.N, q.K, q.lda, q.ldb, q.ldc, tm * BM, tn * BN, q.min_out, nullptr, smem);
  }
}

struct MinOutList {
  int count;
  int32_t* p[kMaxBatch];
};

__global__ void fill_min_outs_kernel(const __grid_constant__ MinOutList l) {
  for (int i = threadIdx.x; i < l.count; i += blockDim.x)
    if (l.p[i] != nullptr) *l.p[i] = kInf;
}

__global__ void fill_i32_kernel(int32_t* dst, int32_t v) { *dst = v; }

// ---- vector x matrix: y[j] = min_k x[k] + B[k][j] (one row of C).  Bound by HBM (B is read
// once), so the kernel is laid out for bandwidth: a CTA owns 32 columns, held by groups of 4
// lanes (8 columns each, one 16-byte load per row); its 128 groups split K, each streaming its
// slice of rows with four loads in flight; x sits in shared memory (duplicated into both
// halfwords once), and the groups' partial minima are combined in shared memory at the end.
// N = 16384 gives 512 CTAs of 512 threads.
constexpr int kGemvLanes = 4, kGemvCols = kGemvLanes * 8, kGemvThreads = 512;
constexpr int kGemvGroups = kGemvThreads / kGemvLanes, kGemvXChunk = 8192, kGemvUnroll = 4;

__global__ void __launch_bounds__(kGemvThreads) minplus_gemv_kernel(const int16_t* __restrict__ x,
                                                                    const int16_t* __restrict__ B, int64_t ldb,
                                                                    int16_t* __restrict__ y, int64_t N, int64_t K,
                                                                    int32_t* min_out) {
  __shared__ uint32_t xs[kGemvXChunk];
  __shared__ uint4 part[kGemvGroups][kGemvLanes];
  const int li = threadIdx.x % kGemvLanes, g = threadIdx.x / kGemvLanes;
  const int64_t col = (int64_t)blockIdx.x * kGemvCols + li * 8;
  const bool full = col + 8 <= N, any = col < N;
  uint32_t acc[4] = {kInf2, kInf2, kInf2, kInf2};
  for (int64_t k0 = 0; k0 < K; k0 += kGemvXChunk) {
    const int kc = (K - k0 < kGemvXChunk) ? (int)(K - k0) : kGemvXChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < kc; i += blockDim.x) xs[i] = (uint32_t)(uint16_t)x[k0 + i] * 0x00010001u;
    __syncthreads();
    const int per = (kc + kGemvGroups - 1) / kGemvGroups;
    const int kb = g * per, ke = (kb + per < kc) ? kb + per : kc;
    const int16_t* bp = B + (k0 + kb) * ldb + col;
    int k = kb;
    if (full) {
      for (; k + kGemvUnroll <= ke; k += kGemvUnroll, bp += kGemvUnroll * ldb) {
        uint4 v[kGemvUnroll];
#pragma unroll
        for (int u = 0; u < kGemvUnroll; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(bp + u * ldb));
#pragma unroll
        for (int u = 0; u < kGemvUnroll; ++u) {
          const uint32_t xw = xs[k + u];
          acc[0] = __viaddmin_s16x2(v[u].x, xw, acc[0]);
          acc[1] = __viaddmin_s16x2(v[u].y, xw, acc[1]);
          acc[2] = __viaddmin_s16x2(v[u].z, xw, acc[2]);
          acc[3] = __viaddmin_s16x2(v[u].w, xw, acc[3]);
        }
      }
    }
    for (; k < ke && any; ++k, bp += ldb) {
      const uint32_t xw = xs[k];
      if (full) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(bp));
        acc[0] = __viaddmin_s16x2(v.x, xw, acc[0]);
        acc[1] = __viaddmin_s16x2(v.y, xw, acc[1]);
        acc[2] = __viaddmin_s16x2(v.z, xw, acc[2]);
        acc[3] = __viaddmin_s16x2(v.w, xw, acc[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t b = (col + e < N) ? (uint32_t)(uint16_t)bp[e] : (uint32_t)kInf;
          const uint32_t sh = 16 * (e & 1);
          const uint32_t cur = (acc[e >> 1] >> sh) & 0xFFFFu;
          const uint32_t cand = b + (xw & 0xFFFFu);
          const uint32_t nv = cand < cur ? cand : cur;
          acc[e >> 1] = (acc[e >> 1] & ~(0xFFFFu << sh)) | (nv << sh);
        }
      }
    }
  }
  part[g][li] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
  __syncthreads();
  // tree over the groups, then the first kGemvLanes threads store
  for (int span = kGemvGroups / 2; span > 0; span >>= 1) {
    if (g < span) {
      uint4 r = part[g][li];
      const uint4 q = part[g + span][li];
      r.x = __vmins2(r.x, q.x);
      r.y = __vmins2(r.y, q.y);
      r.z = __vmins2(r.z, q.z);
      r.w = __vmins2(r.w, q.w);
      part[g][li] = r;
    }
    __syncthreads();
  }
  if (threadIdx.x < kGemvLanes) {
    const uint4 r = part[0][li];
    const uint32_t w4[4] = {r.x, r.y, r.z, r.w};
    int32_t lm = kInf;
    if (full) {
      *reinterpret_cast<uint4*>(y + col) = r;
#pragma unroll
      for (int e = 0; e < 8; ++e) lm = min(lm, (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFF));
    } else if (any) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (col + e < N) {
          const int32_t v = (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
          y[col + e] = (int16_t)v;
          lm = min(lm, v);
        }
    }
    if (min_out != nullptr && lm < kInf) atomicMin(min_out, lm);
  }
}

template <int WHICH>  // 0 plain, 1 ring, 2 batched, 3 split K, 4 plain narrow, 5 split K narrow, 6 stream-K
cudaError_t set_smem_attr() {
  static int done_dev[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done_dev[dev]) return cudaSuccess;
  if (WHICH == 0)
    e = cudaFuncSetAttribute(minplus_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  else if (WHICH == 1)
    e = cudaFuncSetAttribute(minplus_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  else if (WHICH == 3)
    e = cudaFuncSetAttribute(minplus_gemm_splitk_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
  else if (WHICH == 4)
    e = cudaFuncSetAttribute(minplus_gemm_kernel<false, BN_NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(BN_NARROW));
  else if (WHICH == 5)
    e = cudaFuncSetAttribute(minplus_gemm_splitk_kernel<BN_NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(BN_NARROW));
  else if (WHICH == 6)
    e = cudaFuncSetAttribute(minplus_gemm_streamk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
  else
    e = cudaFuncSetAttribute(minplus_gemm_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done_dev[dev] = 1;
  return e;
}

}  // namespace

cudaError_t launch_fill_i32(int32_t* dst, int32_t value, cudaStream_t s) {
  fill_i32_kernel<<<1, 1, 0, s>>>(dst, value);
  return cudaGetLastError();
}

// Split K when the output tiles alone fill less than one wave (2 CTAs per SM): S in {2, 4, 8}, the
// smallest that fills it, with every K slice at least 8 k-tiles deep and none empty.  (Shorter slices
// measured slower: at N = 1024, 8 slices of 128 took 0.051 ms against 0.045 ms for 4 of 256.)
int splitk_factor(int64_t tiles, int64_t K) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t wave = 2 * (int64_t)sms;
  int S = 1;
  while (S < 8 && tiles * S < wave && K >= (int64_t)(2 * S) * 8 * BK) S *= 2;
  if (S > 1) {
    const int64_t kslice = ((K + S - 1) / S + BK - 1) / BK * BK;
    while (S > 1 && (int64_t)(S - 1) * kslice >= K) S /= 2;  // every slice non-empty
  }
  return S;
}

bool splitk_suits(int S, int64_t K) {
  if (S == 1) return true;
  if (S != 2 && S != 4 && S != 8) return false;
  const int64_t kslice = ((K + S - 1) / S + BK - 1) / BK * BK;
  return (int64_t)(S - 1) * kslice < K;
}

int64_t gemm_tiles(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + BN - 1) / BN); }

cudaError_t launch_minplus_gemm(const GemmParams& p, bool ring, cudaStream_t s, int force_splitk, int force_tile) {
  int S = 1;     // ring mode and the diagonal output keep one CTA per tile (no diagonal in the split form)
  int tile = 0;  // 0: BM x BN, 1: BM x BN_NARROW (no ring mode, no diagonal)
  if (force_splitk > 0) {
    if (ring || p.diag_out != nullptr || !splitk_suits(force_splitk, p.K) || force_tile < 0 || force_tile > 1)
      return cudaErrorInvalidValue;
    S = force_splitk;
    tile = force_tile;
  } else if (!ring && p.diag_out == nullptr) {
    rd_tune_entry_t t;
    const int64_t mn = p.M > p.N ? p.M : p.N;
    if (tune_find(RD_TUNE_GEMM_SPLITK, rd_tune_bucket(mn), rd_tune_bucket(p.K), &t) && splitk_suits(t.p[0], p.K)) {
      S = t.p[0];
      tile = t.p[1];
    } else {
      S = splitk_factor(gemm_tiles(p.M, p.N), p.K);
    }
  }
  const int bn = tile ? BN_NARROW : BN;
  const size_t smem = tile ? smem_bytes(BN_NARROW) : SMEM_BYTES;
  const int64_t gx = (p.N + bn - 1) / bn, gy = (p.M + BM - 1) / BM;
  if (gx <= 0 || gy <= 0) return cudaSuccess;
  if (gx > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)gx, (unsigned)gy);
  cudaError_t e;
  if (S > 1) {
    e = tile ? set_smem_attr<5>() : set_smem_attr<3>();
    if (e != cudaSuccess) return e;
    const int64_t kslice = ((p.K + S - 1) / S + BK - 1) / BK * BK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gx, (unsigned)gy, (unsigned)S);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = (unsigned)S;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = tile ? cudaLaunchKernelEx(&cfg, minplus_gemm_splitk_kernel<BN_NARROW>, p, kslice)
             : cudaLaunchKernelEx(&cfg, minplus_gemm_splitk_kernel<BN>, p, kslice);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  if (ring) {
    e = set_smem_attr<1>();
    if (e != cudaSuccess) return e;
    minplus_gemm_kernel<true><<<grid, NT, SMEM_BYTES, s>>>(p);
  } else if (tile) {
    e = set_smem_attr<4>();
    if (e != cudaSuccess) return e;
    minplus_gemm_kernel<false, BN_NARROW><<<grid, NT, smem, s>>>(p);
  } else {
    e = set_smem_attr<0>();
    if (e != cudaSuccess) return e;
    minplus_gemm_kernel<false><<<grid, NT, SMEM_BYTES, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace rd

using namespace rd;

extern "C" rd_status rd_minplus_gemm(const int16_t* A, int64_t lda, const int16_t* B, int64_t ldb, int16_t* C,
                                     int64_t ldc, int64_t M, int64_t N, int64_t K, int32_t* min_out,
                                     cudaStream_t s) {
  if (M < 0 || N < 0 || K < 0) return RD_ERR_ARG;
  if (M > 0 && N > 0) {
    if (!C || !aligned16(C) || ldc < N || ldc % 8 != 0) return RD_ERR_ARG;
    if (K > 0) {
      if (!A || !B || !aligned16(A) || !aligned16(B)) return RD_ERR_ARG;
      if (lda < K || lda % 8 != 0 || ldb < N || ldb % 8 != 0) return RD_ERR_ARG;
    }
  }
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  }
  if (M == 0 || N == 0) return RD_OK;
  if (M == 1) return rd_minplus_gemv(A, B, ldb, C, N, K, min_out, s);  // one row: the bandwidth-bound kernel
  GemmParams p{};
  p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
  p.M = M; p.N = N; p.K = K; p.min_out = min_out; p.diag_out = nullptr;
  e = launch_minplus_gemm(p, false, s);
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}

namespace rd {
namespace {

// Stream-K workspace: two partial tiles per CTA of the largest grid (two CTAs per SM), then the per-tile
// counters.  The counters start at the same offset for every shape, so the zeros one call leaves are the
// zeros the next call counts from, whatever its shape.
struct SkLayout {
  int64_t tiles, grid;
  size_t cnt_bytes, part_bytes;
};
bool sk_layout(int64_t M, int64_t N, int64_t K, SkLayout* L) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms < 1) {
    set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidDevice);
    return false;
  }
  const int64_t gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM, KT = (K + BK - 1) / BK;
  L->tiles = gx * gy;
  const int64_t U = L->tiles * KT;
  L->grid = (U < 2 * (int64_t)sms) ? U : 2 * (int64_t)sms;
  L->cnt_bytes = ((size_t)L->tiles * 4 + 255) / 256 * 256;
  L->part_bytes = (size_t)(2 * sms) * 2 * (size_t)kSkVec * 16;
  return true;
}

}  // namespace
}  // namespace rd

extern "C" rd_status rd_minplus_gemm_streamk_work_bytes(int64_t M, int64_t N, int64_t K, size_t* bytes) {
  if (!bytes || M < 0 || N < 0 || K < 0) return RD_ERR_ARG;
  SkLayout L;
  if (!sk_layout(M, N, K, &L)) return RD_ERR_CUDA;
  *bytes = L.cnt_bytes + L.part_bytes;
  return RD_OK;
}

extern "C" rd_status rd_minplus_gemm_streamk(const int16_t* A, int64_t lda, const int16_t* B, int64_t ldb, int16_t* C,
                                             int64_t ldc, int64_t M, int64_t N, int64_t K, void* work,
                                             size_t work_bytes, int32_t* min_out, cudaStream_t s) {
  if (M < 0 || N < 0 || K < 0) return RD_ERR_ARG;
  if (M > 0 && N > 0) {
    if (!C || !aligned16(C) || ldc < N || ldc % 8 != 0) return RD_ERR_ARG;
    if (K > 0) {
      if (!A || !B || !aligned16(A) || !aligned16(B)) return RD_ERR_ARG;
      if (lda < K || lda % 8 != 0 || ldb < N || ldb % 8 != 0) return RD_ERR_ARG;
    }
  }
  if (M <= 1 || N == 0 || K == 0)  // no stream-K form: one row, an empty result, or no terms
    return rd_minplus_gemm(A, lda, B, ldb, C, ldc, M, N, K, min_out, s);
  SkLayout L;
  if (!sk_layout(M, N, K, &L)) return RD_ERR_CUDA;
  const int64_t units = L.tiles * ((K + BK - 1) / BK);
  if (units * L.grid >= ((int64_t)1 << 32))  // many waves of whole tiles: the one-CTA-per-tile kernel
    return rd_minplus_gemm(A, lda, B, ldb, C, ldc, M, N, K, min_out, s);
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) != 0) return RD_ERR_ARG;
  if (work_bytes < L.cnt_bytes + L.part_bytes) return RD_ERR_NOMEM;
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  }
  GemmParams p{};
  p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
  p.M = M; p.N = N; p.K = K; p.min_out = min_out; p.diag_out = nullptr;
  StreamK sk{};
  sk.gx = (uint32_t)((N + BN - 1) / BN);
  sk.gy = (uint32_t)((M + BM - 1) / BM);
  sk.KT = (uint32_t)((K + BK - 1) / BK);
  sk.U = (uint32_t)units;
  sk.part = static_cast<uint4*>(work);
  sk.cnt = reinterpret_cast<uint32_t*>(static_cast<char*>(work) + L.part_bytes);
  e = set_smem_attr<6>();
  if (e == cudaSuccess) {
    minplus_gemm_streamk_kernel<<<(unsigned)L.grid, NT, SMEM_BYTES, s>>>(p, sk);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}

// ---- the same product by clusters: a cluster of kGvRanks CTAs owns a band of kGvBand columns and
// splits the rows between its CTAs; in a CTA each warp streams whole 512-byte row segments of the band
// (one 16-byte load per lane, four rows in flight), so B is read in long contiguous runs.  The warps'
// partial minima are combined in shared memory, then the CTAs' across the cluster through distributed
// shared memory: CTA r of the cluster finishes 4 of the band's 32 vectors and writes them.  No
// workspace and no atomics on y; the cluster barriers are hardware barriers (no polling).
constexpr int kGvBand = 256, kGvThreads = 256, kGvRanks = 8, kGvXChunk = 4096, kGvUnroll = 4;
constexpr int kGvWarps = kGvThreads / 32, kGvVecs = kGvBand / 8;

__global__ void __launch_bounds__(kGvThreads) minplus_gemv_cluster_kernel(const int16_t* __restrict__ x,
                                                                          const int16_t* __restrict__ B,
                                                                          int64_t ldb, int16_t* __restrict__ y,
                                                                          int64_t N, int64_t K, int32_t* min_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ uint32_t xs[kGvXChunk];
  __shared__ uint4 part[kGvWarps][kGvVecs];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rank = (int)cluster.block_rank();
  const int64_t col = (int64_t)blockIdx.x * kGvBand + lane * 8;
  const bool full = col + 8 <= N, any = col < N;
  // this CTA's rows
  const int64_t per = (K + kGvRanks - 1) / kGvRanks;
  const int64_t r0 = (int64_t)rank * per, r1 = (r0 + per < K) ? r0 + per : K;
  uint32_t acc[4] = {kInf2, kInf2, kInf2, kInf2};
  for (int64_t k0 = r0; k0 < r1; k0 += kGvXChunk) {
    const int kc = (r1 - k0 < kGvXChunk) ? (int)(r1 - k0) : kGvXChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < kc; i += kGvThreads) xs[i] = (uint32_t)(uint16_t)x[k0 + i] * 0x00010001u;
    __syncthreads();
    int k = warp;
    if (full) {
      const int16_t* bp = B + (k0 + k) * ldb + col;
      for (; k + (kGvUnroll - 1) * kGvWarps < kc; k += kGvUnroll * kGvWarps, bp += kGvUnroll * kGvWarps * ldb) {
        uint4 v[kGvUnroll];
#pragma unroll
        for (int u = 0; u < kGvUnroll; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(bp + u * kGvWarps * ldb));
#pragma unroll
        for (int u = 0; u < kGvUnroll; ++u) {
          const uint32_t xw = xs[k + u * kGvWarps];
          acc[0] = __viaddmin_s16x2(v[u].x, xw, acc[0]);
          acc[1] = __viaddmin_s16x2(v[u].y, xw, acc[1]);
          acc[2] = __viaddmin_s16x2(v[u].z, xw, acc[2]);
          acc[3] = __viaddmin_s16x2(v[u].w, xw, acc[3]);
        }
      }
    }
    for (; k < kc && any; k += kGvWarps) {
      const uint32_t xw = xs[k];
      const int16_t* bp = B + (k0 + k) * ldb + col;
      if (full) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(bp));
        acc[0] = __viaddmin_s16x2(v.x, xw, acc[0]);
        acc[1] = __viaddmin_s16x2(v.y, xw, acc[1]);
        acc[2] = __viaddmin_s16x2(v.z, xw, acc[2]);
        acc[3] = __viaddmin_s16x2(v.w, xw, acc[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t b = (col + e < N) ? (uint32_t)(uint16_t)bp[e] : (uint32_t)kInf;
          const uint32_t sh = 16 * (e & 1);
          const uint32_t cur = (acc[e >> 1] >> sh) & 0xFFFFu;
          const uint32_t cand = b + (xw & 0xFFFFu);
          const uint32_t nv = cand < cur ? cand : cur;
          acc[e >> 1] = (acc[e >> 1] & ~(0xFFFFu << sh)) | (nv << sh);
        }
      }
    }
  }
  part[warp][lane] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
  __syncthreads();
  if (warp == 0) {
    uint4 r = part[0][lane];
    for (int w = 1; w < kGvWarps; ++w) {
      const uint4 q = part[w][lane];
      r = make_uint4(__vmins2(r.x, q.x), __vmins2(r.y, q.y), __vmins2(r.z, q.z), __vmins2(r.w, q.w));
    }
    part[0][lane] = r;
  }
  cluster.sync();  // every CTA's band partial is in its shared memory
  constexpr int kPerRank = kGvVecs / kGvRanks;
  if (threadIdx.x < kPerRank) {
    const int vi = rank * kPerRank + threadIdx.x;
    uint4 r = make_uint4(kInf2, kInf2, kInf2, kInf2);
    for (int q = 0; q < kGvRanks; ++q) {
      const uint4 v = *cluster.map_shared_rank(&part[0][vi], q);
      r = make_uint4(__vmins2(r.x, v.x), __vmins2(r.y, v.y), __vmins2(r.z, v.z), __vmins2(r.w, v.w));
    }
    const int64_t c = (int64_t)blockIdx.x * kGvBand + vi * 8;
    const uint32_t w4[4] = {r.x, r.y, r.z, r.w};
    int32_t lm = kInf;
    if (c + 8 <= N) {
      *reinterpret_cast<uint4*>(y + c) = r;
#pragma unroll
      for (int e = 0; e < 8; ++e) lm = min(lm, (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFF));
    } else if (c < N) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (c + e < N) {
          const int32_t v = (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFF);
          y[c + e] = (int16_t)v;
          lm = min(lm, v);
        }
    }
    if (min_out != nullptr && lm < kInf) atomicMin(min_out, lm);
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

// Which GEMV kernel: the cluster one streams long row segments but has N / 256 bands of 8 CTAs;
// below 16 bands the column-strip kernel keeps more CTAs busy.
bool gemv_use_clusters(int64_t N) { return N >= 16 * kGvBand; }

extern "C" rd_status rd_minplus_gemv(const int16_t* x, const int16_t* B, int64_t ldb, int16_t* y, int64_t N,
                                     int64_t K, int32_t* min_out, cudaStream_t s) {
  if (N < 0 || K < 0) return RD_ERR_ARG;
  if (N > 0 && (!y || (K > 0 && (!x || !B || !aligned16(B) || ldb < N || ldb % 8 != 0)))) return RD_ERR_ARG;
  if (N > 0 && !aligned16(y)) return RD_ERR_ARG;
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  }
  if (N == 0) return RD_OK;
  if (gemv_use_clusters(N)) {
    const int64_t bands = (N + kGvBand - 1) / kGvBand;
    if (bands > 0x7FFFFFFF) return RD_ERR_ARG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)bands, kGvRanks, 1);
    cfg.blockDim = dim3(kGvThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = kGvRanks;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, minplus_gemv_cluster_kernel, x, B, ldb, y, N, K, min_out);
  } else {
    const int64_t grid = (N + kGemvCols - 1) / kGemvCols;
    if (grid > 0x7FFFFFFF) return RD_ERR_ARG;
    minplus_gemv_kernel<<<(unsigned)grid, kGemvThreads, 0, s>>>(x, B, ldb, y, N, K, min_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}

extern "C" rd_status rd_minplus_gemm_batched(const rd_gemm_problem* problems, int count, cudaStream_t s) {
  if (count < 0 || count > kMaxBatch || (count > 0 && !problems)) return RD_ERR_ARG;
  if (count == 0) return RD_OK;
  MinOutList mins{};
  mins.count = count;
  int order[kMaxBatch];
  for (int i = 0; i < count; ++i) {
    const rd_gemm_problem& q = problems[i];
    if (q.M < 0 || q.N < 0 || q.K < 0) return RD_ERR_ARG;
    if (q.M > 0 && q.N > 0) {
      if (!q.C || !aligned16(q.C) || q.ldc < q.N || q.ldc % 8 != 0) return RD_ERR_ARG;
      if (q.K > 0 && (!q.A || !q.B || !aligned16(q.A) || !aligned16(q.B) || q.lda < q.K || q.lda % 8 != 0 ||
                      q.ldb < q.N || q.ldb % 8 != 0))
        return RD_ERR_ARG;
    }
    mins.p[i] = q.min_out;
    order[i] = i;
  }
  // schedule order: decreasing K (the cost of one tile), stable
  for (int i = 1; i < count; ++i)
    for (int j = i; j > 0 && problems[order[j]].K > problems[order[j - 1]].K; --j) {
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  BatchParams bp{};
  bp.count = 0;
  bp.tile_start[0] = 0;
  for (int i = 0; i < count; ++i) {
    const rd_gemm_problem& q = problems[order[i]];
    if (q.M == 0 || q.N == 0) continue;
    BatchProblem& b = bp.p[bp.count];
    b.A = q.A;
    b.B = q.B;
    b.C = q.C;
    b.lda = q.lda;
    b.ldb = q.ldb;
    b.ldc = q.ldc;
    b.M = q.M;
    b.N = q.N;
    b.K = q.K;
    b.min_out = q.min_out;
    b.tiles_m = (q.M + BM - 1) / BM;
    b.tiles_n = (q.N + BN - 1) / BN;
    bp.tile_start[bp.count + 1] = bp.tile_start[bp.count] + b.tiles_m * b.tiles_n;
    ++bp.count;
  }
  fill_min_outs_kernel<<<1, 128, 0, s>>>(mins);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  if (bp.count == 0) return RD_OK;
  e = set_smem_attr<2>();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t total = bp.tile_start[bp.count];
  const int64_t grid = total < 2 * (int64_t)sms ? total : 2 * (int64_t)sms;  // two resident CTAs per SM
  minplus_gemm_batched_kernel<<<(unsigned)grid, NT, SMEM_BYTES, s>>>(bp);
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}
