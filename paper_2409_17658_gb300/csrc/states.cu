// states.cu -- correct words (Definition 4) and the transfer matrix A(G)
// (Sec. 4.A, Corollary 6) built on the GPU.
//
// Words are never materialised as a list on the device: each thread turns a
// state index r into its code by unranking against a table T[len][letter] =
// number of correct words of length len whose first letter is `letter`.  That
// makes the enumerator one kernel with no scan and no scratch, and lets the
// transfer builder regenerate the words of its tile in shared memory.
#include <cstring>
#include <string>

#include "rd_internal.cuh"

namespace rd {

namespace {

thread_local std::string g_last_error;

// Definition 4 forbids the vertical factors ad, da, ab, ba, bb; `x` sits directly above `y`.
__host__ __device__ inline bool pair_allowed(int x, int y) {
  // bit (4*x + y) set = forbidden: ad(0,3) da(3,0) ab(0,1) ba(1,0) bb(1,1)
  constexpr uint32_t forbidden = (1u << 3) | (1u << 12) | (1u << 1) | (1u << 4) | (1u << 5);
  return ((forbidden >> (4 * x + y)) & 1u) == 0;
}

struct WordTable {
  int m;
  int64_t t[RD_MAX_M + 1][4];  // t[len][c]: correct words of length len starting with letter c
};

WordTable make_table(int m) {
  WordTable w{};
  w.m = m;
  for (int c = 0; c < 4; ++c) w.t[1][c] = 1;
  for (int len = 2; len <= m; ++len)
    for (int c = 0; c < 4; ++c) {
      int64_t s = 0;
      for (int d = 0; d < 4; ++d)
        if (pair_allowed(c, d)) s += w.t[len - 1][d];
      w.t[len][c] = s;
    }
  return w;
}

// r-th correct word in lexicographic order (a < b < c < d, row 1 most significant).
__device__ inline uint32_t unrank(const WordTable& w, int64_t r) {
  uint32_t code = 0;
  int prev = -1;
  for (int i = 1; i <= w.m; ++i) {
    const int len = w.m - i + 1;
    for (int c = 0; c < 4; ++c) {
      if (prev >= 0 && !pair_allowed(prev, c)) continue;
      const int64_t cnt = w.t[len][c];
      if (r < cnt) {
        code = (code << 2) | (uint32_t)c;
        prev = c;
        break;
      }
      r -= cnt;
    }
  }
  return code;
}

// Rows holding each letter, as bit masks (bit b = row m - b).
struct Masks {
  uint32_t a, b, c, d;
};

__device__ inline Masks word_masks(uint32_t code, int m) {
  Masks k{0, 0, 0, 0};
  for (int bit = 0; bit < m; ++bit) {
    const uint32_t l = (code >> (2 * bit)) & 3u;
    const uint32_t one = 1u << bit;
    k.a |= (l == 0) ? one : 0u;
    k.b |= (l == 1) ? one : 0u;
    k.c |= (l == 2) ? one : 0u;
    k.d |= (l == 3) ? one : 0u;
  }
  return k;
}

__device__ inline int word_weight(const Masks& k) { return 2 * __popc(k.a) + __popc(k.b); }

// "p can follow q", all rows at once.  Row by row (Sec. 4.A):
//   q_i = a -> p_i in {a, c}
//   q_i = b -> p_i = d, or p_i = c with an a directly above or below it in p
//   q_i = c -> p_i in {a, b, d}, or p_i = c with an a above or below it in p
//   q_i = d -> p_i = a
// The first and last rows have one vertical neighbour, which the shifts give
// by construction; for m = 1 there is none.
__device__ inline bool can_follow(const Masks& q, const Masks& p, uint32_t full) {
  const uint32_t near_a = ((p.a << 1) | (p.a >> 1)) & full;
  const uint32_t c_with_a = p.c & near_a;
  const uint32_t bad = (q.a & ~(p.a | p.c)) | (q.b & ~(p.d | c_with_a)) |
                       (q.c & ~(p.a | p.b | p.d | c_with_a)) | (q.d & ~p.a);
  return bad == 0;
}

__global__ void enumerate_kernel(WordTable w, int64_t n, uint32_t* codes, uint8_t* weights) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t code = unrank(w, r);
  codes[r] = code;
  weights[r] = (uint8_t)word_weight(word_masks(code, w.m));
}

// Appendix variant: the last row (bit 0) needs no domination, so q_m = d follows the q_m = c rule.
__device__ inline Masks relax_last_row(Masks q) {
  q.c |= q.d & 1u;
  q.d &= ~1u;
  return q;
}

// Algorithm 3, all rows at once: newly dominated vertices of column p after column q,
// plus the vertex below the strip when p_m = a.
__device__ inline int newly_dominated(const Masks& q, const Masks& p) {
  return __popc(q.a & p.a) + __popc(q.b & p.c) + 2 * __popc(q.c & p.a) + __popc((q.c | q.d) & (p.b | p.c)) +
         3 * __popc(q.d & p.a) + (int)(p.a & 1u);
}

// The destination side of "p can follow q", per word p: the rows where a letter of q is NOT satisfied by
// p (Sec. 4.A, as in can_follow): q has an arc to p iff q.a & na | q.b & nb | q.c & nc | q.d & nd == 0.
struct Refuse {
  uint32_t na, nb, nc, nd;
};

__device__ inline Refuse refuse_masks(const Masks& p, uint32_t full) {
  const uint32_t near_a = ((p.a << 1) | (p.a >> 1)) & full;
  const uint32_t c_with_a = p.c & near_a;
  return Refuse{~(p.a | p.c), ~(p.d | c_with_a), ~(p.a | p.b | p.d | c_with_a), ~p.a};
}

// r-th correct word, unranked against the word table held in shared memory (t[len * 4 + c]; every count
// is below 2^31 for m <= RD_MAX_M).
__device__ inline uint32_t unrank_sm(const int32_t* t, int m, int32_t r) {
  uint32_t code = 0;
  int prev = -1;
  for (int i = 1; i <= m; ++i) {
    const int len = m - i + 1;
    for (int c = 0; c < 4; ++c) {
      if (prev >= 0 && !pair_allowed(prev, c)) continue;
      const int32_t cnt = t[len * 4 + c];
      if (r < cnt) {
        code = (code << 2) | (uint32_t)c;
        prev = c;
        break;
      }
      r -= cnt;
    }
  }
  return code;
}

// A CTA writes a band of `rows` (<= kBuildMaxRows) rows (q) x kBuildCols columns (p), one 16-byte store per
// row and thread: thread t owns columns 8t .. 8t + 7 of the band, keeps those 8 destination words' refusal
// masks and labels in registers, and sweeps the band's rows, whose letter masks it reads from shared memory
// (the same word for every thread: a broadcast).  Per entry: four masked tests, a compare and a select.
// The band's words are unranked once (8 per thread for the columns, one per thread for the rows), so the
// prologue is small against the band's 16-byte stores.  LOSS selects the Appendix variant, whose labels
// 10 p(a) + 5 p(b) - 2 nd(q,p) are stored shifted by 2m (never negative).
constexpr int kBuildThreads = 256;
constexpr int kBuildCols = kBuildThreads * 8;
constexpr int kBuildMaxRows = kBuildThreads;

template <bool LOSS>
__global__ void __launch_bounds__(kBuildThreads) transfer_kernel(WordTable w, int64_t n, int16_t* A, int64_t lda,
                                                                 int64_t ctiles, int rows_per_cta) {
  __shared__ int32_t tab[(RD_MAX_M + 1) * 4];
  __shared__ uint4 qm[kBuildMaxRows];
  const int tid = threadIdx.x;
  for (int i = tid; i < (w.m + 1) * 4; i += kBuildThreads) tab[i] = (int32_t)w.t[i >> 2][i & 3];
  __syncthreads();
  const int64_t q0 = (int64_t)(blockIdx.x / ctiles) * rows_per_cta;
  const int64_t pc = (int64_t)(blockIdx.x % ctiles) * kBuildCols + 8 * tid;
  if (tid < rows_per_cta) {
    const int64_t q = q0 + tid;
    Masks k{0, 0, 0, 0};
    if (q < n) k = word_masks(unrank_sm(tab, w.m, (int32_t)q), w.m);
    qm[tid] = make_uint4(k.a, k.b, k.c, k.d);
  }
  const uint32_t full = (w.m >= 32) ? 0xFFFFFFFFu : ((1u << w.m) - 1u);
  Refuse rf[8];
  Masks pk[8];
  int16_t wt[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t p = pc + e;
    if (p < n) {
      pk[e] = word_masks(unrank_sm(tab, w.m, (int32_t)p), w.m);
      rf[e] = refuse_masks(pk[e], full);
      wt[e] = (int16_t)word_weight(pk[e]);
    } else {
      pk[e] = Masks{0, 0, 0, 0};
      rf[e] = Refuse{~0u, ~0u, ~0u, ~0u};  // every row refuses: no arc into a padding column
      wt[e] = kInf;
    }
  }
  __syncthreads();
  if (pc >= lda) return;
  const int rows = (int)((n - q0 < rows_per_cta) ? (n - q0) : rows_per_cta);
  int16_t* dst = A + q0 * lda + pc;
  for (int r = 0; r < rows; ++r, dst += lda) {
    const uint4 qv = qm[r];
    Masks qf{qv.x, qv.y, qv.z, qv.w};
    if (LOSS) qf = relax_last_row(qf);  // the follow rule of the variant; Algorithm 3 takes q as it is
    uint32_t packed[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const Refuse& f = rf[e + h];
        const uint32_t bad = (qf.a & f.na) | (qf.b & f.nb) | (qf.c & f.nc) | (qf.d & f.nd);
        int label = wt[e + h];
        if (LOSS)
          label = 10 * __popc(pk[e + h].a) + 5 * __popc(pk[e + h].b) -
                  2 * newly_dominated(Masks{qv.x, qv.y, qv.z, qv.w}, pk[e + h]) + 2 * w.m;
        v[h] = (uint32_t)(uint16_t)((bad == 0) ? (int16_t)label : kInf);
      }
      packed[e / 2] = v[0] | (v[1] << 16);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
}

// Rows per CTA of the builder's launch: the widest band (256, 128 or 64 rows) that still gives the GPU at
// least three waves of CTAs (4 resident per SM), so the last wave's idle SMs cost little.
int build_rows_per_cta(int64_t n, int64_t ctiles) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int r = kBuildMaxRows; r > 64; r /= 2)
    if (ctiles * ((n + r - 1) / r) >= 3 * 4 * (int64_t)sms) return r;
  return 64;
}

}  // namespace

void set_cuda_error(cudaError_t e) { g_last_error = cudaGetErrorString(e); }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace rd

using namespace rd;

extern "C" const char* rd_last_cuda_error(void) { return g_last_error.c_str(); }

extern "C" rd_status rd_state_count(int m, int64_t* N) {
  if (m < 1 || m > RD_MAX_M || !N) return RD_ERR_ARG;
  const WordTable w = make_table(m);
  int64_t s = 0;
  for (int c = 0; c < 4; ++c) s += w.t[m][c];
  *N = s;
  return RD_OK;
}

extern "C" rd_status rd_padded_dim(int64_t N, int64_t* Np) {
  if (N < 0 || !Np) return RD_ERR_ARG;
  *Np = (N + 7) / 8 * 8;
  return RD_OK;
}

extern "C" rd_status rd_enumerate_states(int m, uint32_t* codes_dev, uint8_t* weights_dev, cudaStream_t s) {
  int64_t n = 0;
  if (rd_state_count(m, &n) != RD_OK || !codes_dev || !weights_dev) return RD_ERR_ARG;
  const WordTable w = make_table(m);
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  enumerate_kernel<<<(unsigned)blocks, threads, 0, s>>>(w, n, codes_dev, weights_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}

extern "C" rd_status rd_build_transfer(int m, int16_t* A_dev, int64_t lda, cudaStream_t s) {
  int64_t n = 0;
  if (rd_state_count(m, &n) != RD_OK || !A_dev) return RD_ERR_ARG;
  if (lda < n || lda % 8 != 0 || !aligned16(A_dev)) return RD_ERR_ARG;
  const WordTable w = make_table(m);
  const int64_t ctiles = (lda + kBuildCols - 1) / kBuildCols;
  const int rpc = build_rows_per_cta(n, ctiles);
  const int64_t tiles = ctiles * ((n + rpc - 1) / rpc);
  if (tiles > 0x7FFFFFFF) return RD_ERR_ARG;
  transfer_kernel<false><<<(unsigned)tiles, kBuildThreads, 0, s>>>(w, n, A_dev, lda, ctiles, rpc);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}

extern "C" rd_status rd_build_transfer_loss(int m, int16_t* A_dev, int64_t lda, cudaStream_t s) {
  int64_t n = 0;
  if (m < 2 || rd_state_count(m, &n) != RD_OK || !A_dev) return RD_ERR_ARG;
  if (lda < n || lda % 8 != 0 || !aligned16(A_dev)) return RD_ERR_ARG;
  const WordTable w = make_table(m);
  const int64_t ctiles = (lda + kBuildCols - 1) / kBuildCols;
  const int rpc = build_rows_per_cta(n, ctiles);
  const int64_t tiles = ctiles * ((n + rpc - 1) / rpc);
  if (tiles > 0x7FFFFFFF) return RD_ERR_ARG;
  transfer_kernel<true><<<(unsigned)tiles, kBuildThreads, 0, s>>>(w, n, A_dev, lda, ctiles, rpc);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return RD_ERR_CUDA; }
  return RD_OK;
}
