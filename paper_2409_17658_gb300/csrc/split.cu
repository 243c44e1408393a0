// split.cu -- the power step R = A(G) (x) B for a transfer matrix A(G), computed from the row
// rules of Sec. 4.A in two passes over the rows of a grid column, without A(G) itself.
//
// The structure used (Sec. 4.A):
//  * the label of an arc q -> p is the weight of the destination word alone,
//    w(p) = 2 p(a) + p(b);
//  * "p can follow q" is decided row by row: row i of q admits a set S(q_i) of row types of p,
//    where the row type of p_i is its letter, with a c split into c+ (a vertical neighbour in p
//    is an a) and c- (none is):
//        S(a) = {a, c+, c-}   S(b) = {d, c+}   S(c) = {a, b, d, c+}   S(d) = {a}.
// With tau(p) the row types of p,
//     R[q][x] = min over p with tau(p)_i in S(q_i) for every row i of  w(p) + B[p][x].
// Split the rows after row j (h = m - j rows below).  Write rho = tau(p)_{1..j} and
// sigma = tau(p)_{j+1..m}; p is determined by (rho, sigma), and the admissible set is the product of
// an admissible set of rho (fixed by q_{1..j}) and one of sigma (fixed by q_{j+1..m}).  So
//     X[pi][sigma][x] = min over rho admitted by pi of  w(p) + B[p][x],  p = (rho, sigma)    (pass 1)
//     R[q][x]         = min over sigma admitted by q_{j+1..m} of  X[q_{1..j}][sigma][x]       (pass 2)
// for pi a correct word of j letters.  Each entry of R is the minimum of exactly the same sums as in
// the direct product (min is exact and the weight is added once), so the result is identical.
//
// Cost: every row of B and every row of X is read once and written once (X has about 1.6 N rows
// for j = m / 2), and the minima take about 36-48 N^2 operations at m = 9, 10 -- against nnz(A) N
// add-mins over gathered rows of B in the sparse step (121 N^2 at m = 9, 206 N^2 at m = 10).
//
// Kernels: a CTA owns one fiber (pass 1: all p sharing sigma; pass 2: all rows of X sharing pi) and
// a slab of W columns.  It stages the fiber's rows in shared memory (slot = rho resp. sigma rank,
// absent rows RD_INF, plus one all-RD_INF dummy slot that pads every admitted list to a multiple
// of four), then forms each output row as the minimum of its admitted slots with 3-input DPX
// minima, 8 columns (one 16-byte vector) per thread.
#include "rd_internal.cuh"

namespace rd {
namespace {

constexpr int kSplitThreads = 256;
constexpr int kSplitMaxLen = 8;  // rows per part (5^8 row-type codes, 4^8 letter codes)
constexpr int kTauA = 0, kTauB = 1, kTauCp = 2, kTauCm = 3, kTauD = 4;
constexpr int kTauCount = 5;
// bit 4x + y set: the factor xy is excluded by Definition 4 (ad, da, ab, ba, bb)
constexpr uint32_t kForbiddenPairs = (1u << (0 * 4 + 3)) | (1u << (3 * 4 + 0)) | (1u << (0 * 4 + 1)) |
                                     (1u << (1 * 4 + 0)) | (1u << (1 * 4 + 1));
// S(letter) as a bit set over row types, for the letters a, b, c, d
__constant__ uint8_t c_admit[4] = {
    (1u << kTauA) | (1u << kTauCp) | (1u << kTauCm),
    (1u << kTauD) | (1u << kTauCp),
    (1u << kTauA) | (1u << kTauB) | (1u << kTauD) | (1u << kTauCp),
    (1u << kTauA)};

// ---------------------------------------------------------------- codes

// letter of row i (1-based) of a code of `len` letters, row 1 most significant
__host__ __device__ inline int letter_at(uint32_t code, int len, int i) { return (int)((code >> (2 * (len - i))) & 3u); }

__host__ __device__ inline bool correct_code(uint32_t code, int len) {
  for (int i = 1; i < len; ++i)
    if ((kForbiddenPairs >> (4 * letter_at(code, len, i) + letter_at(code, len, i + 1))) & 1u) return false;
  return true;
}

__device__ inline int row_type(uint32_t code, int m, int i) {
  const int x = letter_at(code, m, i);
  if (x == 0) return kTauA;
  if (x == 1) return kTauB;
  if (x == 3) return kTauD;
  const bool up = i > 1 && letter_at(code, m, i - 1) == 0;
  const bool down = i < m && letter_at(code, m, i + 1) == 0;
  return (up || down) ? kTauCp : kTauCm;
}

__device__ inline int word_weight_of(uint32_t code, int m) {
  int w = 0;
  for (int i = 1; i <= m; ++i) {
    const int x = letter_at(code, m, i);
    w += (x == 0) ? 2 : (x == 1) ? 1 : 0;
  }
  return w;
}

// Do the letters `w` (len letters) admit the row types `t` (base 5, first row most significant)?
__device__ inline bool admits(uint32_t w, uint32_t t, int len) {
  for (int i = len; i >= 1; --i) {
    const uint32_t ty = t % kTauCount;
    t /= kTauCount;
    if (!((c_admit[letter_at(w, len, i)] >> ty) & 1u)) return false;
  }
  return true;
}

__host__ __device__ inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// ---------------------------------------------------------------- plan layout

// Host-side bound on the distinct row-type strings of `len` rows: each is a correct word of len
// letters with every c marked + or -.
int64_t type_bound(int len) {
  int64_t t = 0;
  for (uint32_t c = 0; c < (1u << (2 * len)); ++c) {
    if (!correct_code(c, len)) continue;
    int64_t v = 1;
    for (int i = 1; i <= len; ++i)
      if (letter_at(c, len, i) == 2) v *= 2;
    t += v;
  }
  return t;
}

// Host-side bound on the padded admitted-list entries of the correct words of `len` letters: a word
// admits at most prod_i |S(w_i)| row-type strings (|S| = 3, 2, 4, 1 for a, b, c, d) and at most
// `types` of them exist.
int64_t list_bound(int len, int64_t types) {
  const int64_t admit_size[4] = {3, 2, 4, 1};
  int64_t t = 0;
  for (uint32_t c = 0; c < (1u << (2 * len)); ++c) {
    if (!correct_code(c, len)) continue;
    int64_t v = 1;
    for (int i = 1; i <= len; ++i) v *= admit_size[letter_at(c, len, i)];
    t += ((v < types ? v : types) + 3) & ~3ll;
  }
  return t;
}

int64_t correct_count(int len) {
  int64_t n = 0;
  return rd_state_count(len, &n) == RD_OK ? n : -1;
}

struct Layout {
  int m, j, h;
  int64_t N, nPi, nPhi, rhoB, sigB, c1B, c2B;
  size_t totals, codes, wts, rankR, rankS, rankPi, rankPhi, rhoCode, sigCode, piCode, phiCode, c1s, c2s, c1, c2, fiber,
      outrow, bytes;
};

bool make_layout(int m, int j, Layout* L) {
  if (m < 2 || m > RD_MAX_M || j < 1 || j >= m) return false;
  const int h = m - j;
  if (j > kSplitMaxLen || h > kSplitMaxLen) return false;
  L->m = m;
  L->j = j;
  L->h = h;
  L->N = correct_count(m);
  L->nPi = correct_count(j);
  L->nPhi = correct_count(h);
  L->rhoB = type_bound(j);
  L->sigB = type_bound(h);
  L->c1B = list_bound(j, L->rhoB);
  L->c2B = list_bound(h, L->sigB);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  L->totals = take(16 * 4);
  L->codes = take((size_t)L->N * 4);
  L->wts = take((size_t)L->N);
  L->rankR = take((size_t)(ipow(kTauCount, j) + 1) * 4);
  L->rankS = take((size_t)(ipow(kTauCount, h) + 1) * 4);
  L->rankPi = take((size_t)(ipow(4, j) + 1) * 4);
  L->rankPhi = take((size_t)(ipow(4, h) + 1) * 4);
  L->rhoCode = take((size_t)L->rhoB * 4);
  L->sigCode = take((size_t)L->sigB * 4);
  L->piCode = take((size_t)L->nPi * 4);
  L->phiCode = take((size_t)L->nPhi * 4);
  L->c1s = take((size_t)(L->nPi + 1) * 4);
  L->c2s = take((size_t)(L->nPhi + 1) * 4);
  L->c1 = take((size_t)L->c1B * 2);
  L->c2 = take((size_t)L->c2B * 2);
  L->fiber = take((size_t)L->sigB * (size_t)L->rhoB * 4);
  L->outrow = take((size_t)L->nPi * (size_t)L->nPhi * 4);
  L->bytes = off;
  return true;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}
template <typename T>
const T* at(const void* base, size_t off) {
  return reinterpret_cast<const T*>(static_cast<const char*>(base) + off);
}

// ---------------------------------------------------------------- plan kernels

// Each correct word of length m marks the row-type codes of its first j rows and of the rest.
__global__ void split_mark_kernel(const uint32_t* codes, int64_t N, int m, int j, int32_t* flagR, int32_t* flagS) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t code = codes[p];
    uint32_t rc = 0, sc = 0;
    for (int i = 1; i <= j; ++i) rc = rc * kTauCount + row_type(code, m, i);
    for (int i = j + 1; i <= m; ++i) sc = sc * kTauCount + row_type(code, m, i);
    flagR[rc] = 1;
    flagS[sc] = 1;
  }
}

__global__ void correct_flag_kernel(int32_t* flags, int len, int64_t n) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    flags[c] = correct_code((uint32_t)c, len) ? 1 : 0;
}

// In-place exclusive scan of v[0..n) with the total written to v[n]; one CTA.
__global__ void scan_i32_kernel(int32_t* v, int64_t n) {
  __shared__ int32_t warp_sums[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int32_t x = (i < n) ? v[i] : 0;
    int32_t y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) y += t;
    }
    if (lane == 31) warp_sums[warp] = y;
    __syncthreads();
    if (warp == 0) {
      int32_t ws = (lane < nwarps) ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xFFFFFFFFu, ws, o);
        if (lane >= o) ws += t;
      }
      if (lane < nwarps) warp_sums[lane] = ws;
    }
    __syncthreads();
    const int32_t incl = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + y;
    if (i < n) v[i] = incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) v[n] = carry;
}

// inv[rank[c]] = c for every present code c (rank is an exclusive scan of presence flags).
__global__ void invert_kernel(const int32_t* rank, int64_t n, int32_t* inv) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (rank[c + 1] > rank[c]) inv[rank[c]] = (int32_t)c;
}

// Admitted lists: for each letter word w (n_w of them, len letters), the row-type strings t among
// the n_t present ones that it admits, in increasing code order, padded with the dummy slot n_t to a
// multiple of four.  count: cnt[w] = padded length; fill: the entries from start[w].
__global__ void list_count_kernel(const int32_t* wcode, int64_t n_w, const int32_t* tcode, int64_t n_t, int len,
                                  int32_t* cnt) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_w; w += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = 0;
    for (int64_t t = 0; t < n_t; ++t) c += admits((uint32_t)wcode[w], (uint32_t)tcode[t], len) ? 1 : 0;
    cnt[w] = (c + 3) & ~3;
  }
}

__global__ void list_fill_kernel(const int32_t* wcode, int64_t n_w, const int32_t* tcode, int64_t n_t, int len,
                                 const int32_t* start, uint16_t* lst) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_w; w += (int64_t)gridDim.x * blockDim.x) {
    int32_t e = start[w];
    for (int64_t t = 0; t < n_t; ++t)
      if (admits((uint32_t)wcode[w], (uint32_t)tcode[t], len)) lst[e++] = (uint16_t)t;
    while (e < start[w + 1]) lst[e++] = (uint16_t)n_t;
  }
}

// fiber[sigma rank][rho rank] = p * 32 + w(p);  outrow[pi rank][phi rank] = q.
__global__ void split_index_kernel(const uint32_t* codes, int64_t N, int m, int j, const int32_t* rankR,
                                   const int32_t* rankS, int64_t n_rho, const int32_t* rankPi,
                                   const int32_t* rankPhi, int64_t n_phi, int32_t* fiber, int32_t* outrow) {
  const int h = m - j;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t code = codes[p];
    uint32_t rc = 0, sc = 0;
    for (int i = 1; i <= j; ++i) rc = rc * kTauCount + row_type(code, m, i);
    for (int i = j + 1; i <= m; ++i) sc = sc * kTauCount + row_type(code, m, i);
    fiber[(int64_t)rankS[sc] * n_rho + rankR[rc]] = (int32_t)(p * 32 + word_weight_of(code, m));
    const uint32_t pi = code >> (2 * h), phi = code & ((1u << (2 * h)) - 1u);
    outrow[(int64_t)rankPi[pi] * n_phi + rankPhi[phi]] = (int32_t)p;
  }
}

// ---------------------------------------------------------------- the two passes

struct SplitPass {
  const int16_t* in;  // pass 1: B (rows p);  pass 2: X
  int64_t ldin;
  int16_t* out;  // pass 1: X;  pass 2: R
  int64_t ldout;
  int64_t ncols;
  int32_t n_slots;  // rows staged per fiber (rho resp. sigma ranks); slot n_slots is the dummy
  int32_t n_out;    // output rows per fiber (pi resp. phi ranks)
  int32_t n_sigma;
  const int32_t* src;     // pass 1: [sigma][rho] = p * 32 + w(p), or -1
  const int32_t* start;   // [n_out + 1] admitted-list starts (multiples of 4)
  const uint16_t* lst;    // admitted slots
  const int32_t* dst;     // pass 2: [pi][phi] = row q of R, or -1
  int32_t* min_out;
  int32_t* diag_out;
  PowerState* st;  // ring mode: B = power slot k (pass 1), R = slot k + 1 (pass 2)
  int16_t* ring;
  int64_t slot_elems;
  int slots;
};

__device__ __forceinline__ uint32_t min3(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_s16x2(a, b, c); }

template <int W, bool FIRST, bool RING>
__global__ void __launch_bounds__(kSplitThreads) split_pass_kernel(SplitPass a) {
  extern __shared__ uint4 sm[];
  constexpr int LR = W / 8;                 // threads per row of the slab
  constexpr int G = kSplitThreads / LR;     // rows handled side by side
  const int16_t* in = a.in;
  int16_t* out = a.out;
  if (RING) {
    if (*(volatile const int32_t*)&a.st->done) return;
    const int k = *(volatile const int32_t*)&a.st->k;
    if (FIRST)
      in = a.ring + (int64_t)(k % a.slots) * a.slot_elems;
    else
      out = a.ring + (int64_t)((k + 1) % a.slots) * a.slot_elems;
  }
  const int lane = threadIdx.x % LR, g = threadIdx.x / LR;
  const int64_t f = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * W + lane * 8;
  const bool ok = c < a.ncols;
  const uint4 inf4 = make_uint4(kInf2, kInf2, kInf2, kInf2);

  // stage the fiber: slots 0..n_slots (the last one is the RD_INF dummy)
  const int nst = a.n_slots + 1;
  for (int s0 = g; s0 < nst; s0 += 4 * G) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * G;
      v[u] = inf4;
      if (s < a.n_slots && ok) {
        if (FIRST) {
          const int32_t e = __ldg(a.src + f * a.n_slots + s);
          if (e >= 0) {
            const uint4 x = __ldg(reinterpret_cast<const uint4*>(in + (int64_t)(e >> 5) * a.ldin + c));
            const uint32_t w2 = (uint32_t)(e & 31) * 0x00010001u;
            v[u] = make_uint4(__viaddmin_s16x2(x.x, w2, kInf2), __viaddmin_s16x2(x.y, w2, kInf2),
                              __viaddmin_s16x2(x.z, w2, kInf2), __viaddmin_s16x2(x.w, w2, kInf2));
          }
        } else {
          v[u] = __ldg(reinterpret_cast<const uint4*>(in + (f * a.n_sigma + s) * a.ldin + c));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = s0 + u * G;
      if (s < nst) sm[s * LR + lane] = v[u];
    }
  }
  __syncthreads();

  int32_t lmin = kInf, ldiag = kInf;
  for (int o = g; o < a.n_out; o += G) {
    int64_t row;
    if (FIRST) {
      row = (int64_t)o * a.n_sigma + f;
    } else {
      row = __ldg(a.dst + f * a.n_out + o);
      if (row < 0) continue;
    }
    const int e0 = __ldg(a.start + o), e1 = __ldg(a.start + o + 1);
    uint4 acc = inf4;
#pragma unroll 2
    for (int e = e0; e < e1; e += 4) {
      const uint2 ix = __ldg(reinterpret_cast<const uint2*>(a.lst + e));
      const uint4 v0 = sm[(int)(ix.x & 0xFFFFu) * LR + lane];
      const uint4 v1 = sm[(int)(ix.x >> 16) * LR + lane];
      const uint4 v2 = sm[(int)(ix.y & 0xFFFFu) * LR + lane];
      const uint4 v3 = sm[(int)(ix.y >> 16) * LR + lane];
      acc.x = min3(min3(acc.x, v0.x, v1.x), v2.x, v3.x);
      acc.y = min3(min3(acc.y, v0.y, v1.y), v2.y, v3.y);
      acc.z = min3(min3(acc.z, v0.z, v1.z), v2.z, v3.z);
      acc.w = min3(min3(acc.w, v0.w, v1.w), v2.w, v3.w);
    }
    if (!ok) continue;
    if (FIRST) {
      *reinterpret_cast<uint4*>(out + row * a.ldout + c) = acc;
    } else {
      const uint32_t w4[4] = {acc.x, acc.y, acc.z, acc.w};
      if (c + 8 <= a.ncols) {
        *reinterpret_cast<uint4*>(out + row * a.ldout + c) = acc;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (c + e < a.ncols) out[row * a.ldout + c + e] = (int16_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (c + e < a.ncols) {
          const int32_t v = (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
          lmin = min(lmin, v);
          if (c + e == row) ldiag = min(ldiag, v);
        }
      }
    }
  }

  if (!FIRST && (a.min_out != nullptr || a.diag_out != nullptr)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xFFFFFFFFu, lmin, o));
      ldiag = min(ldiag, __shfl_xor_sync(0xFFFFFFFFu, ldiag, o));
    }
    __shared__ int32_t red_m[kSplitThreads / 32], red_d[kSplitThreads / 32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red_m[warp] = lmin;
      red_d[warp] = ldiag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t bm = kInf, bd = kInf;
      for (int w = 0; w < kSplitThreads / 32; ++w) {
        bm = min(bm, red_m[w]);
        bd = min(bd, red_d[w]);
      }
      if (a.min_out != nullptr && bm < *(volatile const int32_t*)a.min_out) atomicMin(a.min_out, bm);
      if (a.diag_out != nullptr && bd < *(volatile const int32_t*)a.diag_out) atomicMin(a.diag_out, bd);
    }
  }
}

size_t pass_smem(int n_slots, int W) { return (size_t)(n_slots + 1) * (size_t)W * 2; }

constexpr size_t kSmemTwoPerSm = 112 * 1024, kSmemMax = 220 * 1024;

int choose_w(int n_slots) {
  const int ws[3] = {128, 64, 32};
  for (int w : ws)
    if (pass_smem(n_slots, w) <= kSmemTwoPerSm) return w;
  for (int w : ws)
    if (pass_smem(n_slots, w) <= kSmemMax) return w;
  return 0;
}

bool valid_w(int W, int n_slots) {
  return (W == 32 || W == 64 || W == 128) && pass_smem(n_slots, W) <= kSmemMax;
}

template <bool FIRST, bool RING>
cudaError_t launch_pass(const SplitPass& a, int W, int64_t fibers, cudaStream_t s) {
  const size_t smem = pass_smem(a.n_slots, W);
  const int64_t slabs = (a.ncols + W - 1) / W;
  const dim3 grid((unsigned)slabs, (unsigned)fibers);
  void (*k)(SplitPass) = nullptr;
  switch (W) {
    case 128: k = split_pass_kernel<128, FIRST, RING>; break;
    case 64: k = split_pass_kernel<64, FIRST, RING>; break;
    default: k = split_pass_kernel<32, FIRST, RING>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kSplitThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// The two passes' fixed operands, from a built plan.
void passes_of(const rd_split_info_t& info, const void* plan, SplitPass* p1, SplitPass* p2) {
  Layout L;
  make_layout(info.m, info.j, &L);
  *p1 = SplitPass{};
  *p2 = SplitPass{};
  p1->ncols = p2->ncols = info.N;
  p1->n_slots = info.n_rho;
  p1->n_out = info.n_pi;
  p1->n_sigma = p2->n_sigma = info.n_sigma;
  p1->src = at<int32_t>(plan, L.fiber);
  p1->start = at<int32_t>(plan, L.c1s);
  p1->lst = at<uint16_t>(plan, L.c1);
  p2->n_slots = info.n_sigma;
  p2->n_out = info.n_phi;
  p2->start = at<int32_t>(plan, L.c2s);
  p2->lst = at<uint16_t>(plan, L.c2);
  p2->dst = at<int32_t>(plan, L.outrow);
}

bool info_ok(const rd_split_info_t* info, const void* plan) {
  if (!info || !plan || !aligned16(plan)) return false;
  Layout L;
  if (!make_layout(info->m, info->j, &L)) return false;
  if (info->N != L.N || info->n_pi != L.nPi || info->n_phi != L.nPhi) return false;
  if (info->n_rho < 1 || info->n_rho > L.rhoB || info->n_sigma < 1 || info->n_sigma > L.sigB) return false;
  return valid_w(info->w1, info->n_rho) && valid_w(info->w2, info->n_sigma);
}

struct SplitCtx {
  SplitPass p1, p2;
  int w1, w2;
  int64_t fibers1, fibers2;
};

cudaError_t split_power_product(const Run& r, const void* ctx, cudaStream_t s) {
  const SplitCtx* c = static_cast<const SplitCtx*>(ctx);
  SplitPass p1 = c->p1, p2 = c->p2;
  p1.st = p2.st = r.st;
  p1.ring = p2.ring = r.ring;
  p1.slot_elems = p2.slot_elems = r.slot_elems;
  p1.slots = p2.slots = r.slots;
  p1.ldin = r.ld;
  p2.ldout = r.ld;
  p2.min_out = &r.st->mu;
  p2.diag_out = &r.st->dmin;
  cudaError_t e = launch_pass<true, true>(p1, c->w1, c->fibers1, s);
  if (e == cudaSuccess) e = launch_pass<false, true>(p2, c->w2, c->fibers2, s);
  return e;
}

rd_status fail(cudaError_t e) {
  set_cuda_error(e);
  return RD_ERR_CUDA;
}

unsigned grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

}  // namespace
}  // namespace rd

using namespace rd;

extern "C" int rd_split_default_j(int m) {
  if (m < 2 || m > RD_MAX_M) return 0;
  const int j = m / 2;
  return (j <= kSplitMaxLen && m - j <= kSplitMaxLen) ? j : 0;
}

extern "C" rd_status rd_split_plan_bytes(int m, int j, size_t* bytes) {
  Layout L;
  if (!bytes || !make_layout(m, j, &L)) return RD_ERR_ARG;
  *bytes = L.bytes;
  return RD_OK;
}

extern "C" rd_status rd_split_plan(int m, int j, void* plan_dev, size_t plan_bytes, rd_split_info_t* info,
                                   cudaStream_t s) {
  Layout L;
  if (!info || !plan_dev || !make_layout(m, j, &L)) return RD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(plan_dev) & 255u) != 0) return RD_ERR_ARG;
  if (plan_bytes < L.bytes) return RD_ERR_NOMEM;
  if (L.N * 32 > 0x7FFFFFFFll) return RD_ERR_ARG;
  void* P = plan_dev;
  const int h = L.h;
  const int64_t n5j = ipow(kTauCount, j), n5h = ipow(kTauCount, h), n4j = ipow(4, j), n4h = ipow(4, h);
  cudaError_t e = cudaSuccess;
  rd_status rc = rd_enumerate_states(m, at<uint32_t>(P, L.codes), at<uint8_t>(P, L.wts), s);
  if (rc != RD_OK) return rc;
  e = cudaMemsetAsync(at<int32_t>(P, L.rankR), 0, (size_t)(n5j + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<int32_t>(P, L.rankS), 0, (size_t)(n5h + 1) * 4, s);
  if (e != cudaSuccess) return fail(e);
  split_mark_kernel<<<grid_for(L.N), 256, 0, s>>>(at<uint32_t>(P, L.codes), L.N, m, j, at<int32_t>(P, L.rankR),
                                                   at<int32_t>(P, L.rankS));
  correct_flag_kernel<<<grid_for(n4j), 256, 0, s>>>(at<int32_t>(P, L.rankPi), j, n4j);
  correct_flag_kernel<<<grid_for(n4h), 256, 0, s>>>(at<int32_t>(P, L.rankPhi), h, n4h);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankR), n5j);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankS), n5h);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankPi), n4j);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankPhi), n4h);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  int32_t cnt[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(&cnt[0], at<int32_t>(P, L.rankR) + n5j, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt[1], at<int32_t>(P, L.rankS) + n5h, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt[2], at<int32_t>(P, L.rankPi) + n4j, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt[3], at<int32_t>(P, L.rankPhi) + n4h, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  const int64_t n_rho = cnt[0], n_sigma = cnt[1];
  // the bounds are exact upper bounds and the prefix / suffix words are the correct words
  if (n_rho < 1 || n_rho > L.rhoB || n_sigma < 1 || n_sigma > L.sigB || cnt[2] != L.nPi || cnt[3] != L.nPhi ||
      n_rho > 0xFFFF || n_sigma > 0xFFFF)
    return RD_ERR_RANGE;
  const int w1 = choose_w((int)n_rho), w2 = choose_w((int)n_sigma);
  if (w1 == 0 || w2 == 0) return RD_ERR_ARG;  // a fiber does not fit in shared memory
  invert_kernel<<<grid_for(n5j), 256, 0, s>>>(at<int32_t>(P, L.rankR), n5j, at<int32_t>(P, L.rhoCode));
  invert_kernel<<<grid_for(n5h), 256, 0, s>>>(at<int32_t>(P, L.rankS), n5h, at<int32_t>(P, L.sigCode));
  invert_kernel<<<grid_for(n4j), 256, 0, s>>>(at<int32_t>(P, L.rankPi), n4j, at<int32_t>(P, L.piCode));
  invert_kernel<<<grid_for(n4h), 256, 0, s>>>(at<int32_t>(P, L.rankPhi), n4h, at<int32_t>(P, L.phiCode));
  list_count_kernel<<<grid_for(L.nPi), 256, 0, s>>>(at<int32_t>(P, L.piCode), L.nPi, at<int32_t>(P, L.rhoCode),
                                                    n_rho, j, at<int32_t>(P, L.c1s));
  list_count_kernel<<<grid_for(L.nPhi), 256, 0, s>>>(at<int32_t>(P, L.phiCode), L.nPhi, at<int32_t>(P, L.sigCode),
                                                     n_sigma, h, at<int32_t>(P, L.c2s));
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.c1s), L.nPi);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.c2s), L.nPhi);
  list_fill_kernel<<<grid_for(L.nPi), 256, 0, s>>>(at<int32_t>(P, L.piCode), L.nPi, at<int32_t>(P, L.rhoCode), n_rho,
                                                   j, at<int32_t>(P, L.c1s), at<uint16_t>(P, L.c1));
  list_fill_kernel<<<grid_for(L.nPhi), 256, 0, s>>>(at<int32_t>(P, L.phiCode), L.nPhi, at<int32_t>(P, L.sigCode),
                                                    n_sigma, h, at<int32_t>(P, L.c2s), at<uint16_t>(P, L.c2));
  e = cudaMemsetAsync(at<int32_t>(P, L.fiber), 0xFF, (size_t)n_sigma * (size_t)n_rho * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<int32_t>(P, L.outrow), 0xFF, (size_t)L.nPi * (size_t)L.nPhi * 4, s);
  if (e != cudaSuccess) return fail(e);
  split_index_kernel<<<grid_for(L.N), 256, 0, s>>>(at<uint32_t>(P, L.codes), L.N, m, j, at<int32_t>(P, L.rankR),
                                                   at<int32_t>(P, L.rankS), n_rho, at<int32_t>(P, L.rankPi),
                                                   at<int32_t>(P, L.rankPhi), L.nPhi, at<int32_t>(P, L.fiber),
                                                   at<int32_t>(P, L.outrow));
  e = cudaGetLastError();
  int32_t tot[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[0], at<int32_t>(P, L.c1s) + L.nPi, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[1], at<int32_t>(P, L.c2s) + L.nPhi, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  *info = rd_split_info_t{};
  info->m = m;
  info->j = j;
  info->N = L.N;
  info->n_rho = (int32_t)n_rho;
  info->n_sigma = (int32_t)n_sigma;
  info->n_pi = (int32_t)L.nPi;
  info->n_phi = (int32_t)L.nPhi;
  info->list1_entries = tot[0];
  info->list2_entries = tot[1];
  info->x_rows = L.nPi * n_sigma;
  info->plan_bytes = L.bytes;
  info->w1 = w1;
  info->w2 = w2;
  return RD_OK;
}

extern "C" rd_status rd_split_minplus(const rd_split_info_t* info, const void* plan_dev, const int16_t* B,
                                      int64_t ldb, int16_t* X_dev, int64_t ldx, int16_t* C, int64_t ldc,
                                      int32_t* min_out, cudaStream_t s) {
  if (!info_ok(info, plan_dev) || !B || !X_dev || !C) return RD_ERR_ARG;
  const int64_t N = info->N;
  if (ldb < N || ldb % 8 != 0 || ldx < N || ldx % 8 != 0 || ldc < N || ldc % 8 != 0) return RD_ERR_ARG;
  if (!aligned16(B) || !aligned16(X_dev) || !aligned16(C)) return RD_ERR_ARG;
  cudaError_t e = cudaSuccess;
  if (min_out) {
    e = launch_fill_i32(min_out, RD_INF, s);
    if (e != cudaSuccess) return fail(e);
  }
  SplitPass p1, p2;
  passes_of(*info, plan_dev, &p1, &p2);
  p1.in = B;
  p1.ldin = ldb;
  p1.out = X_dev;
  p1.ldout = ldx;
  p2.in = X_dev;
  p2.ldin = ldx;
  p2.out = C;
  p2.ldout = ldc;
  p2.min_out = min_out;
  e = launch_pass<true, false>(p1, info->w1, info->n_sigma, s);
  if (e == cudaSuccess) e = launch_pass<false, false>(p2, info->w2, info->n_pi, s);
  if (e != cudaSuccess) return fail(e);
  return RD_OK;
}

extern "C" rd_status rd_power_until_periodic_split(const int16_t* A_dev, int64_t lda, const rd_split_info_t* info,
                                                   const void* plan_dev, int16_t* X_dev, int64_t ldx, int kmax,
                                                   void* work_dev, size_t work_bytes, int64_t* gamma_host,
                                                   int32_t* k_out, int32_t* p_out, int64_t* q_out, cudaStream_t s) {
  if (!A_dev || !info_ok(info, plan_dev) || !X_dev || !work_dev || !gamma_host || !k_out || !p_out || !q_out)
    return RD_ERR_ARG;
  const int64_t N = info->N;
  if (lda < N || lda % 8 != 0 || ldx < N || ldx % 8 != 0 || kmax < 1 || kmax > (1 << 20)) return RD_ERR_ARG;
  if (!aligned16(A_dev) || !aligned16(X_dev) || (reinterpret_cast<uintptr_t>(work_dev) & 255u) != 0)
    return RD_ERR_ARG;
  SplitCtx c{};
  passes_of(*info, plan_dev, &c.p1, &c.p2);
  c.p1.out = X_dev;
  c.p1.ldout = ldx;
  c.p2.in = X_dev;
  c.p2.ldin = ldx;
  c.w1 = info->w1;
  c.w2 = info->w2;
  c.fibers1 = info->n_sigma;
  c.fibers2 = info->n_pi;
  return power_search(A_dev, N, lda, kmax, work_dev, work_bytes, split_power_product, &c, gamma_host, k_out, p_out,
                      q_out, s);
}
