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
// Only the pairs (pi, sigma) for which some word p = (rho, sigma) has rho admitted by pi give a
// finite row of X; X holds those rows only (about 1.28 N of them for j = m / 2).
//
// Kernels: a CTA owns one fiber and a slab of W columns.  A pass-1 fiber is one sigma, its slots the
// words p = (rho, sigma) (at most C_j of them); a pass-2 fiber is one pi, its slots the finite rows
// X[pi][sigma].  The CTA stages the slots' row segments in shared memory (slot 0 is an all-RD_INF
// dummy) and forms the outputs in groups of four that differ only in the letter of the boundary
// row (row j in pass 1, row j + 1 in pass 2).  A row type t of the boundary row feeds exactly the
// letters that admit it,
//     a -> {a, c, d}   b -> {c}   c+ -> {a, b, c}   c- -> {a}   d -> {b, c},
// less the letters for which the group's word, the fiber's boundary or the word itself is not
// correct (those outputs do not exist).  So each (fiber, group) lists its admitted slots in 7
// sub-lists keyed by that set of target letters (only 7 sets occur); a staged vector read once from shared memory
// updates every accumulator of its set, pairs of slots with one 3-input DPX minimum per 32-bit
// word.  Sub-lists are padded to pairs with the dummy; a thread owns 8 columns (one 16-byte vector).
// A fiber's lists, sub-list bounds and output rows are contiguous in the plan and a few KB in size
// for balanced splits: the CTA stages them in shared memory together with the rows, so the folding
// loop reads nothing but shared memory.  When they do not fit (very unbalanced splits), the kernel
// reads them from global memory instead.
#include <initializer_list>
#include <mutex>

#include "power_dev.cuh"
#include "rd_internal.cuh"

namespace rd {
namespace {

constexpr int kSplitThreads = 256;
constexpr int kSplitMaxLen = 8;  // rows per part (5^8 row-type codes, 4^8 letter codes)
constexpr int kTauA = 0, kTauB = 1, kTauCp = 2, kTauCm = 3, kTauD = 4;
constexpr int kTauCount = 5;
// The sets of target letters that occur (as 4-bit masks over a, b, c, d): the letters admitting a row
// type (acd, c, abc, a, bc) less those a neighbouring letter forbids (the correct continuations of
// a, b, c, d are ac, cd, abcd, bcd; in pass 2 two such restrictions meet) -- {a, c, ac, bc, abc, cd,
// acd}.  A group's record holds the starts of its 7 sub-lists and their end.
constexpr int kSets = 7;
constexpr int kRec = 8;
constexpr int kDefaultSlabsPerCta = 8;
__host__ __device__ constexpr int set_index(uint32_t mask) {
  return mask == 0x1 ? 0 : mask == 0x4 ? 1 : mask == 0x5 ? 2 : mask == 0x6 ? 3 : mask == 0x7 ? 4 : mask == 0xC ? 5
       : mask == 0xD ? 6 : -1;
}
// bit 4x + y set: the factor xy is excluded by Definition 4 (ad, da, ab, ba, bb)
constexpr uint32_t kForbiddenPairs = (1u << (0 * 4 + 3)) | (1u << (3 * 4 + 0)) | (1u << (0 * 4 + 1)) |
                                     (1u << (1 * 4 + 0)) | (1u << (1 * 4 + 1));

__host__ __device__ constexpr bool forbidden(int x, int y) { return (kForbiddenPairs >> (4 * x + y)) & 1u; }

// S(letter) as a bit set over row types, for the letters a, b, c, d (Sec. 4.A rules)
__host__ __device__ constexpr uint32_t admit_bits(int letter) {
  return letter == 0   ? (1u << kTauA) | (1u << kTauCp) | (1u << kTauCm)
         : letter == 1 ? (1u << kTauD) | (1u << kTauCp)
         : letter == 2 ? (1u << kTauA) | (1u << kTauB) | (1u << kTauD) | (1u << kTauCp)
                       : (1u << kTauA);
}
// the letters that admit row type t, as a bit set over a, b, c, d
__host__ __device__ constexpr uint32_t targets_of(int t) {
  uint32_t r = 0;
  for (int l = 0; l < 4; ++l)
    if ((admit_bits(l) >> t) & 1u) r |= 1u << l;
  return r;
}
static_assert(targets_of(kTauA) == 0xDu && targets_of(kTauB) == 0x4u && targets_of(kTauCp) == 0x7u &&
                  targets_of(kTauCm) == 0x1u && targets_of(kTauD) == 0x6u,
              "row type -> admitting letters");

// ---------------------------------------------------------------- codes

// letter of row i (1-based) of a code of `len` letters, row 1 most significant
__host__ __device__ inline int letter_at(uint32_t code, int len, int i) { return (int)((code >> (2 * (len - i))) & 3u); }

__host__ __device__ inline bool correct_code(uint32_t code, int len) {
  for (int i = 1; i < len; ++i)
    if (forbidden(letter_at(code, len, i), letter_at(code, len, i + 1))) return false;
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
    if (!((admit_bits(letter_at(w, len, i)) >> ty) & 1u)) return false;
  }
  return true;
}

__host__ __device__ inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// ---------------------------------------------------------------- plan layout

// Host-side bound on the distinct row-type strings of a part of `len` rows: each is a correct word
// of len letters with its c's marked + or -, and only a c in the boundary row (the last row of
// pass 1's part, the first of pass 2's) has a vertical neighbour outside the part; every other mark
// is fixed by the word.
int64_t type_bound(int len, bool boundary_last) {
  int64_t t = 0;
  for (uint32_t c = 0; c < (1u << (2 * len)); ++c) {
    if (!correct_code(c, len)) continue;
    t += letter_at(c, len, boundary_last ? len : 1) == 2 ? 2 : 1;
  }
  return t;
}

// Host-side bound on the list entries of one fiber over all groups of a part of len rows: a group
// word w of len - 1 letters admits at most prod_i |S(w_i)| strings of its rows (|S| = 3, 2, 4, 1 for
// a, b, c, d), each with one of 5 boundary types, and the fiber has at most `slots` slots; each of
// the 7 sub-lists adds at most one padding entry.
int64_t fiber_list_bound(int len, int64_t slots) {
  const int64_t admit_size[4] = {3, 2, 4, 1};
  int64_t t = 0;
  for (uint32_t c = 0; c < (1u << (2 * (len - 1))); ++c) {
    if (!correct_code(c, len - 1)) continue;
    int64_t v = kTauCount;
    for (int i = 1; i <= len - 1; ++i) v *= admit_size[letter_at(c, len - 1, i)];
    t += (v < slots ? v : slots) + kSets;
  }
  return t;
}

int64_t correct_count(int len) {
  if (len == 0) return 1;  // the empty word
  int64_t n = 0;
  return rd_state_count(len, &n) == RD_OK ? n : -1;
}

struct Layout {
  int m, j, h;
  int64_t N, nPi, nPhi, nG1, nG2, rhoB, sigB, l1B, l2B;
  size_t codes, wts, rankR, rankS, rankPi, rankPhi, rankG1, rankG2, rhoCode, sigCode, piCode, g1Code, g2Code, fiber,
      outrow, fstart1, fmem1, frho1, xrank, xsig, fstart2, gls1, l1, go1, ord1, gls2, l2, go2, ord2, counters,
      bytes;
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
  L->nG1 = correct_count(j - 1);
  L->nG2 = correct_count(h - 1);
  L->rhoB = type_bound(j, true);
  L->sigB = type_bound(h, false);
  // a pass-1 fiber has at most C_j slots (rho and sigma fix the letters), a pass-2 fiber at most n_sigma
  L->l1B = L->sigB * fiber_list_bound(j, L->nPi);
  L->l2B = L->nPi * fiber_list_bound(h, L->sigB);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = round_up(off + bytes, 256);
    return o;
  };
  const size_t xcap = (size_t)L->nPi * (size_t)L->sigB;
  L->codes = take((size_t)L->N * 4);
  L->wts = take((size_t)L->N);
  L->rankR = take((size_t)(ipow(kTauCount, j) + 1) * 4);
  L->rankS = take((size_t)(ipow(kTauCount, h) + 1) * 4);
  L->rankPi = take((size_t)(ipow(4, j) + 1) * 4);
  L->rankPhi = take((size_t)(ipow(4, h) + 1) * 4);
  L->rankG1 = take((size_t)(ipow(4, j - 1) + 1) * 4);
  L->rankG2 = take((size_t)(ipow(4, h - 1) + 1) * 4);
  L->rhoCode = take((size_t)L->rhoB * 4);
  L->sigCode = take((size_t)L->sigB * 4);
  L->piCode = take((size_t)L->nPi * 4);
  L->g1Code = take((size_t)L->nG1 * 4);
  L->g2Code = take((size_t)L->nG2 * 4);
  L->fiber = take((size_t)L->sigB * (size_t)L->rhoB * 4);
  L->outrow = take((size_t)L->nPi * (size_t)L->nPhi * 4);
  L->fstart1 = take((size_t)(L->sigB + 1) * 4);
  L->fmem1 = take((size_t)L->N * 4);
  L->frho1 = take((size_t)L->N * 4);
  L->xrank = take((xcap + 1) * 4);
  L->xsig = take(xcap * 4);
  L->fstart2 = take((size_t)(L->nPi + 1) * 4);
  L->gls1 = take(((size_t)L->sigB * (size_t)L->nG1 * kRec + 1) * 4);
  L->l1 = take((size_t)L->l1B * 2);
  L->go1 = take((size_t)L->sigB * (size_t)L->nG1 * 4 * 4);
  L->ord1 = take((size_t)L->sigB * (size_t)L->nG1 * 2);
  L->gls2 = take(((size_t)L->nPi * (size_t)L->nG2 * kRec + 1) * 4);
  L->l2 = take((size_t)L->l2B * 2);
  L->go2 = take((size_t)L->nPi * (size_t)L->nG2 * 4 * 4);
  L->ord2 = take((size_t)L->nPi * (size_t)L->nG2 * 2);
  L->counters = take(32 * 4);  // [0, 8): counters of the build; [16, 24): the readback stage
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

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- plan kernels

// Each correct word of length m marks the row-type codes of its first j rows and of the rest.
__global__ void split_mark_kernel(const uint32_t* codes, int64_t N, int m, int j, int32_t* flagR, int32_t* flagS) {
  GRID_STRIDE(p, N) {
    const uint32_t code = codes[p];
    uint32_t rc = 0, sc = 0;
    for (int i = 1; i <= j; ++i) rc = rc * kTauCount + row_type(code, m, i);
    for (int i = j + 1; i <= m; ++i) sc = sc * kTauCount + row_type(code, m, i);
    flagR[rc] = 1;
    flagS[sc] = 1;
  }
}

__global__ void correct_flag_kernel(int32_t* flags, int len, int64_t n) {
  GRID_STRIDE(c, n) flags[c] = correct_code((uint32_t)c, len) ? 1 : 0;
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
  GRID_STRIDE(c, n) {
    if (rank[c + 1] > rank[c]) inv[rank[c]] = (int32_t)c;
  }
}

// fiber[sigma rank][rho rank] = p * 32 + w(p);  outrow[pi rank][phi rank] = q.
__global__ void split_index_kernel(const uint32_t* codes, int64_t N, int m, int j, const int32_t* rankR,
                                   const int32_t* rankS, int64_t n_rho, const int32_t* rankPi,
                                   const int32_t* rankPhi, int64_t n_phi, int32_t* fiber, int32_t* outrow) {
  const int h = m - j;
  GRID_STRIDE(p, N) {
    const uint32_t code = codes[p];
    uint32_t rc = 0, sc = 0;
    for (int i = 1; i <= j; ++i) rc = rc * kTauCount + row_type(code, m, i);
    for (int i = j + 1; i <= m; ++i) sc = sc * kTauCount + row_type(code, m, i);
    fiber[(int64_t)rankS[sc] * n_rho + rankR[rc]] = (int32_t)(p * 32 + word_weight_of(code, m));
    const uint32_t pi = code >> (2 * h), phi = code & ((1u << (2 * h)) - 1u);
    outrow[(int64_t)rankPi[pi] * n_phi + rankPhi[phi]] = (int32_t)p;
  }
}

// Pass-1 fibers in compact form: the words of fiber sigma in increasing rho rank.
__global__ void fiber_count_kernel(const int32_t* fiber, int64_t n_sigma, int64_t n_rho, int32_t* cnt) {
  GRID_STRIDE(s, n_sigma) {
    int32_t c = 0;
    for (int64_t r = 0; r < n_rho; ++r) c += fiber[s * n_rho + r] >= 0 ? 1 : 0;
    cnt[s] = c;
  }
}

__global__ void fiber_fill_kernel(const int32_t* fiber, int64_t n_sigma, int64_t n_rho, const int32_t* start,
                                  int32_t* mem, int32_t* rho_of, int32_t* max_slots) {
  GRID_STRIDE(s, n_sigma) {
    int32_t e = start[s];
    for (int64_t r = 0; r < n_rho; ++r) {
      const int32_t v = fiber[s * n_rho + r];
      if (v < 0) continue;
      mem[e] = v;
      rho_of[e] = (int32_t)r;
      ++e;
    }
    atomicMax(max_slots, e - start[s]);
  }
}

// xflag[pi][sigma] = 1 when some word of fiber sigma has its rho admitted by pi (a finite row of X).
__global__ void xflag_kernel(const int32_t* piCode, int64_t n_pi, int64_t n_sigma, const int32_t* fstart1,
                             const int32_t* frho1, const int32_t* rhoCode, int j, int32_t* xflag) {
  GRID_STRIDE(i, n_pi * n_sigma) {
    const int64_t pi = i / n_sigma, s = i % n_sigma;
    int32_t fin = 0;
    for (int32_t e = fstart1[s]; e < fstart1[s + 1] && !fin; ++e)
      fin = admits((uint32_t)piCode[pi], (uint32_t)rhoCode[frho1[e]], j) ? 1 : 0;
    xflag[i] = fin;
  }
}

// The sigma of each finite row of X, and the pass-2 fiber starts (X rows of pi are contiguous).
__global__ void xsig_kernel(const int32_t* xrank, int64_t n_pi, int64_t n_sigma, int32_t* xsig, int32_t* fstart2,
                            int32_t* max_slots) {
  GRID_STRIDE(i, n_pi * n_sigma) {
    if (xrank[i + 1] > xrank[i]) xsig[xrank[i]] = (int32_t)(i % n_sigma);
    if (i % n_sigma == 0) {
      const int64_t pi = i / n_sigma;
      fstart2[pi] = xrank[i];
      atomicMax(max_slots, xrank[i + n_sigma] - xrank[i]);
      if (pi == n_pi - 1) fstart2[n_pi] = xrank[n_pi * n_sigma];
    }
  }
}

// One (fiber, group) of a pass: enumerate its slots, and for each slot admitted on the group's rows
// give the set of target letters (the letters admitting the boundary type that give an existing
// output).  FILL = false counts entries per set (each padded to even) into cnt[8 (f G + g) + set]
// (entry 7 stays 0, so after the scan it is the record's end) and raises *bad for a set outside the
// 7; FILL = true writes the 1-based slot numbers from start and pads with the dummy slot 0.
struct GroupArgs {
  int first;  // 1: pass 1 (boundary = last row of the part), 0: pass 2 (boundary = first row)
  int len;    // rows of the part (j resp. h)
  int64_t n_fibers, n_groups;
  const int32_t* gcode;    // group words (len - 1 letters)
  const int32_t* fstart;   // slot ranges of the fibers (pass 1: into frho; pass 2: X rows)
  const int32_t* slot_tc;  // pass 1: rho rank of each member; pass 2: sigma rank of each X row
  const int32_t* tcode;    // row-type code of a rho / sigma rank
  const int32_t* piCode;   // pass 2: the fiber's word pi (its last letter borders the part)
};

__device__ inline uint32_t allowed_letters(const GroupArgs& a, int64_t f, uint32_t gw) {
  const int glen = a.len - 1;
  uint32_t allow = 0;
  for (int l = 0; l < 4; ++l) {
    bool ok;
    if (a.first)
      ok = glen == 0 || !forbidden(letter_at(gw, glen, glen), l);
    else
      ok = (glen == 0 || !forbidden(l, letter_at(gw, glen, 1))) && !forbidden((int)(a.piCode[f] & 3), l);
    if (ok) allow |= 1u << l;
  }
  return allow;
}

template <bool FILL>
__global__ void group_lists_kernel(GroupArgs a, int32_t* cnt_or_start, uint16_t* lst, int32_t* bad) {
  GRID_STRIDE(i, a.n_fibers * a.n_groups) {
    const int64_t f = i / a.n_groups, g = i % a.n_groups;
    const uint32_t gw = (uint32_t)a.gcode[g];
    const int glen = a.len - 1;
    const uint32_t allow = allowed_letters(a, f, gw);
    int32_t pos[kRec];
    for (int s = 0; s < kRec; ++s) pos[s] = FILL ? cnt_or_start[i * kRec + s] : 0;
    const uint32_t p = (uint32_t)ipow(kTauCount, glen);
    for (int32_t e = a.fstart[f]; e < a.fstart[f + 1]; ++e) {
      const uint32_t tc = (uint32_t)a.tcode[a.slot_tc[e]];
      const int t = a.first ? (int)(tc % kTauCount) : (int)(tc / p);
      const uint32_t rest = a.first ? tc / kTauCount : tc % p;
      if (!admits(gw, rest, glen)) continue;
      const uint32_t set = targets_of(t) & allow;
      if (set == 0) continue;
      const int si = set_index(set);
      if (si < 0) {
        if (!FILL) atomicExch(bad, 1);
        continue;
      }
      if (FILL)
        lst[pos[si]++] = (uint16_t)(e - a.fstart[f] + 1);
      else
        ++pos[si];
    }
    if (FILL) {
      for (int s = 0; s < kSets; ++s)
        if (pos[s] & 1) lst[pos[s]] = 0;
    } else {
      for (int s = 0; s < kSets; ++s) cnt_or_start[i * kRec + s] = (pos[s] + 1) & ~1;
      cnt_or_start[i * kRec + kSets] = 0;
    }
  }
}

// Each fiber's groups in the order the kernel deals them to its lane sets (back and forth): by their
// sub-list lengths compared lexicographically, the target sets taken in the order abc, acd, ac, a, c, bc,
// cd, longer first (ties by index).  A warp runs each sub-list loop for as long as the longest of its
// groups' sub-lists, so groups that share a warp should have similar sub-lists; groups of similar size
// stay together too, so the back-and-forth dealing still balances the lane sets.  A model of the plans
// (warp work over the groups' mean): m = 8 pass 2 1.39, m = 9 pass 2 1.20, against 1.76 and 1.70 for the
// order by total length alone.
//
// The order as one 64-bit key per group, smaller first: the seven sub-list lengths in the set order above,
// each as 511 minus the length capped at 511 (9 bits), the first set in the top bits.  Lengths above 511
// (only very unbalanced splits have such groups) tie, which only changes the order among them.
__device__ inline uint64_t group_key(const int32_t* r) {
  const int order[kSets] = {4, 6, 2, 0, 1, 3, 5};  // set indexes of abc, acd, ac, a, c, bc, cd
  uint64_t key = 0;
  for (int k = 0; k < kSets; ++k) {
    const int sidx = order[k];
    const int32_t len = r[sidx + 1] - r[sidx];
    key = (key << 9) | (uint64_t)(511 - (len < 511 ? len : 511));
  }
  return key;
}

// Correct words of length len at compile time, by their last letter: a may follow a or c, b may follow c
// or d, c anything, d anything but a (Definition 4 forbids ad, da, ab, ba, bb).
constexpr int64_t correct_count_ce(int len) {
  int64_t a = 1, b = 1, c = 1, d = 1;
  for (int i = 1; i < len; ++i) {
    const int64_t a2 = a + c, b2 = c + d, c2 = a + b + c + d, d2 = b + c + d;
    a = a2; b = b2; c = c2; d = d2;
  }
  return len == 0 ? 1 : a + b + c + d;
}
static_assert(correct_count_ce(3) == 33 && correct_count_ce(9) == 21909, "word count recurrence");
// group_order_kernel keeps one 8-byte key per group of a fiber (at most C_(kSplitMaxLen - 1) groups) in
// dynamic shared memory without raising the 48 KB default limit.
static_assert(8 * correct_count_ce(kSplitMaxLen - 1) <= 48 * 1024, "group keys exceed 48 KB of shared memory");

// One CTA per fiber: the groups' keys in shared memory, then each group's rank (the groups with a smaller
// key, or an equal key and a smaller index) is its place in the order.
__global__ void group_order_kernel(const int32_t* gls, int64_t n_groups, uint16_t* ord) {
  extern __shared__ uint64_t keys[];
  const int64_t f = blockIdx.x;
  const int32_t* r = gls + f * n_groups * kRec;
  for (int64_t g = threadIdx.x; g < n_groups; g += blockDim.x) keys[g] = group_key(r + g * kRec);
  __syncthreads();
  uint16_t* o = ord + f * n_groups;
  for (int64_t g = threadIdx.x; g < n_groups; g += blockDim.x) {
    const uint64_t kg = keys[g];
    int64_t rank = 0;
    for (int64_t h = 0; h < n_groups; ++h) rank += (keys[h] < kg || (keys[h] == kg && h < g)) ? 1 : 0;
    o[rank] = (uint16_t)g;
  }
}

// The list entries of each fiber (its records are contiguous), maximum into *out.
__global__ void fiber_list_max_kernel(const int32_t* gls, int64_t n_fibers, int64_t n_groups, int32_t* out) {
  GRID_STRIDE(f, n_fibers) {
    atomicMax(out, gls[(f + 1) * n_groups * kRec] - gls[f * n_groups * kRec]);
  }
}

// Output rows of the groups: go[4 (f G + g) + l] = the row written for letter l at the boundary,
// or -1.  Pass 1: the X row of (pi = group + l, sigma = f) when it is finite (a step of xrank).
// Pass 2: the row q of R of the word pi_f + (l + group) when that word is correct.
__global__ void group_out_kernel(GroupArgs a, const int32_t* rank_w, const int32_t* xrank, int64_t n_sigma,
                                 const int32_t* outrow, int64_t n_phi, int32_t* go) {
  GRID_STRIDE(i, a.n_fibers * a.n_groups) {
    const int64_t f = i / a.n_groups, g = i % a.n_groups;
    const uint32_t gw = (uint32_t)a.gcode[g];
    const int glen = a.len - 1;
    const uint32_t allow = allowed_letters(a, f, gw);
    for (int l = 0; l < 4; ++l) {
      int32_t row = -1;
      if ((allow >> l) & 1u) {
        if (a.first) {
          const int64_t x = (int64_t)rank_w[(gw << 2) | (uint32_t)l] * n_sigma + f;
          if (xrank[x + 1] > xrank[x]) row = xrank[x];
        } else {
          row = outrow[f * n_phi + rank_w[((uint32_t)l << (2 * glen)) | gw]];
        }
      }
      go[i * 4 + l] = row;
    }
  }
}

// ---------------------------------------------------------------- the two passes

struct SplitPass {
  const int16_t* in;  // pass 1: B (rows p);  pass 2: X
  int64_t ldin;
  int16_t* out;  // pass 1: X;  pass 2: R
  int64_t ldout;
  int64_t ncols;           // columns of this launch (a chunk of the N columns)
  int64_t in_rows, out_rows;  // rows of `in` and `out` (pass 1: N and X rows; pass 2: X rows and N)
  int64_t in_col0, out_col0;  // first column of the chunk in `in` resp. `out` (X holds one chunk at column 0)
  int32_t n_groups;
  int32_t norm;           // ring mode: pass 1 reduces the next offset step mu into st->mu, pass 2 writes
                          // the power normalised by it, with its hash and range flag (no normaliser pass)
  int32_t max_slots;      // shared-memory rows = max_slots + 1 (row 0 is the dummy)
  int32_t max_list;       // list entries of one fiber at most
  int32_t slabs_per_cta;  // column slabs one CTA sweeps with its fiber staged once
  int32_t fiber_x;        // 1: blockIdx.x is the fiber and blockIdx.y the slab group (the launch's choice)
  const int32_t* fstart;  // [fibers + 1] slot ranges: pass 1 into fmem, pass 2 X rows
  const int32_t* fmem;    // pass 1: p * 32 + w(p) per slot
  const int32_t* gls;     // [8 (fibers G) + 1] per (fiber, group): the 7 sub-list starts (even), then the end
  const uint16_t* lst;    // 1-based slot numbers, 0 = dummy
  const int32_t* go;      // [(fibers G) * 4] output rows per boundary letter, or -1
  const uint16_t* ord;    // [fibers G] each fiber's groups in dealing order (group_order_kernel)
  int32_t* min_out;
  int32_t* diag_out;
  PowerState* st;  // ring mode: B = power slot k (pass 1), R = slot k + 1 (pass 2)
  int16_t* ring;
  int64_t slot_elems;
  int slots;
};

__device__ __forceinline__ uint32_t min3(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_s16x2(a, b, c); }

// Checked builds (-DRD_CHECKED, rd_split_check_flags): every index the passes take from plan data -- input
// rows, staged-row numbers in the lists, group numbers and sub-list bounds, output rows -- is tested against
// its buffer; a failed test ORs its bit into g_split_check and the access is skipped (an RD_INF row read
// instead, no write).  In other builds split_ok is constant true and the tests compile away.
constexpr unsigned kChkInRow = 1, kChkSlot = 2, kChkGroup = 4, kChkOutRow = 8;
#ifdef RD_CHECKED
__device__ unsigned int g_split_check = 0;
__device__ __forceinline__ bool split_ok(bool c, unsigned bit) {
  if (!c) atomicOr(&g_split_check, bit);
  return c;
}
#else
__device__ __forceinline__ bool split_ok(bool, unsigned) { return true; }
#endif

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int SET>
__device__ __forceinline__ void fold_pair(uint4 (&acc)[4], const uint4& v0, const uint4& v1) {
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    if ((SET >> l) & 1) {
      acc[l].x = min3(acc[l].x, v0.x, v1.x);
      acc[l].y = min3(acc[l].y, v0.y, v1.y);
      acc[l].z = min3(acc[l].z, v0.z, v1.z);
      acc[l].w = min3(acc[l].w, v0.w, v1.w);
    }
  }
}

// Four rows into the accumulators of SET: the minimum of three rows once, then one 3-input minimum per
// accumulator word (1 + |SET| instructions per word instead of 2 |SET|, one dependent step per word).
template <int SET>
__device__ __forceinline__ void fold_quad(uint4 (&acc)[4], const uint4& v0, const uint4& v1, const uint4& v2,
                                          const uint4& v3) {
  const uint4 t = make_uint4(min3(v0.x, v1.x, v2.x), min3(v0.y, v1.y, v2.y), min3(v0.z, v1.z, v2.z),
                             min3(v0.w, v1.w, v2.w));
  fold_pair<SET>(acc, t, v3);
}

// Folds the sub-list [e0, e1) (even bounds) of target set SET into the group's accumulators.  SCALED:
// the list entries are byte offsets of the staged rows (slot x 16 LR, the list as staged in shared
// memory), so a row's address is one add and one mask or shift away.
template <int SET, int LR, bool SCALED>
__device__ __forceinline__ void fold_sublist(uint4 (&acc)[4], const uint4* sm, const uint32_t* pairs, int e0, int e1,
                                             int lane, uint32_t nst) {
  int p = e0 >> 1;
  const int pe = e1 >> 1;
  if constexpr (SCALED) {
    const char* base = reinterpret_cast<const char*>(sm);
    const uint32_t lane2 = (uint32_t)lane * 16u * 0x00010001u;  // the lane's offset, in both halves
    for (; p + 2 <= pe; p += 2) {
      const uint32_t i0 = pairs[p] + lane2, i1 = pairs[p + 1] + lane2;
      const uint4 v0 = *reinterpret_cast<const uint4*>(base + (i0 & 0xFFFFu));
      const uint4 v1 = *reinterpret_cast<const uint4*>(base + (i0 >> 16));
      const uint4 v2 = *reinterpret_cast<const uint4*>(base + (i1 & 0xFFFFu));
      const uint4 v3 = *reinterpret_cast<const uint4*>(base + (i1 >> 16));
      fold_quad<SET>(acc, v0, v1, v2, v3);
    }
    if (p < pe) {
      const uint32_t i0 = pairs[p] + lane2;
      fold_pair<SET>(acc, *reinterpret_cast<const uint4*>(base + (i0 & 0xFFFFu)),
                     *reinterpret_cast<const uint4*>(base + (i0 >> 16)));
    }
  } else {
  for (; p + 2 <= pe; p += 2) {
    uint32_t i0 = pairs[p], i1 = pairs[p + 1];
    if (!split_ok((i0 & 0xFFFFu) < nst && (i0 >> 16) < nst && (i1 & 0xFFFFu) < nst && (i1 >> 16) < nst, kChkSlot))
      i0 = i1 = 0;  // the RD_INF dummy row
    const uint4 v0 = sm[(int)(i0 & 0xFFFFu) * LR + lane];
    const uint4 v1 = sm[(int)(i0 >> 16) * LR + lane];
    const uint4 v2 = sm[(int)(i1 & 0xFFFFu) * LR + lane];
    const uint4 v3 = sm[(int)(i1 >> 16) * LR + lane];
    fold_pair<SET>(acc, v0, v1);
    fold_pair<SET>(acc, v2, v3);
  }
  if (p < pe) {
    uint32_t i0 = pairs[p];
    if (!split_ok((i0 & 0xFFFFu) < nst && (i0 >> 16) < nst, kChkSlot)) i0 = 0;
    fold_pair<SET>(acc, sm[(int)(i0 & 0xFFFFu) * LR + lane], sm[(int)(i0 >> 16) * LR + lane]);
  }
  }
}

// Shared memory of one CTA: the staged rows, then the fiber's sub-list bounds (uint16, local to the
// fiber's list), its output rows (int32), its list (uint16), its words (pass 1, int32) and its group
// order (uint16), each part 16-byte aligned.
struct PassSmem {
  size_t gls, go, lst, mem, ord, bytes;
};
__host__ __device__ inline PassSmem pass_smem_layout(int max_slots, int n_groups, int max_list, int W, bool words) {
  PassSmem p;
  const size_t data = (size_t)(max_slots + 1) * (size_t)W * 2;
  p.gls = data;
  p.go = p.gls + (size_t)n_groups * kRec * 2;
  p.lst = p.go + (size_t)n_groups * 4 * 4;
  p.mem = p.lst + ((size_t)max_list * 2 + 15) / 16 * 16;
  p.ord = p.mem + (words ? ((size_t)max_slots * 4 + 15) / 16 * 16 : 0);  // words: pass 1 only
  p.bytes = p.ord + ((size_t)n_groups * 2 + 15) / 16 * 16;
  return p;
}

// One (fiber f, slab group) of a pass: the body of split_pass_kernel.  sm: the dynamic shared memory
// (pass_smem bytes).
template <int W, bool FIRST, bool RING, bool STAGED>
__device__ __forceinline__ void split_pass_body(const SplitPass& a, const int64_t f, const int64_t slab_group,
                                                uint4* sm) {
  constexpr int LR = W / 8;              // threads per row of the slab
  constexpr int G = kSplitThreads / LR;  // groups (resp. staged rows) handled side by side
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
  in += a.in_col0;
  out += a.out_col0;
  const int lane = threadIdx.x % LR, gi = threadIdx.x / LR;
  const uint4 inf4 = make_uint4(kInf2, kInf2, kInf2, kInf2);

  // stage the fiber's metadata once: sub-list bounds relative to the fiber's first list entry,
  // output rows, the list itself (its bounds are even, so it moves as 32-bit pairs) and, in pass 1,
  // the words of the fiber
  const PassSmem lay = pass_smem_layout(a.max_slots, a.n_groups, a.max_list, W, FIRST);
  char* smb = reinterpret_cast<char*>(sm);
  uint16_t* sgls = reinterpret_cast<uint16_t*>(smb + lay.gls);
  int4* sgo = reinterpret_cast<int4*>(smb + lay.go);
  uint32_t* slst = reinterpret_cast<uint32_t*>(smb + lay.lst);
  int32_t* smem_words = reinterpret_cast<int32_t*>(smb + lay.mem);
  uint16_t* sord = reinterpret_cast<uint16_t*>(smb + lay.ord);
  const uint16_t* gord = a.ord + f * a.n_groups;
  const int64_t r0 = f * a.n_groups * kRec;
  const int32_t base = __ldg(a.gls + r0);
  const int4* go4 = reinterpret_cast<const int4*>(a.go) + f * a.n_groups;
  const uint32_t* glst = reinterpret_cast<const uint32_t*>(a.lst) + (base >> 1);
  const int32_t f0 = __ldg(a.fstart + f);
  const int nst = __ldg(a.fstart + f + 1) - f0 + 1;  // row 0 is the dummy, rows 1..n the slots
#ifdef RD_CHECKED
  const int list_pairs = (__ldg(a.gls + r0 + (int64_t)a.n_groups * kRec) - base) >> 1;
#else
  constexpr int list_pairs = 0;  // used by the checks only
#endif
  if (STAGED) {
    const int nb = a.n_groups * kRec;
    for (int i = threadIdx.x; i < nb; i += kSplitThreads) sgls[i] = (uint16_t)(__ldg(a.gls + r0 + i) - base);
    for (int i = threadIdx.x; i < a.n_groups; i += kSplitThreads) sgo[i] = __ldg(go4 + i);
    const int npairs = (__ldg(a.gls + r0 + nb) - base) >> 1;
    constexpr uint32_t kRowBytes = (uint32_t)W * 2;  // staged rows fit in 64 KB (stageable), so offsets fit 16 bits
    for (int i = threadIdx.x; i < npairs; i += kSplitThreads) {
      uint32_t q = __ldg(glst + i);
      if (!split_ok((q & 0xFFFFu) < (uint32_t)nst && (q >> 16) < (uint32_t)nst, kChkSlot)) q = 0;
      slst[i] = (q & 0xFFFFu) * kRowBytes | ((q >> 16) * kRowBytes) << 16;
    }
    if (FIRST)
      for (int i = threadIdx.x; i < nst - 1; i += kSplitThreads) smem_words[i] = __ldg(a.fmem + f0 + i);
    for (int i = threadIdx.x; i < a.n_groups; i += kSplitThreads) sord[i] = gord[i];
  }
  const uint32_t* pairs = STAGED ? slst : glst;
  int32_t lmin = kInf, ldiag = kInf;
  uint32_t m2 = kInf2;  // halfword minima of the full vectors written (pass 2)
  uint32_t mv = kInf2;  // pass 1 with norm: halfword minima of the staged values
  unsigned long long hsum = 0;  // pass 2 with norm: hash of the normalised power (as the normaliser's)
  uint32_t nbad = 0;            // pass 2 with norm: a normalised entry left [0, RD_MAX_FINITE]
  uint32_t fmax = 0;            // pass 2 with norm: halfword maxima of the finite normalised entries
  int32_t mu = 0;
  if (RING && !FIRST && a.norm) {
    const int32_t mr = *(volatile const int32_t*)&a.st->mu;  // complete: pass 1 has finished
    mu = (mr >= kInf) ? 0 : mr;
  }
  const uint32_t mu2 = (uint32_t)mu * 0x00010001u;

  const int64_t slabs = (a.ncols + W - 1) / W;
  const int64_t sb_end = min(slabs, (slab_group + 1) * a.slabs_per_cta);
  for (int64_t sb = slab_group * a.slabs_per_cta; sb < sb_end; ++sb) {
    const int64_t c = sb * W + lane * 8;
    const bool ok = c < a.ncols;
    __syncthreads();  // the metadata is staged / the previous slab has been consumed
    // every row segment of the slab goes in flight at once (asynchronous 16-byte copies, no registers)
#pragma unroll 1
    for (int s = gi; s < nst; s += G) {
      const int32_t e = (s < 1) ? -1 : FIRST ? (STAGED ? smem_words[s - 1] : __ldg(a.fmem + f0 + s - 1)) : f0 + s - 1;
      if (ok && e >= 0 && split_ok((int64_t)(FIRST ? (e >> 5) : e) < a.in_rows, kChkInRow))
        cp_async16(&sm[s * LR + lane], in + (int64_t)(FIRST ? (e >> 5) : e) * a.ldin + c);
      else
        sm[s * LR + lane] = inf4;
    }
    cp_async_wait_all();
    if (FIRST && ok) {
      // pass 1 stages w(p) + B[p]: each thread adds the weights to the vectors it copied itself
#pragma unroll 1
      for (int s = gi + (gi < 1 ? G : 0); s < nst; s += G) {
        const int32_t e = STAGED ? smem_words[s - 1] : __ldg(a.fmem + f0 + s - 1);
        const uint4 x = sm[s * LR + lane];
        const uint32_t w2 = (uint32_t)(e & 31) * 0x00010001u;
        const uint4 v = make_uint4(__viaddmin_s16x2(x.x, w2, kInf2), __viaddmin_s16x2(x.y, w2, kInf2),
                                   __viaddmin_s16x2(x.z, w2, kInf2), __viaddmin_s16x2(x.w, w2, kInf2));
        sm[s * LR + lane] = v;
        if (RING && a.norm) {
          // min of A(G) (x) P = min over p, x of w(p) + P[p][x] (every word has a predecessor)
          uint32_t t[4] = {v.x, v.y, v.z, v.w};
          if (c + 8 > a.ncols) mask_tail(t, (int)(a.ncols - c));  // lanes past the chunk / N
          mv = min3(min3(mv, t[0], t[1]), min3(t[2], t[3], kInf2), kInf2);
        }
      }
    }
    __syncthreads();

    // groups in the plan's order, dealt to the lane sets back and forth (0..G-1, G-1..0, ...)
    for (int round0 = 0; round0 < a.n_groups; round0 += G) {
      const int idx = round0 + (((round0 / G) & 1) ? (G - 1 - gi) : gi);
      if (idx >= a.n_groups) continue;
      int g = STAGED ? sord[idx] : __ldg(gord + idx);
      if (!split_ok(g < a.n_groups, kChkGroup)) continue;
      uint4 acc[4] = {inf4, inf4, inf4, inf4};
      // the group's record: the starts of its 7 sub-lists and their end
      int b[kRec];
      if (STAGED) {
        const uint4 q = reinterpret_cast<const uint4*>(sgls)[g];
        b[0] = q.x & 0xFFFF; b[1] = q.x >> 16; b[2] = q.y & 0xFFFF; b[3] = q.y >> 16;
        b[4] = q.z & 0xFFFF; b[5] = q.z >> 16; b[6] = q.w & 0xFFFF; b[7] = q.w >> 16;
      } else {
        const int4* r4 = reinterpret_cast<const int4*>(a.gls + r0) + 2 * g;
        const int4 q0 = __ldg(r4), q1 = __ldg(r4 + 1);
        b[0] = q0.x - base; b[1] = q0.y - base; b[2] = q0.z - base; b[3] = q0.w - base;
        b[4] = q1.x - base; b[5] = q1.y - base; b[6] = q1.z - base; b[7] = q1.w - base;
      }
      {
        bool rec_ok = b[0] >= 0 && b[7] <= 2 * list_pairs;
#pragma unroll
        for (int q = 0; q < kRec - 1; ++q) rec_ok = rec_ok && b[q] <= b[q + 1];
        if (!split_ok(rec_ok, kChkGroup)) continue;
      }
      // most sub-lists are empty (about 2 of the 7 hold entries at m = 9), and the plan's group order gives a
      // warp's lane sets the same pattern, so in pass 2 an empty one is skipped by one test instead of a loop
      // header (m = 10: 10.39 -> 10.30 ms per product).  Pass 1 keeps the plain loops: at its 48-register
      // bound the tests cost it spills (m = 10 product 10.70 ms with them in both passes).
      if (FIRST || b[0] != b[1]) fold_sublist<0x1, LR, STAGED>(acc, sm, pairs, b[0], b[1], lane, (uint32_t)nst);
      if (FIRST || b[1] != b[2]) fold_sublist<0x4, LR, STAGED>(acc, sm, pairs, b[1], b[2], lane, (uint32_t)nst);
      if (FIRST || b[2] != b[3]) fold_sublist<0x5, LR, STAGED>(acc, sm, pairs, b[2], b[3], lane, (uint32_t)nst);
      if (FIRST || b[3] != b[4]) fold_sublist<0x6, LR, STAGED>(acc, sm, pairs, b[3], b[4], lane, (uint32_t)nst);
      if (FIRST || b[4] != b[5]) fold_sublist<0x7, LR, STAGED>(acc, sm, pairs, b[4], b[5], lane, (uint32_t)nst);
      if (FIRST || b[5] != b[6]) fold_sublist<0xC, LR, STAGED>(acc, sm, pairs, b[5], b[6], lane, (uint32_t)nst);
      if (FIRST || b[6] != b[7]) fold_sublist<0xD, LR, STAGED>(acc, sm, pairs, b[6], b[7], lane, (uint32_t)nst);
      if (!ok) continue;
      const int4 rows = STAGED ? sgo[g] : __ldg(go4 + g);
      const int32_t row4[4] = {rows.x, rows.y, rows.z, rows.w};
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int64_t row = row4[l];
        if (row < 0 || !split_ok(row < a.out_rows, kChkOutRow)) continue;
        if (FIRST) {
          *reinterpret_cast<uint4*>(out + row * a.ldout + c) = acc[l];
        } else {
          uint32_t w4[4] = {acc[l].x, acc[l].y, acc[l].z, acc[l].w};
          if ((uint64_t)(row - a.out_col0 - c) < 8) {  // diagonal minimum of the raw product
            const int e = (int)(row - a.out_col0 - c);
            ldiag = min(ldiag, (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFFu));
          }
          if (RING && a.norm) {
            // P = R - mu on finite entries, range-checked, hashed per 16-byte chunk as the normaliser does
            uint32_t hw[4], sub[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t isinf = __vcmpeq2(w4[q], kInf2);
              sub[q] = __vsub2(w4[q], mu2) & ~isinf;  // 0 in the RD_INF lanes
              hw[q] = sub[q] | (kInf2 & isinf);
            }
            const int valid = (c + 8 <= a.ncols) ? 8 : (int)(a.ncols - c);
            uint32_t chk[4] = {hw[0], hw[1], hw[2], hw[3]};
            if (valid < 8) {
              mask_tail(chk, valid);
#pragma unroll
              for (int q = 0; q < 4; ++q) nbad |= __vcmpgtu2(chk[q], 0x1FFF1FFFu) & ~__vcmpeq2(chk[q], kInf2);
            } else {
              // the range check as a running maximum of the finite entries, tested once at the end
#pragma unroll
              for (int q = 0; q < 4; ++q) fmax = __vmaxu2(fmax, sub[q]);
            }
            hsum += chunk_hash(row, a.out_col0 + c, chk);
#pragma unroll
            for (int q = 0; q < 4; ++q) w4[q] = hw[q];
            acc[l] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          }
          if (c + 8 <= a.ncols) {
            *reinterpret_cast<uint4*>(out + row * a.ldout + c) = acc[l];
            if (!(RING && a.norm)) m2 = min3(min3(m2, acc[l].x, acc[l].y), acc[l].z, acc[l].w);  // min_out
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              if (c + e < a.ncols) {
                const int32_t v = (int32_t)((w4[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
                out[row * a.ldout + c + e] = (int16_t)v;
                lmin = min(lmin, v);
              }
            }
          }
        }
      }
    }
  }

  // the block reductions below use the start of the staged-row buffer, dead once every warp has folded the
  // last slab
  __syncthreads();
  unsigned long long* red_h = reinterpret_cast<unsigned long long*>(sm);
  int32_t* red_v = reinterpret_cast<int32_t*>(red_h + kSplitThreads / 32);
  int32_t* red_m = red_v + kSplitThreads / 32;
  int32_t* red_d = red_m + kSplitThreads / 32;
  if (RING && a.norm) {
    if (FIRST) {
      int32_t v = (int32_t)min(mv & 0xFFFFu, mv >> 16);
      for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
      if ((threadIdx.x & 31) == 0) red_v[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        int32_t bm = kInf;
        for (int w = 0; w < kSplitThreads / 32; ++w) bm = min(bm, red_v[w]);
        if (bm < kInf && bm < *(volatile const int32_t*)&a.st->mu) atomicMin(&a.st->mu, bm);
      }
    } else {
      nbad |= __vcmpgtu2(fmax, 0x1FFF1FFFu);
      for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xFFFFFFFFu, hsum, o);
      if ((threadIdx.x & 31) == 0) red_h[threadIdx.x >> 5] = hsum;
      const int any_bad = __syncthreads_or(nbad != 0);
      if (threadIdx.x == 0) {
        unsigned long long h = 0;
        for (int w = 0; w < kSplitThreads / 32; ++w) h += red_h[w];
        atomicAdd(&a.st->hacc, h);
        if (any_bad) atomicOr(&a.st->range_bad, 1);
      }
    }
  }

  if (!FIRST && (a.min_out != nullptr || a.diag_out != nullptr)) {
    lmin = min(lmin, (int32_t)min(m2 & 0xFFFFu, m2 >> 16));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xFFFFFFFFu, lmin, o));
      ldiag = min(ldiag, __shfl_xor_sync(0xFFFFFFFFu, ldiag, o));
    }
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

template <int W, bool FIRST, bool RING, bool STAGED>
__global__ void __launch_bounds__(kSplitThreads, FIRST ? 5 : 4) split_pass_kernel(SplitPass a) {
  extern __shared__ uint4 sm[];
  const int64_t f = a.fiber_x ? blockIdx.x : blockIdx.y;
  const int64_t slab_group = a.fiber_x ? blockIdx.y : blockIdx.x;
  split_pass_body<W, FIRST, RING, STAGED>(a, f, slab_group, sm);
}

constexpr size_t kSmemLimit = 220 * 1024;

// Shared memory of a launch: rows and metadata when they fit (staged), else the rows alone.
// Staging needs the fiber's list positions to fit the uint16 offsets, and the staged rows to fit 64 KB
// (the staged list holds their byte offsets in 16 bits).
bool stageable(int max_list, int max_slots, int W, size_t bytes, size_t limit) {
  return max_list <= 0xFFFF && (size_t)(max_slots + 1) * (size_t)W * 2 <= 65536 && bytes <= limit;
}

size_t pass_smem(int max_slots, int n_groups, int max_list, int W, bool words, bool* staged) {
  const size_t full = pass_smem_layout(max_slots, n_groups, max_list, W, words).bytes;
  *staged = stageable(max_list, max_slots, W, full, kSmemLimit);
  return *staged ? full : (size_t)(max_slots + 1) * (size_t)W * 2;
}

// Slab width: the widest of 256, 128, 64 columns whose staged fiber leaves room for 3 CTAs per SM (narrower
// slabs put more groups in a warp and cost shared-memory bank conflicts; at 256 a warp folds one group at a
// time, so its lanes never diverge: m = 8 0.186 -> 0.144 ms and m = 9 1.147 -> 1.109 ms tuned), else the
// widest that fits 2 or 1; then the same for the rows alone.
int choose_w(int max_slots, int n_groups, int max_list, bool words) {
  const int ws[4] = {256, 128, 64, 32};
  const size_t limits[3] = {72 * 1024, 112 * 1024, kSmemLimit};
  for (size_t lim : limits)
    for (int w : ws)
      if (stageable(max_list, max_slots, w, pass_smem_layout(max_slots, n_groups, max_list, w, words).bytes, lim))
        return w;
  for (size_t lim : limits)
    for (int w : ws)
      if ((size_t)(max_slots + 1) * (size_t)w * 2 <= lim) return w;
  return 0;
}

bool valid_w(int W, int max_slots) {
  return (W == 32 || W == 64 || W == 128 || W == 256) && (size_t)(max_slots + 1) * (size_t)W * 2 <= kSmemLimit;
}

// The pass kernels' dynamic shared-memory limit, raised once per device to kSmemLimit (the limit is
// a ceiling: occupancy follows each launch's own request).  rd_split_plan does it, so that no
// attribute call falls inside a stream capture of the steps.
template <bool FIRST, bool RING>
cudaError_t raise_limits() {
  void (*ks[8])(SplitPass) = {split_pass_kernel<256, FIRST, RING, true>,  split_pass_kernel<128, FIRST, RING, true>,
                              split_pass_kernel<64, FIRST, RING, true>,   split_pass_kernel<32, FIRST, RING, true>,
                              split_pass_kernel<256, FIRST, RING, false>, split_pass_kernel<128, FIRST, RING, false>,
                              split_pass_kernel<64, FIRST, RING, false>,  split_pass_kernel<32, FIRST, RING, false>};
  for (auto k : ks) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

std::mutex g_limits_mu;
uint64_t g_limits_done = 0;  // one bit per device

cudaError_t ensure_limits() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_limits_mu);
  if (dev < 64 && ((g_limits_done >> dev) & 1u)) return cudaSuccess;
  e = raise_limits<true, false>();
  if (e == cudaSuccess) e = raise_limits<false, false>();
  if (e == cudaSuccess) e = raise_limits<true, true>();
  if (e == cudaSuccess) e = raise_limits<false, true>();
  if (e == cudaSuccess && dev < 64) g_limits_done |= 1ull << dev;
  return e;
}

template <bool FIRST, bool RING>
cudaError_t launch_pass(const SplitPass& a, int W, int64_t fibers, cudaStream_t s) {
  bool staged = false;
  const size_t smem = pass_smem(a.max_slots, a.n_groups, a.max_list, W, FIRST, &staged);
  const int64_t slabs = (a.ncols + W - 1) / W;
  // Fibers along x, so that the CTAs resident on an SM belong to different fibers (different slot and
  // list counts) and their staging and folding phases drift apart instead of running in step.
  const int64_t groups = (slabs + a.slabs_per_cta - 1) / a.slabs_per_cta;
  SplitPass b = a;
  b.fiber_x = groups <= 65535 ? 1 : 0;
  const dim3 grid = b.fiber_x ? dim3((unsigned)fibers, (unsigned)groups) : dim3((unsigned)groups, (unsigned)fibers);
  void (*k)(SplitPass) = nullptr;
  if (staged) {
    switch (W) {
      case 256: k = split_pass_kernel<256, FIRST, RING, true>; break;
      case 128: k = split_pass_kernel<128, FIRST, RING, true>; break;
      case 64: k = split_pass_kernel<64, FIRST, RING, true>; break;
      default: k = split_pass_kernel<32, FIRST, RING, true>; break;
    }
  } else {
    switch (W) {
      case 256: k = split_pass_kernel<256, FIRST, RING, false>; break;
      case 128: k = split_pass_kernel<128, FIRST, RING, false>; break;
      case 64: k = split_pass_kernel<64, FIRST, RING, false>; break;
      default: k = split_pass_kernel<32, FIRST, RING, false>; break;
    }
  }
  cudaError_t e = ensure_limits();
  if (e != cudaSuccess) return e;
  k<<<grid, kSplitThreads, smem, s>>>(b);
  return cudaGetLastError();
}

// Both passes over the columns in chunks of info.chunk_cols (all N at once when 0): X holds one chunk.
template <bool RING>
cudaError_t run_passes(SplitPass p1, SplitPass p2, const rd_split_info_t& info, cudaStream_t s) {
  const int64_t N = info.N;
  const int64_t cw = info.chunk_cols > 0 ? info.chunk_cols : N;
  cudaError_t e = cudaSuccess;
  for (int64_t c0 = 0; c0 < N && e == cudaSuccess; c0 += cw) {
    const int64_t w = (N - c0 < cw) ? (N - c0) : cw;
    p1.ncols = p2.ncols = w;
    p1.in_col0 = c0;
    p1.out_col0 = 0;
    p2.in_col0 = 0;
    p2.out_col0 = c0;
    e = launch_pass<true, RING>(p1, info.w1, info.n_sigma, s);
    if (e == cudaSuccess) e = launch_pass<false, RING>(p2, info.w2, info.n_pi, s);
  }
  return e;
}

// The two passes' fixed operands, from a built plan.
void passes_of(const rd_split_info_t& info, const void* plan, SplitPass* p1, SplitPass* p2) {
  Layout L;
  make_layout(info.m, info.j, &L);
  *p1 = SplitPass{};
  *p2 = SplitPass{};
  p1->ncols = p2->ncols = info.N;
  p1->in_rows = p2->out_rows = info.N;
  p1->out_rows = p2->in_rows = info.x_rows;
  p1->n_groups = (int32_t)L.nG1;
  p1->max_slots = info.slots1;
  p1->max_list = info.lmax1;
  p1->slabs_per_cta = info.k1;
  p1->fstart = at<int32_t>(plan, L.fstart1);
  p1->fmem = at<int32_t>(plan, L.fmem1);
  p1->gls = at<int32_t>(plan, L.gls1);
  p1->lst = at<uint16_t>(plan, L.l1);
  p1->go = at<int32_t>(plan, L.go1);
  p1->ord = at<uint16_t>(plan, L.ord1);
  p2->n_groups = (int32_t)L.nG2;
  p2->max_slots = info.slots2;
  p2->max_list = info.lmax2;
  p2->slabs_per_cta = info.k2;
  p2->fstart = at<int32_t>(plan, L.fstart2);
  p2->gls = at<int32_t>(plan, L.gls2);
  p2->lst = at<uint16_t>(plan, L.l2);
  p2->go = at<int32_t>(plan, L.go2);
  p2->ord = at<uint16_t>(plan, L.ord2);
}

bool info_ok(const rd_split_info_t* info, const void* plan) {
  if (!info || !plan || !aligned16(plan)) return false;
  Layout L;
  if (!make_layout(info->m, info->j, &L)) return false;
  if (info->N != L.N || info->n_pi != L.nPi || info->n_phi != L.nPhi) return false;
  if (info->n_rho < 1 || info->n_rho > L.rhoB || info->n_sigma < 1 || info->n_sigma > L.sigB) return false;
  if (info->slots1 < 1 || info->slots1 > L.nPi || info->slots2 < 1 || info->slots2 > info->n_sigma) return false;
  if (info->x_rows < 1 || info->x_rows > (int64_t)L.nPi * info->n_sigma) return false;
  if (info->lmax1 < 0 || info->lmax2 < 0 || info->k1 < 1 || info->k1 > 64 || info->k2 < 1 || info->k2 > 64)
    return false;
  if (info->chunk_cols < 0 || info->chunk_cols % 128 != 0) return false;
  return valid_w(info->w1, info->slots1) && valid_w(info->w2, info->slots2);
}

// Columns X must hold: one chunk, or all N.
int64_t x_cols(const rd_split_info_t& info) { return info.chunk_cols > 0 ? info.chunk_cols : info.N; }

struct SplitCtx {
  SplitPass p1, p2;
  rd_split_info_t info;
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
  // Unchunked, pass 1 sees every entry before pass 2 starts and reduces the offset step itself, and
  // pass 2 writes the normalised power; in column chunks the normaliser pass does it after both.
  p1.norm = p2.norm = split_normalises(c->info) ? 1 : 0;
  p2.min_out = p2.norm ? nullptr : &r.st->mu;
  p2.diag_out = &r.st->dmin;
  return run_passes<true>(p1, p2, c->info, s);
}

rd_status fail(cudaError_t e) {
  set_cuda_error(e);
  return RD_ERR_CUDA;
}

}  // namespace

bool split_normalises(const rd_split_info_t& info) { return info.chunk_cols == 0; }

bool split_ring_ok(const SplitRing& d, int64_t N) {
  return info_ok(&d.info, d.plan) && d.info.N == N && d.X != nullptr && aligned16(d.X) && d.ldx >= x_cols(d.info) &&
         d.ldx % 8 == 0;
}

cudaError_t split_ring_product(const SplitRing& d, PowerState* st, int16_t* ring, int64_t slot_elems, int slots,
                               int64_t ld, cudaStream_t s) {
  SplitCtx c{};
  passes_of(d.info, d.plan, &c.p1, &c.p2);
  c.p1.out = d.X;
  c.p1.ldout = d.ldx;
  c.p2.in = d.X;
  c.p2.ldin = d.ldx;
  c.info = d.info;
  Run r{};
  r.st = st;
  r.ring = ring;
  r.slot_elems = slot_elems;
  r.slots = slots;
  r.N = d.info.N;
  r.ld = ld;
  return split_power_product(r, &c, s);
}

namespace {

unsigned grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

// Flags and exclusive ranks of the correct words of len letters (len may be 0), total in rank[4^len].
void rank_correct(int32_t* rank, int len, cudaStream_t s) {
  const int64_t n = ipow(4, len);
  correct_flag_kernel<<<grid_for(n), 256, 0, s>>>(rank, len, n);
  scan_i32_kernel<<<1, 1024, 0, s>>>(rank, n);
}

cudaError_t read_i32(const int32_t* dev, int32_t* host, int n, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(host, dev, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Up to 8 scattered device int32 values gathered into one readback (one host round trip instead of n).
struct Gather8 {
  const int32_t* src[8];
  int n;
};
__global__ void gather_i32_kernel(Gather8 g, int32_t* dst) {
  if ((int)threadIdx.x < g.n) dst[threadIdx.x] = *g.src[threadIdx.x];
}
cudaError_t read_gathered_i32(std::initializer_list<const int32_t*> srcs, int32_t* stage_dev, int32_t* host,
                              cudaStream_t s) {
  Gather8 g{};
  if (srcs.size() > 8) return cudaErrorInvalidValue;
  for (const int32_t* p : srcs) g.src[g.n++] = p;
  gather_i32_kernel<<<1, 32, 0, s>>>(g, stage_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? read_i32(stage_dev, host, g.n, s) : e;
}

}  // namespace

bool split_width_fits(int W, int max_slots) { return valid_w(W, max_slots); }

}  // namespace rd

using namespace rd;

extern "C" int rd_split_default_j(int m) {
  if (m < 2 || m > RD_MAX_M) return 0;
  // The lower half gets the extra row up to m = 10 and the upper half from m = 11 on: at m = 11 the split
  // after row 5 gives pass-2 fibers of up to 1085 slots (32-column slabs), after row 6 fibers of at most
  // 848, and the product takes 137 ms against 161 ms (tuned 135 against 153); for m = 5, 7, 9 the two
  // choices are within 2 % of each other.
  const int j = (m >= 11) ? m - m / 2 : m / 2;
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
  const int64_t n5j = ipow(kTauCount, j), n5h = ipow(kTauCount, h);
  int32_t* counters = at<int32_t>(P, L.counters);
  cudaError_t e0 = ensure_limits();
  if (e0 != cudaSuccess) return fail(e0);
  rd_status rc = rd_enumerate_states(m, at<uint32_t>(P, L.codes), at<uint8_t>(P, L.wts), s);
  if (rc != RD_OK) return rc;
  cudaError_t e = cudaMemsetAsync(at<int32_t>(P, L.rankR), 0, (size_t)(n5j + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<int32_t>(P, L.rankS), 0, (size_t)(n5h + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 8 * 4, s);
  if (e != cudaSuccess) return fail(e);
  split_mark_kernel<<<grid_for(L.N), 256, 0, s>>>(at<uint32_t>(P, L.codes), L.N, m, j, at<int32_t>(P, L.rankR),
                                                   at<int32_t>(P, L.rankS));
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankR), n5j);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.rankS), n5h);
  // the correct words of j, h, j - 1 and h - 1 letters; the last two are the output groups
  rank_correct(at<int32_t>(P, L.rankPi), j, s);
  rank_correct(at<int32_t>(P, L.rankPhi), h, s);
  rank_correct(at<int32_t>(P, L.rankG1), j - 1, s);
  rank_correct(at<int32_t>(P, L.rankG2), h - 1, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  int32_t cnt[6] = {0, 0, 0, 0, 0, 0};
  const int32_t* totals[6] = {at<int32_t>(P, L.rankR) + n5j,         at<int32_t>(P, L.rankS) + n5h,
                              at<int32_t>(P, L.rankPi) + ipow(4, j), at<int32_t>(P, L.rankPhi) + ipow(4, h),
                              at<int32_t>(P, L.rankG1) + ipow(4, j - 1), at<int32_t>(P, L.rankG2) + ipow(4, h - 1)};
  int32_t* stage = counters + 16;
  e = read_gathered_i32({totals[0], totals[1], totals[2], totals[3], totals[4], totals[5]}, stage, cnt, s);
  if (e != cudaSuccess) return fail(e);
  const int64_t n_rho = cnt[0], n_sigma = cnt[1];
  // the type counts are within their bounds, and the letter words counted are the correct words
  if (n_rho < 1 || n_rho > L.rhoB || n_sigma < 1 || n_sigma > L.sigB || cnt[2] != L.nPi || cnt[3] != L.nPhi ||
      cnt[4] != L.nG1 || cnt[5] != L.nG2 || L.nPi >= 0xFFFF || n_sigma >= 0xFFFF)
    return RD_ERR_RANGE;
  invert_kernel<<<grid_for(n5j), 256, 0, s>>>(at<int32_t>(P, L.rankR), n5j, at<int32_t>(P, L.rhoCode));
  invert_kernel<<<grid_for(n5h), 256, 0, s>>>(at<int32_t>(P, L.rankS), n5h, at<int32_t>(P, L.sigCode));
  invert_kernel<<<grid_for(ipow(4, j)), 256, 0, s>>>(at<int32_t>(P, L.rankPi), ipow(4, j), at<int32_t>(P, L.piCode));
  invert_kernel<<<grid_for(ipow(4, j - 1)), 256, 0, s>>>(at<int32_t>(P, L.rankG1), ipow(4, j - 1),
                                                         at<int32_t>(P, L.g1Code));
  invert_kernel<<<grid_for(ipow(4, h - 1)), 256, 0, s>>>(at<int32_t>(P, L.rankG2), ipow(4, h - 1),
                                                         at<int32_t>(P, L.g2Code));
  e = cudaMemsetAsync(at<int32_t>(P, L.fiber), 0xFF, (size_t)n_sigma * (size_t)n_rho * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<int32_t>(P, L.outrow), 0xFF, (size_t)L.nPi * (size_t)L.nPhi * 4, s);
  if (e != cudaSuccess) return fail(e);
  split_index_kernel<<<grid_for(L.N), 256, 0, s>>>(at<uint32_t>(P, L.codes), L.N, m, j, at<int32_t>(P, L.rankR),
                                                   at<int32_t>(P, L.rankS), n_rho, at<int32_t>(P, L.rankPi),
                                                   at<int32_t>(P, L.rankPhi), L.nPhi, at<int32_t>(P, L.fiber),
                                                   at<int32_t>(P, L.outrow));
  // pass-1 fibers in compact form, then the finite rows of X and the pass-2 fibers
  fiber_count_kernel<<<grid_for(n_sigma), 256, 0, s>>>(at<int32_t>(P, L.fiber), n_sigma, n_rho,
                                                       at<int32_t>(P, L.fstart1));
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.fstart1), n_sigma);
  fiber_fill_kernel<<<grid_for(n_sigma), 256, 0, s>>>(at<int32_t>(P, L.fiber), n_sigma, n_rho,
                                                      at<int32_t>(P, L.fstart1), at<int32_t>(P, L.fmem1),
                                                      at<int32_t>(P, L.frho1), counters + 0);
  const int64_t nx = L.nPi * n_sigma;
  xflag_kernel<<<grid_for(nx), 256, 0, s>>>(at<int32_t>(P, L.piCode), L.nPi, n_sigma, at<int32_t>(P, L.fstart1),
                                             at<int32_t>(P, L.frho1), at<int32_t>(P, L.rhoCode), j,
                                             at<int32_t>(P, L.xrank));
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.xrank), nx);
  xsig_kernel<<<grid_for(nx), 256, 0, s>>>(at<int32_t>(P, L.xrank), L.nPi, n_sigma, at<int32_t>(P, L.xsig),
                                            at<int32_t>(P, L.fstart2), counters + 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  int32_t c3[3] = {0, 0, 0};
  e = read_gathered_i32({counters, counters + 1, at<int32_t>(P, L.xrank) + nx}, stage, c3, s);
  if (e != cudaSuccess) return fail(e);
  const int32_t slots1 = c3[0], slots2 = c3[1], x_rows = c3[2];
  if (slots1 < 1 || slots1 > L.nPi || slots2 < 1 || slots2 > n_sigma || x_rows < 1) return RD_ERR_RANGE;

  GroupArgs g1{};
  g1.first = 1;
  g1.len = j;
  g1.n_fibers = n_sigma;
  g1.n_groups = L.nG1;
  g1.gcode = at<int32_t>(P, L.g1Code);
  g1.fstart = at<int32_t>(P, L.fstart1);
  g1.slot_tc = at<int32_t>(P, L.frho1);
  g1.tcode = at<int32_t>(P, L.rhoCode);
  GroupArgs g2{};
  g2.first = 0;
  g2.len = h;
  g2.n_fibers = L.nPi;
  g2.n_groups = L.nG2;
  g2.gcode = at<int32_t>(P, L.g2Code);
  g2.fstart = at<int32_t>(P, L.fstart2);
  g2.slot_tc = at<int32_t>(P, L.xsig);
  g2.tcode = at<int32_t>(P, L.sigCode);
  g2.piCode = at<int32_t>(P, L.piCode);
  const int64_t nrec1 = n_sigma * L.nG1, nrec2 = L.nPi * L.nG2;
  group_lists_kernel<false><<<grid_for(nrec1), 256, 0, s>>>(g1, at<int32_t>(P, L.gls1), nullptr, counters + 4);
  group_lists_kernel<false><<<grid_for(nrec2), 256, 0, s>>>(g2, at<int32_t>(P, L.gls2), nullptr, counters + 4);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.gls1), nrec1 * kRec);
  scan_i32_kernel<<<1, 1024, 0, s>>>(at<int32_t>(P, L.gls2), nrec2 * kRec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  // the longest fiber lists (read only from the scanned counts, so safe to take before the checks below)
  fiber_list_max_kernel<<<grid_for(n_sigma), 256, 0, s>>>(at<int32_t>(P, L.gls1), n_sigma, L.nG1, counters + 2);
  fiber_list_max_kernel<<<grid_for(L.nPi), 256, 0, s>>>(at<int32_t>(P, L.gls2), L.nPi, L.nG2, counters + 3);
  int32_t tot[5] = {0, 0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = read_gathered_i32({at<int32_t>(P, L.gls1) + nrec1 * kRec, at<int32_t>(P, L.gls2) + nrec2 * kRec, counters + 4,
                           counters + 2, counters + 3},
                          stage, tot, s);
  if (e != cudaSuccess) return fail(e);
  // a target set outside the 7 would be a slip in the rules above: refuse the plan
  if (tot[0] > L.l1B || tot[1] > L.l2B || tot[2] != 0) return RD_ERR_RANGE;
  const int32_t lm[2] = {tot[3], tot[4]};
  const int w1 = choose_w(slots1, (int)L.nG1, lm[0], true), w2 = choose_w(slots2, (int)L.nG2, lm[1], false);
  if (w1 == 0 || w2 == 0) return RD_ERR_ARG;  // a fiber does not fit in shared memory
  group_lists_kernel<true><<<grid_for(nrec1), 256, 0, s>>>(g1, at<int32_t>(P, L.gls1), at<uint16_t>(P, L.l1), nullptr);
  group_lists_kernel<true><<<grid_for(nrec2), 256, 0, s>>>(g2, at<int32_t>(P, L.gls2), at<uint16_t>(P, L.l2), nullptr);
  group_order_kernel<<<(unsigned)n_sigma, 128, (size_t)L.nG1 * 8, s>>>(at<int32_t>(P, L.gls1), L.nG1,
                                                                     at<uint16_t>(P, L.ord1));
  group_order_kernel<<<(unsigned)L.nPi, 128, (size_t)L.nG2 * 8, s>>>(at<int32_t>(P, L.gls2), L.nG2,
                                                                   at<uint16_t>(P, L.ord2));
  group_out_kernel<<<grid_for(nrec1), 256, 0, s>>>(g1, at<int32_t>(P, L.rankPi), at<int32_t>(P, L.xrank), n_sigma,
                                                   nullptr, 0, at<int32_t>(P, L.go1));
  group_out_kernel<<<grid_for(nrec2), 256, 0, s>>>(g2, at<int32_t>(P, L.rankPhi), nullptr, 0,
                                                   at<int32_t>(P, L.outrow), L.nPhi, at<int32_t>(P, L.go2));
  e = cudaGetLastError();
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
  info->x_rows = x_rows;
  info->plan_bytes = L.bytes;
  info->w1 = w1;
  info->w2 = w2;
  info->slots1 = slots1;
  info->slots2 = slots2;
  info->lmax1 = lm[0];
  info->lmax2 = lm[1];
  info->k1 = kDefaultSlabsPerCta;
  info->k2 = kDefaultSlabsPerCta;
  info->chunk_cols = 0;
  rd_tune_entry_t t;  // a tuned launch shape for this (m, j), when its widths fit this plan
  if (tune_find(RD_TUNE_SPLIT, m, j, &t) && valid_w(t.p[0], slots1) && valid_w(t.p[2], slots2)) {
    info->w1 = t.p[0];
    info->k1 = t.p[1];
    info->w2 = t.p[2];
    info->k2 = t.p[3];
  }
  return RD_OK;
}

extern "C" rd_status rd_split_minplus(const rd_split_info_t* info, const void* plan_dev, const int16_t* B,
                                      int64_t ldb, int16_t* X_dev, int64_t ldx, int16_t* C, int64_t ldc,
                                      int32_t* min_out, cudaStream_t s) {
  if (!info_ok(info, plan_dev) || !B || !X_dev || !C) return RD_ERR_ARG;
  const int64_t N = info->N;
  if (ldb < N || ldb % 8 != 0 || ldx < x_cols(*info) || ldx % 8 != 0 || ldc < N || ldc % 8 != 0) return RD_ERR_ARG;
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
  e = run_passes<false>(p1, p2, *info, s);
  if (e != cudaSuccess) return fail(e);
  return RD_OK;
}

namespace rd {
namespace {

// Plain passes over an N x N power (row-major, leading dimension ld a multiple of 8, 16-byte aligned rows),
// blocks striding over rows and threads over 16-byte chunks; entries past column N are padding and ignored.
__device__ __forceinline__ uint32_t tail_keep(int64_t j0, int64_t N, int q) {
  // halfword mask of word q of the chunk at column j0: 0xFFFF for columns < N
  const int64_t c = j0 + 2 * q;
  return (c < N ? 0x0000FFFFu : 0u) | (c + 1 < N ? 0xFFFF0000u : 0u);
}

__global__ void plain_min_kernel(const int16_t* __restrict__ X, int64_t N, int64_t ld, int32_t* out) {
  uint32_t m2 = kInf2;
  const int64_t cpr = (N + 7) / 8;
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x)
    for (int64_t c = threadIdx.x; c < cpr; c += blockDim.x) {
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(X + i * ld + c * 8));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t keep = tail_keep(c * 8, N, q);
        m2 = __vminu2(m2, (w[q] & keep) | (kInf2 & ~keep));
      }
    }
  int32_t m = (int32_t)min(m2 & 0xFFFFu, m2 >> 16);
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0 && m < kInf) atomicMin(out, m);
}

// dst = src - mu on finite entries (the search's normalisation of a power); padding columns copied as they are
__global__ void plain_normalise_kernel(const int16_t* __restrict__ src, int16_t* __restrict__ dst, int64_t N,
                                       int64_t ld, const int32_t* mu_dev) {
  const int32_t mu_raw = *mu_dev;
  const uint32_t mu2 = (uint32_t)((mu_raw >= kInf) ? 0 : mu_raw) * 0x00010001u;
  const int64_t cpr = (N + 7) / 8;
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x)
    for (int64_t c = threadIdx.x; c < cpr; c += blockDim.x) {
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(src + i * ld + c * 8));
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t isinf = __vcmpeq2(w[q], kInf2);
        w[q] = __vsub2(w[q], mu2 & ~isinf);
      }
      *reinterpret_cast<uint4*>(dst + i * ld + c * 8) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// *flag = 1 when a and b differ in some entry of the N x N matrix
__global__ void plain_differ_kernel(const int16_t* __restrict__ a, const int16_t* __restrict__ b, int64_t N,
                                    int64_t ld, int32_t* flag) {
  uint32_t d = 0;
  const int64_t cpr = (N + 7) / 8;
  for (int64_t i = blockIdx.x; i < N; i += gridDim.x)
    for (int64_t c = threadIdx.x; c < cpr; c += blockDim.x) {
      const uint4 x = __ldcg(reinterpret_cast<const uint4*>(a + i * ld + c * 8));
      const uint4 y = __ldcg(reinterpret_cast<const uint4*>(b + i * ld + c * 8));
      d |= ((x.x ^ y.x) & tail_keep(c * 8, N, 0)) | ((x.y ^ y.y) & tail_keep(c * 8, N, 1)) |
           ((x.z ^ y.z) & tail_keep(c * 8, N, 2)) | ((x.w ^ y.w) & tail_keep(c * 8, N, 3));
    }
  if (__syncthreads_or(d != 0) && threadIdx.x == 0) atomicOr(flag, 1);
}

// The search stopped at P_j with P_i (i < j) its only hash match, out of the ring.  Re-derive P_i from A(G)
// in the two ring slots that do not hold P_j -- A(G) rebuilt, normalised, then i - 1 row-split products each
// normalised, the same arithmetic as the search -- and compare it with P_j entry by entry.  The search state's
// scalar fields serve as device scratch (the search has stopped).
rd_status verify_far_pair(const rd_split_info_t& info, const void* plan, int16_t* X, int64_t ldx, int64_t lda,
                          void* work_dev, int kmax, int slots, int i, int j, bool* equal, cudaStream_t s) {
  const int64_t N = info.N;
  PowerState* st = reinterpret_cast<PowerState*>(work_dev);
  int16_t* ring = reinterpret_cast<int16_t*>(static_cast<char*>(work_dev) + state_bytes(kmax));
  const int64_t se = (int64_t)(slot_bytes(N, lda) / 2);
  int16_t* pj = ring + (int64_t)(j % slots) * se;
  int16_t* cur = ring + (int64_t)((j + 1) % slots) * se;
  int16_t* nxt = ring + (int64_t)((j + 2) % slots) * se;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(sms * 8);
  rd_status rc = rd_build_transfer(info.m, cur, lda, s);
  if (rc != RD_OK) return rc;
  cudaError_t e = launch_fill_i32(&st->mu, kInf, s);
  if (e == cudaSuccess) {
    plain_min_kernel<<<grid, 256, 0, s>>>(cur, N, lda, &st->mu);
    plain_normalise_kernel<<<grid, 256, 0, s>>>(cur, nxt, N, lda, &st->mu);  // P_1
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(e);
  int16_t* p = nxt;
  int16_t* q = cur;
  for (int t = 1; t < i; ++t) {  // P_(t+1) from P_t
    rc = rd_split_minplus(&info, plan, p, lda, X, ldx, q, lda, &st->mu, s);
    if (rc != RD_OK) return rc;
    plain_normalise_kernel<<<grid, 256, 0, s>>>(q, q, N, lda, &st->mu);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e);
    int16_t* t2 = p;
    p = q;
    q = t2;
  }
  e = launch_fill_i32(&st->dmin, 0, s);
  if (e == cudaSuccess) {
    plain_differ_kernel<<<grid, 256, 0, s>>>(p, pj, N, lda, &st->dmin);
    e = cudaGetLastError();
  }
  int32_t differ = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&differ, &st->dmin, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  *equal = differ == 0;
  return RD_OK;
}

}  // namespace
}  // namespace rd

extern "C" rd_status rd_power_until_periodic_split(const int16_t* A_dev, int64_t lda, const rd_split_info_t* info,
                                                   const void* plan_dev, int16_t* X_dev, int64_t ldx, int kmax,
                                                   void* work_dev, size_t work_bytes, int64_t* gamma_host,
                                                   int32_t* k_out, int32_t* p_out, int64_t* q_out, cudaStream_t s) {
  if (!A_dev || !info_ok(info, plan_dev) || !X_dev || !work_dev || !gamma_host || !k_out || !p_out || !q_out)
    return RD_ERR_ARG;
  const int64_t N = info->N;
  if (lda < N || lda % 8 != 0 || ldx < x_cols(*info) || ldx % 8 != 0 || kmax < 1 || kmax > (1 << 20))
    return RD_ERR_ARG;
  if (!aligned16(A_dev) || !aligned16(X_dev) || (reinterpret_cast<uintptr_t>(work_dev) & 255u) != 0)
    return RD_ERR_ARG;
  SplitCtx c{};
  passes_of(*info, plan_dev, &c.p1, &c.p2);
  c.p1.out = X_dev;
  c.p1.ldout = ldx;
  c.p2.in = X_dev;
  c.p2.ldin = ldx;
  c.info = *info;
  rd_status rc = power_search(A_dev, N, lda, kmax, work_dev, work_bytes, split_power_product, &c, gamma_host, k_out,
                              p_out, q_out, s, split_normalises(*info));
  if (rc != RD_ERR_NOMEM) return rc;
  // Stopped with a hash match out of the ring?  Then verify it by re-deriving the earlier power.
  PowerState h{};
  cudaError_t e = cudaMemcpyAsync(&h, work_dev, sizeof(PowerState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  if (!(h.done == 3 && h.err == kErrRing && h.slots >= 3 && h.found_i >= 1 && h.found_j > h.found_i)) return rc;
  bool equal = false;
  rc = verify_far_pair(*info, plan_dev, X_dev, ldx, lda, work_dev, kmax, h.slots, h.found_i, h.found_j, &equal, s);
  if (rc != RD_OK) return rc;
  if (!equal) return RD_ERR_NOMEM;  // a hash collision with a power that has left the ring
  int64_t off_i = 0, off_j = 0;
  const int64_t* off = reinterpret_cast<const int64_t*>(static_cast<const char*>(work_dev) + kStateHeader);
  e = cudaMemcpyAsync(&off_i, off + h.found_i, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&off_j, off + h.found_j, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e);
  *k_out = h.found_i;
  *p_out = h.found_j - h.found_i;
  *q_out = off_j - off_i;
  return RD_OK;
}

extern "C" rd_status rd_split_check_flags(uint32_t* flags, int reset) {
  if (!flags) return RD_ERR_ARG;
  *flags = 0;
#ifdef RD_CHECKED
  unsigned int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_split_check, sizeof(v));
  if (e == cudaSuccess && reset) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_split_check, &zero, sizeof(zero));
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return RD_ERR_CUDA;
  }
  *flags = v;
  return RD_OK;
#else
  (void)reset;
  return RD_NOT_FOUND;
#endif
}
