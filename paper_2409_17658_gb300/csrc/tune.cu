// tune.cu -- the tuning table and the autotuners of the launch shapes.
//
// A launch shape (the output tile and split-K factor of the dense product, the slab widths and slabs per CTA of the
// row-split passes, the rows per block of the sparse step) changes how long a product takes, never
// what it computes.  The table maps (mode, size class) to the shape the autotuner measured fastest
// on this GPU; the launchers consult it and fall back to their built-in rules.  The table is one
// process-wide array under a mutex; the autotuners time their candidates with CUDA events on the
// caller's stream.
#include <mutex>

#include "rd_internal.cuh"

namespace rd {
namespace {

struct Table {
  std::mutex mu;
  rd_tune_entry_t e[RD_TUNE_MAX];
  int n = 0;
};

Table& table() {
  static Table t;
  return t;
}

bool same_key(const rd_tune_entry_t& a, const rd_tune_entry_t& b) {
  return a.mode == b.mode && a.key == b.key && a.aux == b.aux;
}

bool is_pow2_le8(int v) { return v == 1 || v == 2 || v == 4 || v == 8; }

bool entry_ok(const rd_tune_entry_t& t) {
  switch (t.mode) {
    case RD_TUNE_GEMM_SPLITK:
      return t.key >= 0 && t.key <= 63 && t.aux >= 0 && t.aux <= 63 && is_pow2_le8(t.p[0]) &&
             (t.p[1] == 0 || t.p[1] == 1);
    case RD_TUNE_SPLIT:
      return t.key >= 2 && t.key <= RD_MAX_M && t.aux >= 1 && t.aux < t.key &&
             (t.p[0] == 32 || t.p[0] == 64 || t.p[0] == 128 || t.p[0] == 256) && t.p[1] >= 1 && t.p[1] <= 64 &&
             (t.p[2] == 32 || t.p[2] == 64 || t.p[2] == 128 || t.p[2] == 256) && t.p[3] >= 1 && t.p[3] <= 64;
    case RD_TUNE_SPARSE_R:
      return t.key >= 0 && t.key <= 63 && t.aux == 0 && is_pow2_le8(t.p[0]);
    default:
      return false;
  }
}

// Mean milliseconds of `reps` calls of f after one warm-up call, or a negative value on failure.
template <class F>
float time_calls(F&& f, int reps, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t s, rd_status* rc) {
  *rc = f();
  if (*rc != RD_OK) return -1.f;
  cudaError_t e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    *rc = f();
    if (*rc != RD_OK) return -1.f;
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    *rc = RD_ERR_CUDA;
    return -1.f;
  }
  return ms / (float)reps;
}

struct Events {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    return e;
  }
  ~Events() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

bool tune_find(int mode, int key, int aux, rd_tune_entry_t* out) {
  Table& t = table();
  std::lock_guard<std::mutex> g(t.mu);
  for (int i = 0; i < t.n; ++i)
    if (t.e[i].mode == mode && t.e[i].key == key && t.e[i].aux == aux) {
      *out = t.e[i];
      return true;
    }
  return false;
}

bool tune_put(const rd_tune_entry_t& e) {
  if (!entry_ok(e)) return false;
  Table& t = table();
  std::lock_guard<std::mutex> g(t.mu);
  for (int i = 0; i < t.n; ++i)
    if (same_key(t.e[i], e)) {
      t.e[i] = e;
      return true;
    }
  if (t.n >= RD_TUNE_MAX) return false;
  t.e[t.n++] = e;
  return true;
}

}  // namespace rd

using namespace rd;

extern "C" int rd_tune_bucket(int64_t x) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) < x) ++b;
  return b;
}

extern "C" rd_status rd_tune_set(const rd_tune_entry_t* entries, int count) {
  if (count < 0 || count > RD_TUNE_MAX || (count > 0 && !entries)) return RD_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!entry_ok(entries[i])) return RD_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (same_key(entries[i], entries[j])) return RD_ERR_ARG;
  }
  Table& t = table();
  std::lock_guard<std::mutex> g(t.mu);
  for (int i = 0; i < count; ++i) t.e[i] = entries[i];
  t.n = count;
  return RD_OK;
}

extern "C" rd_status rd_tune_get(rd_tune_entry_t* entries, int cap, int* count) {
  if (cap < 0 || (cap > 0 && !entries) || !count) return RD_ERR_ARG;
  Table& t = table();
  std::lock_guard<std::mutex> g(t.mu);
  for (int i = 0; i < t.n && i < cap; ++i) entries[i] = t.e[i];
  *count = t.n;
  return RD_OK;
}

extern "C" rd_status rd_tune_lookup(int mode, int key, int aux, rd_tune_entry_t* out) {
  if (!out) return RD_ERR_ARG;
  return tune_find(mode, key, aux, out) ? RD_OK : RD_NOT_FOUND;
}

extern "C" rd_status rd_tune_gemm(const int16_t* A, int64_t lda, const int16_t* B, int64_t ldb, int16_t* C,
                                  int64_t ldc, int64_t M, int64_t N, int64_t K, int reps, rd_tune_entry_t* best,
                                  cudaStream_t s) {
  if (M < 2 || N < 1 || K < 1 || reps < 1 || !A || !B || !C) return RD_ERR_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return RD_ERR_ARG;
  if (lda < K || lda % 8 != 0 || ldb < N || ldb % 8 != 0 || ldc < N || ldc % 8 != 0) return RD_ERR_ARG;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles_wide = gemm_tiles(M, N), tiles_narrow = ((M + 127) / 128) * ((N + 127) / 128);
  Events ev;
  cudaError_t ce = ev.create();
  if (ce != cudaSuccess) {
    set_cuda_error(ce);
    return RD_ERR_CUDA;
  }
  GemmParams p{};
  p.A = A;
  p.lda = lda;
  p.B = B;
  p.ldb = ldb;
  p.C = C;
  p.ldc = ldc;
  p.M = M;
  p.N = N;
  p.K = K;
  rd_tune_entry_t t{};
  t.mode = RD_TUNE_GEMM_SPLITK;
  t.key = rd_tune_bucket(M > N ? M : N);
  t.aux = rd_tune_bucket(K);
  t.ms = -1.f;
  const int cands[4] = {1, 2, 4, 8};
  for (int tile = 0; tile < 2; ++tile) {
    // the wide tile runs 2 CTAs per SM, the narrow one 3
    const int64_t tiles = tile ? tiles_narrow : tiles_wide, wave = (tile ? 3 : 2) * (int64_t)sms;
    for (int S : cands) {
      if (!splitk_suits(S, K) || (S > 1 && tiles * S > 4 * wave)) continue;
      if (tile && tiles > 4 * wave) continue;  // the narrow tile only for products of a few waves
      rd_status rc = RD_OK;
      const float ms = time_calls(
          [&]() -> rd_status {
            const cudaError_t e = launch_minplus_gemm(p, false, s, S, tile);
            if (e != cudaSuccess) {
              set_cuda_error(e);
              return RD_ERR_CUDA;
            }
            return RD_OK;
          },
          reps, ev.e0, ev.e1, s, &rc);
      if (rc != RD_OK) return rc;
      if (t.ms < 0.f || ms < t.ms) {
        t.p[0] = S;
        t.p[1] = tile;
        t.ms = ms;
      }
    }
  }
  if (!tune_put(t)) return RD_ERR_NOMEM;  // the table is full
  if (best) *best = t;
  return RD_OK;
}

extern "C" rd_status rd_tune_split(rd_split_info_t* info, const void* plan_dev, const int16_t* B, int64_t ldb,
                                   int16_t* X_dev, int64_t ldx, int16_t* C, int64_t ldc, int reps,
                                   rd_tune_entry_t* best, cudaStream_t s) {
  if (!info || reps < 1) return RD_ERR_ARG;
  Events ev;
  cudaError_t ce = ev.create();
  if (ce != cudaSuccess) {
    set_cuda_error(ce);
    return RD_ERR_CUDA;
  }
  rd_split_info_t trial = *info;
  auto product = [&]() -> rd_status { return rd_split_minplus(&trial, plan_dev, B, ldb, X_dev, ldx, C, ldc, nullptr, s); };
  // the shape as given first: it validates the arguments and is the time to beat
  rd_status rc = RD_OK;
  float best_ms = time_calls(product, reps, ev.e0, ev.e1, s, &rc);
  if (rc != RD_OK) return rc;
  const int ws[4] = {32, 64, 128, 256}, ks[6] = {1, 2, 4, 8, 16, 32};
  for (int pass = 1; pass <= 2; ++pass) {
    const int slots = pass == 1 ? info->slots1 : info->slots2;
    for (int w : ws) {
      if (!split_width_fits(w, slots)) continue;
      for (int k : ks) {
        trial = *info;
        if (pass == 1) {
          if (w == info->w1 && k == info->k1) continue;
          trial.w1 = w;
          trial.k1 = k;
        } else {
          if (w == info->w2 && k == info->k2) continue;
          trial.w2 = w;
          trial.k2 = k;
        }
        const float ms = time_calls(product, reps, ev.e0, ev.e1, s, &rc);
        if (rc != RD_OK) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          *info = trial;  // the next candidates vary around the best so far
        }
      }
    }
  }
  rd_tune_entry_t t{};
  t.mode = RD_TUNE_SPLIT;
  t.key = info->m;
  t.aux = info->j;
  t.p[0] = info->w1;
  t.p[1] = info->k1;
  t.p[2] = info->w2;
  t.p[3] = info->k2;
  t.ms = best_ms;
  if (!tune_put(t)) return RD_ERR_NOMEM;
  if (best) *best = t;
  return RD_OK;
}
