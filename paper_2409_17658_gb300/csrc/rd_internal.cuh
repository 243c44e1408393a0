// rd_internal.cuh -- definitions shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "rd.h"

namespace rd {

constexpr int16_t kInf = RD_INF;
constexpr uint32_t kInf2 = 0x3FFF3FFFu;  // RD_INF in both halfwords
constexpr int kMaxFinite = RD_MAX_FINITE;
constexpr int kMaxCand = 8;

// Device-resident bookkeeping of one rd_power_until_periodic run.  It lives at
// the front of the caller's work buffer; the per-power arrays follow it.
struct PowerState {
  int32_t k;            // index of the latest finished normalised power P_k
  int32_t done;         // 0 running, 1 relation found, 2 kmax reached, 3 error
  int32_t err;          // kErr* bits: range, ring too short, too many hash candidates, device wait timed out
  int32_t kmax;
  int32_t mu;           // atomicMin target: min of the raw product being formed
  int32_t dmin;         // atomicMin target: min of its diagonal
  uint32_t blocks_done; // arrival counter of the compare kernel
  int32_t ncand;
  int32_t cand[kMaxCand];
  int32_t mismatch[kMaxCand];
  int32_t found_i, found_j;
  int64_t found_q;
  unsigned long long hacc;  // hash accumulator of the power being normalised
  int32_t range_bad;
  int32_t slots;
  // the multi-run step kernel: items finished per dependency level of this run in the current launch, and
  // (in the first run's state) the launch's item queue and its count of CTAs that have left the queue
  uint32_t lvl_done[4];
  uint32_t queue;
  uint32_t exited;
  // the smallest earlier power whose hash matches the new one but which has left the ring (kFarNone: none);
  // when no power in the ring matches exactly, the search stops with kErrRing and found_i = far_i,
  // found_j = the new power, so a caller that can re-derive that power may still verify the relation
  int32_t far_i;
};
constexpr int32_t kFarNone = 0x7FFFFFFF;

constexpr size_t kStateHeader = 256;
static_assert(sizeof(PowerState) <= kStateHeader, "state header too large");

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// PowerState::err bits and the status a stopped search reports for them.
constexpr int32_t kErrRange = 1, kErrRing = 2, kErrCandidates = 4, kErrTimeout = 8;
inline rd_status status_from_err(int32_t err) {
  if (err & kErrRange) return RD_ERR_RANGE;
  if (err & kErrTimeout) return RD_ERR_TIMEOUT;
  return RD_ERR_NOMEM;
}

// Layout of the work buffer: [header][offset int64 x (kmax+1)][gamma int64 x (kmax+1)]
// [hash u64 x (kmax+1)] padded to 256 B, then the ring of power slots.
inline size_t state_bytes(int kmax) { return round_up(kStateHeader + 3 * 8 * (size_t)(kmax + 1), 256); }
inline size_t slot_bytes(int64_t N, int64_t ld) { return round_up((size_t)N * (size_t)ld * 2, 256); }

__host__ __device__ inline int64_t* st_offset(PowerState* st) {
  return reinterpret_cast<int64_t*>(reinterpret_cast<char*>(st) + kStateHeader);
}
__host__ __device__ inline int64_t* st_gamma(PowerState* st) { return st_offset(st) + (st->kmax + 1); }
__host__ __device__ inline unsigned long long* st_hash(PowerState* st) {
  return reinterpret_cast<unsigned long long*>(st_gamma(st) + (st->kmax + 1));
}

// Operands of one (min,+) product.  In ring mode the left operand and the
// result are power slots chosen on the device from st->k.
struct GemmParams {
  const int16_t* A;
  int64_t lda;
  const int16_t* B;
  int64_t ldb;
  int16_t* C;
  int64_t ldc;
  int64_t M, N, K;
  int32_t* min_out;   // nullable; atomicMin of all result entries
  int32_t* diag_out;  // nullable; atomicMin of the diagonal entries
  PowerState* st;     // ring mode only
  int16_t* ring;
  int64_t slot_elems;
  int slots;
};

// Launchers implemented in the .cu files.
// force_splitk > 0 (not in ring mode): split K by exactly that factor, with tile shape force_tile (0: 128 x
// 256, 1: 128 x 128) -- the autotuner's trials; else the tuning table's factor and tile for the product's
// size class, else the built-in rule (the wide tile).
cudaError_t launch_minplus_gemm(const GemmParams& p, bool ring, cudaStream_t s, int force_splitk = 0,
                                int force_tile = 0);
bool splitk_suits(int S, int64_t K);         // S in {1, 2, 4, 8} and every K slice non-empty
int64_t gemm_tiles(int64_t M, int64_t N);  // output tiles (CTAs of an unsplit launch)

// The tuning table (tune.cu): lookup and insert-or-replace by (mode, key, aux).
bool tune_find(int mode, int key, int aux, rd_tune_entry_t* out);
bool tune_put(const rd_tune_entry_t& e);

// Row-split passes (split.cu): whether slab width W fits with max_slots staged rows.
bool split_width_fits(int W, int max_slots);
cudaError_t launch_fill_i32(int32_t* dst, int32_t value, cudaStream_t s);

// One run of the period search (power.cu): the device state, the ring of powers and the operand.
struct Run {
  PowerState* st;
  int16_t* ring;
  int64_t slot_elems;
  int slots;
  int64_t N, ld;
  const int16_t* A;
  int grid;
};

// Enqueues R = (next raw power) into the ring slot of power st->k + 1, with min and diag-min into
// st->mu and st->dmin.  `ctx` carries the product's own operands.
typedef cudaError_t (*ProductFn)(const Run& r, const void* ctx, cudaStream_t s);

cudaError_t dense_power_product(const Run& r, const void* ctx, cudaStream_t s);

// `normalised`: the product itself writes the normalised power, its hash and range flag into the
// state (the row-split step), so the normaliser pass is skipped.  `lookahead`: keep a block of steps
// queued ahead of the host's check (uses page-locked host memory, made once per thread and device);
// false reads the state after each block with no allocation at all.
rd_status power_search(const int16_t* A_dev, int64_t N, int64_t lda, int kmax, void* work_dev, size_t work_bytes,
                       ProductFn product, const void* ctx, int64_t* gamma_host, int32_t* k_out, int32_t* p_out,
                       int64_t* q_out, cudaStream_t s, bool normalised = false, bool lookahead = true);

// A built row-split plan with its intermediate (split.cu), and the ring-mode product it runs: the
// next power A(G) (x) P_k, already normalised, into the slot of power st->k + 1, with its minimum
// (the offset step), raw diagonal minimum, hash and range flag in st -- everything the normaliser
// pass would add, so runs stepped by it skip that pass.
struct SplitRing {
  rd_split_info_t info;
  const void* plan;
  int16_t* X;
  int64_t ldx;
};
bool split_ring_ok(const SplitRing& d, int64_t N);
bool split_normalises(const rd_split_info_t& info);  // the ring product writes the normalised power
cudaError_t split_ring_product(const SplitRing& d, PowerState* st, int16_t* ring, int64_t slot_elems, int slots,
                               int64_t ld, cudaStream_t s);

// One period-search run as the multi-run kernels see it (power_multi.cu).
struct RunDesc {
  PowerState* st;
  int16_t* ring;
  int64_t slot_elems;
  int slots;
  int64_t N, ld;
  const int16_t* A;
  const int64_t* start;
  const uint32_t* rec;
  int64_t nb_unused, slabs_unused;  // filled in by the launcher
  const SplitRing* split;           // non-null: the row-split step instead of the sparse one
  int32_t normalised;               // the product writes the normalised power (no normaliser pass)
};
constexpr int kMaxRunsPerStep = 16;
cudaError_t runs_first(const RunDesc* runs, int count, int R, int kmax, cudaStream_t s);
cudaError_t runs_step(const RunDesc* runs, int count, int R, cudaStream_t s);

void set_cuda_error(cudaError_t e);
bool aligned16(const void* p);

// A relation record (rd_relation_t) and its gamma[0..j] pass the checks every record of a transfer
// matrix satisfies (power.cu; rd_gamma_R_import states them).
bool relation_ok(const rd_relation_t* rel, const int64_t* gamma);

}  // namespace rd
