// power_multi.cu -- several period searches (Algorithm 2) advanced together.
//
// Each run is its own transfer matrix with its own work buffer (state + ring), exactly as in
// rd_power_until_periodic_sparse / _split.  The runs form groups that advance side by side:
//  * every run stepped by the sparse step belongs to one group whose step is ONE launch of
//    multi_step_kernel, a persistent kernel that walks a list of work items of all its runs in
//    dependency levels (products, normaliser, finalize, compare; see below);
//  * every run stepped by the row split is a group of its own, stepped by its two pass launches and
//    its finalize and compare launches (inside the shared kernel its passes ran 40 % slower: one register
//    budget and one code image for every kind of item).
// rd_power_until_periodic_multi gives each group a stream of its own, forked from the caller's and joined
// after a block of steps, and captures a block of steps of all groups into one CUDA graph, so the groups'
// chains of steps run concurrently and small runs fill the gaps of the large ones.  Runs that have
// stopped exit at kernel entry, so the same launch sequence stays valid until the last run stops.
#include <cstdlib>
#include <cstring>

#include "power_dev.cuh"
#include "rd_internal.cuh"
#include "sparse_tile.cuh"

namespace rd {
namespace {

constexpr int kMaxRuns = 16;
constexpr int kMultiThreads = 128;  // product CTA width: a slab of 2048 columns

struct MultiRun {
  PowerState* st;
  int16_t* ring;
  int64_t slot_elems;
  int slots;
  int64_t N, ld;
  const int16_t* A;
  const int64_t* start;
  const uint32_t* rec;
  int64_t nb, slabs;
  const SplitRing* split;  // non-null: this run's product is the row-split step
  int32_t normalised;      // its product writes the normalised power (no normaliser pass)
};

struct MultiParams {
  int count;
  int nsmall;                       // runs that share the flattened product launch
  int small[kMaxRuns];              // their indexes in r[]
  int64_t cta_start[kMaxRuns + 1];  // prefix sums of nb * slabs over the small runs
  MultiRun r[kMaxRuns];
};

// Runs at least this large get a product launch of their own (a 2-D grid with direct
// parameters): their CTAs are short enough that looking the run up would cost a
// noticeable share of each CTA's time.
constexpr int64_t kOwnLaunchN = 4096;

__global__ void multi_init_kernel(const __grid_constant__ MultiParams mp, int kmax) {
  const MultiRun& q = mp.r[blockIdx.y];
  init_state_body(q.st, kmax, q.slots);
}

__global__ void multi_reduce_kernel(const __grid_constant__ MultiParams mp) {
  const MultiRun& q = mp.r[blockIdx.y];
  reduce_min_diag_body(q.A, q.N, q.ld, q.st);
}

template <bool COPY>
__global__ void multi_normalise_kernel(const __grid_constant__ MultiParams mp) {
  const MultiRun& q = mp.r[blockIdx.y];
  if (!COPY && q.normalised) return;  // the row-split product wrote the normalised power itself
  normalise_hash_body<COPY>(q.A, q.st, q.ring, q.slot_elems, q.slots, q.N, q.ld);
}

__global__ void multi_finalize_kernel(const __grid_constant__ MultiParams mp) { finalize_body(mp.r[blockIdx.y].st); }

__global__ void multi_compare_kernel(const __grid_constant__ MultiParams mp) {
  const MultiRun& q = mp.r[blockIdx.y];
  compare_resolve_body(q.st, q.ring, q.slot_elems, q.slots, q.N, q.ld);
}

// Small runs: CTA -> (run, slab, row block); row blocks vary fastest so a wave sweeps one slab.
template <int R>
__global__ void __launch_bounds__(128) multi_sparse_product_kernel(const __grid_constant__ MultiParams mp) {
  const int64_t c = blockIdx.x;
  int lo = 0, hi = mp.nsmall - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mp.cta_start[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  const MultiRun& q = mp.r[mp.small[lo]];
  if (*(volatile const int32_t*)&q.st->done) return;
  const int64_t local = c - mp.cta_start[lo];
  const int64_t slab = local / q.nb, b = local % q.nb;
  const int k = *(volatile const int32_t*)&q.st->k;
  SparseArgs a{};
  a.M = q.N;
  a.start = q.start;
  a.rec = q.rec;
  a.ldb = q.ld;
  a.ldc = q.ld;
  a.Ncols = q.N;
  a.min_out = &q.st->mu;
  a.diag_out = &q.st->dmin;
  const int16_t* B = q.ring + (int64_t)(k % q.slots) * q.slot_elems;
  int16_t* C = q.ring + (int64_t)((k + 1) % q.slots) * q.slot_elems;
  sparse_tile_body<R>(a, B, C, b, slab);
}

// Large runs: one 2-D launch each, run parameters passed directly.
template <int R>
__global__ void __launch_bounds__(128) own_sparse_product_kernel(SparseArgs a) {
  if (*(volatile const int32_t*)&a.st->done) return;
  const int k = *(volatile const int32_t*)&a.st->k;
  const int16_t* B = a.ring + (int64_t)(k % a.slots) * a.slot_elems;
  int16_t* C = a.ring + (int64_t)((k + 1) % a.slots) * a.slot_elems;
  sparse_tile_body<R>(a, B, C, blockIdx.x, blockIdx.y);
}

template <int R>
cudaError_t launch_products(const MultiParams& mp, cudaStream_t s) {
  for (int i = 0; i < mp.count; ++i) {
    const MultiRun& q = mp.r[i];
    if (q.split != nullptr) {
      const cudaError_t e = split_ring_product(*q.split, q.st, q.ring, q.slot_elems, q.slots, q.ld, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if (q.N < kOwnLaunchN) continue;
    SparseArgs a{};
    a.M = q.N;
    a.start = q.start;
    a.rec = q.rec;
    a.ldb = q.ld;
    a.ldc = q.ld;
    a.Ncols = q.N;
    a.min_out = &q.st->mu;
    a.diag_out = &q.st->dmin;
    a.st = q.st;
    a.ring = q.ring;
    a.slot_elems = q.slot_elems;
    a.slots = q.slots;
    if (q.nb > 0x7FFFFFFF || q.slabs > 65535) return cudaErrorInvalidConfiguration;
    own_sparse_product_kernel<R><<<dim3((unsigned)q.nb, (unsigned)q.slabs), kMultiThreads, 0, s>>>(a);
  }
  const int64_t total = mp.cta_start[mp.nsmall];
  if (total > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if (total > 0) multi_sparse_product_kernel<R><<<(unsigned)total, kMultiThreads, 0, s>>>(mp);
  return cudaGetLastError();
}

cudaError_t launch_multi_product(int R, const MultiParams& mp, cudaStream_t s) {
  switch (R) {
    case 1: return launch_products<1>(mp, s);
    case 2: return launch_products<2>(mp, s);
    case 4: return launch_products<4>(mp, s);
    case 8: return launch_products<8>(mp, s);
    default: return cudaErrorInvalidValue;
  }
}

// The step as launches per phase (products, normaliser, finalize, compare) for the runs of mp.
cudaError_t enqueue_phase_step(int R, const MultiParams& mp, int grid, cudaStream_t s) {
  cudaError_t e = launch_multi_product(R, mp, s);
  if (e != cudaSuccess) return e;
  const dim3 g((unsigned)grid, (unsigned)mp.count);
  bool all_normalised = true;  // row-split products that wrote the normalised power need no normaliser pass
  for (int i = 0; i < mp.count; ++i) all_normalised = all_normalised && mp.r[i].normalised;
  if (!all_normalised) multi_normalise_kernel<false><<<g, 256, 0, s>>>(mp);
  multi_finalize_kernel<<<dim3(1, (unsigned)mp.count), 32, 0, s>>>(mp);
  multi_compare_kernel<<<g, 256, 0, s>>>(mp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- the sparse runs' step as one launch
//
// One launch of multi_step_kernel advances every sparse-step run of a group by one power.  Its work is a
// list of items in four dependency levels per run:
//   level 0  the product's (row block, slab) tiles, R = A (x) P_k with min and diagonal minimum;
//   level 1  the normaliser's parts (P_(k+1) = R - mu, its hash and range flag);
//   level 2  finalize: one item (offsets, gamma, hash table, candidates);
//   level 3  the exact compare's parts; the last one advances k.
// The list holds every run's level-0 items (largest run first), then level 1 (smallest first), then
// levels 2 and 3.  CTAs take items in list order from a counter in the first run's state; an item waits
// until its run's previous level has finished, a wait bounded by time (after about a second it marks its
// run timed out and skips its work).  Every item an item waits for sits earlier in the list and was taken
// by a running CTA that waits only for items earlier still, so the launch always progresses.  The last CTA
// to leave clears the counters for the next launch.

enum : int32_t { kItemSparse = 0, kItemNormalise = 1, kItemFinalize = 2, kItemCompare = 3 };
constexpr int kStepThreads = 256;
constexpr int kStepMaxSeg = 4 * kMaxRuns;
constexpr uint64_t kStepWaitNs = 1000000000ull;  // the default bound of a wait: one second

struct StepSeg {
  int32_t run, kind;  // kind = the item's level
  int64_t begin, count;
};

struct StepRun {
  PowerState* st;
  int16_t* ring;
  int64_t slot_elems;
  int32_t slots;
  int64_t N, ld;
  const int64_t* start;
  const uint32_t* rec;
  int64_t nb;         // row blocks of the product's tiles
  int64_t parts;      // parts of the normaliser and of the compare
  uint32_t need[4];   // items of each level
};

struct StepList {
  int32_t count, nseg, R;
  int64_t total;
  uint64_t wait_ns;  // bound of a wait between levels
  StepSeg seg[kStepMaxSeg];
  StepRun r[kMaxRuns];
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until level `lvl` of the run has `need` finished items; false when `wait_ns` ran out.
__device__ __forceinline__ bool step_wait(PowerState* st, int lvl, uint32_t need, uint64_t wait_ns) {
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint64_t t0 = global_ns();
    while (*(volatile const uint32_t*)&st->lvl_done[lvl] < need) {
      if (global_ns() - t0 > wait_ns) {
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  const int ok = ok_sh;
  __syncthreads();
  return ok != 0;
}

template <int R>
__device__ __forceinline__ void step_sparse_item(const StepRun& q, int64_t local, uint32_t* srec) {
  if (*(volatile const int32_t*)&q.st->done) return;
  const int k = *(volatile const int32_t*)&q.st->k;
  SparseArgs a{};
  a.M = q.N;
  a.start = q.start;
  a.rec = q.rec;
  a.ldb = q.ld;
  a.ldc = q.ld;
  a.Ncols = q.N;
  a.min_out = &q.st->mu;
  a.diag_out = &q.st->dmin;
  const int16_t* B = q.ring + (int64_t)(k % q.slots) * q.slot_elems;
  int16_t* C = q.ring + (int64_t)((k + 1) % q.slots) * q.slot_elems;
  sparse_tile_body<R>(a, B, C, local % q.nb, local / q.nb, srec);
}

template <int R>
__global__ void __launch_bounds__(kStepThreads) multi_step_kernel(const __grid_constant__ StepList L) {
  __shared__ __align__(16) uint32_t srec[kChunk * record_words(R)];
  __shared__ int64_t item_sh;
  PowerState* st0 = L.r[0].st;
  for (;;) {
    if (threadIdx.x == 0) item_sh = (int64_t)atomicAdd(&st0->queue, 1u);
    __syncthreads();
    const int64_t it = item_sh;
    __syncthreads();
    if (it >= L.total) break;
    int si = 0;
    while (si + 1 < L.nseg && L.seg[si + 1].begin <= it) ++si;
    const StepSeg& sg = L.seg[si];
    const StepRun& q = L.r[sg.run];
    const int64_t local = it - sg.begin;
    const int lvl = sg.kind;
    // a run that has stopped does no work, so its items need not wait
    const bool stopped = *(volatile const int32_t*)&q.st->done != 0;
    if (lvl > 0 && !stopped && !step_wait(q.st, lvl - 1, q.need[lvl - 1], L.wait_ns)) {
      if (threadIdx.x == 0) {
        atomicOr(&q.st->err, kErrTimeout);
        atomicExch(&q.st->done, 3);
      }
    } else {
      switch (lvl) {
        case kItemSparse: step_sparse_item<R>(q, local, srec); break;
        case kItemNormalise:
          normalise_hash_body<false>(nullptr, q.st, q.ring, q.slot_elems, q.slots, q.N, q.ld, local, q.parts);
          break;
        case kItemFinalize:
          if (threadIdx.x < 32) finalize_body(q.st);
          break;
        default:
          compare_resolve_body(q.st, q.ring, q.slot_elems, q.slots, q.N, q.ld, local, q.parts);
          break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&q.st->lvl_done[lvl], 1u);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st0->exited, 1u) == gridDim.x - 1) {
      __threadfence();
      for (int r = 0; r < L.count; ++r)
        for (int l = 0; l < 4; ++l) L.r[r].st->lvl_done[l] = 0;
      st0->queue = 0;
      st0->exited = 0;
      __threadfence();
    }
  }
}

// The step of the sparse-step runs of mp as one launch of multi_step_kernel with `ctas` CTAs (0: as many as
// fit on the GPU); *used is false (nothing launched) when R is not 1 or 2 or mp holds a row-split run.
// wait_ns bounds each wait between levels; stall >= 0 makes that run's level 0 count one item more than
// it has, so its level-1 items wait until the bound runs out (the timeout path, exercised by a test).
cudaError_t launch_sparse_step(int R, const MultiParams& mp, int ctas, uint64_t wait_ns, int stall, cudaStream_t s,
                               bool* used) {
  *used = false;
  if (mp.count < 1 || !(R == 1 || R == 2)) return cudaSuccess;
  for (int i = 0; i < mp.count; ++i)
    if (mp.r[i].split != nullptr) return cudaSuccess;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  StepList L{};
  L.count = mp.count;
  L.R = R;
  for (int i = 0; i < mp.count; ++i) {
    const MultiRun& d = mp.r[i];
    StepRun& q = L.r[i];
    q.st = d.st;
    q.ring = d.ring;
    q.slot_elems = d.slot_elems;
    q.slots = d.slots;
    q.N = d.N;
    q.ld = d.ld;
    q.start = d.start;
    q.rec = d.rec;
    q.nb = (d.N + R - 1) / R;
    q.parts = d.N < 4 * (int64_t)sms ? d.N : 4 * (int64_t)sms;
    const int64_t slabs = (d.N + kStepThreads * 16 - 1) / (kStepThreads * 16);
    q.need[0] = (uint32_t)(q.nb * slabs);
    q.need[1] = (uint32_t)q.parts;
    q.need[2] = 1;
    q.need[3] = (uint32_t)q.parts;
  }
  L.wait_ns = wait_ns;
  int order[kMaxRuns];
  for (int i = 0; i < mp.count; ++i) order[i] = i;
  for (int i = 1; i < mp.count; ++i)
    for (int j = i; j > 0 && mp.r[order[j]].N > mp.r[order[j - 1]].N; --j) {
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  int64_t at = 0;
  auto add = [&](int run, int32_t kind, int64_t n) {
    L.seg[L.nseg] = StepSeg{run, kind, at, n};
    ++L.nseg;
    at += n;
  };
  for (int o = 0; o < mp.count; ++o) add(order[o], kItemSparse, L.r[order[o]].need[0]);
  for (int o = mp.count - 1; o >= 0; --o) add(order[o], kItemNormalise, L.r[order[o]].need[1]);
  for (int i = 0; i < mp.count; ++i) add(i, kItemFinalize, 1);
  for (int i = 0; i < mp.count; ++i) add(i, kItemCompare, L.r[i].need[3]);
  L.total = at;
  if (stall >= 0 && stall < mp.count) L.r[stall].need[0] += 1;
  void (*k)(StepList) = (R == 1) ? multi_step_kernel<1> : multi_step_kernel<2>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kStepThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = (ctas > 0 && ctas < per_sm * sms) ? ctas : per_sm * sms;
  k<<<grid, kStepThreads, 0, s>>>(L);
  e = cudaGetLastError();
  if (e == cudaSuccess) *used = true;
  return e;
}

// The step as one launch per group where the group suits it, or when RD_MULTI_STEP=launches is set (to
// compare the two forms), as launches per phase.
bool one_launch_step_wanted() {
  const char* v = getenv("RD_MULTI_STEP");
  return !(v && strcmp(v, "launches") == 0);
}

cudaError_t enqueue_group_step(int R, const MultiParams& g, int grid, int ctas, cudaStream_t s,
                               uint64_t wait_ns = kStepWaitNs, int stall = -1) {
  if (one_launch_step_wanted()) {
    bool used = false;
    const cudaError_t e = launch_sparse_step(R, g, ctas, wait_ns, stall, s, &used);
    if (e != cudaSuccess || used) return e;
  }
  return enqueue_phase_step(R, g, grid, s);
}

// A subset of the runs of mp as its own MultiParams.
MultiParams subset(const MultiParams& mp, const int* idx, int n, int R) {
  MultiParams g{};
  g.count = n;
  for (int i = 0; i < n; ++i) {
    g.r[i] = mp.r[idx[i]];
    const MultiRun& q = g.r[i];
    (void)R;
    if (q.N < kOwnLaunchN && q.split == nullptr) {
      g.small[g.nsmall] = i;
      g.cta_start[g.nsmall + 1] = g.cta_start[g.nsmall] + q.nb * q.slabs;
      ++g.nsmall;
    }
  }
  return g;
}

// The runs as groups: all sparse-step runs together (first, when there are any), each row-split run alone.
int make_groups(const MultiParams& mp, int R, MultiParams* groups) {
  int sparse_idx[kMaxRuns], ns = 0, ng = 0;
  for (int i = 0; i < mp.count; ++i)
    if (mp.r[i].split == nullptr) sparse_idx[ns++] = i;
  if (ns > 0) groups[ng++] = subset(mp, sparse_idx, ns, R);
  for (int i = 0; i < mp.count; ++i)
    if (mp.r[i].split != nullptr) groups[ng++] = subset(mp, &i, 1, R);
  return ng;
}

// One step of every run on one stream: the row-split runs' launches, then the sparse runs' one launch.
cudaError_t enqueue_multi_step(int R, const MultiParams& mp, int grid, cudaStream_t s) {
  MultiParams groups[kMaxRuns];
  const int ng = make_groups(mp, R, groups);
  cudaError_t e = cudaSuccess;
  for (int gi = ng - 1; gi >= 0 && e == cudaSuccess; --gi) e = enqueue_group_step(R, groups[gi], grid, 0, s);
  return e;
}

cudaError_t enqueue_multi_first(const MultiParams& mp, int kmax, int grid, cudaStream_t s) {
  const dim3 g((unsigned)grid, (unsigned)mp.count);
  multi_init_kernel<<<dim3(1, (unsigned)mp.count), 256, 0, s>>>(mp, kmax);
  multi_reduce_kernel<<<g, 256, 0, s>>>(mp);
  multi_normalise_kernel<true><<<g, 256, 0, s>>>(mp);
  multi_finalize_kernel<<<dim3(1, (unsigned)mp.count), 32, 0, s>>>(mp);
  multi_compare_kernel<<<g, 256, 0, s>>>(mp);
  return cudaGetLastError();
}

rd_status fail_cuda(cudaError_t e) {
  set_cuda_error(e);
  return RD_ERR_CUDA;
}

}  // namespace

// Internal entry points for the query server: the first power of some runs, and
// one step of some runs, described by RunDesc (the MultiRun layout).
static_assert(sizeof(RunDesc) == sizeof(MultiRun), "RunDesc mirrors MultiRun");

static void fill_params(const RunDesc* runs, int count, int R, MultiParams* mp) {
  *mp = MultiParams{};
  mp->count = count;
  for (int i = 0; i < count; ++i) {
    MultiRun& q = mp->r[i];
    const RunDesc& d = runs[i];
    q.st = d.st;
    q.ring = d.ring;
    q.slot_elems = d.slot_elems;
    q.slots = d.slots;
    q.N = d.N;
    q.ld = d.ld;
    q.A = d.A;
    q.start = d.start;
    q.rec = d.rec;
    q.split = d.split;
    q.normalised = (d.split != nullptr && split_normalises(d.split->info)) ? 1 : 0;
    q.nb = (d.N + R - 1) / R;
    q.slabs = (d.N + kMultiThreads * 16 - 1) / (kMultiThreads * 16);
    if (d.N < kOwnLaunchN && d.split == nullptr) {
      mp->small[mp->nsmall] = i;
      mp->cta_start[mp->nsmall + 1] = mp->cta_start[mp->nsmall] + q.nb * q.slabs;
      ++mp->nsmall;
    }
  }
}

static int streaming_grid() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;
}

cudaError_t runs_first(const RunDesc* runs, int count, int R, int kmax, cudaStream_t s) {
  if (count < 1 || count > kMaxRuns) return cudaErrorInvalidValue;
  MultiParams mp;
  fill_params(runs, count, R, &mp);
  return enqueue_multi_first(mp, kmax, streaming_grid(), s);
}

cudaError_t runs_step(const RunDesc* runs, int count, int R, cudaStream_t s) {
  if (count < 1 || count > kMaxRuns) return cudaErrorInvalidValue;
  MultiParams mp;
  fill_params(runs, count, R, &mp);
  return enqueue_multi_step(R, mp, streaming_grid(), s);
}

}  // namespace rd

using namespace rd;

extern "C" rd_status rd_power_until_periodic_multi_bounded(rd_power_run* runs, int count, int R, int kmax,
                                                           int graph_steps, uint32_t wait_ms, int32_t stall_run,
                                                           cudaStream_t s) {
  if (!runs || count < 1 || count > kMaxRuns || kmax < 1 || kmax > (1 << 20) || graph_steps < 0) return RD_ERR_ARG;
  if (wait_ms < 1 || wait_ms > 60000 || stall_run < -1 || stall_run >= count) return RD_ERR_ARG;
  const uint64_t wait_ns = (uint64_t)wait_ms * 1000000ull;
  if (!(R == 1 || R == 2 || R == 4 || R == 8)) return RD_ERR_ARG;
  MultiParams mp{};
  mp.count = count;
  mp.cta_start[0] = 0;
  SplitRing split_rings[kMaxRuns];
  int64_t maxN = 0;
  for (int i = 0; i < count; ++i) {
    rd_power_run& u = runs[i];
    u.k = 0;
    u.p = 0;
    u.q = 0;
    u.status = RD_ERR_ARG;
    const bool split = u.split_info != nullptr;
    if (!u.A || !u.work || !u.gamma_host || (!split && (!u.block_start || !u.records))) return RD_ERR_ARG;
    if (u.N < 1 || u.lda < u.N || u.lda % 8 != 0 || !aligned16(u.A) || (!split && !aligned16(u.records)) ||
        (reinterpret_cast<uintptr_t>(u.work) & 255u) != 0)
      return RD_ERR_ARG;
    if (split) {
      split_rings[i] = SplitRing{*u.split_info, u.split_plan, u.split_X, u.split_ldx};
      if (!split_ring_ok(split_rings[i], u.N)) return RD_ERR_ARG;
    }
    const size_t sb = state_bytes(kmax), pb = slot_bytes(u.N, u.lda);
    if (u.work_bytes < sb + 2 * pb) return RD_ERR_NOMEM;
    const size_t slots64 = (u.work_bytes - sb) / pb;
    MultiRun& q = mp.r[i];
    q.st = reinterpret_cast<PowerState*>(u.work);
    q.ring = reinterpret_cast<int16_t*>(static_cast<char*>(u.work) + sb);
    q.slot_elems = (int64_t)(pb / 2);
    q.slots = (int)(slots64 > (size_t)kmax + 1 ? (size_t)kmax + 1 : slots64);
    q.N = u.N;
    q.ld = u.lda;
    q.A = u.A;
    q.start = u.block_start;
    q.rec = u.records;
    q.split = split ? &split_rings[i] : nullptr;
    q.normalised = (split && split_normalises(split_rings[i].info)) ? 1 : 0;
    q.nb = (u.N + R - 1) / R;
    q.slabs = (u.N + kMultiThreads * 16 - 1) / (kMultiThreads * 16);
    if (u.N < kOwnLaunchN && !split) {
      mp.small[mp.nsmall] = i;
      mp.cta_start[mp.nsmall + 1] = mp.cta_start[mp.nsmall] + q.nb * q.slabs;
      ++mp.nsmall;
    }
    if (u.N > maxN) maxN = u.N;
  }
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 4;  // blocks per run for the streaming kernels, as in the single-run path
  MultiParams groups[kMaxRuns];
  const int ng = make_groups(mp, R, groups);
  // the stalled run's place in the sparse group (the group lists its runs in the order of runs[])
  int stall_in_group = -1;
  if (stall_run >= 0 && mp.r[stall_run].split == nullptr) {
    stall_in_group = 0;
    for (int i = 0; i < stall_run; ++i) stall_in_group += mp.r[i].split == nullptr ? 1 : 0;
  }
  // the sparse runs' one-launch step shares the GPU with row-split groups: two CTAs per SM then, so their
  // waits between levels hold few of the slots the row-split passes use (m = 1..9 on GB300: 8, 19, 38, 76,
  // 152, 304 and 608 CTAs took 132, 69, 45.8, 43.9, 43.4, 42.7 and 43.3 ms)
  const int sparse_ctas = ng > 1 ? 2 * sms : 0;

  // Graph capture needs a stream other than the legacy default one: a private stream w ordered after `s`
  // by events (and `s` after it at the end), and one stream per group forked from w and joined back to it
  // after each block of steps.
  cudaStream_t w = nullptr;
  cudaStream_t br[kMaxRuns] = {};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxRuns] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking);
  for (int g = 0; g < ng && e == cudaSuccess; ++g) {
    e = cudaStreamCreateWithFlags(&br[g], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join[g], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev_in, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w, ev_in, 0);
  if (e == cudaSuccess) e = enqueue_multi_first(mp, kmax, grid, w);
  // `steps` steps of every group, each group's chain on its own stream between a fork from w and a join to w
  auto enqueue_block = [&](int steps) {
    cudaError_t x = cudaEventRecord(ev_fork, w);
    for (int g = 0; g < ng && x == cudaSuccess; ++g) {
      x = cudaStreamWaitEvent(br[g], ev_fork, 0);
      for (int i = 0; i < steps && x == cudaSuccess; ++i)
        x = enqueue_group_step(R, groups[g], grid, groups[g].r[0].split ? 0 : sparse_ctas, br[g], wait_ns,
                               groups[g].r[0].split ? -1 : stall_in_group);
      if (x == cudaSuccess) x = cudaEventRecord(ev_join[g], br[g]);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(w, ev_join[g], 0);
    }
    return x;
  };
  if (e == cudaSuccess && graph_steps > 0) {
    e = cudaStreamBeginCapture(w, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = enqueue_block(graph_steps);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(w, &g);
      if (e == cudaSuccess) e = e2;
      graph = g;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  }
  // Host loop: replay (or enqueue) blocks of steps until every run has stopped.
  const int per_check = graph_steps > 0 ? graph_steps : ((maxN >= 2048) ? 1 : 8);
  PowerState h[kMaxRuns];
  int enqueued = 1;
  while (e == cudaSuccess) {
    for (int i = 0; i < count && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(&h[i], mp.r[i].st, sizeof(PowerState), cudaMemcpyDeviceToHost, w);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w);
    if (e != cudaSuccess) break;
    bool all_done = true;
    for (int i = 0; i < count; ++i) all_done = all_done && (h[i].done != 0);
    if (all_done || enqueued >= kmax) break;
    e = exec ? cudaGraphLaunch(exec, w) : enqueue_block(per_check);
    enqueued += per_check;
  }
  rd_status rc = RD_OK;
  if (e != cudaSuccess) rc = fail_cuda(e);
  for (int i = 0; i < count && rc == RD_OK; ++i) {
    rd_power_run& u = runs[i];
    e = cudaMemcpyAsync(u.gamma_host, static_cast<char*>(u.work) + kStateHeader + 8 * (size_t)(kmax + 1),
                        8 * (size_t)(kmax + 1), cudaMemcpyDeviceToHost, w);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w);
    if (e != cudaSuccess) {
      rc = fail_cuda(e);
      break;
    }
    const int last = (h[i].done == 1) ? h[i].found_j : h[i].k;
    for (int k = 0; k <= kmax; ++k)
      if (k < 1 || k > last) u.gamma_host[k] = RD_GAMMA_UNSET;
    if (h[i].done == 1) {
      u.k = h[i].found_i;
      u.p = h[i].found_j - h[i].found_i;
      u.q = h[i].found_q;
      u.status = RD_OK;
    } else if (h[i].done == 3) {
      u.status = status_from_err(h[i].err);
    } else {
      u.status = RD_NOT_FOUND;
    }
  }
  if (ev_out && w) {
    cudaEventRecord(ev_out, w);
    cudaStreamWaitEvent(s, ev_out, 0);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (ev_fork) cudaEventDestroy(ev_fork);
  for (int g = 0; g < ng; ++g) {
    if (ev_join[g]) cudaEventDestroy(ev_join[g]);
    if (br[g]) cudaStreamDestroy(br[g]);
  }
  if (w) cudaStreamDestroy(w);
  return rc;
}

extern "C" rd_status rd_power_until_periodic_multi(rd_power_run* runs, int count, int R, int kmax, int graph_steps,
                                                   cudaStream_t s) {
  return rd_power_until_periodic_multi_bounded(runs, count, R, kmax, graph_steps, 1000, -1, s);
}
