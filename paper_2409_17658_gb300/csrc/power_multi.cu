// power_multi.cu -- several period searches (Algorithm 2) advanced together.
//
// Each run is its own transfer matrix with its own work buffer (state + ring),
// exactly as in rd_power_until_periodic_sparse.  A step of ALL runs is four
// launches: the dense x sparse products (one launch over the concatenated CTA lists
// of the small runs, one 2-D launch per large run), then the normaliser/hash,
// finalize and compare of every run side by side (blockIdx.y = run).  Runs that have stopped exit at kernel entry, so the same
// launch sequence stays valid until the last run stops; it is captured once
// into a CUDA graph of several steps and replayed, so small matrices (m <= 5,
// whose steps are launch-bound) ride along with the large ones at no cost.
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

cudaError_t enqueue_multi_step(int R, const MultiParams& mp, int grid, cudaStream_t s) {
  cudaError_t e = launch_multi_product(R, mp, s);
  if (e != cudaSuccess) return e;
  const dim3 g((unsigned)grid, (unsigned)mp.count);
  multi_normalise_kernel<false><<<g, 256, 0, s>>>(mp);
  multi_finalize_kernel<<<dim3(1, (unsigned)mp.count), 32, 0, s>>>(mp);
  multi_compare_kernel<<<g, 256, 0, s>>>(mp);
  return cudaGetLastError();
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

extern "C" rd_status rd_power_until_periodic_multi(rd_power_run* runs, int count, int R, int kmax, int graph_steps,
                                                   cudaStream_t s) {
  if (!runs || count < 1 || count > kMaxRuns || kmax < 1 || kmax > (1 << 20) || graph_steps < 0) return RD_ERR_ARG;
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

  // Graph capture needs a stream other than the legacy default one: use a private stream
  // ordered after `s` by events, and order `s` after it at the end.
  cudaStream_t w = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev_in, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(w, ev_in, 0);
  if (e == cudaSuccess) e = enqueue_multi_first(mp, kmax, grid, w);
  if (e == cudaSuccess && graph_steps > 0) {
    e = cudaStreamBeginCapture(w, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; i < graph_steps && e == cudaSuccess; ++i) e = enqueue_multi_step(R, mp, grid, w);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(w, &g);
    if (e == cudaSuccess) e = e2;
    graph = g;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  }
  // Host loop: replay (or launch) steps until every run has stopped.
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
    if (exec) {
      e = cudaGraphLaunch(exec, w);
    } else {
      for (int i = 0; i < per_check && e == cudaSuccess; ++i) e = enqueue_multi_step(R, mp, grid, w);
    }
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
  if (w) cudaStreamDestroy(w);
  return rc;
}
