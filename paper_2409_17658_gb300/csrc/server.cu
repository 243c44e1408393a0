// server.cu -- a query server for gamma_R(P_m box C_n) with continuous batching.
//
// Queries (m, n) arrive from any host thread.  A worker thread owns one CUDA
// stream and a table of period-search jobs, one per m still being searched:
//   * a query whose m has a known relation (k, p, q) is answered on the host at
//     once (Prop. 7: gamma(n) = gamma(k + (n - k) mod p) + q floor((n - k)/p));
//   * a query whose gamma(n) has already been produced by a running job (power
//     n computed) is answered at once as well;
//   * otherwise it waits on the job for its m, which is created on first need.
// Jobs are admitted while their device footprint (A(G), the work buffer, and the
// block-sparse form of A(G), or for m >= 8 the row-split plan and its
// intermediate) fits the HBM budget; the others wait and are admitted as
// running jobs finish and free their memory.  Every step advances ALL admitted
// jobs together with the multi-run launches (one product launch for the small
// ones plus one per large one, then the normaliser/finalize/compare side by
// side), so jobs that arrive while others are running share the GPU with them;
// a round gives a cheap job several steps for each step of the costliest one.
// After each step the worker reads back each job's state and gamma table and
// answers what it can; a job whose relation is found is retired (its relation
// cached for the life of the server) and its memory freed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxStepsPerRound = 16;

struct Query {
  int m = 0;
  int64_t n = 0;
  Clock::time_point t_submit;
  Clock::time_point t_done;
  bool done = false;
  int64_t answer = 0;
  rd_status status = RD_OK;
};

struct Final {
  bool valid = false;
  bool found = false;
  rd_status status = RD_OK;
  int k = 0, p = 0, j = 0;
  int64_t q = 0;
  std::vector<int64_t> gamma;
};

struct Job {
  int m = 0;
  int64_t N = 0, ld = 0;
  int16_t* A = nullptr;
  int64_t* start = nullptr;
  uint32_t* rec = nullptr;
  void* work = nullptr;
  void* plan = nullptr;       // row-split plan (large jobs)
  int16_t* X = nullptr;       // its intermediate
  rd::SplitRing split{};
  size_t work_bytes = 0, footprint = 0, need = 0;
  rd::RunDesc run{};
  double cost = 1.0;  // bytes one product moves: B rows (sparse: entries x N x 2; row split: 4 (N + X rows) N)
  int k_known = 0;
  std::vector<int64_t> gamma;
  std::vector<uint64_t> waiting;
};

}  // namespace

struct rd_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> incoming;
  std::unordered_map<uint64_t, Query> queries;
  uint64_t next_ticket = 1;
  Final final_[RD_MAX_M + 1];
  std::vector<Job*> active, pending;  // worker-owned
  size_t budget = 0;
  std::atomic<size_t> used{0}, peak{0};  // device bytes held by admitted jobs
  int kmax = 256, R = 2, slots = 8, device = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  bool stop = false;
  rd_server_stats_t stats{};
};

namespace {

int64_t closed_form(const Final& f, int64_t n) {
  if (n <= f.j) return f.gamma[(size_t)n];
  const int64_t t = (n - f.k) / f.p;
  return f.gamma[(size_t)(f.k + (n - f.k) % f.p)] + f.q * t;
}

// Under sv->mu.
void answer(rd_server* sv, uint64_t ticket, int64_t value, rd_status st) {
  auto it = sv->queries.find(ticket);
  if (it == sv->queries.end()) return;
  it->second.answer = value;
  it->second.status = st;
  it->second.done = true;
  it->second.t_done = Clock::now();
  sv->stats.answered += 1;
}

void free_job(rd_server* sv, Job* j) {
  if (j->A) cudaFree(j->A);
  if (j->start) cudaFree(j->start);
  if (j->rec) cudaFree(j->rec);
  if (j->work) cudaFree(j->work);
  if (j->plan) cudaFree(j->plan);
  if (j->X) cudaFree(j->X);
  j->A = nullptr;
  j->start = nullptr;
  j->rec = nullptr;
  j->work = nullptr;
  j->plan = nullptr;
  j->X = nullptr;
  sv->used -= j->footprint;
  j->footprint = 0;
}

// Large jobs (C_m >= kSplitN) step with the row-split product; smaller ones with the sparse one,
// all of whose products share one launch.
constexpr int64_t kSplitN = 4096;

// The row-split operands of a large job: its plan and intermediate, after A and the work buffer.
rd_status admit_split(rd_server* sv, Job* j, size_t base) {
  const int sj = rd_split_default_j(j->m);
  size_t pbytes = 0;
  rd_status rc = rd_split_plan_bytes(j->m, sj, &pbytes);
  if (rc != RD_OK) return RD_ERR_CUDA;
  if (sv->used + pbytes > sv->budget) {
    j->need = base + pbytes;
    free_job(sv, j);
    return (j->need > sv->budget) ? RD_ERR_ARG : RD_ERR_NOMEM;
  }
  if (cudaMalloc(&j->plan, pbytes) != cudaSuccess) return RD_ERR_CUDA;
  j->footprint += pbytes;
  sv->used += pbytes;
  rc = rd_split_plan(j->m, sj, j->plan, pbytes, &j->split.info, sv->stream);
  if (rc != RD_OK) return RD_ERR_CUDA;
  const size_t xbytes = (size_t)j->split.info.x_rows * (size_t)j->ld * 2;
  if (sv->used + xbytes > sv->budget) {
    j->need = j->footprint + xbytes;  // exact now; retry when that much is free
    free_job(sv, j);
    return (j->need > sv->budget) ? RD_ERR_ARG : RD_ERR_NOMEM;
  }
  if (cudaMalloc(&j->X, xbytes) != cudaSuccess) return RD_ERR_CUDA;
  j->footprint += xbytes;
  sv->used += xbytes;
  j->split.plan = j->plan;
  j->split.X = j->X;
  j->split.ldx = j->ld;
  j->cost = 4.0 * (double)(j->N + j->split.info.x_rows) * (double)j->N;
  return RD_OK;
}

// Allocate and build one job's operands; RD_OK, RD_ERR_NOMEM (does not fit now: j->need
// says how much it needs), or another error (the job cannot run at all).
rd_status admit(rd_server* sv, Job* j) {
  rd_state_count(j->m, &j->N);
  rd_padded_dim(j->N, &j->ld);
  const size_t a_bytes = (size_t)j->N * (size_t)j->ld * 2;
  rd_power_work_bytes(j->N, j->ld, sv->kmax, sv->slots, &j->work_bytes);
  const bool use_split = j->N >= kSplitN && rd_split_default_j(j->m) > 0;
  const int64_t nb = (j->N + sv->R - 1) / sv->R;
  const size_t start_bytes = use_split ? 0 : (size_t)(nb + 1) * 8;
  const size_t base = a_bytes + j->work_bytes + start_bytes;
  if (j->need == 0) j->need = base;
  if (j->need > sv->budget) return RD_ERR_ARG;  // never fits: reported to its queries as RD_ERR_NOMEM
  if (sv->used + j->need > sv->budget) return RD_ERR_NOMEM;
  cudaError_t e = cudaMalloc(&j->A, a_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&j->work, j->work_bytes);
  if (e == cudaSuccess && !use_split) e = cudaMalloc(&j->start, start_bytes);
  j->footprint = base;
  sv->used += base;
  rd_status rc = (e == cudaSuccess) ? RD_OK : RD_ERR_CUDA;
  if (rc == RD_OK) rc = rd_build_transfer(j->m, j->A, j->ld, sv->stream);
  if (use_split && rc == RD_OK) {
    rc = admit_split(sv, j, base);
    if (rc == RD_ERR_NOMEM || rc == RD_ERR_ARG) return rc;  // freed already
  }
  int64_t entries = 0;
  if (!use_split && rc == RD_OK) rc = rd_sparse_count(j->A, j->ld, j->N, j->N, sv->R, j->start, &entries, sv->stream);
  const size_t rec_bytes = use_split ? 0 : (size_t)(entries > 0 ? entries : 1) * 4 * rd_sparse_record_words(sv->R);
  if (!use_split && rc == RD_OK && sv->used + rec_bytes > sv->budget) {
    j->need = base + rec_bytes;  // exact now; retry when that much is free
    free_job(sv, j);
    return (j->need > sv->budget) ? RD_ERR_ARG : RD_ERR_NOMEM;
  }
  if (!use_split && rc == RD_OK) {
    e = cudaMalloc(&j->rec, rec_bytes);
    if (e != cudaSuccess) rc = RD_ERR_CUDA;
    else {
      j->footprint += rec_bytes;
      sv->used += rec_bytes;
    }
  }
  if (!use_split && rc == RD_OK) rc = rd_sparse_build(j->A, j->ld, j->N, j->N, sv->R, j->start, j->rec, sv->stream);
  if (!use_split) j->cost = 2.0 * (double)(entries > 0 ? entries : 1) * (double)j->N;
  if (rc == RD_OK) {
    const size_t sb = rd::state_bytes(sv->kmax), pb = rd::slot_bytes(j->N, j->ld);
    j->run.st = reinterpret_cast<rd::PowerState*>(j->work);
    j->run.ring = reinterpret_cast<int16_t*>(static_cast<char*>(j->work) + sb);
    j->run.slot_elems = (int64_t)(pb / 2);
    const size_t s64 = (j->work_bytes - sb) / pb;
    j->run.slots = (int)(s64 > (size_t)sv->kmax + 1 ? (size_t)sv->kmax + 1 : s64);
    j->run.N = j->N;
    j->run.ld = j->ld;
    j->run.A = j->A;
    j->run.start = j->start;
    j->run.rec = j->rec;
    j->run.split = use_split ? &j->split : nullptr;
    e = rd::runs_first(&j->run, 1, sv->R, sv->kmax, sv->stream);
    if (e != cudaSuccess) rc = RD_ERR_CUDA;
  }
  if (rc != RD_OK) {
    free_job(sv, j);
    return RD_ERR_CUDA;
  }
  sv->peak = std::max(sv->peak.load(), sv->used.load());
  j->gamma.assign((size_t)sv->kmax + 1, RD_GAMMA_UNSET);
  return RD_OK;
}

Job* find_job(rd_server* sv, int m) {
  for (Job* j : sv->active)
    if (j->m == m) return j;
  for (Job* j : sv->pending)
    if (j->m == m) return j;
  return nullptr;
}

void retire(rd_server* sv, Job* j, const rd::PowerState& h) {
  Final f;
  f.valid = true;
  f.found = (h.done == 1);
  f.status = (h.done == 1 || h.done == 2) ? RD_OK : rd::status_from_err(h.err);
  f.k = h.found_i;
  f.p = h.found_j - h.found_i;
  f.q = h.found_q;
  f.j = (h.done == 1) ? h.found_j : h.k;
  f.gamma = j->gamma;
  std::lock_guard<std::mutex> lock(sv->mu);
  for (uint64_t t : j->waiting) {
    auto it = sv->queries.find(t);
    if (it == sv->queries.end()) continue;
    const int64_t n = it->second.n;
    if (f.status != RD_OK) answer(sv, t, 0, f.status);
    else if (n <= f.j) answer(sv, t, f.gamma[(size_t)n], RD_OK);
    else if (f.found) answer(sv, t, closed_form(f, n), RD_OK);
    else answer(sv, t, 0, RD_NOT_FOUND);
  }
  j->waiting.clear();
  sv->final_[j->m] = std::move(f);
  sv->stats.jobs_completed += 1;
  sv->cv_done.notify_all();
}

void worker_main(rd_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<rd::PowerState> hdr;
  for (;;) {
    std::vector<uint64_t> batch;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      if (sv->active.empty() && sv->pending.empty())
        sv->cv_work.wait_for(lock, std::chrono::milliseconds(50),
                             [&] { return sv->stop || !sv->incoming.empty(); });
      if (sv->stop) break;
      batch.assign(sv->incoming.begin(), sv->incoming.end());
      sv->incoming.clear();
      // route the new queries
      bool any = false;
      for (uint64_t t : batch) {
        Query& q = sv->queries[t];
        const Final& f = sv->final_[q.m];
        if (f.valid) {
          if (f.status != RD_OK) answer(sv, t, 0, f.status);
          else if (q.n <= f.j) answer(sv, t, f.gamma[(size_t)q.n], RD_OK);
          else if (f.found) answer(sv, t, closed_form(f, q.n), RD_OK);
          else answer(sv, t, 0, RD_NOT_FOUND);
          any = true;
          continue;
        }
        Job* j = find_job(sv, q.m);
        if (j && q.n <= j->k_known) {
          answer(sv, t, j->gamma[(size_t)q.n], RD_OK);
          any = true;
          continue;
        }
        if (!j) {
          j = new Job();
          j->m = q.m;
          sv->pending.push_back(j);
        }
        j->waiting.push_back(t);
      }
      if (any) sv->cv_done.notify_all();
    }
    // admission, FIFO, by device footprint
    for (size_t i = 0; i < sv->pending.size() && (int)sv->active.size() < rd::kMaxRunsPerStep;) {
      Job* j = sv->pending[i];
      const rd_status rc = admit(sv, j);
      if (rc == RD_OK) {
        sv->active.push_back(j);
        sv->pending.erase(sv->pending.begin() + (long)i);
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stats.jobs_admitted += 1;
        continue;
      }
      if (rc == RD_ERR_NOMEM) break;  // wait for memory; keep arrival order
      // cannot run at all: fail its queries
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        for (uint64_t t : j->waiting) answer(sv, t, 0, RD_ERR_NOMEM);
        sv->cv_done.notify_all();
      }
      sv->pending.erase(sv->pending.begin() + (long)i);
      delete j;
    }
    if (sv->active.empty()) continue;
    // One round: every admitted job advances, a cheap job by several steps (up to
    // kMaxStepsPerRound, in proportion to how much cheaper its product is than the
    // costliest one) so that small searches are not held to the pace of a large one.
    double cmax = 0.0;
    for (Job* j : sv->active) cmax = std::max(cmax, j->cost);
    std::vector<int> reps(sv->active.size());
    int rounds = 1;
    for (size_t i = 0; i < sv->active.size(); ++i) {
      const double r = cmax / sv->active[i]->cost;
      reps[i] = r >= kMaxStepsPerRound ? kMaxStepsPerRound : (r < 1.0 ? 1 : (int)r);
      rounds = std::max(rounds, reps[i]);
    }
    cudaError_t e = cudaSuccess;
    for (int sub = 0; sub < rounds && e == cudaSuccess; ++sub) {
      std::vector<rd::RunDesc> runs;
      for (size_t i = 0; i < sv->active.size(); ++i)
        if (reps[i] > sub) runs.push_back(sv->active[i]->run);
      e = rd::runs_step(runs.data(), (int)runs.size(), sv->R, sv->stream);
    }
    hdr.resize(sv->active.size());
    for (size_t i = 0; i < sv->active.size() && e == cudaSuccess; ++i) {
      Job* j = sv->active[i];
      e = cudaMemcpyAsync(&hdr[i], j->run.st, sizeof(rd::PowerState), cudaMemcpyDeviceToHost, sv->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->gamma.data(), static_cast<char*>(j->work) + rd::kStateHeader + 8 * (size_t)(sv->kmax + 1),
                            8 * (size_t)(sv->kmax + 1), cudaMemcpyDeviceToHost, sv->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->stats.steps += 1;
    }
    if (e != cudaSuccess) {
      rd::set_cuda_error(e);
      std::lock_guard<std::mutex> lock(sv->mu);
      for (Job* j : sv->active)
        for (uint64_t t : j->waiting) answer(sv, t, 0, RD_ERR_CUDA);
      sv->cv_done.notify_all();
      for (Job* j : sv->active) {
        free_job(sv, j);
        delete j;
      }
      sv->active.clear();
      continue;
    }
    std::vector<Job*> still;
    for (size_t i = 0; i < sv->active.size(); ++i) {
      Job* j = sv->active[i];
      const rd::PowerState& h = hdr[i];
      j->k_known = (h.done == 1) ? h.found_j : h.k;
      if (h.done) {
        free_job(sv, j);  // its gamma table is on the host already
        retire(sv, j, h);
        delete j;
        continue;
      }
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        std::vector<uint64_t> left;
        for (uint64_t t : j->waiting) {
          auto it = sv->queries.find(t);
          if (it != sv->queries.end() && it->second.n <= j->k_known) answer(sv, t, j->gamma[(size_t)it->second.n], RD_OK);
          else left.push_back(t);
        }
        if (left.size() != j->waiting.size()) sv->cv_done.notify_all();
        j->waiting.swap(left);
      }
      still.push_back(j);
    }
    sv->active.swap(still);
  }
  for (Job* j : sv->active) {
    free_job(sv, j);
    delete j;
  }
  for (Job* j : sv->pending) delete j;
  sv->active.clear();
  sv->pending.clear();
}

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

}  // namespace

extern "C" rd_status rd_server_create(size_t hbm_budget_bytes, int kmax, rd_server** out) {
  if (!out || kmax < 8 || kmax > 4096 || hbm_budget_bytes == 0) return RD_ERR_ARG;
  rd_server* sv = new rd_server();
  sv->budget = hbm_budget_bytes;
  sv->kmax = kmax;
  cudaError_t e = cudaGetDevice(&sv->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    rd::set_cuda_error(e);
    delete sv;
    return RD_ERR_CUDA;
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return RD_OK;
}

extern "C" rd_status rd_server_submit(rd_server* sv, int count, const int32_t* m, const int64_t* n,
                                      uint64_t* tickets) {
  if (!sv || count < 0 || (count > 0 && (!m || !n || !tickets))) return RD_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (m[i] < 1 || m[i] > RD_MAX_M || n[i] < 3) return RD_ERR_ARG;
  const auto now = Clock::now();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    for (int i = 0; i < count; ++i) {
      const uint64_t t = sv->next_ticket++;
      Query q;
      q.m = m[i];
      q.n = n[i];
      q.t_submit = now;
      sv->queries.emplace(t, q);
      sv->incoming.push_back(t);
      tickets[i] = t;
    }
    sv->stats.submitted += (uint64_t)count;
  }
  sv->cv_work.notify_one();
  return RD_OK;
}

extern "C" rd_status rd_server_wait(rd_server* sv, int count, const uint64_t* tickets, double timeout_s,
                                    int64_t* gamma, int32_t* status, double* latency_s) {
  if (!sv || count < 0 || (count > 0 && (!tickets || !gamma || !status))) return RD_ERR_ARG;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                           timeout_s > 0 ? timeout_s : 0.0));
  std::unique_lock<std::mutex> lock(sv->mu);
  for (int i = 0; i < count; ++i) {
    auto it = sv->queries.find(tickets[i]);
    if (it == sv->queries.end()) return RD_ERR_ARG;
    const bool ok = sv->cv_done.wait_until(lock, deadline, [&] { return it->second.done; });
    if (!ok) return RD_ERR_TIMEOUT;
  }
  for (int i = 0; i < count; ++i) {
    auto it = sv->queries.find(tickets[i]);
    gamma[i] = it->second.answer;
    status[i] = (int32_t)it->second.status;
    if (latency_s) latency_s[i] = seconds(it->second.t_done - it->second.t_submit);
    sv->queries.erase(it);
  }
  return RD_OK;
}

extern "C" rd_status rd_server_stats(rd_server* sv, rd_server_stats_t* out) {
  if (!sv || !out) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  *out = sv->stats;
  out->bytes_in_use = sv->used.load();
  out->bytes_peak = sv->peak.load();
  return RD_OK;
}

extern "C" rd_status rd_server_export(rd_server* sv, int m, rd_relation_t* rel, int64_t* gamma, int64_t cap) {
  if (!sv || m < 1 || m > RD_MAX_M || !rel) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  const Final& f = sv->final_[m];
  if (!f.valid) return RD_NOT_FOUND;
  if (f.status != RD_OK) return f.status;
  *rel = rd_relation_t{};
  rel->m = m;
  rel->found = f.found ? 1 : 0;
  rel->k = f.found ? f.k : 0;
  rel->p = f.found ? f.p : 0;
  rel->q = f.found ? f.q : 0;
  rel->j = f.j;
  if (!gamma) return RD_OK;
  if (cap < (int64_t)f.j + 1) return RD_ERR_ARG;
  gamma[0] = RD_GAMMA_UNSET;
  for (int n = 1; n <= f.j; ++n) gamma[n] = f.gamma[(size_t)n];
  return RD_OK;
}

extern "C" rd_status rd_server_import(rd_server* sv, const rd_relation_t* rel, const int64_t* gamma) {
  if (!sv || !rd::relation_ok(rel, gamma)) return RD_ERR_ARG;
  Final f;
  f.valid = true;
  f.found = rel->found == 1;
  f.status = RD_OK;
  f.k = rel->k;
  f.p = rel->p;
  f.q = rel->q;
  f.j = rel->j;
  f.gamma.assign(gamma, gamma + rel->j + 1);
  f.gamma[0] = RD_GAMMA_UNSET;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->final_[rel->m] = std::move(f);
  return RD_OK;
}

extern "C" rd_status rd_server_destroy(rd_server* sv) {
  if (!sv) return RD_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  if (sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
  return RD_OK;
}
