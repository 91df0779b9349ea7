// Serving engine: continuous batching of top-k n-gram jobs on one GPU.
//
// Callers submit jobs (a corpus already on the device, host offsets, the
// job's parameters). A scheduler thread admits pending jobs whenever a slot
// is free and the job's tables fit the device-memory budget (sizes come from
// a dry-run plan) - by default the job with the least estimated work first
// (corpus bytes times passes, plus its counter arrays), with the wait counted
// in so that no job starves, and on a stream whose priority falls with the
// job's work, so that at every kernel boundary the GPU's block scheduler
// starts a small job's pass before a large job's next one; with
// IG_SRV_FIFO in arrival order on default-priority streams. It gives each
// admitted job its own plan and stream, and then advances every active job
// one pass at a time: whenever a
// job's previous step has completed on the GPU it enqueues the job's next
// pass (or its final top-k). Jobs at different passes therefore have work in
// flight on the device at the same time, each job's candidate and count
// tables stay resident between its passes, and a job that arrives while
// others run is admitted as soon as memory and a slot free up. With
// max_active = 1 the same engine runs one job per launch, in order.
//
// A job's result does not depend on what else runs: each job owns every
// table it touches (its plan), and the kernels are deterministic.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ig_internal.cuh"

namespace ig {
bool plan_passes_done(const ig_plan* pl);
uint32_t plan_row_bytes(const ig_plan* pl);
ig_status plan_enqueue_next(ig_plan* pl, cudaEvent_t ev);
ig_status plan_last_status(ig_plan* pl);
bool plan_regrow_and_restart(ig_plan* pl);
ig_status plan_enqueue_topk(ig_plan* pl, uint8_t* keys_host, uint64_t* counts_host, uint32_t cap, uint32_t* rows,
                            cudaEvent_t ev);
void set_last_error(const std::string& msg);
}  // namespace ig

namespace {

using Clock = std::chrono::steady_clock;

// IG_SRV_LARGE_ALONE default: jobs that stream at least this many bytes over
// all their passes (about 15 ms of scans on a GB300) run alone
constexpr double kLargeWork = 2e9;

enum JobState { kPending = 0, kPasses = 1, kTopk = 2, kDone = 3 };

struct Job {
  uint64_t id = 0;
  ig_params p{};
  ig_tuning t{};
  bool has_tuning = false;
  const void* data = nullptr;
  std::vector<uint64_t> offsets;
  uint32_t m = 0;
  uint64_t bytes = 0;  // device bytes charged against the budget
  double work = 0;     // estimated work: bytes streamed over all passes
  uint32_t behind = 0; // jobs already running when it was admitted
  bool large = false;  // IG_SRV_LARGE_ALONE: runs with no other job beside it
  ig_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  uint8_t* keys_pinned = nullptr;
  uint64_t* counts_pinned = nullptr;
  int state = kPending;
  bool inflight = false;
  ig_status status = IG_OK;
  std::string err;
  std::vector<uint8_t> keys;
  std::vector<uint64_t> counts;
  uint32_t rows = 0, row_bytes = 0;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct ig_server {
  ig_server_config cfg{};
  int device = 0;
  // pinned host buffers for results, kept for reuse (pinning is slow and
  // freeing pinned memory can synchronise the device): size -> buffers
  std::multimap<size_t, void*> pinned_free;
  std::mutex pinned_mu;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  bool stop = false;
  uint32_t active = 0, peak_active = 0;
  uint32_t large_active = 0;  // a large job is running alone
  uint64_t mem_used = 0, peak_mem = 0, submitted = 0, completed = 0, failed = 0;
  std::thread worker;
};

namespace {

// A pinned buffer of at least `bytes` (sizes rounded up to powers of two).
void* pinned_take(ig_server* sv, size_t bytes) {
  size_t sz = 4096;
  while (sz < bytes) sz <<= 1;
  {
    std::lock_guard<std::mutex> lock(sv->pinned_mu);
    auto it = sv->pinned_free.find(sz);
    if (it != sv->pinned_free.end()) {
      void* p = it->second;
      sv->pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, sz) != cudaSuccess) return nullptr;
  return p;
}

void pinned_give(ig_server* sv, void* p, size_t bytes) {
  if (!p) return;
  size_t sz = 4096;
  while (sz < bytes) sz <<= 1;
  std::lock_guard<std::mutex> lock(sv->pinned_mu);
  sv->pinned_free.emplace(sz, p);
}

size_t keys_bytes(const Job* jb) { return std::max<size_t>((size_t)jb->p.k * jb->row_bytes, 1); }

void release_job_resources(ig_server* sv, Job* jb) {
  if (jb->plan) intergrams_free(jb->plan);  // synchronises the job's stream
  jb->plan = nullptr;
  if (jb->ev) cudaEventDestroy(jb->ev);
  jb->ev = nullptr;
  if (jb->stream) cudaStreamDestroy(jb->stream);
  jb->stream = nullptr;
  pinned_give(sv, jb->keys_pinned, keys_bytes(jb));
  jb->keys_pinned = nullptr;
  pinned_give(sv, jb->counts_pinned, sizeof(uint64_t) * jb->p.k);
  jb->counts_pinned = nullptr;
}

void finish_job(ig_server* sv, Job* jb, ig_status st, const std::string& err) {
  const Clock::time_point done = Clock::now();  // the job's last GPU step has completed
  if (st == IG_OK && jb->rows) {
    jb->keys.assign(jb->keys_pinned, jb->keys_pinned + (size_t)jb->rows * jb->row_bytes);
    jb->counts.assign(jb->counts_pinned, jb->counts_pinned + jb->rows);
  }
  release_job_resources(sv, jb);
  std::lock_guard<std::mutex> lock(sv->mu);
  jb->status = st;
  jb->err = err;
  jb->state = kDone;
  jb->t_done = done;
  sv->mem_used -= jb->bytes;
  sv->active -= 1;
  if (jb->large) sv->large_active -= 1;
  if (st == IG_OK) sv->completed += 1;
  else sv->failed += 1;
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

// Work classes for stream priorities: below 1 GB, below 8 GB of bytes
// streamed, and the rest.
int stream_priority(const ig_server* sv, const Job* jb) {
  if (sv->cfg.flags & IG_SRV_FIFO) return 0;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
  if (sv->cfg.flags & IG_SRV_OLDEST_FIRST) {
    // admitted behind `active - 1` older jobs: one level below each
    return std::min(least, greatest + (int)jb->behind);
  }
  if (jb->work < 1e9) return greatest;
  if (jb->work < 8e9) return (least + greatest) / 2;
  return least;
}

// Create the job's plan, stream and result buffers (scheduler thread).
ig_status admit_job(ig_server* sv, Job* jb, std::string* err) {
  if (cudaStreamCreateWithPriority(&jb->stream, cudaStreamNonBlocking, stream_priority(sv, jb)) != cudaSuccess ||
      cudaEventCreateWithFlags(&jb->ev, cudaEventDisableTiming) != cudaSuccess) {
    *err = "stream/event creation failed";
    return IG_ECUDA;
  }
  ig_params p = jb->p;
  p.flags = (p.flags & ~(IG_F_HOST_INPUT | IG_F_GRAPH | IG_F_DRY_RUN)) | IG_F_OFFSETS_HOST | IG_F_ASYNC_ALLOC;
  ig_status st = intergrams_plan(&p, jb->data, jb->offsets.data(), jb->m, jb->stream,
                                 jb->has_tuning ? &jb->t : nullptr, &jb->plan);
  if (st != IG_OK) {
    *err = intergrams_last_error();
    return st;
  }
  jb->row_bytes = ig::plan_row_bytes(jb->plan);
  jb->keys_pinned = static_cast<uint8_t*>(pinned_take(sv, keys_bytes(jb)));
  jb->counts_pinned = static_cast<uint64_t*>(pinned_take(sv, sizeof(uint64_t) * jb->p.k));
  if (!jb->keys_pinned || !jb->counts_pinned) {
    *err = "pinned host allocation failed";
    return IG_ENOMEM;
  }
  return IG_OK;
}

void scheduler(ig_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<Job*> running;
  for (;;) {
    std::vector<Job*> admit;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      if (sv->stop && sv->pending.empty() && running.empty()) break;
      // admission while a slot is free and the budget allows: arrival order
      // (IG_SRV_FIFO), else the least work first, each job's work discounted
      // by its wait (it halves for every 100 ms waited, so none starves)
      while (!sv->pending.empty() && sv->active < sv->cfg.max_active && sv->large_active == 0) {
        auto pick = sv->pending.begin();
        if (!(sv->cfg.flags & (IG_SRV_FIFO | IG_SRV_OLDEST_FIRST))) {
          const Clock::time_point now = Clock::now();
          double best = 0;
          for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
            const double waited = std::chrono::duration<double>(now - (*it)->t_submit).count();
            const double key = (*it)->work / (1.0 + 10.0 * waited);
            if (it == sv->pending.begin() || key < best) {
              best = key;
              pick = it;
            }
          }
        }
        Job* jb = *pick;
        if (sv->mem_used + jb->bytes > sv->cfg.mem_budget && sv->active > 0) break;
        // a large job waits for the GPU to drain, then runs alone (the jobs
        // picked after it wait with it, so it cannot starve)
        jb->large = (sv->cfg.flags & IG_SRV_LARGE_ALONE) &&
                    jb->work >= (sv->cfg.large_work ? (double)sv->cfg.large_work : kLargeWork);
        if (jb->large && sv->active > 0) break;
        if (jb->large) sv->large_active += 1;
        sv->pending.erase(pick);
        sv->mem_used += jb->bytes;
        sv->peak_mem = std::max(sv->peak_mem, sv->mem_used);
        jb->behind = sv->active;
        sv->active += 1;
        sv->peak_active = std::max(sv->peak_active, sv->active);
        admit.push_back(jb);
      }
      if (running.empty() && admit.empty()) {
        sv->cv_work.wait_for(lock, std::chrono::milliseconds(2));
        continue;
      }
    }
    for (Job* jb : admit) {
      jb->t_admit = Clock::now();
      std::string err;
      const ig_status st = admit_job(sv, jb, &err);
      if (st != IG_OK) finish_job(sv, jb, st, err);
      else running.push_back(jb);
    }
    bool progressed = !admit.empty();
    // a job handed to finish_job may be deleted by its waiter at once, so it
    // leaves the running list in the same step and is not touched again
    for (auto it = running.begin(); it != running.end();) {
      Job* jb = *it;
      bool finished = false;
      if (jb->inflight) {
        const cudaError_t q = cudaEventQuery(jb->ev);
        if (q == cudaErrorNotReady) {
          ++it;
          continue;
        }
        jb->inflight = false;
        progressed = true;
        if (q != cudaSuccess) {
          finish_job(sv, jb, IG_ECUDA, cudaGetErrorString(q));
          finished = true;
        } else if (jb->state == kPasses) {
          ig_status st = ig::plan_last_status(jb->plan);
          if (st == IG_ETABLE_FULL && ig::plan_regrow_and_restart(jb->plan)) {
            // its survivor lists grew: charge the job's new size, run it again
            uint64_t b = 0;
            intergrams_plan_device_bytes(jb->plan, &b);
            std::lock_guard<std::mutex> lock(sv->mu);
            if (b > jb->bytes) {
              sv->mem_used += b - jb->bytes;
              sv->peak_mem = std::max(sv->peak_mem, sv->mem_used);
              jb->bytes = b;
            }
            st = IG_OK;
          }
          if (st != IG_OK) {
            finish_job(sv, jb, st, intergrams_last_error());
            finished = true;
          }
        } else if (jb->state == kTopk) {
          finish_job(sv, jb, IG_OK, "");
          finished = true;
        }
      }
      if (!finished) {
        // the job's previous step is complete: enqueue its next one
        ig_status st;
        if (!ig::plan_passes_done(jb->plan)) {
          jb->state = kPasses;
          st = ig::plan_enqueue_next(jb->plan, jb->ev);
        } else {
          jb->state = kTopk;
          st = ig::plan_enqueue_topk(jb->plan, jb->keys_pinned, jb->counts_pinned, jb->p.k, &jb->rows, jb->ev);
        }
        if (st != IG_OK) {
          finish_job(sv, jb, st, intergrams_last_error());
          finished = true;
        } else {
          jb->inflight = true;
          progressed = true;
        }
      }
      if (finished) it = running.erase(it);
      else ++it;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

ig_status intergrams_server_create(const ig_server_config* cfg, ig_server** out) {
  ig::set_last_error("");
  if (!out) return IG_EINVAL;
  *out = nullptr;
  ig_server* sv = new (std::nothrow) ig_server();
  if (!sv) return IG_ENOMEM;
  if (cfg) sv->cfg = *cfg;
  if (sv->cfg.max_active == 0) sv->cfg.max_active = 8;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return IG_ECUDA;
  }
  if (sv->cfg.mem_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete sv;
      return IG_ECUDA;
    }
    sv->cfg.mem_budget = (uint64_t)(free_b * 0.8);
  }
  // keep freed job tables cached in the stream-ordered pool between jobs
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  sv->worker = std::thread(scheduler, sv);
  *out = sv;
  return IG_OK;
}

ig_status intergrams_server_submit(ig_server* sv, const ig_params* p, const void* data, const uint64_t* offsets,
                                   uint32_t m, const ig_tuning* tuning, uint64_t* job_id) {
  ig::set_last_error("");
  if (!sv || !p || !offsets || !job_id) {
    ig::set_last_error("NULL argument");
    return IG_EINVAL;
  }
  // size the job's tables with a dry-run plan (also validates the arguments)
  ig_params dp = *p;
  dp.flags = (dp.flags & ~(IG_F_HOST_INPUT | IG_F_GRAPH)) | IG_F_OFFSETS_HOST | IG_F_DRY_RUN;
  ig_plan* dry = nullptr;
  ig_status st = intergrams_plan(&dp, data, offsets, m, nullptr, tuning, &dry);
  if (st != IG_OK) return st;
  uint64_t bytes = 0;
  intergrams_plan_device_bytes(dry, &bytes);
  intergrams_free(dry);
  std::lock_guard<std::mutex> lock(sv->mu);
  if (bytes > sv->cfg.mem_budget) {
    ig::set_last_error("job needs more device memory than the server budget");
    return IG_ENOMEM;
  }
  Job* jb = new (std::nothrow) Job();
  if (!jb) return IG_ENOMEM;
  jb->id = sv->next_id++;
  jb->p = *p;
  if (tuning) {
    jb->t = *tuning;
    jb->has_tuning = true;
  }
  jb->data = data;
  jb->offsets.assign(offsets, offsets + (size_t)m + 1);
  jb->m = m;
  jb->bytes = bytes;
  {
    const uint32_t b = std::min(p->base_n, p->n);
    const double passes = (double)(p->n - b + 1);
    const double sym_bytes = (double)offsets[m] * (p->symbol_bits == 2 ? 0.25 : 1.0);
    const double sigma = p->symbol_bits == 2 ? 4.0 : 256.0;
    // the corpus is streamed once per pass; each candidate pass also reads
    // its sigma * Z counters a few times in the selection
    jb->work = sym_bytes * passes + (passes - 1) * 3.0 * 2.0 * sigma * (double)p->candidates;
  }
  jb->t_submit = Clock::now();
  sv->jobs[jb->id] = jb;
  sv->pending.push_back(jb);
  sv->submitted += 1;
  sv->cv_work.notify_all();
  *job_id = jb->id;
  return IG_OK;
}

ig_status intergrams_server_wait(ig_server* sv, uint64_t job_id, int64_t timeout_us, uint8_t* keys_out,
                                 uint64_t* counts_out, uint32_t capacity, uint32_t* k_out, double* latency_s) {
  ig::set_last_error("");
  if (!sv || !k_out) return IG_EINVAL;
  *k_out = 0;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) {
    ig::set_last_error("unknown job id");
    return IG_EINVAL;
  }
  Job* jb = it->second;
  auto done = [&] { return jb->state == kDone; };
  if (timeout_us < 0) sv->cv_done.wait(lock, done);
  else if (!sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done)) return IG_ETIMEOUT;
  // rows of a finished job: only what finish_job copied out (nothing if it failed)
  uint32_t r = jb->status == IG_OK ? std::min(capacity, jb->rows) : 0u;
  r = std::min<uint64_t>(r, jb->counts.size());
  if (jb->row_bytes) r = std::min<uint64_t>(r, jb->keys.size() / jb->row_bytes);
  if (keys_out && r) std::memcpy(keys_out, jb->keys.data(), (size_t)r * jb->row_bytes);
  if (counts_out && r) std::memcpy(counts_out, jb->counts.data(), sizeof(uint64_t) * r);
  *k_out = r;
  if (latency_s) *latency_s = std::chrono::duration<double>(jb->t_done - jb->t_submit).count();
  const ig_status st = jb->status;
  if (st != IG_OK) ig::set_last_error(jb->err);
  sv->jobs.erase(it);
  delete jb;
  return st;
}

ig_status intergrams_server_stats(ig_server* sv, ig_server_stats* out) {
  if (!sv || !out) return IG_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->active = sv->active;
  out->peak_active = sv->peak_active;
  out->pending = (uint32_t)sv->pending.size();
  out->mem_used = sv->mem_used;
  out->peak_mem = sv->peak_mem;
  out->mem_budget = sv->cfg.mem_budget;
  return IG_OK;
}

void intergrams_server_destroy(ig_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& kv : sv->jobs) delete kv.second;
  for (auto& kv : sv->pinned_free) cudaFreeHost(kv.second);
  delete sv;
}

}  // extern "C"
