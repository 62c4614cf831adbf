// Continuous-batching server for time-stepping jobs (a native request loop around ark_step).
//
// Jobs (tree, p, constant coefficients, dt, steps, g, initial state) arrive at given times.
// The loop admits a waiting job as soon as an active slot is free and the device-memory
// budget allows its operators (unless a resident factorization of an identical operator can
// be shared) plus its work buffers and state; admitted jobs advance one ARK step at a time,
// each on its own CUDA stream with up to two steps in flight, so steps of different jobs
// overlap on the GPU and a new job joins while others run.  Finished jobs copy their state
// back and release their memory; factorizations without users stay cached until memory is
// needed.  Every step is bracketed by CUDA events for the latency statistics.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "hps_internal.cuh"

namespace {

constexpr int kRing = 4;      // event pairs per job (steps in flight <= kInFlight < kRing)
constexpr int kInFlight = 2;

struct OpKey {
  hps_tree tree;
  int p;
  double c[5];
  double gdt;
  bool operator==(const OpKey &o) const {
    return std::memcmp(&tree, &o.tree, sizeof(tree)) == 0 && p == o.p && std::memcmp(c, o.c, sizeof(c)) == 0 &&
           gdt == o.gdt;
  }
};

struct CacheEntry {
  OpKey key;
  hps_handle *base = nullptr;
  int users = 0;
  size_t bytes = 0;
  double last_use = 0.0;
};

enum JobState { kWaiting = 0, kActive = 1, kDone = 2, kRejected = 3 };

struct Job {
  hps_job_desc d;
  int state = kWaiting;
  int status = HPS_OK;
  CacheEntry *ce = nullptr;
  hps_handle *h = nullptr;
  cudaStream_t st = nullptr;
  double *du = nullptr;
  int64_t N = 0;
  size_t bytes = 0;
  int enq = 0, done = 0;
  cudaEvent_t ev[2 * kRing] = {};
  std::vector<float> step_ms;
  double admit_s = 0.0, finish_s = 0.0;
  bool shared_ops = false;
};

}  // namespace

struct hps_server {
  size_t budget = 0, used = 0, peak_used = 0;
  int max_active = 1;
  std::vector<std::unique_ptr<Job>> jobs;
  std::vector<std::unique_ptr<CacheEntry>> cache;
  double makespan_s = 0.0;
  int max_concurrent = 0;
  int builds = 0, cache_hits = 0;
};

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void release_job(hps_server *S, Job &J) {
  if (J.h) hps_free(J.h);
  J.h = nullptr;
  if (J.du) cudaFree(J.du);
  J.du = nullptr;
  for (auto &e : J.ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (J.st) cudaStreamDestroy(J.st);
  J.st = nullptr;
  if (J.ce) --J.ce->users;
  J.ce = nullptr;
  S->used -= J.bytes;
}

// frees cached factorizations without users, least recently used first, until `need` fits
void evict(hps_server *S, size_t need) {
  for (;;) {
    if (S->used + need <= S->budget) return;
    CacheEntry *victim = nullptr;
    for (auto &c : S->cache)
      if (c->base && c->users == 0 && (!victim || c->last_use < victim->last_use)) victim = c.get();
    if (!victim) return;
    hps_free(victim->base);
    victim->base = nullptr;
    S->used -= victim->bytes;
  }
}

CacheEntry *find_entry(hps_server *S, const OpKey &k) {
  for (auto &c : S->cache)
    if (c->base && c->key == k) return c.get();
  return nullptr;
}

// tries to admit J; returns false when it has to wait for memory or a slot
bool admit(hps_server *S, Job &J, double t) {
  const hps_job_desc &d = J.d;
  OpKey key{};
  key.tree = d.tree;
  key.p = d.p;
  key.c[0] = d.c_a11; key.c[1] = d.c_a22; key.c[2] = d.c_a1; key.c[3] = d.c_a2; key.c[4] = d.c_a0;
  key.gdt = 0.25 * d.dt;
  size_t ops = 0, work = 0;
  if (hps::bytes_split(&d.tree, d.p, HPS_COEF_CONST, 0, &ops, &work)) {
    J.state = kRejected;
    J.status = HPS_EINVAL;
    return true;
  }
  int64_t N = 0;
  hps_sizes(&d.tree, d.p, &N, nullptr, nullptr);
  CacheEntry *ce = find_entry(S, key);
  const size_t need_job = work + (size_t)N * sizeof(double);
  const size_t need = need_job + (ce ? 0 : ops);
  if (need > S->budget) {  // can never fit
    J.state = kRejected;
    J.status = HPS_ENOMEM;
    return true;
  }
  if (S->used + need > S->budget) {
    if (ce) ++ce->users;  // pinned: the factorization this job will share must not be evicted
    evict(S, need);
    if (ce) --ce->users;
  }
  if (S->used + need > S->budget) return false;
  if (cudaStreamCreateWithFlags(&J.st, cudaStreamNonBlocking) != cudaSuccess) {
    J.state = kRejected;
    J.status = HPS_ECUDA;
    return true;
  }
  auto reject = [&](int e) {
    J.status = e;
    J.state = kRejected;
    release_job(S, J);
    return true;
  };
  if (!ce) {  // build and cache the factorization of this operator
    hps_coeffs c{};
    c.kind = HPS_COEF_CONST;
    c.c_a11 = d.c_a11; c.c_a22 = d.c_a22; c.c_a1 = d.c_a1; c.c_a2 = d.c_a2; c.c_a0 = d.c_a0;
    hps_handle *base = nullptr;
    const int e = hps_build(&d.tree, d.p, &c, key.gdt, 0, (hps_stream_t)J.st, &base);
    if (e) return reject(e);
    auto entry = std::make_unique<CacheEntry>();
    entry->key = key;
    entry->base = base;
    entry->bytes = ops;
    ce = entry.get();
    S->cache.push_back(std::move(entry));
    S->used += ops;
    ++S->builds;
  } else {
    ++S->cache_hits;
    J.shared_ops = true;
  }
  ce->last_use = t;
  ++ce->users;
  J.ce = ce;
  J.bytes = need_job;
  S->used += need_job;
  S->peak_used = std::max(S->peak_used, S->used);
  if (int e = hps::clone_handle(ce->base, J.st, &J.h)) return reject(e);
  J.h->graph_mode = true;  // a fresh handle: no recorded graphs to discard
  if (cudaMalloc(&J.du, (size_t)N * sizeof(double)) != cudaSuccess) return reject(HPS_ENOMEM);
  J.N = N;
  for (auto &e : J.ev)
    if (cudaEventCreate(&e) != cudaSuccess) return reject(HPS_ECUDA);
  cudaMemcpyAsync(J.du, d.u0, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, J.st);
  J.state = kActive;
  J.admit_s = t;
  J.step_ms.reserve(d.steps);
  return true;
}

}  // namespace

extern "C" {

int hps_server_create(size_t mem_budget_bytes, int max_active, hps_server **out) {
  if (!out || max_active < 1 || mem_budget_bytes == 0) return HPS_EINVAL;
  hps_server *S = new (std::nothrow) hps_server();
  if (!S) return HPS_ENOMEM;
  S->budget = mem_budget_bytes;
  S->max_active = max_active;
  *out = S;
  return HPS_OK;
}

int hps_server_submit(hps_server *S, const hps_job_desc *d, int *job_id) {
  if (!S || !d || !d->u0 || !d->u_out || d->steps < 0 || !(d->dt > 0.0) || d->g_kind < HPS_G_NONE ||
      d->g_kind > HPS_G_BURGERS || !(d->arrival_s >= 0.0))
    return HPS_EINVAL;
  auto J = std::make_unique<Job>();
  J->d = *d;
  if (job_id) *job_id = (int)S->jobs.size();
  S->jobs.push_back(std::move(J));
  return HPS_OK;
}

int hps_server_run(hps_server *S) {
  if (!S) return HPS_EINVAL;
  std::vector<Job *> order;
  for (auto &j : S->jobs)
    if (j->state == kWaiting) order.push_back(j.get());
  std::stable_sort(order.begin(), order.end(), [](Job *a, Job *b) { return a->d.arrival_s < b->d.arrival_s; });
  const auto t0 = std::chrono::steady_clock::now();
  size_t next = 0;  // first job not yet admitted (admission in arrival order)
  std::vector<Job *> active;
  int err = HPS_OK;
  while (next < order.size() || !active.empty()) {
    bool progressed = false;
    const double t = now_s(t0);
    // 1. completed steps and finished jobs
    for (size_t i = 0; i < active.size();) {
      Job &J = *active[i];
      while (J.done < J.enq && cudaEventQuery(J.ev[2 * (J.done % kRing) + 1]) == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, J.ev[2 * (J.done % kRing)], J.ev[2 * (J.done % kRing) + 1]);
        J.step_ms.push_back(ms);
        ++J.done;
        progressed = true;
      }
      if (J.done == J.d.steps) {
        cudaMemcpyAsync(J.d.u_out, J.du, (size_t)J.N * sizeof(double), cudaMemcpyDeviceToHost, J.st);
        if (cudaStreamSynchronize(J.st) != cudaSuccess) J.status = HPS_ECUDA;
        const int st = hps_status(J.h, (hps_stream_t)J.st);
        if (st && !J.status) J.status = st;
        J.finish_s = now_s(t0);
        J.state = kDone;
        release_job(S, J);
        active.erase(active.begin() + i);
        progressed = true;
        continue;
      }
      ++i;
    }
    // 2. admissions (in arrival order; a job that must wait for memory holds the queue)
    while (next < order.size() && order[next]->d.arrival_s <= t && (int)active.size() < S->max_active) {
      Job &J = *order[next];
      if (!admit(S, J, t)) break;
      ++next;
      progressed = true;
      if (J.state == kActive) active.push_back(&J);
    }
    S->max_concurrent = std::max(S->max_concurrent, (int)active.size());
    if (next < order.size() && active.empty() && order[next]->d.arrival_s <= t && S->used == 0) {
      // nothing runs and the head job still does not fit: it never will
      order[next]->state = kRejected;
      order[next]->status = HPS_ENOMEM;
      ++next;
    }
    // 3. keep up to kInFlight steps queued per job
    for (Job *Jp : active) {
      Job &J = *Jp;
      while (J.enq < J.d.steps && J.enq - J.done < kInFlight) {
        const int slot = J.enq % kRing;
        hps_ark_terms terms{};
        terms.g_kind = J.d.g_kind;
        terms.g_param[0] = J.d.g_param[0];
        terms.g_param[1] = J.d.g_param[1];
        cudaEventRecord(J.ev[2 * slot], J.st);
        const int e = ark_step(J.h, J.du, J.d.t0 + J.enq * J.d.dt, J.d.dt, &terms, (hps_stream_t)J.st);
        cudaEventRecord(J.ev[2 * slot + 1], J.st);
        if (e) {
          err = e;
          J.status = e;
        }
        ++J.enq;
        progressed = true;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  S->makespan_s = now_s(t0);
  return err;
}

int hps_server_job_stats(hps_server *S, int job_id, hps_job_stats *out) {
  if (!S || !out || job_id < 0 || job_id >= (int)S->jobs.size()) return HPS_EINVAL;
  const Job &J = *S->jobs[job_id];
  std::memset(out, 0, sizeof(*out));
  out->state = J.state;
  out->status = J.status;
  out->arrival_s = J.d.arrival_s;
  out->admit_s = J.admit_s;
  out->finish_s = J.finish_s;
  out->steps_done = (int)J.step_ms.size();
  out->shared_operators = J.shared_ops ? 1 : 0;
  out->work_bytes = J.bytes;
  if (!J.step_ms.empty()) {
    std::vector<float> v = J.step_ms;
    std::sort(v.begin(), v.end());
    double s = 0.0;
    for (float x : v) s += x;
    out->step_ms_mean = s / v.size();
    out->step_ms_p50 = v[v.size() / 2];
    out->step_ms_p99 = v[std::min(v.size() - 1, (size_t)(0.99 * v.size()))];
  }
  return HPS_OK;
}

int hps_server_summary(hps_server *S, hps_server_stats *out) {
  if (!S || !out) return HPS_EINVAL;
  std::memset(out, 0, sizeof(*out));
  std::vector<float> all;
  double dof_stages = 0.0;
  for (auto &jp : S->jobs) {
    const Job &J = *jp;
    if (J.state == kDone) ++out->jobs_done;
    if (J.state == kRejected) ++out->jobs_rejected;
    all.insert(all.end(), J.step_ms.begin(), J.step_ms.end());
    dof_stages += (double)J.N * 5.0 * (double)J.step_ms.size();
  }
  out->makespan_s = S->makespan_s;
  out->dof_stages_per_s = S->makespan_s > 0 ? dof_stages / S->makespan_s : 0.0;
  out->steps = (int64_t)all.size();
  if (!all.empty()) {
    std::sort(all.begin(), all.end());
    out->step_ms_p50 = all[all.size() / 2];
    out->step_ms_p99 = all[std::min(all.size() - 1, (size_t)(0.99 * all.size()))];
  }
  out->max_concurrent = S->max_concurrent;
  out->peak_bytes = S->peak_used;
  out->factorizations_built = S->builds;
  out->factorizations_shared = S->cache_hits;
  return HPS_OK;
}

void hps_server_free(hps_server *S) {
  if (!S) return;
  cudaDeviceSynchronize();
  for (auto &j : S->jobs)
    if (j->state == kActive) release_job(S, *j);
  for (auto &c : S->cache)
    if (c->base) hps_free(c->base);
  delete S;
}

}  // extern "C"
