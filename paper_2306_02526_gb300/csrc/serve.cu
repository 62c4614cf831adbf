// Continuous-batching server for time-stepping jobs (a native request loop around ark_step).
//
// Jobs (tree, p, constant or nodal coefficients, dt, steps, g, sources and boundary data through a
// per-step callback, initial state) arrive at given times.
// The loop admits a waiting job as soon as an active slot is free and the device-memory
// budget allows its operators (unless a resident factorization of an identical operator can
// be shared) plus its work buffers and state; admitted jobs advance one ARK step at a time,
// each on its own CUDA stream with up to two steps in flight, so steps of different jobs
// overlap on the GPU and a new job joins while others run.  Finished jobs copy their state
// back and release their memory; factorizations without users stay cached until memory is
// needed.  Every step is bracketed by CUDA events for the latency statistics.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "hps_internal.cuh"

namespace {

constexpr int kRing = 4;      // event pairs per job (steps in flight <= kInFlight < kRing)
constexpr int kInFlight = 2;

// The operator of a job: tree, p, gamma dt and its coefficients -- five constants, or (nodal) a
// hash of the five arrays, equal keys then compared entry by entry against the stored arrays.
struct OpKey {
  hps_tree tree;
  int p;
  double c[5];
  double gdt;
  int nodal;
  uint64_t chash;
  bool operator==(const OpKey &o) const {
    return std::memcmp(&tree, &o.tree, sizeof(tree)) == 0 && p == o.p && std::memcmp(c, o.c, sizeof(c)) == 0 &&
           gdt == o.gdt && nodal == o.nodal && chash == o.chash;
  }
};

struct CacheEntry {
  OpKey key;
  std::vector<double> coef;  // nodal: the five coefficient arrays (5 x N_int, zeros for NULL)
  hps_handle *base = nullptr;
  int users = 0;
  size_t bytes = 0;
  double last_use = 0.0;
};

enum JobState { kWaiting = 0, kActive = 1, kDone = 2, kRejected = 3 };

struct Job {
  hps_job_desc d;
  OpKey key{};
  int64_t N_int = 0, N_bd = 0;
  double a11max = 0.0, a22max = 0.0;  // largest |a11|, |a22| over the points (stiffness)
  int state = kWaiting;
  int status = HPS_OK;
  CacheEntry *ce = nullptr;
  hps_handle *h = nullptr;
  cudaStream_t st = nullptr;
  double *du = nullptr;
  double *dq = nullptr, *df = nullptr;  // terms callback: the step's q (6 x N_int) and f (6 x N_bd)
  int64_t N = 0;
  size_t bytes = 0;
  int enq = 0, done = 0;
  cudaEvent_t ev[2 * kRing] = {};
  std::vector<float> step_ms;
  double admit_s = 0.0, finish_s = 0.0;
  bool shared_ops = false;
  struct Group *grp = nullptr;  // batched serving: the batch it is (or will be) a column of
  // eviction with checkpoint / resume: after `evict_after` steps the job's state u and its step
  // count (hence t = t0 + steps dt) go to host memory, its device memory and slot are released,
  // and it queues again; re-admitted, it resumes from the checkpoint
  int evict_after = -1;
  int evictions = 0;
  std::vector<double> ckpt;
  bool pending_evict() const { return evict_after >= 0 && evictions == 0; }
  const double *state_in() const { return evictions > 0 ? ckpt.data() : d.u0; }
};

// Batched serving: jobs of one operation advanced together as the columns of one state.
struct Group {
  OpKey key;
  bool with_terms = false;             // members fill q and f before every step
  double *Q = nullptr, *F = nullptr;   // 6 x N_int x cap, 6 x N_bd x cap (stage-major, columns fastest)
  double *qs = nullptr, *fs = nullptr; // one member's fill (6 x N_int, 6 x N_bd)
  int64_t N_int = 0, N_bd = 0;
  int g_kind = 0;
  double g_param[2] = {0.0, 0.0};
  CacheEntry *ce = nullptr;
  hps_handle *h = nullptr;
  cudaStream_t st = nullptr;
  double *U = nullptr, *U2 = nullptr;  // N x cap each: the state (R columns) and the repack target
  double *col = nullptr;               // N: one job's state on its way in or out
  int *d_map = nullptr;                // cap: repack map (new column -> old column or -1)
  int cap = 0, R = 0;
  int refine = 1;                      // FP64 refinement sweeps per implicit solve of this batch
  int64_t N = 0;
  size_t bytes = 0;
  std::vector<Job *> members, pending;
  int enq = 0, done = 0;
  cudaEvent_t ev[2 * kRing] = {};
  int64_t col_steps = 0, steps = 0;    // sum over steps of the member count; steps run
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
  int batch_cols = 0, refine = 1;  // batching on when batch_cols > 0
  std::vector<std::unique_ptr<Group>> groups;
  int groups_formed = 0;
  int64_t batch_col_steps = 0, batch_step_count = 0;  // batched steps run and their member counts
};

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void release_job(hps_server *S, Job &J) {
  if (J.h) hps_free(J.h);
  J.h = nullptr;
  for (double **p : {&J.du, &J.dq, &J.df})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
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

const double *coef_array(const hps_job_desc &d, int c) {
  const double *a[5] = {d.a11, d.a22, d.a1, d.a2, d.a0};
  return a[c];
}
bool job_nodal(const hps_job_desc &d) { return d.a11 || d.a22 || d.a1 || d.a2 || d.a0; }

// FNV-1a over the bit patterns of the five arrays (a NULL array as zeros)
uint64_t coef_hash(const hps_job_desc &d, int64_t n) {
  uint64_t h = 1469598103934665603ull;
  for (int c = 0; c < 5; ++c) {
    const double *a = coef_array(d, c);
    for (int64_t i = 0; i < n; ++i) {
      uint64_t b = 0;
      if (a) std::memcpy(&b, a + i, sizeof b);
      for (int k = 0; k < 8; ++k) {
        h ^= (b >> (8 * k)) & 0xffu;
        h *= 1099511628211ull;
      }
    }
  }
  return h;
}

// the job's arrays hold exactly the stored values (bit patterns; NULL = zeros)
bool coef_same(const std::vector<double> &stored, const hps_job_desc &d, int64_t n) {
  if ((int64_t)stored.size() != 5 * n) return false;
  for (int c = 0; c < 5; ++c) {
    const double *a = coef_array(d, c);
    const double *s = stored.data() + c * n;
    if (a) {
      if (std::memcmp(a, s, (size_t)n * sizeof(double)) != 0) return false;
    } else {
      for (int64_t i = 0; i < n; ++i)
        if (std::signbit(s[i]) || s[i] != 0.0) return false;
    }
  }
  return true;
}

// the operator of J is that of cache entry c
bool same_operator(const CacheEntry &c, const Job &J) {
  return c.key == J.key && (!J.key.nodal || coef_same(c.coef, J.d, J.N_int));
}

CacheEntry *find_entry(hps_server *S, const Job &J) {
  for (auto &c : S->cache)
    if (c->base && same_operator(*c, J)) return c.get();
  return nullptr;
}

// Builds J's factorization on `st` (nodal coefficients staged to the device for the build) and
// caches it with `ops` bytes.
int build_entry(hps_server *S, const Job &J, cudaStream_t st, size_t ops, CacheEntry **out) {
  const hps_job_desc &d = J.d;
  hps_coeffs c{};
  double *dc = nullptr;
  if (J.key.nodal) {
    const int64_t n = J.N_int;
    if (cudaMalloc(&dc, 5 * (size_t)n * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    for (int k = 0; k < 5; ++k) {
      const double *a = coef_array(d, k);
      if (a)
        cudaMemcpyAsync(dc + k * n, a, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
      else
        cudaMemsetAsync(dc + k * n, 0, (size_t)n * sizeof(double), st);
    }
    c.kind = HPS_COEF_NODAL;
    c.a11 = dc; c.a22 = dc + n; c.a1 = dc + 2 * n; c.a2 = dc + 3 * n; c.a0 = dc + 4 * n;
  } else {
    c.kind = HPS_COEF_CONST;
    c.c_a11 = d.c_a11; c.c_a22 = d.c_a22; c.c_a1 = d.c_a1; c.c_a2 = d.c_a2; c.c_a0 = d.c_a0;
  }
  hps_handle *base = nullptr;
  int e = hps_build(&d.tree, d.p, &c, J.key.gdt, 0, (hps_stream_t)st, &base);
  if (dc) {
    if (cudaStreamSynchronize(st) != cudaSuccess && !e) e = HPS_ECUDA;
    cudaFree(dc);
  }
  if (e) {
    if (base) hps_free(base);
    return e;
  }
  auto entry = std::make_unique<CacheEntry>();
  entry->key = J.key;
  if (J.key.nodal) {
    entry->coef.assign(5 * (size_t)J.N_int, 0.0);
    for (int k = 0; k < 5; ++k)
      if (const double *a = coef_array(d, k)) std::memcpy(entry->coef.data() + k * J.N_int, a, (size_t)J.N_int * 8);
  }
  entry->base = base;
  entry->bytes = ops;
  *out = entry.get();
  S->cache.push_back(std::move(entry));
  S->used += ops;
  ++S->builds;
  return HPS_OK;
}

// extra device bytes of a nodal build (the staged coefficient arrays, freed after it)
size_t build_extra(const Job &J) { return J.key.nodal ? 5 * (size_t)J.N_int * sizeof(double) : 0; }
// device bytes of one (q, f) pair of a step
size_t terms_bytes(const Job &J) { return 6 * (size_t)(J.N_int + J.N_bd) * sizeof(double); }

// tries to admit J; returns false when it has to wait for memory or a slot
bool admit(hps_server *S, Job &J, double t) {
  const hps_job_desc &d = J.d;
  size_t ops = 0, work = 0;
  if (hps::bytes_split(&d.tree, d.p, J.key.nodal ? HPS_COEF_NODAL : HPS_COEF_CONST, 0, &ops, &work)) {
    J.state = kRejected;
    J.status = HPS_EINVAL;
    return true;
  }
  int64_t N = 0;
  hps_sizes(&d.tree, d.p, &N, nullptr, nullptr);
  CacheEntry *ce = find_entry(S, J);
  const size_t need_job = work + (size_t)N * sizeof(double) + (d.terms ? terms_bytes(J) : 0);
  const size_t need = need_job + (ce ? 0 : ops + build_extra(J));
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
    if (int e = build_entry(S, J, J.st, ops, &ce)) return reject(e);
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
  if (d.terms && (cudaMalloc(&J.dq, 6 * (size_t)J.N_int * sizeof(double)) != cudaSuccess ||
                  cudaMalloc(&J.df, 6 * (size_t)std::max<int64_t>(1, J.N_bd) * sizeof(double)) != cudaSuccess))
    return reject(HPS_ENOMEM);
  J.N = N;
  for (auto &e : J.ev)
    if (cudaEventCreate(&e) != cudaSuccess) return reject(HPS_ECUDA);
  cudaMemcpyAsync(J.du, J.state_in(), (size_t)N * sizeof(double), cudaMemcpyHostToDevice, J.st);
  J.state = kActive;
  J.enq = J.done;  // a resumed job continues with its next step
  J.admit_s = t;
  J.step_ms.reserve(d.steps);
  return true;
}


// ---- batched serving -----------------------------------------------------------------------
// dst[i Rd + j] = src[i Rs + map[j]] (map[j] < 0: zero), the columns of a batch after members
// joined or left
__global__ void k_repack(int64_t N, const double *__restrict__ src, int Rs, double *__restrict__ dst, int Rd,
                         const int *__restrict__ map) {
  const int64_t n = N * Rd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pt = i / Rd;
    const int j = (int)(i - pt * Rd), s = map[j];
    dst[i] = s >= 0 ? src[pt * Rs + s] : 0.0;
  }
}
// one column of an N x R state from / to a contiguous vector
__global__ void k_col(int64_t N, double *__restrict__ U, int R, int j, double *__restrict__ v, int to_state) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (to_state) U[i * R + j] = v[i];
    else v[i] = U[i * R + j];
  }
}

// one member's fill into column j of a batch's stage-major term array: dst[r R + j] = src[r]
__global__ void k_put_col(int64_t rows, const double *__restrict__ src, double *__restrict__ dst, int R, int j) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    dst[r * R + j] = src[r];
}

// Refinement sweeps for the mixed-precision step of an operation when the caller leaves the choice
// to the server: by the stiffness sigma = gamma dt max(a11 / hx^2, a22 / hy^2) 4 lambda(p), lambda(p)
// = 0.047 (p - 1)^4 the spectral radius of the 1-D Chebyshev second-derivative matrix on [-1, 1]
// with Dirichlet ends; the FP32 sweep's error, and with it the number of sweeps that bring the
// solve to FP64 accuracy, grows with sigma: 1 sweep up to sigma = 1e5 (measured: heat on 32 x 32
// leaves with p = 16 and dt = 0.01, sigma = 2.4e4, stays within 2e-11 of the FP64 step over ten
// steps with one sweep), then one more per factor 100.  Nodal coefficients: the largest |a11|, |a22|.
int auto_refine(const Job &J) {
  const hps_job_desc &d = J.d;
  const double hx = (d.tree.x1 - d.tree.x0) / d.tree.n1, hy = (d.tree.y1 - d.tree.y0) / d.tree.n2;
  const double lam = 0.047 * std::pow((double)(d.p - 1), 4.0);
  const double sigma = 0.25 * d.dt * std::max(J.a11max / (hx * hx), J.a22max / (hy * hy)) * 4.0 * lam;
  int r = 1;
  for (double s = 1e5; sigma > s && r < 4; s *= 100.0) ++r;
  return r;
}

// The key of a submitted job (the hash and maxima of nodal coefficients read once, at submission).
void job_key(Job &J) {
  const hps_job_desc &d = J.d;
  OpKey key{};
  key.tree = d.tree;
  key.p = d.p;
  key.gdt = 0.25 * d.dt;
  if (job_nodal(d)) {
    key.nodal = 1;
    key.chash = coef_hash(d, J.N_int);
    J.a11max = J.a22max = 0.0;
    for (int64_t i = 0; i < J.N_int; ++i) {
      if (d.a11) J.a11max = std::max(J.a11max, std::fabs(d.a11[i]));
      if (d.a22) J.a22max = std::max(J.a22max, std::fabs(d.a22[i]));
    }
  } else {
    key.c[0] = d.c_a11; key.c[1] = d.c_a22; key.c[2] = d.c_a1; key.c[3] = d.c_a2; key.c[4] = d.c_a0;
    J.a11max = std::fabs(d.c_a11);
    J.a22max = std::fabs(d.c_a22);
  }
  J.key = key;
}

// J's steps are the operation of batch G: its operator, its g, and terms on both or neither
bool same_op(const Group &G, const Job &J) {
  const hps_job_desc &d = J.d;
  return G.ce && same_operator(*G.ce, J) && G.g_kind == d.g_kind && G.g_param[0] == d.g_param[0] &&
         G.g_param[1] == d.g_param[1] && G.with_terms == (d.terms != nullptr);
}

void release_group(hps_server *S, Group &G) {
  if (G.st) cudaStreamSynchronize(G.st);
  if (G.h) hps_free(G.h);
  for (double *p : {G.U, G.U2, G.col, G.Q, G.F, G.qs, G.fs})
    if (p) cudaFree(p);
  if (G.d_map) cudaFree(G.d_map);
  for (auto &e : G.ev)
    if (e) cudaEventDestroy(e);
  if (G.st) cudaStreamDestroy(G.st);
  if (G.ce) --G.ce->users;
  S->used -= G.bytes;
  S->batch_col_steps += G.col_steps;
  S->batch_step_count += G.steps;
  G = Group{};
}

// A new (empty) batch for job J's operation: its factorization (shared through the cache), a
// handle reserved for `cap` columns and the state buffers.  The batch's bytes are measured as the
// device memory its allocations took.  Returns false when the budget does not hold it (J waits).
bool create_group(hps_server *S, const Job &J, double t, Group **out, int *reject) {
  const hps_job_desc &d = J.d;
  const OpKey key = J.key;
  *reject = HPS_OK;
  size_t ops = 0, work = 0;
  if (hps::bytes_split(&d.tree, d.p, key.nodal ? HPS_COEF_NODAL : HPS_COEF_CONST, 0, &ops, &work)) {
    *reject = HPS_EINVAL;
    return false;
  }
  int64_t N = 0;
  hps_sizes(&d.tree, d.p, &N, nullptr, nullptr);
  const int cap = S->batch_cols;
  // estimate before allocating: FP64 operators if not cached + about 160 bytes per point and
  // column of batched work vectors and states + the single-column work of the handle
  CacheEntry *ce = find_entry(S, J);
  const size_t est = (ce ? 0 : ops + build_extra(J)) + work + (size_t)N * cap * 160 + (size_t)N * 8 +
                     (d.terms ? terms_bytes(J) * (cap + 1) : 0);
  if (est > S->budget) {
    *reject = HPS_ENOMEM;
    return false;
  }
  if (S->used + est > S->budget) {
    if (ce) ++ce->users;
    evict(S, est);
    for (auto &g : S->groups)  // idle batches hold memory too
      if (S->used + est > S->budget && g->h && g->members.empty() && g->pending.empty()) release_group(S, *g);
    if (ce) --ce->users;
  }
  if (S->used + est > S->budget) return false;
  auto G = std::make_unique<Group>();
  G->key = key;
  G->g_kind = d.g_kind;
  G->g_param[0] = d.g_param[0];
  G->g_param[1] = d.g_param[1];
  G->cap = cap;
  G->N = N;
  G->N_int = J.N_int;
  G->N_bd = J.N_bd;
  G->with_terms = d.terms != nullptr;
  G->refine = S->refine >= 0 ? S->refine : auto_refine(J);
  auto fail = [&](int e) -> bool {
    *reject = e;
    release_group(S, *G);
    return false;
  };
  if (cudaStreamCreateWithFlags(&G->st, cudaStreamNonBlocking) != cudaSuccess) return fail(HPS_ECUDA);
  if (!ce) {
    if (int e = build_entry(S, J, G->st, ops, &ce)) return fail(e);
  } else {
    ++S->cache_hits;
  }
  ce->last_use = t;
  ++ce->users;
  G->ce = ce;
  size_t free0 = 0, free1 = 0, total = 0;
  cudaDeviceSynchronize();
  cudaMemGetInfo(&free0, &total);
  if (int e = hps::clone_handle(ce->base, G->st, &G->h)) return fail(e);
  if (int e = hps_batch_reserve(G->h, cap)) return fail(e);
  G->h->graph_mode = true;
  if (cudaMalloc(&G->U, (size_t)N * cap * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&G->U2, (size_t)N * cap * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&G->col, (size_t)N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&G->d_map, (size_t)cap * sizeof(int)) != cudaSuccess)
    return fail(HPS_ENOMEM);
  if (G->with_terms) {
    const size_t nb = (size_t)std::max<int64_t>(1, J.N_bd);
    if (cudaMalloc(&G->Q, 6 * (size_t)J.N_int * cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G->F, 6 * nb * cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G->qs, 6 * (size_t)J.N_int * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G->fs, 6 * nb * sizeof(double)) != cudaSuccess)
      return fail(HPS_ENOMEM);
  }
  for (auto &e : G->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(HPS_ECUDA);
  cudaDeviceSynchronize();
  cudaMemGetInfo(&free1, &total);
  G->bytes = free0 > free1 ? free0 - free1 : est;
  if (S->used + G->bytes > S->budget) {  // the measured size breaks the budget: give it back, wait
    release_group(S, *G);
    return false;
  }
  S->used += G->bytes;
  S->peak_used = std::max(S->peak_used, S->used);
  ++S->groups_formed;
  S->groups.push_back(std::move(G));
  *out = S->groups.back().get();
  return true;
}

inline int round4i(int n) { return (n + 3) & ~3; }

// A step boundary of G (none of its steps in flight): members that have run all their steps copy
// their column out and leave, waiting members join, and the columns are repacked into R = the
// member count rounded up to 4 (at most cap).
int group_boundary(Group &G, std::chrono::steady_clock::time_point t0, std::vector<Job *> &evicted) {
  std::vector<Job *> stay;
  std::vector<int> from;  // old column of each member of the new layout (-1: a joining job)
  bool changed = false;
  const unsigned nb = (unsigned)std::min<int64_t>((G.N + 255) / 256, 4096);
  for (int j = 0; j < (int)G.members.size(); ++j) {
    Job &J = *G.members[j];
    if (J.pending_evict() && J.done >= J.evict_after && J.done < J.d.steps) {  // checkpoint and queue again
      k_col<<<nb, 256, 0, G.st>>>(G.N, G.U, G.R, j, G.col, 0);
      J.ckpt.resize((size_t)G.N);
      cudaMemcpyAsync(J.ckpt.data(), G.col, (size_t)G.N * sizeof(double), cudaMemcpyDeviceToHost, G.st);
      if (cudaStreamSynchronize(G.st) != cudaSuccess && !J.status) J.status = HPS_ECUDA;
      ++J.evictions;
      J.state = kWaiting;
      J.grp = nullptr;
      evicted.push_back(&J);
      changed = true;
      continue;
    }
    if (J.done >= J.d.steps) {
      k_col<<<nb, 256, 0, G.st>>>(G.N, G.U, G.R, j, G.col, 0);
      cudaMemcpyAsync(J.d.u_out, G.col, (size_t)G.N * sizeof(double), cudaMemcpyDeviceToHost, G.st);
      if (cudaStreamSynchronize(G.st) != cudaSuccess && !J.status) J.status = HPS_ECUDA;
      const int st = hps_status(G.h, (hps_stream_t)G.st);
      if (st && !J.status) J.status = st;
      J.finish_s = now_s(t0);
      J.state = kDone;
      J.grp = nullptr;
      changed = true;
    } else {
      stay.push_back(&J);
      from.push_back(j);
    }
  }
  while (!G.pending.empty() && (int)stay.size() < G.cap) {
    stay.push_back(G.pending.front());
    from.push_back(-1);
    G.pending.erase(G.pending.begin());
    changed = true;
  }
  if (!changed) return HPS_OK;
  const int Rn = stay.empty() ? 0 : std::min(G.cap, round4i((int)stay.size()));
  if (Rn > 0) {
    std::vector<int> map(Rn, -1);
    for (size_t i = 0; i < stay.size(); ++i) map[i] = from[i];
    if (cudaMemcpyAsync(G.d_map, map.data(), Rn * sizeof(int), cudaMemcpyHostToDevice, G.st) != cudaSuccess)
      return HPS_ECUDA;
    if (G.R > 0) {
      k_repack<<<(unsigned)std::min<int64_t>((G.N * Rn + 255) / 256, 8192), 256, 0, G.st>>>(G.N, G.U, G.R, G.U2, Rn,
                                                                                            G.d_map);
    } else {
      cudaMemsetAsync(G.U2, 0, (size_t)G.N * Rn * sizeof(double), G.st);
    }
    std::swap(G.U, G.U2);
    if (G.with_terms) {  // columns moved: every member fills its own before the next step
      cudaMemsetAsync(G.Q, 0, 6 * (size_t)G.N_int * Rn * sizeof(double), G.st);
      cudaMemsetAsync(G.F, 0, 6 * (size_t)G.N_bd * Rn * sizeof(double), G.st);
    }
    const double now = now_s(t0);
    for (size_t i = 0; i < stay.size(); ++i) {
      if (from[i] >= 0) continue;
      Job &J = *stay[i];
      cudaMemcpyAsync(G.col, J.state_in(), (size_t)G.N * sizeof(double), cudaMemcpyHostToDevice, G.st);
      k_col<<<nb, 256, 0, G.st>>>(G.N, G.U, Rn, (int)i, G.col, 1);
      J.admit_s = now;
      J.step_ms.reserve(J.d.steps);
    }
  }
  G.members = stay;
  G.R = Rn;
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

int run_batched(hps_server *S) {
  std::vector<Job *> order;
  for (auto &j : S->jobs)
    if (j->state == kWaiting) order.push_back(j.get());
  std::stable_sort(order.begin(), order.end(), [](Job *a, Job *b) { return a->d.arrival_s < b->d.arrival_s; });
  const auto t0 = std::chrono::steady_clock::now();
  size_t next = 0;
  int err = HPS_OK;
  auto in_flight_jobs = [&]() {
    int n = 0;
    for (auto &g : S->groups) n += (int)(g->members.size() + g->pending.size());
    return n;
  };
  for (;;) {
    const int busy = in_flight_jobs();
    if (next >= order.size() && busy == 0) break;
    bool progressed = false;
    const double t = now_s(t0);
    // 1. completed steps
    for (auto &gp : S->groups) {
      Group &G = *gp;
      while (G.done < G.enq && cudaEventQuery(G.ev[2 * (G.done % kRing) + 1]) == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, G.ev[2 * (G.done % kRing)], G.ev[2 * (G.done % kRing) + 1]);
        for (Job *J : G.members) {
          J->step_ms.push_back(ms);
          ++J->done;
        }
        G.col_steps += (int64_t)G.members.size();
        ++G.steps;
        ++G.done;
        progressed = true;
      }
    }
    // 2. admissions in arrival order: into a batch of the same operation with a free column, else a
    // new batch (memory permitting; a job that must wait for memory holds the queue)
    while (next < order.size() && order[next]->d.arrival_s <= t && in_flight_jobs() < S->max_active) {
      Job &J = *order[next];
      Group *G = nullptr;
      for (auto &g : S->groups)
        if (g->h && same_op(*g, J) && (int)(g->members.size() + g->pending.size()) < g->cap) {
          G = g.get();
          J.shared_ops = true;
          break;
        }
      if (!G) {
        int rej = HPS_OK;
        const int builds = S->builds;
        if (!create_group(S, J, t, &G, &rej)) {
          if (rej || in_flight_jobs() == 0) {  // it never fits: reject, the rest still runs
            J.state = kRejected;
            J.status = rej ? rej : HPS_ENOMEM;
            ++next;
            progressed = true;
            continue;
          }
          break;
        }
        J.shared_ops = false;
        if (S->builds == builds) J.shared_ops = true, --S->cache_hits;  // (create_group counted the cache hit)
      }
      if (J.shared_ops) ++S->cache_hits;  // a running batch of its operation: operators shared
      G->pending.push_back(&J);
      J.grp = G;
      J.state = kActive;
      J.N = G->N;
      J.bytes = G->bytes / G->cap;
      ++next;
      progressed = true;
    }
    S->max_concurrent = std::max(S->max_concurrent, in_flight_jobs());
    // 3. step boundaries and steps
    for (auto &gp : S->groups) {
      Group &G = *gp;
      if (!G.h) continue;
      bool leaving = false;
      for (Job *J : G.members) leaving |= J->done >= J->d.steps || (J->pending_evict() && J->done >= J->evict_after);
      if (G.done == G.enq && (leaving || !G.pending.empty())) {
        std::vector<Job *> evicted;
        if (int e = group_boundary(G, t0, evicted)) err = e;
        for (Job *J : evicted) order.push_back(J);  // queued again (admissible at once)
        progressed = true;
      }
      if (G.members.empty() || !G.pending.empty()) continue;  // joiners get in once the queue drains
      int room = 1 << 30;
      for (Job *J : G.members)
        room = std::min(room, (J->pending_evict() ? std::min(J->evict_after, J->d.steps) : J->d.steps) - J->done);
      room -= G.enq - G.done;
      while (G.enq - G.done < kInFlight && room > 0) {
        const int slot = G.enq % kRing;
        hps_ark_terms terms{};
        terms.g_kind = G.g_kind;
        terms.g_param[0] = G.g_param[0];
        terms.g_param[1] = G.g_param[1];
        cudaEventRecord(G.ev[2 * slot], G.st);
        if (G.with_terms) {  // each member's q and f at its own time, into its column
          const int64_t ahead = G.enq - G.done;
          const unsigned nbq = (unsigned)std::min<int64_t>((6 * G.N_int + 255) / 256, 4096);
          const unsigned nbf = (unsigned)std::min<int64_t>((6 * G.N_bd + 255) / 256, 4096);
          for (size_t j = 0; j < G.members.size(); ++j) {
            Job &J = *G.members[j];
            const double tj = J.d.t0 + (double)(J.done + ahead) * J.d.dt;
            const int e = J.d.terms(J.d.terms_user, tj, J.d.dt, G.qs, G.fs, (hps_stream_t)G.st);
            if (e && !J.status) J.status = e;
            k_put_col<<<nbq, 256, 0, G.st>>>(6 * G.N_int, G.qs, G.Q, G.R, (int)j);
            if (G.N_bd > 0) k_put_col<<<nbf, 256, 0, G.st>>>(6 * G.N_bd, G.fs, G.F, G.R, (int)j);
          }
          terms.q = G.Q;
          terms.f = G.F;
        }
        const int e = ark_step_batch(G.h, G.R, G.U, 0.0, 4.0 * G.key.gdt, &terms, G.refine, (hps_stream_t)G.st);
        cudaEventRecord(G.ev[2 * slot + 1], G.st);
        if (e) {
          err = e;
          for (Job *J : G.members) J->status = e;
        }
        ++G.enq;
        --room;
        progressed = true;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  S->makespan_s = now_s(t0);
  for (auto &g : S->groups)
    if (g->h) release_group(S, *g);
  S->groups.clear();
  return err;
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
  int64_t N = 0, N_int = 0, N_bd = 0;
  if (hps_sizes(&d->tree, d->p, &N, &N_int, &N_bd)) return HPS_EINVAL;
  auto J = std::make_unique<Job>();
  J->d = *d;
  J->N_int = N_int;
  J->N_bd = N_bd;
  job_key(*J);
  if (job_id) *job_id = (int)S->jobs.size();
  S->jobs.push_back(std::move(J));
  return HPS_OK;
}

int hps_server_evict_after(hps_server *S, int job_id, int steps) {
  if (!S || job_id < 0 || job_id >= (int)S->jobs.size() || steps < 0) return HPS_EINVAL;
  S->jobs[job_id]->evict_after = steps;
  return HPS_OK;
}

int hps_server_set_batching(hps_server *S, int max_cols, int refine) {
  if (!S || max_cols < 0 || max_cols > 64 || refine < -1 || refine > 8) return HPS_EINVAL;
  S->batch_cols = max_cols;
  S->refine = refine;
  return HPS_OK;
}

int hps_server_run(hps_server *S) {
  if (!S) return HPS_EINVAL;
  if (S->batch_cols > 0) return run_batched(S);
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
      if (J.pending_evict() && J.done >= J.evict_after && J.done == J.enq && J.done < J.d.steps) {
        // checkpoint (u, steps done) to host memory, release the job's memory and slot, queue again
        J.ckpt.resize((size_t)J.N);
        cudaMemcpyAsync(J.ckpt.data(), J.du, (size_t)J.N * sizeof(double), cudaMemcpyDeviceToHost, J.st);
        if (cudaStreamSynchronize(J.st) != cudaSuccess) J.status = HPS_ECUDA;
        ++J.evictions;
        J.state = kWaiting;
        release_job(S, J);
        order.push_back(&J);
        active.erase(active.begin() + i);
        progressed = true;
        continue;
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
      while (J.enq < J.d.steps && J.enq - J.done < kInFlight && !(J.pending_evict() && J.enq >= J.evict_after)) {
        const int slot = J.enq % kRing;
        hps_ark_terms terms{};
        terms.g_kind = J.d.g_kind;
        terms.g_param[0] = J.d.g_param[0];
        terms.g_param[1] = J.d.g_param[1];
        const double tn = J.d.t0 + J.enq * J.d.dt;
        if (J.d.terms) {  // q and f of this step, ordered on the job's stream before it
          if (const int e = J.d.terms(J.d.terms_user, tn, J.d.dt, J.dq, J.df, (hps_stream_t)J.st)) {
            err = e;
            J.status = e;
            J.d.steps = J.enq;  // no further steps: the job ends with its steps in flight
            break;
          }
          terms.q = J.dq;
          terms.f = J.df;
        }
        cudaEventRecord(J.ev[2 * slot], J.st);
        const int e = ark_step(J.h, J.du, tn, J.d.dt, &terms, (hps_stream_t)J.st);
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
  out->evictions = J.evictions;
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
  out->batches_formed = S->groups_formed;
  out->mean_batch_cols = S->batch_step_count > 0 ? (double)S->batch_col_steps / S->batch_step_count : 0.0;
  return HPS_OK;
}

void hps_server_free(hps_server *S) {
  if (!S) return;
  cudaDeviceSynchronize();
  for (auto &g : S->groups)
    if (g->h) release_group(S, *g);
  for (auto &j : S->jobs)
    if (j->state == kActive && !j->grp) release_job(S, *j);
  for (auto &c : S->cache)
    if (c->base) hps_free(c->base);
  delete S;
}

}  // extern "C"
