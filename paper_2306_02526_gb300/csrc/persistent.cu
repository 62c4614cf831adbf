// All merge levels of one sweep direction in one cooperative (persistent) kernel.
//
// The upward sweep is 2L-1 dependent mat-vec tasks (per level: w3 = X d, then
// h^t = [h^a_1; h^b_2] + Tcat w3) and the downward sweep L tasks (u3 = S u_b + w3); each
// task is tiny next to a kernel launch on the lower levels.  Here one CTA grid sized to be
// resident on all SMs walks the task list; a grid-wide barrier separates consecutive tasks.
// Within a task the work items are (node group, row tile, column chunk); column chunks of
// one output tile are added by the CTA that finishes last, in chunk order (deterministic,
// nothing waits).  Every wait is bounded: a barrier that does not complete within the time
// limit sets the handle's error word and all CTAs return (hps_status reports HPS_ETIMEOUT).
#include <algorithm>
#include <cstdlib>

#include "hps_internal.cuh"

namespace hps {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded grid barrier (generation counter).  Returns false if the wait timed out here or
// another CTA reported an error.
__device__ bool grid_barrier(unsigned *bar, int *err, unsigned expect, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(bar + 1);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == expect - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire(bar + 1) == gen) {
        if (ld_acquire(reinterpret_cast<const unsigned *>(err))) { ok = 0; break; }
        if (global_ns() - t0 > limit_ns) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && !ld_acquire(reinterpret_cast<const unsigned *>(err));
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double load_x(const MTask &T, const PArgs &A, const double *hC, const double *w3, int k,
                                         int c) {
  switch (T.kind) {
    case 0: return hC[(int64_t)(2 * k + 1) * T.nbc + T.j3b + c] - hC[(int64_t)(2 * k) * T.nbc + T.j3a + c];
    case 1: return w3[(int64_t)k * T.n3 + c];
    default: return A.gvec[box_bd(A.g, T.origin[2 * k], T.origin[2 * k + 1], T.a, T.c, c)];
  }
}

__device__ __forceinline__ void epilogue(const MTask &T, const PArgs &A, const double *hC, double *w3, double *h,
                                         int k, int r, double v) {
  switch (T.kind) {
    case 0: w3[(int64_t)k * T.n3 + r] = v; break;
    case 1: h[(int64_t)k * T.nb + r] = hC[(int64_t)(2 * k) * T.nbc + T.hsrc[r]] + v; break;
    default:
      A.gvec[iface_bd(A.g, T.origin[2 * k], T.origin[2 * k + 1], T.a, T.c, T.split, r)] =
          v + w3[(int64_t)k * T.n3 + r];
  }
}

__global__ void __launch_bounds__(kPThreads) k_merge_persistent(PArgs A) {
  extern __shared__ double xs[];
  __shared__ int s_last;
  if (A.selftest) {  // a barrier that can never complete: exercises the bounded wait
    grid_barrier(A.bar, A.err, gridDim.x + 1, A.limit_ns);
    return;
  }
  for (int t = 0; t < A.ntasks; ++t) {
    if (A.stamps && blockIdx.x == 0 && threadIdx.x == 0) A.stamps[t] = global_ns();
    const MTask T = A.tasks[t];
    const double *hC = A.h[T.lvl + 1];
    double *w3 = A.w3[T.lvl];
    double *h = A.h[T.lvl];
    for (int64_t item = blockIdx.x; item < T.items; item += gridDim.x) {
      const int ks = (int)(item % T.ksplit);
      const int64_t rest = item / T.ksplit;
      const int tile = (int)(rest % T.row_tiles), ng = (int)(rest / T.row_tiles);
      const int node0 = ng * T.npc, nn = min(T.npc, T.nodes - node0);
      const int c0 = ks * T.kchunk, klen = min(T.kchunk, T.K - c0);
      __syncthreads();  // xs of the previous item is no longer read
      for (int idx = threadIdx.x; idx < nn * klen; idx += blockDim.x)
        xs[idx] = load_x(T, A, hC, w3, node0 + idx / klen, c0 + idx % klen);
      __syncthreads();
      int lo, r;
      if (T.npc > 1) {
        lo = threadIdx.x / T.M;
        r = threadIdx.x % T.M;
      } else {
        lo = 0;
        r = tile * T.rows_cta + threadIdx.x;
      }
      const bool active = lo < nn && r < T.M && (T.npc > 1 || threadIdx.x < T.rows_cta);
      const int k = node0 + lo;
      double acc = 0.0;
      if (active) {
        const double *a = T.AT + (int64_t)k * T.str + (int64_t)c0 * T.ld + r;
        const double *x = xs + lo * klen;
#pragma unroll 8
        for (int c = 0; c < klen; ++c) acc = fma(__ldg(a + (int64_t)c * T.ld), x[c], acc);
      }
      if (T.ksplit == 1) {
        if (active) epilogue(T, A, hC, w3, h, k, r, acc);
        continue;
      }
      // split columns: publish the partial sum; the last CTA of this tile adds them in order
      if (active) __stcg(A.partial + ((int64_t)ks * T.nodes + k) * T.M + r, acc);
      __threadfence();
      __syncthreads();
      unsigned *cnt = A.counters + (int64_t)ng * T.row_tiles + tile;
      if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1u) == (unsigned)(T.ksplit - 1);
      __syncthreads();
      if (s_last) {
        __threadfence();
        if (active) {
          double s = 0.0;
#pragma unroll 8
          for (int j = 0; j < T.ksplit; ++j) s += __ldcg(A.partial + ((int64_t)j * T.nodes + k) * T.M + r);
          epilogue(T, A, hC, w3, h, k, r, s);
        }
        if (threadIdx.x == 0) atomicExch(cnt, 0u);
      }
    }
    if (t + 1 < A.ntasks && !grid_barrier(A.bar, A.err, gridDim.x, A.limit_ns)) return;
  }
  if (A.stamps) {  // the end of the last task: every CTA is done once all have arrived here
    if (grid_barrier(A.bar, A.err, gridDim.x, A.limit_ns) && blockIdx.x == 0 && threadIdx.x == 0)
      A.stamps[A.ntasks] = global_ns();
  }
}

MTask plan_task(int kind, int lvl, int M, int K, int nodes, int target) {
  MTask T{};
  T.kind = kind;
  T.lvl = lvl;
  T.M = M;
  T.K = K;
  T.nodes = nodes;
  if (M <= kPThreads / 2) {
    T.npc = std::max(1, std::min(nodes, kPThreads / M));
    T.rows_cta = M;
    T.row_tiles = 1;
  } else {
    T.npc = 1;
    T.rows_cta = kPThreads;
    T.row_tiles = (M + kPThreads - 1) / kPThreads;
  }
  T.node_groups = (nodes + T.npc - 1) / T.npc;
  const int base = T.node_groups * T.row_tiles;
  int ks = 1;
  if (base < target) ks = std::min({(target + base - 1) / base, std::max(1, K / 32), kMaxSplit});
  T.kchunk = (K + ks - 1) / ks;
  while (T.npc * T.kchunk > kPSmemDoubles) T.kchunk = (T.kchunk + 1) / 2;
  T.ksplit = (K + T.kchunk - 1) / T.kchunk;
  T.items = (int64_t)base * T.ksplit;
  return T;
}

}  // namespace

int persistent_grid(hps_handle *H) {
  if (H->pgrid) return H->pgrid;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_merge_persistent, kPThreads,
                                                    kPSmemDoubles * sizeof(double)) != cudaSuccess ||
      bps < 1)
    return 0;
  int per_sm = 4;  // tuning knob: HPS_PERSISTENT_CTAS_PER_SM (1..8)
  if (const char *env = std::getenv("HPS_PERSISTENT_CTAS_PER_SM")) per_sm = std::max(1, std::min(8, std::atoi(env)));
  H->pgrid = H->num_sms * std::min(bps, per_sm);
  return H->pgrid;
}

// Task lists of one operator set: upward (w3, h per level, leaves to root) and downward.
int build_tasks(hps_handle *H, OpSet &ops) {
  if (!persistent_grid(H)) return HPS_ECUDA;
  const int target = H->fp64_plan_target * H->num_sms;  // the same split plan as the per-level path
  std::vector<MTask> up, down;
  for (int l = H->L - 1; l >= 0; --l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    MTask w = plan_task(0, l, lv.n3, lv.n3, lv.nodes, target);
    w.AT = mo.X; w.ld = mo.ldX; w.str = mo.strX;
    w.nbc = lv.nbc; w.j3a = lv.j3a; w.j3b = lv.j3b; w.n3 = lv.n3;
    up.push_back(w);
    if (l > 0) {
      MTask t = plan_task(1, l, lv.nb, lv.n3, lv.nodes, target);
      t.AT = mo.Tcat; t.ld = mo.ldT; t.str = mo.strT;
      t.nbc = lv.nbc; t.n3 = lv.n3; t.hsrc = lv.d_hsrc; t.nb = lv.nb;
      up.push_back(t);
    }
  }
  for (int l = 0; l < H->L; ++l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    MTask d = plan_task(2, l, lv.n3, lv.nb, lv.nodes, target);
    d.AT = mo.S; d.ld = mo.ldS; d.str = mo.strS;
    d.n3 = lv.n3; d.origin = lv.d_origin; d.a = lv.a; d.c = lv.c; d.split = lv.split;
    down.push_back(d);
  }
  size_t part = 0, cnt = 0;
  for (const auto *v : {&up, &down})
    for (const MTask &T : *v) {
      if (T.ksplit > 1) part = std::max(part, (size_t)T.ksplit * T.nodes * T.M);
      cnt = std::max(cnt, (size_t)T.node_groups * T.row_tiles);
    }
  H->ppartial_len = std::max(H->ppartial_len, part);
  H->pcounter_len = std::max(H->pcounter_len, cnt);
  ops.n_up = (int)up.size();
  ops.n_down = (int)down.size();
  if (cudaMalloc(&ops.d_up, std::max<size_t>(1, up.size()) * sizeof(MTask)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(ops.d_up);
  if (cudaMalloc(&ops.d_down, std::max<size_t>(1, down.size()) * sizeof(MTask)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(ops.d_down);
  cudaMemcpy(ops.d_up, up.data(), up.size() * sizeof(MTask), cudaMemcpyHostToDevice);
  cudaMemcpy(ops.d_down, down.data(), down.size() * sizeof(MTask), cudaMemcpyHostToDevice);
  return HPS_OK;
}

static PArgs make_args(hps_handle *H, const MTask *tasks, int ntasks, double *gvec) {
  PArgs A{};
  A.tasks = tasks;
  A.ntasks = ntasks;
  for (int l = 0; l <= H->L && l < kMaxLevels; ++l) {
    A.h[l] = H->h[l];
    if (l < H->L) A.w3[l] = H->w3[l];
  }
  A.g = H->g;
  A.gvec = gvec;
  A.partial = H->ppartial;
  A.counters = H->pcounters;
  A.bar = H->pbar;
  A.err = H->perr;
  A.limit_ns = 2000000000ull;  // 2 s: far above any level's work, short enough to report a fault
  return A;
}

static int launch_persistent(hps_handle *H, PArgs &A, cudaStream_t st) {
  void *args[] = {&A};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_merge_persistent, dim3(H->pgrid),
                                                    dim3(kPThreads), args, kPSmemDoubles * sizeof(double), st);
  return e == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

int merge_persistent(hps_handle *H, const OpSet &ops, bool upward, double *gvec, cudaStream_t st) {
  PArgs A = make_args(H, upward ? ops.d_up : ops.d_down, upward ? ops.n_up : ops.n_down, gvec);
  if (H->stamp_tasks && H->pstamps && A.ntasks < 64) A.stamps = H->pstamps + (upward ? 0 : 64);
  if (A.ntasks == 0) return HPS_OK;
  const int slot = upward ? kMergeUpFused : kMergeDownFused;
  H->trace.begin(slot, st);
  const int e = launch_persistent(H, A, st);
  H->trace.end(slot, st);
  return e;
}

int selftest_barrier(hps_handle *H, cudaStream_t st) {
  PArgs A = make_args(H, nullptr, 0, nullptr);
  A.selftest = 1;
  A.limit_ns = 1000000ull;  // 1 ms
  cudaMemsetAsync(H->pbar, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(H->perr, 0, sizeof(int), st);
  if (int e = launch_persistent(H, A, st)) return e;
  int herr = 0;
  cudaMemcpyAsync(&herr, H->perr, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;
  cudaMemsetAsync(H->pbar, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(H->perr, 0, sizeof(int), st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;
  return herr ? HPS_ETIMEOUT : HPS_OK;
}

}  // namespace hps
