// Many independent instances stepped together: one call advances every instance (its own tree,
// p, coefficients and R columns) by one batched mixed-precision ARK step, each instance on an
// internal stream forked from and joined back into the caller's stream, so the per-level kernels
// of different instances run concurrently on the GPU.  In graph mode the whole multi-instance
// step -- every instance's kernel sequence as one branch -- is recorded into ONE CUDA graph on the
// second call with the same arguments and replayed afterwards: one graph launch per step for all
// instances, whatever their tree sizes.  In lockstep mode the instances' FP32 sweeps share their
// merge launches: one grouped launch per tree level and merge operator for all instances (upward
// levels counted from each tree's leaves, downward from the roots), the leaf parts, residuals and
// epilogues still per instance on its own stream.
#include <cstring>
#include <new>
#include <vector>

#include "hps_internal.cuh"

struct hps_multi {
  std::vector<hps_handle *> h;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaEvent_t merged = nullptr;  // the grouped merges of a lockstep sweep are done
  bool graph = false;
  bool lockstep = false;
  cudaStream_t cap = nullptr;
  std::vector<uint64_t> key;  // arguments of the recorded graph
  bool seen = false;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void drop_graph(hps_multi *M) {
  if (M->exec) cudaGraphExecDestroy(M->exec);
  M->exec = nullptr;
  M->seen = false;
  M->key.clear();
}

uint64_t bits(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
}

// the instances' steps, forked from `st` and joined back into it
int enqueue(hps_multi *M, double *const *u, const int *R, const hps_ark_terms *terms, double dt, int refine,
            cudaStream_t st) {
  if (cudaEventRecord(M->fork, st) != cudaSuccess) return HPS_ECUDA;
  int err = HPS_OK;
  if (M->lockstep) {
    const int n = (int)M->h.size();
    for (int i = 0; i < n; ++i)
      if (cudaStreamWaitEvent(M->st[i], M->fork, 0) != cudaSuccess) return HPS_ECUDA;
    err = hps::ark_batch_lockstep(M->h.data(), n, u, R, terms, dt, refine, hps::ark_table(), st, M->st.data(),
                                  M->join.data(), M->merged);
    for (int i = 0; i < n; ++i)
      if (cudaEventRecord(M->join[i], M->st[i]) != cudaSuccess || cudaStreamWaitEvent(st, M->join[i], 0) != cudaSuccess)
        return HPS_ECUDA;
    return err;
  }
  for (size_t i = 0; i < M->h.size(); ++i) {
    if (cudaStreamWaitEvent(M->st[i], M->fork, 0) != cudaSuccess) return HPS_ECUDA;
    const int e = ark_step_batch(M->h[i], R[i], u[i], 0.0, dt, terms ? &terms[i] : nullptr, refine,
                                 (hps_stream_t)M->st[i]);
    if (e && !err) err = e;
    if (cudaEventRecord(M->join[i], M->st[i]) != cudaSuccess) return HPS_ECUDA;
    if (cudaStreamWaitEvent(st, M->join[i], 0) != cudaSuccess) return HPS_ECUDA;
  }
  return err;
}

}  // namespace

extern "C" {

int hps_multi_create(hps_handle *const *handles, int n, hps_multi **out) {
  if (!handles || n < 1 || !out) return HPS_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!handles[i]) return HPS_EINVAL;
  hps_multi *M = new (std::nothrow) hps_multi();
  if (!M) return HPS_ENOMEM;
  M->h.assign(handles, handles + n);
  M->st.assign(n, nullptr);
  M->join.assign(n, nullptr);
  bool ok = cudaEventCreateWithFlags(&M->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&M->merged, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i)
    ok = cudaStreamCreateWithFlags(&M->st[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&M->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    hps_multi_free(M);
    return HPS_ECUDA;
  }
  *out = M;
  return HPS_OK;
}

int hps_multi_set_graph(hps_multi *M, int enable) {
  if (!M) return HPS_EINVAL;
  cudaDeviceSynchronize();
  drop_graph(M);
  M->graph = enable != 0;
  for (hps_handle *h : M->h) h->graph_mode = false;  // the instances' own graphs would nest
  return HPS_OK;
}

int hps_multi_set_lockstep(hps_multi *M, int enable) {
  if (!M) return HPS_EINVAL;
  if (enable)
    for (hps_handle *h : M->h)
      if (h->batch.groups != 1) return HPS_EINVAL;
  cudaDeviceSynchronize();
  drop_graph(M);
  M->lockstep = enable != 0;
  return HPS_OK;
}

int hps_multi_ark_step(hps_multi *M, double *const *u, const int *R, const hps_ark_terms *terms, double dt, int refine,
                       hps_stream_t stream) {
  if (!M || !u || !R || !(dt > 0.0) || refine < 0 || refine > 8) return HPS_EINVAL;
  const size_t n = M->h.size();
  for (size_t i = 0; i < n; ++i)
    if (!u[i] || R[i] < 1 || R[i] > M->h[i]->batch.Rmax) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!M->graph || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return enqueue(M, u, R, terms, dt, refine, st);
  std::vector<uint64_t> key;
  key.reserve(n * 8 + 2);
  key.push_back(bits(dt));
  key.push_back((uint64_t)refine);
  for (size_t i = 0; i < n; ++i) {
    key.push_back((uint64_t)u[i]);
    key.push_back((uint64_t)R[i]);
    const hps_ark_terms *t = terms ? &terms[i] : nullptr;
    key.push_back((uint64_t)(t ? t->q : nullptr));
    key.push_back((uint64_t)(t ? t->f : nullptr));
    key.push_back((uint64_t)(t ? t->g_kind : 0));
    key.push_back(bits(t ? t->g_param[0] : 0.0));
    key.push_back(bits(t ? t->g_param[1] : 0.0));
  }
  if (M->exec && key == M->key) return cudaGraphLaunch(M->exec, st) == cudaSuccess ? HPS_OK : HPS_ECUDA;
  if (!(M->seen && key == M->key)) {  // first call with these arguments: eager
    drop_graph(M);
    M->key = key;
    M->seen = true;
    return enqueue(M, u, R, terms, dt, refine, st);
  }
  if (!M->cap && cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking) != cudaSuccess) return HPS_ECUDA;
  cudaGraph_t g = nullptr;
  int e = HPS_OK;
  if (cudaStreamBeginCapture(M->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) e = HPS_ECUDA;
  if (e == HPS_OK) {
    e = enqueue(M, u, R, terms, dt, refine, M->cap);
    if (cudaStreamEndCapture(M->cap, &g) != cudaSuccess && e == HPS_OK) e = HPS_ECUDA;
  }
  if (e == HPS_OK && cudaGraphInstantiate(&M->exec, g, 0) != cudaSuccess) e = HPS_ECUDA;
  if (g) cudaGraphDestroy(g);
  if (e != HPS_OK) {
    drop_graph(M);
    cudaGetLastError();
    return e;
  }
  return cudaGraphLaunch(M->exec, st) == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

void hps_multi_free(hps_multi *M) {
  if (!M) return;
  cudaDeviceSynchronize();
  drop_graph(M);
  if (M->cap) cudaStreamDestroy(M->cap);
  for (cudaStream_t s : M->st)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : M->join)
    if (e) cudaEventDestroy(e);
  if (M->fork) cudaEventDestroy(M->fork);
  if (M->merged) cudaEventDestroy(M->merged);
  delete M;
}

}  // extern "C"
