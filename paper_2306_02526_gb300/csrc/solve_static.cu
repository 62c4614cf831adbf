// hps_solve_static: hps_solve whose per-call work vectors live in one fixed device array
// instead of the buffers hps_build allocated with the handle.
//
// Who needs it: code that must not allocate device memory at solve time -- a real-time or
// embedded loop whose memory budget is fixed up front, a host that forbids cudaMalloc after
// start-up, or a caller whose allocator is not available on the thread that solves.  The
// operators still come from a handle built earlier; this entry point itself allocates
// nothing (no cudaMalloc, cudaFree or allocating library call).
#include "hps_internal.cuh"

namespace {

constexpr size_t kStaticScratchDoubles = size_t(2) << 20;  // 2,097,152 doubles = 16 MiB
constexpr int kMaxDevices = 64;

// Every GPU that loads libhps.so holds this array until the process exits.
static __device__ __align__(256) double g_solve_scratch[kStaticScratchDoubles];

// Device address of g_solve_scratch per device ordinal, looked up once per device.
double *g_scratch_addr[kMaxDevices] = {};

inline size_t round256(size_t n) { return (n + 31) & ~size_t(31); }  // 32 doubles = 256 bytes

// Carries a timeout recorded in this call's error word (inside the static array) into the
// handle's own error word, which hps_status reads; an earlier unreported timeout is kept.
__global__ void k_fold_error(const int *__restrict__ call_err, int *__restrict__ handle_err) {
  if (threadIdx.x == 0 && *call_err != 0) *handle_err = *call_err;
}

}  // namespace

extern "C" int hps_solve_static(hps_handle *H, const double *rhs, const double *f, double *u, hps_stream_t stream) {
  if (!H || !rhs || !u) return HPS_EINVAL;
  constexpr int kMaxLevels = 32;
  if (H->L + 1 > kMaxLevels) return HPS_EINVAL;
  // the handle's work vectors: leaf particular solutions, fluxes per level, w3 per merge level
  size_t need = round256((size_t)H->g.N_int);
  for (int l = 0; l <= H->L; ++l) {
    need += round256((size_t)H->lev[l].nodes * H->lev[l].nb);
    if (l < H->L) need += round256((size_t)H->lev[l].nodes * H->lev[l].n3);
  }
  need += round256(H->partial_len);  // split-K partial sums of the top merge levels
  // the persistent merge kernel's partial sums, tile counters, barrier and error word
  const size_t cnt_d = (H->pcounter_len + 1) / 2;
  need += round256(H->ppartial_len) + round256(cnt_d) + 32;
  if (need > kStaticScratchDoubles) return HPS_ESCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HPS_ECUDA;
  if (!g_scratch_addr[dev]) {  // set-up on the first call on this device (before any stream capture)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_solve_scratch) != cudaSuccess || !p) return HPS_ECUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  double *base = g_scratch_addr[dev];
  // point the handle's work vectors into the static array for this call, then restore them
  double *saved_w = H->wleaf, *saved_partial = H->partial, *saved_pp = H->ppartial;
  unsigned *saved_cnt = H->pcounters, *saved_bar = H->pbar;
  int *saved_err = H->perr;
  double *saved_h[kMaxLevels], *saved_w3[kMaxLevels];
  size_t off = 0;
  H->wleaf = base + off;
  off += round256((size_t)H->g.N_int);
  for (int l = 0; l <= H->L; ++l) {
    saved_h[l] = H->h[l];
    H->h[l] = base + off;
    off += round256((size_t)H->lev[l].nodes * H->lev[l].nb);
    if (l < H->L) {
      saved_w3[l] = H->w3[l];
      H->w3[l] = base + off;
      off += round256((size_t)H->lev[l].nodes * H->lev[l].n3);
    }
  }
  H->partial = H->partial_len ? base + off : nullptr;
  off += round256(H->partial_len);
  H->ppartial = base + off;
  off += round256(H->ppartial_len);
  H->pcounters = reinterpret_cast<unsigned *>(base + off);
  off += round256(cnt_d);
  H->pbar = reinterpret_cast<unsigned *>(base + off);
  H->perr = reinterpret_cast<int *>(base + off + 16);
  off += 32;
  cudaStream_t st = (cudaStream_t)stream;
  // counters, barrier and error word must start at zero (they keep the last call's values)
  int e = HPS_OK;
  if (cudaMemsetAsync(H->pcounters, 0, round256(cnt_d) * sizeof(double) + 32 * sizeof(double), st) != cudaSuccess)
    e = HPS_ECUDA;
  if (e == HPS_OK) e = hps::set_boundary(H, u, f, st);
  if (e == HPS_OK) {
    hps::Combo c{};
    c.ptr[0] = rhs;
    c.coef[0] = 1.0;
    c.n = 1;
    e = hps::sweep(H, H->impl, c, nullptr, u, u, nullptr, st);
  }
  if (e == HPS_OK && H->persistent) {  // the bounded waits of the persistent merge kernel report here
    k_fold_error<<<1, 32, 0, st>>>(H->perr, saved_err);
    if (cudaPeekAtLastError() != cudaSuccess) e = HPS_ECUDA;
  }
  H->wleaf = saved_w;
  H->partial = saved_partial;
  H->ppartial = saved_pp;
  H->pcounters = saved_cnt;
  H->pbar = saved_bar;
  H->perr = saved_err;
  for (int l = 0; l <= H->L; ++l) {
    H->h[l] = saved_h[l];
    if (l < H->L) H->w3[l] = saved_w3[l];
  }
  return e;
}
