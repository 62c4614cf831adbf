// Internal declarations shared by the translation units of libhps.so.
// Layout conventions are those documented in include/hps.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hps.h"

namespace hps {

constexpr int kMaxP = 32;          // Chebyshev points per leaf side
constexpr int kMaxBd = 24576;      // largest box boundary (doubles staged in shared memory)
constexpr int kCombo = 16;         // terms of a right-hand-side linear combination

// Sizes of the global vector (include/hps.h ordering).
struct GridDims {
  int n1, n2, m, p;
  int64_t N_int, N_v, N_h, N, N_bd;
};

__host__ __device__ inline int64_t vseg(const GridDims &g, int line, int iy, int j0) {
  return g.N_int + ((int64_t)line * g.n2 + iy) * g.m + j0;
}
__host__ __device__ inline int64_t hseg(const GridDims &g, int line, int ix, int i0) {
  return g.N_int + g.N_v + ((int64_t)line * g.n1 + ix) * g.m + i0;
}

// Global index of position `pos` of the boundary of the a x c box at leaf (ix0, iy0);
// box order: south (ascending x), east (ascending y), north (ascending x), west (ascending y).
__host__ __device__ inline int64_t box_bd(const GridDims &g, int ix0, int iy0, int a, int c, int pos) {
  const int m = g.m, am = a * m, cm = c * m;
  if (pos < am) return hseg(g, iy0, ix0 + pos / m, pos % m);
  pos -= am;
  if (pos < cm) return vseg(g, ix0 + a, iy0 + pos / m, pos % m);
  pos -= cm;
  if (pos < am) return hseg(g, iy0 + c, ix0 + pos / m, pos % m);
  pos -= am;
  return vseg(g, ix0, iy0 + pos / m, pos % m);
}

// Global index of position `pos` of the interface a node's split creates.
__host__ __device__ inline int64_t iface_bd(const GridDims &g, int ix0, int iy0, int a, int c, int split, int pos) {
  const int m = g.m;
  if (split == 0) return vseg(g, ix0 + a / 2, iy0 + pos / m, pos % m);
  return hseg(g, iy0 + c / 2, ix0 + pos / m, pos % m);
}

// Kernel slots for launch counting and optional CUDA-event timing (hps_trace_*).
enum Slot {
  kLeafUp = 0, kMergeUpW3, kMergeUpH, kMergeDown, kLeafDown, kLeafEval, kSetBoundary, kMergeUpFused,
  kMergeDownFused, kResidual, kJump, kFinish, kClose, kNumSlots
};

constexpr int kMaxLevels = 32;
constexpr int kPThreads = 256;       // threads per CTA of the persistent merge kernel
constexpr int kPSmemDoubles = 4096;  // its vector staging (32 KB)
constexpr int kMaxSplit = 64;        // column chunks of one output tile (all merge paths)

// One mat-vec task of the persistent merge kernel (all nodes of one level, one operator kind).
struct MTask {
  int kind;  // 0: w3 = X d,  1: h = [h^a_1; h^b_2] + Tcat w3,  2: u3 = S u_b + w3 (scattered)
  int lvl;
  int M, K, nodes, npc, rows_cta, row_tiles, node_groups, ksplit, kchunk;
  int64_t items;
  const double *AT;
  int ld;
  int64_t str;
  int nbc, j3a, j3b, n3, nb;
  const int *hsrc;
  const int *origin;
  int a, c, split;
};

struct PArgs {
  const MTask *tasks;
  int ntasks;
  int selftest;
  double *h[kMaxLevels];
  double *w3[kMaxLevels];
  GridDims g;
  double *gvec;
  double *partial;
  unsigned *counters;
  unsigned *bar;  // [count, generation]
  int *err;
  unsigned long long limit_ns;
  unsigned long long *stamps;  // optional: globaltimer at the start of every task and at the end
};

// One level of the uniform binary tree (all boxes on a level have the same shape).
struct Level {
  int nodes = 0, a = 0, c = 0;
  int split = -1;     // 0: vertical cut (x), 1: horizontal cut (y), -1: leaf level
  int nb = 0;         // boundary points of a box on this level: 2(a+c)m
  int n3 = 0;         // interface points of the cut (merge levels)
  int nbc = 0;        // boundary points of a child box
  int j3a = 0, j3b = 0;  // offset of the interface in the alpha / beta child boundary
  int *d_origin = nullptr;  // nodes x (ix0, iy0)
  int *d_hsrc = nullptr;    // nb: parent boundary position -> child*nbc + position in child
  int *d_cmap = nullptr;    // 2 nbc: child*nbc + position -> parent position, or nb + interface position
  std::vector<int> origin, hsrc, cmap;
};

// Merge operators of one level, FP64, row-major, per node (stride) or shared (stride 0).
struct MergeOps {
  double *X = nullptr, *S = nullptr, *Tcat = nullptr;
  int ldX = 0, ldS = 0, ldT = 0;
  int64_t strX = 0, strS = 0, strT = 0;
};

struct OpSet {
  bool identity = false;
  double *Ainv = nullptr, *Sleaf = nullptr;
  int ldA = 0, ldSl = 0;
  int64_t strA = 0, strSl = 0;
  std::vector<MergeOps> merge;  // index = level (0 .. L-1)
  MTask *d_up = nullptr, *d_down = nullptr;  // persistent task lists
  int n_up = 0, n_down = 0;
};

// FP32 copy of an operator set (same layouts, leading dimensions and strides as the FP64 one).
struct Op32 {
  float *p = nullptr;
  int ld = 0;        // rows padded to a multiple of 4 floats (16-byte column loads)
  int64_t str = 0;   // per node, 0 when shared
};
struct OpSet32 {
  Op32 Ainv, Sleaf;
  std::vector<Op32> X, S, Tcat;  // per level
};

// Work buffers of one column group of the batched mixed-precision path (up to Rmax columns).
// Vectors with R columns are stored RHS-fastest: entry (point i, column j) at i*R + j.
struct BatchWork {
  int Rmax = 0;
  double *u = nullptr;  // the group's columns of the caller's u (grouped calls only)
  double *ustage = nullptr, *Rb = nullptr, *KL = nullptr, *KE = nullptr, *r = nullptr;  // FP64
  float *g32 = nullptr, *w32 = nullptr, *r32 = nullptr;
  std::vector<float *> h32, w332;  // per level
  float *partial32 = nullptr;
  size_t partial_len = 0;          // floats
  unsigned *tile_count = nullptr;  // split-K tiles: CTAs done (re-armed by the last one)
  size_t tile_count_len = 0;
  unsigned *flow_sync = nullptr;   // dataflow merge kernels: ticket counter + node flags
  size_t flow_len = 0;
  cudaStream_t stream = nullptr;   // grouped calls: the group's own stream
  cudaEvent_t done = nullptr;
  cudaEvent_t first = nullptr;     // grouped ARK steps: the explicit first stage is done
  double *slope = nullptr;         // batched slope form: kappa_1..6, J ([N][R] each), scaled f ([N_bd][R])
  size_t slope_len = 0;            // doubles
  double *slope_g = nullptr;       // ... with g: lambda_1..6, U ([N][R] each), gamma dt L lambda_1..6 ([N_int][R])
};

// The batched path: FP32 operator copies (shared by all groups) and G column groups.  With
// G > 1 the columns of a call are split into G groups that run on their own streams, so that
// one group's FP64 residual kernels (bound by the FP64 pipe) overlap another group's FP32
// sweeps (bound by the FP32 pipe and L2).
struct Batch {
  int Rmax = 0, groups = 1;
  int fp64_ctas_per_sm = 0;  // 0: one CTA per leaf; else a persistent grid of that many per SM
  int flow_levels = 0;       // lower merge levels run as one dataflow kernel (0: one launch per level)
  int flow_n3_max = 32;      // ... those with interfaces of at most this many points
  bool gemv2 = false;        // upper merge levels: in-CTA + cluster split-K (else split-K partials)
  bool even_odd = true;      // FP64 leaf kernels by the even-odd decomposition (even p)
  bool leaf_split = false;   // stage right-hand side as its own streaming pass before the leaf apply
  bool offset_groups = true; // grouped ARK steps: each group starts one phase after the previous
  int last_cta_max_split = 0;   // split-K sums by the last CTA of each tile up to this split depth (0: never)
  bool fast_diag = true;     // leaf apply by fast diagonalization where the handle has it
  bool fuse_epilogue = true;  // stage epilogue written by the last leaf kernel of the stage solve
  bool fuse_jump = true;      // residual: flux jumps from the even-odd leaf kernel (no k_b_jump)
  bool fold_scale = true;     // even-odd leaf kernels: scales folded into the half matrices
  bool sa_close = true;       // step close from the last stage value (stiffly accurate table)
  bool edge_projection = true;  // step close by per-line tridiagonal solves for the edge values
  int tile_cols_apply[3] = {0, 0, 0};  // w3, h, down applies: register-tile columns (0: plan_tile_cols)
  int eo_cols = 12;           // even-odd FP64 leaf kernels: columns per pass (3 CTAs per SM at p = 16)
  int plan_target = 2;       // split-K plans: CTAs per SM aimed at
  int plan_kmin = 32;        // split-K plans: smallest K chunk
  int plan_npc_max = 1 << 30;  // split-K plans: most nodes per CTA
  int plan_tile_cols = 2;    // merge applies: register-tile columns per thread (8, 4 or 2)
  bool tensor_leaf = true;   // shared leaf operator applied by 3xTF32 warp MMA (else FP32 FFMA)
  unsigned *afrag_hi = nullptr, *afrag_lo = nullptr;  // its TF32 fragments
  int umma_leaf = 1;         // per-node leaf operators on the tcgen05 tensor cores (3xTF32): 1 first sweep, 2 all;
                             // 3: BF16 trial (first sweep one BF16 product, refinement sweeps FP32 FFMA)
  float *ainv_k = nullptr;   // their TF32 hi / lo split, K-major: [leaf][hi, lo][row][ainv_ldk]
  int ainv_ldk = 0;
  uint64_t ainv_map[16] = {};  // its TMA tensor map (CUtensorMap, 128 bytes)
  bool one_column_merge = true; // per-node merge applies with one column streamed without staging
  bool one_column_merge_sum = true; // ... and their split-K sums by the last CTA (else k_b_reduce)
  int stream_leaf = 3;       // one to four columns: leaf operators streamed by bulk copies, CTAs per SM (0: off)
  int stream_chunk_kb = 24;  // ... in chunks of about this many KB
  int sub_levels = 0;        // lowest merge levels of the upward sweep fused per subtree (0: per level)
  bool pdl = false;          // merge applies launched as programmatic dependents of the kernel before
  bool prefetch_next = false;
  bool b1_roll = false;
  bool stream_prefetch = true;  // streaming downward leaf apply: per-leaf loads ahead of the products  // one-column merge applies: rolling operator loads
  int b1_kw = 8;         // one-column merge applies: most warps splitting K in a CTA  // merge applies prefetch the next apply's operator into L2
  int eo_threads = 0;        // threads per CTA of the FP64 even-odd leaf kernel (0: 128 for one column per pass, else 256)
  void *ainv_bf = nullptr;       // BF16 trial: their BF16 copy, K-major [leaf][row][round8(q)]
  uint64_t ainv_map_bf[16] = {}; // its TMA tensor map
  OpSet32 impl32, ident32;
  std::vector<BatchWork> work;
  cudaEvent_t fork = nullptr;
};

// A kernel sequence recorded into a CUDA graph (hps_set_graph), replayed for equal arguments.
struct GraphEntry {
  static constexpr int kKey = 8;
  static constexpr int kEventPairs = 1024;  // enough for every kernel of one batched ARK step
  bool seen = false;   // the key ran once eagerly (kernels loaded, attributes set)
  bool valid = false;  // exec holds the graph of this key
  uint64_t key[kKey] = {};
  cudaGraphExec_t exec = nullptr;
  int64_t launches[16] = {};         // launches per kernel slot in one replay (>= kNumSlots)
  std::vector<cudaEvent_t> ev;       // timing event pairs recorded inside the graph
  std::vector<int> ev_slot;
  int nev = 0;
  bool pending = false;              // the last replay's events are not read yet
  void destroy();
};

struct Trace {
  int64_t launches[kNumSlots] = {};
  int64_t timed[kNumSlots] = {};
  double ms[kNumSlots] = {};
  unsigned mask = 0;
  std::vector<cudaEvent_t> pool;   // pairs (start, end)
  std::vector<int> pair_slot;
  size_t used = 0;                 // pairs in flight
  int open_slot = -1;
  GraphEntry *capturing = nullptr; // set while a graph is being recorded
  void begin(int slot, cudaStream_t st);
  void end(int slot, cudaStream_t st);
  void drain();                    // synchronizes the recorded events, accumulates ms
  void release();
};

// Factored inverse of the constant-coefficient leaf operator (fastdiag.cu): V_x, V_x^-1, V_y,
// V_y^-1 and 1 / (c - gamma dt (lam_y + lam_x)), each m x mp (rows padded to a multiple of 4).
struct FastDiag {
  bool on = false;
  int mp = 0;
  double *d64 = nullptr;
  float *d32 = nullptr;
};

struct Combo {
  const double *ptr[kCombo];
  double coef[kCombo];
  int n;
};

}  // namespace hps

struct hps_handle {
  hps_tree tree;
  hps::GridDims g;
  int p, m, q, b, L;
  double hx, hy, gamma_dt;
  bool shared;
  int coef_kind;
  double cst[5];
  double *d_coef = nullptr;   // 5 x N_int (NODAL)
  double *d_D = nullptr;      // D1x, D1y, Dxx, Dyy: 4 p*p doubles, row-major
  // edge projection (step close): Thomas factors of the per-line tridiagonal systems,
  // [w_x, 1/b_x] (n1 - 1 each) then [w_y, 1/b_y] (n2 - 1 each); off-diagonals lo (v_{L-1}), up (v_{L+1})
  double *d_proj = nullptr;
  double proj_lo[2] = {0.0, 0.0}, proj_up[2] = {0.0, 0.0};
  hps::FastDiag fd;           // factored A_ii^-1 (constant coefficients)
  std::vector<hps::Level> lev;  // 0 (root) .. L (leaves)
  hps::OpSet impl, ident;
  // work buffers
  double *ustage = nullptr, *R = nullptr, *KL = nullptr, *KE = nullptr, *wleaf = nullptr;
  double *gbuf = nullptr;  // N_int: the caller's g of one stage (HPS_G_USER), allocated at first use
  std::vector<double *> h;    // per level: nodes x nb
  std::vector<double *> w3;   // per merge level: nodes x n3
  double *partial = nullptr;  // split-K partial sums of the merge applies
  size_t partial_len = 0;
  int num_sms = 0;
  std::vector<void *> allocs;
  hps::Trace trace;
  bool persistent = false;    // merge levels by the persistent kernel (else one launch per task)
  int fp64_plan_target = 3;   // FP64 merge applies: split columns until this many CTAs per SM
  double *host_stage = nullptr;  // device copy of the states of ark_step(_batch)_host
  size_t host_stage_len = 0;
  double *slope_k = nullptr;     // slope form: 6 scaled slopes (N each) and the interface right-hand side
  double *slope_l = nullptr;     // slope form with g: 6 explicit slopes, a stage value (N each), their dt L (6 N_int), scratch
  int pgrid = 0;              // its CTA count (co-resident)
  double *ppartial = nullptr; // its split-column partial sums
  size_t ppartial_len = 0;
  unsigned *pcounters = nullptr;  // last-CTA counters (self-resetting)
  size_t pcounter_len = 0;
  unsigned *pbar = nullptr;   // grid barrier [count, generation]
  int *perr = nullptr;        // bounded-wait error word
  unsigned long long *pstamps = nullptr;  // per-task time stamps (up: [0, 64), down: [64, 128))
  bool stamp_tasks = false;
  bool graph_mode = false;
  cudaStream_t cap_stream = nullptr;
  hps::GraphEntry g_ark, g_solve, g_ark_b, g_solve_b;
  hps::Batch batch;
};

namespace hps {

// ---- build (build.cu) --------------------------------------------------------------
int build_operators(hps_handle *H, OpSet &ops, double gamma_dt, bool identity, cudaStream_t st);

// ---- solve (sweep.cu) ----------------------------------------------------------------
struct Epilogue {          // fused ARK stage epilogue at the leaves (a5)
  double *KL = nullptr;    // dt L u_i = (u_i - R_i) / gamma
  double *KE = nullptr;    // dt (q_i + g(u_i))
  const double *Rsaved = nullptr;
  const double *q = nullptr;
  double inv_gamma = 0.0, dt = 0.0;
  int g_kind = 0;
  double gp0 = 0.0, gp1 = 0.0;
};

int sweep(hps_handle *H, const OpSet &ops, const Combo &rhs, double *Rsave, double *gvec,
          double *out_interior, const Epilogue *ep, cudaStream_t st, const double *jump = nullptr);
int set_boundary(hps_handle *H, double *gvec, const double *f, cudaStream_t st);
size_t partial_doubles(const hps_handle *H);  // split-K scratch the merge applies need
void drain_graph(hps_handle *H, GraphEntry &e);  // read the timing events of the last replay

// ---- persistent merge kernel (persistent.cu) ---------------------------------------------
int persistent_grid(hps_handle *H);
int build_tasks(hps_handle *H, OpSet &ops);
int merge_persistent(hps_handle *H, const OpSet &ops, bool upward, double *gvec, cudaStream_t st);
int selftest_barrier(hps_handle *H, cudaStream_t st);

// ---- handle services (api.cu) ----------------------------------------------------------------
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the CURRENT device (the
// attribute is per device; requests above 32 KB are raised explicitly, since the 48 KB default
// also has to hold the kernel's static shared memory).  Remembers the largest value set per (kernel, device) under a lock,
// so every host thread and every device gets the attribute before its first large launch.
// HPS_OK, or HPS_ECUDA when the runtime refuses the value.
int smem_optin(const void *kernel, size_t bytes);
int alloc_work(hps_handle *H, cudaStream_t st);
int clone_handle(const hps_handle *base, cudaStream_t st, hps_handle **out);
int bytes_split(const hps_tree *tree, int p, int coeff_kind, int flags, size_t *ops, size_t *work);

// ---- batched mixed-precision path (batched.cu) ---------------------------------------------
int fastdiag_build(hps_handle *H, const std::vector<double> &Dh, cudaStream_t st);
bool fastdiag_factor(int p, const double *Dh, const double *cst, double gdt, bool check_all,
                     std::vector<double> (&F)[5], double *max_err);
int batch_reserve(hps_handle *H, int R, int groups);
int batch_option(hps_handle *H, int opt, const int *set, int *get);
// edge projection of the step close (batched.cu): u interior = combination `c`, u boundary as
// given, shared-edge values from flux continuity; rhs: [N][R] scratch
int edge_projection(hps_handle *H, int R, const Combo &c, double *u, double *rhs, cudaStream_t st,
                    const double *J = nullptr);  // J: interface right-hand side (global vector) or null
// r = -(flux jump of u) at every shared-edge point, (west/south flux) - (east/north flux) negated
int flux_jump_rhs(hps_handle *H, int R, const double *u, double *r, cudaStream_t st);

int batch_autotune(hps_handle *H, int R, int refine, cudaStream_t st, hps_tune_result *res, int max_res, int *n_res);
void batch_release(hps_handle *H);
int solve_batch(hps_handle *H, int R, const double *rhs, const double *f, double *u, int refine, cudaStream_t st);
struct ArkTable {
  double A[6][6], Ah[6][6], b[6];
};
// one ARK step in slope form (g = 0, or a preset g with time-independent boundary data), FP64 (slope.cu)
int ark_slope(hps_handle *H, double *u, double dt, const hps_ark_terms *terms, const ArkTable &tb, cudaStream_t st);
int ark_slope_batch(hps_handle *H, int R, double *u, double dt, const hps_ark_terms *terms, int refine,
                    const ArkTable &tb, cudaStream_t st);
ArkTable ark_table();  // the method's ARK tables (api.cu)
int ark_batch_lockstep(hps_handle *const *h, int n, double *const *u, const int *R, const hps_ark_terms *terms,
                       double dt, int refine, const ArkTable &tb, cudaStream_t st, const cudaStream_t *sts,
                       const cudaEvent_t *evs, cudaEvent_t evm);
int ark_batch(hps_handle *H, int R, double *u, double dt, const hps_ark_terms *terms, int refine, const ArkTable &tb,
              cudaStream_t st);
int leaf_eval(hps_handle *H, const double *u, double *KL, double *KE, const double *q, double dt,
              int g_kind, double gp0, double gp1, cudaStream_t st);

}  // namespace hps
