// Batched mixed-precision path: R right-hand sides per sweep, FP32 applies, FP64 refinement.
//
// Every implicit stage solve A u = b (eq. ``sparse_A``) is done as
//   u = solve32(b);  repeat `refine` times:  r = b - A u (FP64);  u += solve32(r)
// where solve32 is the HPS sweep with FP32 operators, FP32 work vectors and FP32
// accumulation, and the residual is formed in FP64 against the leaf collocation operators
// (interior rows: R - (u - gamma dt L u) by leaf-local differentiation; shared-edge rows: the
// flux jump, entered in the sweep as the right-hand side of the interface equations).
// Vectors with R columns are stored RHS-fastest (point i, column j at i*R + j); the FP32
// applies compute 4 columns per thread from one operator load.
#include <algorithm>

#include "hps_internal.cuh"

namespace hps {

namespace {

constexpr int kBT = 256;
constexpr int kBSmemFloats = 8192;  // vector staging of the merge applies (32 KB)

__host__ __device__ inline int round4(int r) { return (r + 3) & ~3; }

// flux (D_bi w)_e of column j of an interior field W[node*Rp + j] (float)
__device__ float flux32(int e, int j, int Rp, const float *W, const float *D1x, const float *D1y, int p, int m) {
  const int side = e / m, t = e % m;
  float s = 0.f;
  if (side == 0 || side == 2) {
    const float *d = D1y + (side == 0 ? 0 : (p - 1) * p);
    for (int jj = 1; jj <= m; ++jj) s = fmaf(d[jj], W[((jj - 1) * m + t) * Rp + j], s);
  } else {
    const float *d = D1x + (side == 1 ? (p - 1) * p : 0);
    for (int ii = 1; ii <= m; ++ii) s = fmaf(d[ii], W[(t * m + ii - 1) * Rp + j], s);
  }
  return s;
}

// ---- leaf applies (FP32, R columns) ------------------------------------------------------
// Register tile per thread: 4 consecutive rows (one 16-byte operator load per column of the
// transposed operator) x TC columns of the right-hand sides (TC/4 16-byte shared loads).

template <int TC>
__device__ __forceinline__ void tile_fma(float (&acc)[4][TC], const float4 a, const float *x) {
  float xv[TC];
#pragma unroll
  for (int t = 0; t < TC; t += 4) {
    const float4 v = *reinterpret_cast<const float4 *>(x + t);
    xv[t] = v.x; xv[t + 1] = v.y; xv[t + 2] = v.z; xv[t + 3] = v.w;
  }
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    acc[0][t] = fmaf(a.x, xv[t], acc[0][t]);
    acc[1][t] = fmaf(a.y, xv[t], acc[1][t]);
    acc[2][t] = fmaf(a.z, xv[t], acc[2][t]);
    acc[3][t] = fmaf(a.w, xv[t], acc[3][t]);
  }
}

template <int TC>
__global__ void __launch_bounds__(kBT) k_b_leaf_up(GridDims g, int R, const int *__restrict__ origin, Combo rhs,
                                                   double *__restrict__ Rsave, const float *__restrict__ AinvT,
                                                   int ldA, int64_t strA, int identity, const double *__restrict__ Dg,
                                                   float *__restrict__ w32, float *__restrict__ h32) {
  extern __shared__ float smf[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, Rp = round4(R);
  float *D1x = smf, *D1y = smf + p * p, *Rs = smf + round4(2 * p * p), *Ws = Rs + q * Rp;
  const int k = blockIdx.x;
  const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) smf[i] = (float)Dg[i];
  for (int idx = threadIdx.x; idx < q * Rp; idx += blockDim.x) {
    const int r = idx / Rp, j = idx % Rp;
    double v = 0.0;
    if (j < R) {
      for (int t = 0; t < rhs.n; ++t) v = fma(rhs.coef[t], rhs.ptr[t][(l0 + r) * R + j], v);
      if (Rsave) Rsave[(l0 + r) * R + j] = v;
    }
    Rs[idx] = (float)v;
  }
  __syncthreads();
  const int QQ = (q + 3) / 4, CG = Rp / TC;
  for (int it = threadIdx.x; it < QQ * CG; it += blockDim.x) {
    const int r0 = 4 * (it % QQ), j0 = TC * (it / QQ);
    float acc[4][TC];
    if (identity) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[e][t] = r0 + e < q ? Rs[(r0 + e) * Rp + j0 + t] : 0.f;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
      const float *a = AinvT + (int64_t)k * strA + r0;
#pragma unroll 2
      for (int c = 0; c < q; ++c)
        tile_fma<TC>(acc, __ldg(reinterpret_cast<const float4 *>(a + (int64_t)c * ldA)), Rs + c * Rp + j0);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (r0 + e < q)
#pragma unroll
        for (int t = 0; t < TC; ++t) Ws[(r0 + e) * Rp + j0 + t] = acc[e][t];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * R; idx += blockDim.x) {
    const int r = idx / R, j = idx % R;
    w32[((int64_t)k * q + r) * R + j] = Ws[r * Rp + j];
  }
  for (int idx = threadIdx.x; idx < b * R; idx += blockDim.x) {
    const int e = idx / R, j = idx % R;
    h32[((int64_t)k * b + e) * R + j] = flux32(e, j, Rp, Ws, D1x, D1y, p, m);
  }
}

template <int TC>
__global__ void __launch_bounds__(kBT) k_b_leaf_down(GridDims g, int R, const int *__restrict__ origin,
                                                     const float *__restrict__ SlT, int ldS, int64_t strS, int identity,
                                                     const float *__restrict__ w32, float *__restrict__ g32) {
  extern __shared__ float ub[];  // [b][Rp]
  const int m = g.m, q = m * m, b = 4 * m, Rp = round4(R);
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int idx = threadIdx.x; idx < b * Rp; idx += blockDim.x) {
    const int e = idx / Rp, j = idx % Rp;
    ub[idx] = j < R ? g32[box_bd(g, ix, iy, 1, 1, e) * R + j] : 0.f;
  }
  __syncthreads();
  const int QQ = (q + 3) / 4, CG = Rp / TC;
  for (int it = threadIdx.x; it < QQ * CG; it += blockDim.x) {
    const int r0 = 4 * (it % QQ), j0 = TC * (it / QQ);
    float acc[4][TC];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
    if (!identity) {
      const float *a = SlT + (int64_t)k * strS + r0;
#pragma unroll 2
      for (int c = 0; c < b; ++c)
        tile_fma<TC>(acc, __ldg(reinterpret_cast<const float4 *>(a + (int64_t)c * ldS)), ub + c * Rp + j0);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + e;
      if (r >= q) continue;
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        const int j = j0 + t;
        if (j < R) g32[(l0 + r) * R + j] = w32[((int64_t)k * q + r) * R + j] + acc[e][t];
      }
    }
  }
}

// Narrow variants (R <= 4) for streaming per-leaf operators: the columns of the operator are
// split over KS thread slices per row quad so that a whole CTA keeps 16-byte loads in flight;
// the slices are added in a fixed order through shared memory.
__device__ __forceinline__ void quad_apply_sliced(const float *a, int ld, int K, const float *x, int Rp, int QQ,
                                                  int KS, float *part /*[KS][4*QQ][4]*/) {
  for (int t = threadIdx.x; t < QQ * KS; t += blockDim.x) {
    const int rq = t % QQ, ks = t / QQ;
    const int c0 = (int)((int64_t)K * ks / KS), c1 = (int)((int64_t)K * (ks + 1) / KS);
    float acc[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[e][u] = 0.f;
    const float *ar = a + 4 * rq;
#pragma unroll 8
    for (int c = c0; c < c1; ++c) tile_fma<4>(acc, __ldg(reinterpret_cast<const float4 *>(ar + (int64_t)c * ld)), x + c * Rp);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      *reinterpret_cast<float4 *>(part + ((int64_t)ks * 4 * QQ + 4 * rq + e) * 4) =
          make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
  }
}

__global__ void __launch_bounds__(kBT) k_b_leaf_up_narrow(GridDims g, int R, const int *__restrict__ origin,
                                                          Combo rhs, double *__restrict__ Rsave,
                                                          const float *__restrict__ AinvT, int ldA, int64_t strA,
                                                          int identity, const double *__restrict__ Dg,
                                                          float *__restrict__ w32, float *__restrict__ h32) {
  extern __shared__ float smf[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, QQ = (q + 3) / 4, KS = max(1, kBT / QQ);
  float *D1x = smf, *D1y = smf + p * p, *Rs = smf + round4(2 * p * p), *Ws = Rs + 4 * q, *part = Ws + 4 * q;
  const int k = blockIdx.x;
  const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) smf[i] = (float)Dg[i];
  for (int idx = threadIdx.x; idx < q * 4; idx += blockDim.x) {
    const int r = idx / 4, j = idx % 4;
    double v = 0.0;
    if (j < R) {
      for (int t = 0; t < rhs.n; ++t) v = fma(rhs.coef[t], rhs.ptr[t][(l0 + r) * R + j], v);
      if (Rsave) Rsave[(l0 + r) * R + j] = v;
    }
    Rs[idx] = (float)v;
  }
  __syncthreads();
  if (identity) {
    for (int idx = threadIdx.x; idx < q * 4; idx += blockDim.x) Ws[idx] = Rs[idx];
  } else {
    quad_apply_sliced(AinvT + (int64_t)k * strA, ldA, q, Rs, 4, QQ, KS, part);
    __syncthreads();
    for (int idx = threadIdx.x; idx < q * 4; idx += blockDim.x) {
      float s = 0.f;
      for (int ks = 0; ks < KS; ++ks) s += part[(int64_t)ks * 16 * QQ + idx];
      Ws[idx] = s;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * R; idx += blockDim.x) {
    const int r = idx / R, j = idx % R;
    w32[((int64_t)k * q + r) * R + j] = Ws[r * 4 + j];
  }
  for (int idx = threadIdx.x; idx < b * R; idx += blockDim.x) {
    const int e = idx / R, j = idx % R;
    h32[((int64_t)k * b + e) * R + j] = flux32(e, j, 4, Ws, D1x, D1y, p, m);
  }
}

__global__ void __launch_bounds__(kBT) k_b_leaf_down_narrow(GridDims g, int R, const int *__restrict__ origin,
                                                            const float *__restrict__ SlT, int ldS, int64_t strS,
                                                            int identity, const float *__restrict__ w32,
                                                            float *__restrict__ g32) {
  extern __shared__ float smf[];
  const int m = g.m, q = m * m, b = 4 * m, QQ = (q + 3) / 4, KS = max(1, kBT / QQ);
  float *ub = smf, *part = smf + 4 * b;
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int idx = threadIdx.x; idx < b * 4; idx += blockDim.x) {
    const int e = idx / 4, j = idx % 4;
    ub[idx] = j < R ? g32[box_bd(g, ix, iy, 1, 1, e) * R + j] : 0.f;
  }
  __syncthreads();
  if (!identity) quad_apply_sliced(SlT + (int64_t)k * strS, ldS, b, ub, 4, QQ, KS, part);
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * R; idx += blockDim.x) {
    const int r = idx / R, j = idx % R;
    float s = w32[((int64_t)k * q + r) * R + j];
    if (!identity)
      for (int ks = 0; ks < KS; ++ks) s += part[(int64_t)ks * 16 * QQ + r * 4 + j];
    g32[(l0 + r) * R + j] = s;
  }
}

// ---- merge applies (FP32, R columns) -------------------------------------------------------
struct BPlan {
  int M, K, nodes, R, Rp, TC, MQ, CG;
  int npc, quads_cta, row_tiles, node_groups, ksplit, kchunk;
};

BPlan plan_b(int M, int K, int nodes, int R, int target) {
  BPlan P;
  P.M = M;
  P.K = K;
  P.nodes = nodes;
  P.R = R;
  P.Rp = round4(R);
  P.TC = P.Rp % 8 == 0 ? 8 : 4;
  P.MQ = (M + 3) / 4;
  P.CG = P.Rp / P.TC;
  const int per = P.MQ * P.CG;
  if (per <= kBT / 2) {
    P.npc = std::max(1, std::min(nodes, kBT / per));
    P.quads_cta = P.MQ;
    P.row_tiles = 1;
  } else {
    P.npc = 1;
    P.quads_cta = std::max(1, kBT / P.CG);
    P.row_tiles = (P.MQ + P.quads_cta - 1) / P.quads_cta;
  }
  P.node_groups = (nodes + P.npc - 1) / P.npc;
  const int base = P.node_groups * P.row_tiles;
  int ks = 1;
  if (base < target) ks = std::min({(target + base - 1) / base, std::max(1, K / 32), kMaxSplit});
  P.kchunk = (K + ks - 1) / ks;
  while ((int64_t)P.npc * P.kchunk * P.Rp > kBSmemFloats) P.kchunk = (P.kchunk + 1) / 2;
  P.ksplit = (K + P.kchunk - 1) / P.kchunk;
  return P;
}

struct BXDiff {  // d = h^b_3 - h^a_3 (+ interface right-hand side)
  const float *hC;
  int nbc, j3a, j3b, R;
  const double *jump;
  GridDims g;
  const int *origin;
  int a, c, split;
  __device__ float operator()(int k, int cc, int j) const {
    float v = hC[((int64_t)(2 * k + 1) * nbc + j3b + cc) * R + j] - hC[((int64_t)(2 * k) * nbc + j3a + cc) * R + j];
    if (jump) v += (float)jump[iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, cc) * R + j];
    return v;
  }
};
struct BXVec {
  const float *v;
  int n, R;
  __device__ float operator()(int k, int c, int j) const { return v[((int64_t)k * n + c) * R + j]; }
};
struct BXBd {
  GridDims g;
  const int *origin;
  int a, c, R;
  const float *gv;
  __device__ float operator()(int k, int pos, int j) const {
    return gv[box_bd(g, origin[2 * k], origin[2 * k + 1], a, c, pos) * R + j];
  }
};
struct BEStore {
  float *out;
  int n, R;
  __device__ void operator()(int k, int r, int j, float v) const { out[((int64_t)k * n + r) * R + j] = v; }
};
struct BEFlux {
  const int *hsrc;
  const float *hC;
  int nbc, nb, R;
  float *h;
  __device__ void operator()(int k, int r, int j, float v) const {
    h[((int64_t)k * nb + r) * R + j] = hC[((int64_t)(2 * k) * nbc + hsrc[r]) * R + j] + v;
  }
};
struct BEScatter {
  GridDims g;
  const int *origin;
  int a, c, split, n3, R;
  const float *w3;
  float *gv;
  __device__ void operator()(int k, int r, int j, float v) const {
    gv[iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r) * R + j] = v + w3[((int64_t)k * n3 + r) * R + j];
  }
};

template <int TC, class XL, class EP>
__global__ void __launch_bounds__(kBT) k_b_gemv(BPlan P, const float *__restrict__ AT, int ld, int64_t str, XL xl,
                                                EP ep, float *__restrict__ partial) {
  extern __shared__ float xs[];  // [nn][klen][Rp]
  const int ng = blockIdx.x / P.row_tiles, tile = blockIdx.x % P.row_tiles;
  const int node0 = ng * P.npc, nn = min(P.npc, P.nodes - node0);
  const int ks = blockIdx.y, c0 = ks * P.kchunk, klen = min(P.kchunk, P.K - c0);
  const int Rp = P.Rp;
  for (int idx = threadIdx.x; idx < nn * klen * Rp; idx += blockDim.x) {
    const int lo = idx / (klen * Rp), rem = idx % (klen * Rp), c = rem / Rp, j = rem % Rp;
    xs[idx] = j < P.R ? xl(node0 + lo, c0 + c, j) : 0.f;
  }
  __syncthreads();
  int lo, rq, cg;
  if (P.npc > 1) {
    const int per = P.MQ * P.CG;
    lo = threadIdx.x / per;
    const int rem = threadIdx.x % per;
    cg = rem / P.MQ;
    rq = rem % P.MQ;
    if (lo >= nn) return;
  } else {
    lo = 0;
    cg = threadIdx.x / P.quads_cta;
    rq = tile * P.quads_cta + threadIdx.x % P.quads_cta;
    if (cg >= P.CG || rq >= P.MQ) return;
  }
  const int k = node0 + lo, r0 = 4 * rq, j0 = TC * cg;
  const float *a = AT + (int64_t)k * str + (int64_t)c0 * ld + r0;
  const float *x = xs + (int64_t)lo * klen * Rp + j0;
  float acc[4][TC];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
#pragma unroll 4
  for (int c = 0; c < klen; ++c)
    tile_fma<TC>(acc, __ldg(reinterpret_cast<const float4 *>(a + (int64_t)c * ld)), x + c * Rp);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = r0 + e;
    if (r >= P.M) continue;
    if (P.ksplit == 1) {
#pragma unroll
      for (int t = 0; t < TC; ++t)
        if (j0 + t < P.R) ep(k, r, j0 + t, acc[e][t]);
    } else {
      float *dst = partial + (((int64_t)ks * P.nodes + k) * P.M + r) * Rp + j0;
#pragma unroll
      for (int t = 0; t < TC; t += 4)
        *reinterpret_cast<float4 *>(dst + t) = make_float4(acc[e][t], acc[e][t + 1], acc[e][t + 2], acc[e][t + 3]);
    }
  }
}

template <class EP>
__global__ void k_b_reduce(BPlan P, const float *__restrict__ partial, EP ep) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)P.nodes * P.M * P.R) return;
  const int j = (int)(idx % P.R);
  const int64_t kr = idx / P.R;
  const int r = (int)(kr % P.M), k = (int)(kr / P.M);
  float s = 0.f;
#pragma unroll 8
  for (int ks = 0; ks < P.ksplit; ++ks) s += partial[(((int64_t)ks * P.nodes + k) * P.M + r) * P.Rp + j];
  ep(k, r, j, s);
}

template <class XL, class EP>
int launch_b(hps_handle *H, int slot, const BPlan &P, const float *AT, int ld, int64_t str, XL xl, EP ep,
             cudaStream_t st) {
  const size_t smem = (size_t)P.npc * P.kchunk * P.Rp * sizeof(float);
  if (P.ksplit > 1 && (size_t)P.ksplit * P.nodes * P.M * P.Rp > H->batch.partial_len) return HPS_EINVAL;
  H->trace.begin(slot, st);
  const dim3 grid(P.node_groups * P.row_tiles, P.ksplit);
  if (P.TC == 8)
    k_b_gemv<8, XL, EP><<<grid, kBT, smem, st>>>(P, AT, ld, str, xl, ep, H->batch.partial32);
  else
    k_b_gemv<4, XL, EP><<<grid, kBT, smem, st>>>(P, AT, ld, str, xl, ep, H->batch.partial32);
  if (P.ksplit > 1) {
    const int64_t n = (int64_t)P.nodes * P.M * P.R;
    k_b_reduce<EP><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, H->batch.partial32, ep);
  }
  H->trace.end(slot, st);
  return HPS_OK;
}

// ---- FP64 leaf kernels: residual, stage epilogue, explicit first stage ---------------------
enum { kResid = 0, kEpilogue = 1, kEval = 2 };

struct Leaf64Args {
  int mode, R;
  const double *u;      // [N][R]
  const double *Rb;     // [N_int][R] stage right-hand side (kResid, kEpilogue)
  double *out0, *out1;  // kResid: r; kEpilogue / kEval: KL, KE
  const double *q;      // [N_int][R] or null
  const double *coef;   // 5 x N_int or null (constants in cst)
  double cst[5];
  int64_t N_int;
  double gdt, inv_gamma, dt;
  int g_kind;
  double gp0, gp1;
  int need_d1, need_d2;  // first / second derivatives needed (zero terms are skipped)
};

__global__ void __launch_bounds__(kBT) k_b_leaf64(GridDims g, const int *__restrict__ origin, Leaf64Args A,
                                                  const double *__restrict__ Dg) {
  extern __shared__ double sd[];
  const int p = g.p, m = g.m, q = m * m, pp = p * p, R = A.R;
  const int Rc = max(1, min(R, 4096 / pp));
  double *D1x = sd, *D1y = sd + pp, *Dxx = sd + 2 * pp, *Dyy = sd + 3 * pp, *U = sd + 4 * pp;  // U [pp][Rc]
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int i = threadIdx.x; i < 4 * pp; i += blockDim.x) sd[i] = Dg[i];
  for (int j0 = 0; j0 < R; j0 += Rc) {
    const int rc = min(Rc, R - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < pp * rc; idx += blockDim.x) {
      const int node = idx / rc, jj = idx % rc;
      const int i = node % p, j = node / p;
      const bool ei = (i == 0 || i == p - 1), ej = (j == 0 || j == p - 1);
      double v = 0.0;
      int64_t gi = -1;
      if (!ei && !ej) gi = l0 + (j - 1) * m + (i - 1);
      else if (ei && !ej) gi = vseg(g, ix + (i == 0 ? 0 : 1), iy, j - 1);
      else if (!ei && ej) gi = hseg(g, iy + (j == 0 ? 0 : 1), ix, i - 1);
      if (gi >= 0) v = A.u[gi * R + j0 + jj];
      U[node * Rc + jj] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < q * rc; idx += blockDim.x) {
      const int rr = idx / rc, jj = idx % rc;
      const int i = rr % m + 1, j = rr / m + 1;
      const int64_t gi = l0 + rr;
      const int col = j0 + jj;
      const double uu = U[(j * p + i) * Rc + jj];
      double ux = 0.0, uy = 0.0, uxx = 0.0, uyy = 0.0;
      if (A.need_d1 || A.need_d2) {
        for (int kk = 0; kk < p; ++kk) {
          const double vx = U[(j * p + kk) * Rc + jj], vy = U[(kk * p + i) * Rc + jj];
          if (A.need_d1) {
            ux = fma(D1x[i * p + kk], vx, ux);
            uy = fma(D1y[j * p + kk], vy, uy);
          }
          if (A.need_d2) {
            uxx = fma(Dxx[i * p + kk], vx, uxx);
            uyy = fma(Dyy[j * p + kk], vy, uyy);
          }
        }
      }
      const int64_t o = gi * R + col;
      double Lu = 0.0;
      if (A.mode != kEpilogue) {
        double c[5];
        for (int t = 0; t < 5; ++t) c[t] = A.coef ? A.coef[t * A.N_int + gi] : A.cst[t];
        Lu = c[0] * uxx + c[1] * uyy + c[2] * ux + c[3] * uy + c[4] * uu;
      }
      if (A.mode == kResid) {
        A.out0[o] = A.Rb[o] - (uu - A.gdt * Lu);
      } else {
        double e;
        switch (A.g_kind) {
          case HPS_G_ALLEN_CAHN: e = A.gp0 * (uu - uu * uu * uu); break;
          case HPS_G_FISHER: e = A.gp0 * uu * (1.0 - uu); break;
          case HPS_G_BURGERS: e = -uu * (A.gp0 * ux + A.gp1 * uy); break;
          default: e = 0.0;
        }
        if (A.q) e += A.q[o];
        A.out0[o] = A.mode == kEval ? A.dt * Lu : (uu - A.Rb[o]) * A.inv_gamma;
        A.out1[o] = A.dt * e;
      }
    }
  }
}

// The modes without derivatives (stage epilogue of a g without derivatives; residual of the
// identity operator) touch interior points only, which are contiguous: one flat pass.
__global__ void k_b_pointwise(int64_t n, Leaf64Args A) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const double uu = A.u[o];
  if (A.mode == kResid) {  // gamma dt = 0
    A.out0[o] = A.Rb[o] - uu;
    return;
  }
  double e;
  switch (A.g_kind) {
    case HPS_G_ALLEN_CAHN: e = A.gp0 * (uu - uu * uu * uu); break;
    case HPS_G_FISHER: e = A.gp0 * uu * (1.0 - uu); break;
    default: e = 0.0;
  }
  if (A.q) e += A.q[o];
  A.out0[o] = (uu - A.Rb[o]) * A.inv_gamma;
  A.out1[o] = A.dt * e;
}

// r = -(flux from the west/south leaf - flux from the east/north leaf) at every shared edge point
__global__ void k_b_jump(GridDims g, int R, const double *__restrict__ u, double *__restrict__ r,
                         const double *__restrict__ Dg) {
  const int p = g.p, m = g.m, q = m * m;
  const double *D1x = Dg, *D1y = Dg + p * p;
  const int64_t nv = (int64_t)(g.n1 - 1) * g.n2 * m, nh = (int64_t)(g.n2 - 1) * g.n1 * m;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (nv + nh) * R) return;
  const int col = (int)(idx % R);
  int64_t pt = idx / R;
  double fa = 0.0, fb = 0.0;
  int64_t gi;
  if (pt < nv) {  // vertical line L = 1..n1-1, leaf row iy, node jn
    const int jn = (int)(pt % m) + 1;
    const int64_t s = pt / m;
    const int iy = (int)(s % g.n2), L = (int)(s / g.n2) + 1;
    gi = vseg(g, L, iy, jn - 1);
    const int64_t lw = ((int64_t)iy * g.n1 + (L - 1)) * q, le = ((int64_t)iy * g.n1 + L) * q;
    for (int k = 0; k < p; ++k) {
      const int64_t iw = k == 0 ? vseg(g, L - 1, iy, jn - 1) : k == p - 1 ? gi : lw + (jn - 1) * m + (k - 1);
      const int64_t ie = k == 0 ? gi : k == p - 1 ? vseg(g, L + 1, iy, jn - 1) : le + (jn - 1) * m + (k - 1);
      fa = fma(D1x[(p - 1) * p + k], u[iw * R + col], fa);
      fb = fma(D1x[k], u[ie * R + col], fb);
    }
  } else {  // horizontal line L = 1..n2-1, leaf column ix, node in
    pt -= nv;
    const int in = (int)(pt % m) + 1;
    const int64_t s = pt / m;
    const int ix = (int)(s % g.n1), L = (int)(s / g.n1) + 1;
    gi = hseg(g, L, ix, in - 1);
    const int64_t ls = ((int64_t)(L - 1) * g.n1 + ix) * q, ln = ((int64_t)L * g.n1 + ix) * q;
    for (int k = 0; k < p; ++k) {
      const int64_t is = k == 0 ? hseg(g, L - 1, ix, in - 1) : k == p - 1 ? gi : ls + (k - 1) * m + (in - 1);
      const int64_t inn = k == 0 ? gi : k == p - 1 ? hseg(g, L + 1, ix, in - 1) : ln + (k - 1) * m + (in - 1);
      fa = fma(D1y[(p - 1) * p + k], u[is * R + col], fa);
      fb = fma(D1y[k], u[inn * R + col], fb);
    }
  }
  r[gi * R + col] = -(fa - fb);
}

// compact boundary position of global point gi, or -1 if gi is not on the outer boundary
__device__ __forceinline__ int64_t bd_pos(const GridDims &g, int64_t gi) {
  const int64_t nv = (int64_t)g.n2 * g.m, nh = (int64_t)g.n1 * g.m;
  if (gi < g.N_int) return -1;
  if (gi < g.N_int + g.N_v) {
    const int64_t off = gi - g.N_int;
    const int64_t line = off / nv;
    if (line == 0) return off;
    if (line == g.n1) return nv + (off - (int64_t)g.n1 * nv);
    return -1;
  }
  const int64_t off = gi - g.N_int - g.N_v;
  const int64_t line = off / nh;
  if (line == 0) return 2 * nv + off;
  if (line == g.n2) return 2 * nv + nh + (off - (int64_t)g.n2 * nh);
  return -1;
}

__global__ void k_b_set_boundary32(GridDims g, int R, float *__restrict__ g32, const double *__restrict__ f) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.N_bd * R) return;
  const int64_t kk = idx / R;
  const int j = (int)(idx % R);
  const int64_t nv = (int64_t)g.n2 * g.m, nh = (int64_t)g.n1 * g.m;
  int64_t gi;
  if (kk < nv) gi = g.N_int + kk;
  else if (kk < 2 * nv) gi = g.N_int + (int64_t)g.n1 * nv + (kk - nv);
  else if (kk < 2 * nv + nh) gi = g.N_int + g.N_v + (kk - 2 * nv);
  else gi = g.N_int + g.N_v + (int64_t)g.n2 * nh + (kk - 2 * nv - nh);
  g32[gi * R + j] = f ? (float)f[idx] : 0.f;
}

// u (FP64) from the FP32 sweep result: assign or add; interior points optionally; shared-edge
// points always; outer-boundary points set to f exactly (assign) or left alone (add).
__global__ void k_b_finish(GridDims g, int R, const float *__restrict__ g32, double *__restrict__ u, int assign,
                           int interior, const double *__restrict__ f) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.N * R) return;
  const int64_t gi = idx / R;
  if (gi < g.N_int) {
    if (!interior) return;
    u[idx] = assign ? (double)g32[idx] : u[idx] + (double)g32[idx];
    return;
  }
  const int64_t kk = bd_pos(g, gi);
  if (kk >= 0) {
    if (assign) u[idx] = f ? f[kk * R + idx % R] : 0.0;
    return;
  }
  u[idx] = assign ? (double)g32[idx] : u[idx] + (double)g32[idx];
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- host orchestration --------------------------------------------------------------------
__global__ void k_relayout(const double *__restrict__ src, int ld64, int64_t str64, int rows, int cols, int64_t nops,
                           float *__restrict__ dst, int ld32) {
  const int64_t total = nops * cols * (int64_t)ld32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / ((int64_t)cols * ld32);
    const int64_t rem = i % ((int64_t)cols * ld32);
    const int c = (int)(rem / ld32), r = (int)(rem % ld32);
    dst[i] = r < rows ? (float)src[node * str64 + (int64_t)c * ld64 + r] : 0.f;
  }
}

// FP32 copy of a transposed operator (rows x cols per node) with rows padded to 4 floats.
int convert_op(hps_handle *H, const double *src, int ld64, int64_t str64, int rows, int cols, int64_t nops, Op32 &o) {
  if (!src) return HPS_OK;
  o.ld = round4(rows);
  o.str = nops > 1 || str64 ? (int64_t)cols * o.ld : 0;
  const int64_t total = std::max<int64_t>(1, nops) * cols * (int64_t)o.ld;
  if (cudaMalloc(&o.p, total * sizeof(float)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(o.p);
  k_relayout<<<(unsigned)std::min<int64_t>(8192, (total + 255) / 256), 256>>>(src, ld64, str64, rows, cols,
                                                                              std::max<int64_t>(1, nops), o.p, o.ld);
  return HPS_OK;
}

int convert_opset(hps_handle *H, const OpSet &ops, OpSet32 &o32, bool shared) {
  const int L = H->L, q = H->q, b = H->b;
  const int64_t nleaf = shared ? 1 : H->lev[L].nodes;
  if (!ops.identity) {
    if (int e = convert_op(H, ops.Ainv, ops.ldA, ops.strA, q, q, nleaf, o32.Ainv)) return e;
    if (int e = convert_op(H, ops.Sleaf, ops.ldSl, ops.strSl, q, b, nleaf, o32.Sleaf)) return e;
  }
  o32.X.assign(L, Op32());
  o32.S.assign(L, Op32());
  o32.Tcat.assign(L, Op32());
  for (int l = 0; l < L; ++l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const int64_t nops = shared ? 1 : lv.nodes;
    if (int e = convert_op(H, mo.X, mo.ldX, mo.strX, lv.n3, lv.n3, nops, o32.X[l])) return e;
    if (int e = convert_op(H, mo.S, mo.ldS, mo.strS, lv.n3, lv.nb, nops, o32.S[l])) return e;
    if (l > 0)
      if (int e = convert_op(H, mo.Tcat, mo.ldT, mo.strT, lv.nb, lv.n3, nops, o32.Tcat[l])) return e;
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

size_t partial_floats(hps_handle *H, int R) {
  size_t mx = 0;
  for (int l = 0; l < H->L; ++l) {
    const Level &lv = H->lev[l];
    const BPlan P[3] = {plan_b(lv.n3, lv.n3, lv.nodes, R, 2 * H->num_sms), plan_b(lv.nb, lv.n3, lv.nodes, R, 2 * H->num_sms),
                        plan_b(lv.n3, lv.nb, lv.nodes, R, 2 * H->num_sms)};
    for (const BPlan &pl : P)
      if (pl.ksplit > 1) mx = std::max(mx, (size_t)pl.ksplit * pl.nodes * pl.M * pl.Rp);
  }
  return mx;
}

// One FP32 sweep on R columns: leaf applies, merges up (with an optional FP64 interface
// right-hand side), merges down into g32 (whose outer boundary the caller has set), leaf solves.
int sweep32(hps_handle *H, const OpSet &ops, const OpSet32 &o32, int R, const Combo &rhs, double *Rsave,
            const double *jump, cudaStream_t st) {
  Batch &B = H->batch;
  const int L = H->L, p = H->p, q = H->q, b = H->b, Rp = round4(R);
  const Level &leaf = H->lev[L];
  const int target = 2 * H->num_sms;
  const bool tc8 = Rp % 8 == 0;
  const bool narrow = Rp == 4 && !H->shared;  // streaming per-leaf operators, one column group
  const int QQ = (q + 3) / 4, KS = std::max(1, kBT / QQ);
  if (narrow) {
    const size_t smem = (size_t)(round4(2 * p * p) + 8 * q + KS * 16 * QQ) * sizeof(float);
    static size_t set = 0;
    if (smem > 48 * 1024 && smem > set) {
      cudaFuncSetAttribute(k_b_leaf_up_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      set = smem;
    }
    H->trace.begin(kLeafUp, st);
    k_b_leaf_up_narrow<<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, o32.Ainv.p, o32.Ainv.ld,
                                                      o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
    H->trace.end(kLeafUp, st);
  } else {
    const size_t smem = (size_t)(round4(2 * p * p) + 2 * q * Rp) * sizeof(float);
    static size_t set = 0;
    if (smem > 48 * 1024 && smem > set) {
      cudaFuncSetAttribute(k_b_leaf_up<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_b_leaf_up<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      set = smem;
    }
    H->trace.begin(kLeafUp, st);
    if (tc8)
      k_b_leaf_up<8><<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, o32.Ainv.p, o32.Ainv.ld,
                                                    o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
    else
      k_b_leaf_up<4><<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, o32.Ainv.p, o32.Ainv.ld,
                                                    o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
    H->trace.end(kLeafUp, st);
  }
  for (int l = L - 1; l >= 0; --l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const BPlan Pw = plan_b(lv.n3, lv.n3, lv.nodes, R, target);
    if (int e = launch_b(H, kMergeUpW3, Pw, o32.X[l].p, o32.X[l].ld, o32.X[l].str,
                         BXDiff{B.h32[l + 1], lv.nbc, lv.j3a, lv.j3b, R, jump, H->g, lv.d_origin, lv.a, lv.c, lv.split},
                         BEStore{B.w332[l], lv.n3, R}, st))
      return e;
    if (l > 0) {
      const BPlan Ph = plan_b(lv.nb, lv.n3, lv.nodes, R, target);
      if (int e = launch_b(H, kMergeUpH, Ph, o32.Tcat[l].p, o32.Tcat[l].ld, o32.Tcat[l].str, BXVec{B.w332[l], lv.n3, R},
                           BEFlux{lv.d_hsrc, B.h32[l + 1], lv.nbc, lv.nb, R, B.h32[l]}, st))
        return e;
    }
  }
  for (int l = 0; l < L; ++l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const BPlan Pd = plan_b(lv.n3, lv.nb, lv.nodes, R, target);
    if (int e = launch_b(H, kMergeDown, Pd, o32.S[l].p, o32.S[l].ld, o32.S[l].str, BXBd{H->g, lv.d_origin, lv.a, lv.c, R, B.g32},
                         BEScatter{H->g, lv.d_origin, lv.a, lv.c, lv.split, lv.n3, R, B.w332[l], B.g32}, st))
      return e;
  }
  H->trace.begin(kLeafDown, st);
  if (narrow)
    k_b_leaf_down_narrow<<<leaf.nodes, kBT, (size_t)(4 * b + KS * 16 * QQ) * sizeof(float), st>>>(
        H->g, R, leaf.d_origin, o32.Sleaf.p, o32.Sleaf.ld, o32.Sleaf.str, ops.identity ? 1 : 0, B.w32, B.g32);
  else if (tc8)
    k_b_leaf_down<8><<<leaf.nodes, kBT, (size_t)b * Rp * sizeof(float), st>>>(
        H->g, R, leaf.d_origin, o32.Sleaf.p, o32.Sleaf.ld, o32.Sleaf.str, ops.identity ? 1 : 0, B.w32, B.g32);
  else
    k_b_leaf_down<4><<<leaf.nodes, kBT, (size_t)b * Rp * sizeof(float), st>>>(
        H->g, R, leaf.d_origin, o32.Sleaf.p, o32.Sleaf.ld, o32.Sleaf.str, ops.identity ? 1 : 0, B.w32, B.g32);
  H->trace.end(kLeafDown, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

Leaf64Args leaf64_args(hps_handle *H, int mode, int R) {
  Leaf64Args A{};
  A.mode = mode;
  A.R = R;
  A.coef = H->d_coef;
  for (int i = 0; i < 5; ++i) A.cst[i] = H->cst[i];
  A.N_int = H->g.N_int;
  A.gdt = H->gamma_dt;
  return A;
}

int leaf64(hps_handle *H, Leaf64Args A, cudaStream_t st) {
  // which derivatives the mode needs; terms with zero constant coefficients are skipped
  const bool nodal = H->d_coef != nullptr;
  const bool L_needed = A.mode == kEval || (A.mode == kResid && A.gdt != 0.0);
  const bool d1_L = nodal || H->cst[2] != 0.0 || H->cst[3] != 0.0;
  const bool d2_L = nodal || H->cst[0] != 0.0 || H->cst[1] != 0.0;
  A.need_d1 = (L_needed && d1_L) || (A.mode != kResid && A.g_kind == HPS_G_BURGERS);
  A.need_d2 = L_needed && d2_L;
  const int slot = A.mode == kResid ? kResidual : kLeafEval;
  if (!A.need_d1 && !A.need_d2 && A.mode != kEval) {
    const int64_t n = H->g.N_int * A.R;
    H->trace.begin(slot, st);
    k_b_pointwise<<<blocks(n), 256, 0, st>>>(n, A);
    H->trace.end(slot, st);
    return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
  }
  const int p = H->p, pp = p * p;
  const int Rc = std::max(1, std::min(A.R, 4096 / pp));
  const size_t smem = (size_t)(4 * pp + pp * Rc) * sizeof(double);
  static size_t set = 0;
  if (smem > 48 * 1024 && smem > set) {
    cudaFuncSetAttribute(k_b_leaf64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    set = smem;
  }
  const Level &leaf = H->lev[H->L];
  H->trace.begin(slot, st);
  k_b_leaf64<<<leaf.nodes, kBT, smem, st>>>(H->g, leaf.d_origin, A, H->d_D);
  H->trace.end(slot, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Residual of the stage system for u (FP64) into B.r: interior rows (gdt = the operator's
// gamma dt; 0 for the identity) and shared-edge flux jumps.
int residual(hps_handle *H, int R, const double *u, const double *Rb, double gdt, cudaStream_t st) {
  Batch &B = H->batch;
  Leaf64Args A = leaf64_args(H, kResid, R);
  A.u = u;
  A.Rb = Rb;
  A.out0 = B.r;
  A.gdt = gdt;
  if (int e = leaf64(H, A, st)) return e;
  const int64_t npts = ((int64_t)(H->g.n1 - 1) * H->g.n2 + (int64_t)(H->g.n2 - 1) * H->g.n1) * H->m;
  if (npts > 0) {
    H->trace.begin(kJump, st);
    k_b_jump<<<blocks(npts * R), 256, 0, st>>>(H->g, R, u, B.r, H->d_D);
    H->trace.end(kJump, st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Solve A u = [rhs (given by combination `c`, saved to Rsave if non-null); 0; f] with refinement.
int refined_solve(hps_handle *H, const OpSet &ops, const OpSet32 &o32, int R, const Combo &c, double *Rsave,
                  const double *Rb, const double *f, double *u, int refine, double gdt, cudaStream_t st) {
  Batch &B = H->batch;
  const GridDims &g = H->g;
  k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, B.g32, f);
  if (int e = sweep32(H, ops, o32, R, c, Rsave, nullptr, st)) return e;
  k_b_finish<<<blocks(g.N * R), 256, 0, st>>>(g, R, B.g32, u, 1, 1, f);
  for (int it = 0; it < refine; ++it) {
    if (int e = residual(H, R, u, Rb, gdt, st)) return e;
    k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, B.g32, nullptr);
    Combo cr{};
    cr.n = 1;
    cr.ptr[0] = B.r;
    cr.coef[0] = 1.0;
    if (int e = sweep32(H, ops, o32, R, cr, nullptr, B.r, st)) return e;
    k_b_finish<<<blocks(g.N * R), 256, 0, st>>>(g, R, B.g32, u, 0, 1, nullptr);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

void add_term_b(Combo &c, const double *p, double coef) {
  if (coef == 0.0) return;
  c.ptr[c.n] = p;
  c.coef[c.n] = coef;
  ++c.n;
}

}  // namespace

int batch_reserve(hps_handle *H, int R) {
  Batch &B = H->batch;
  if (R <= 0 || R > 64) return HPS_EINVAL;
  if (R <= B.Rmax) return HPS_OK;
  cudaDeviceSynchronize();
  if (B.impl32.X.empty()) {  // FP32 operator copies (once)
    if (int e = convert_opset(H, H->impl, B.impl32, H->shared)) return e;
    if (int e = convert_opset(H, H->ident, B.ident32, true)) return e;
  }
  // (re)allocate the R-column work vectors; old ones stay in the handle's list until hps_free
  const GridDims &g = H->g;
  auto da = [&](auto **ptr, size_t n) -> int {
    if (cudaMalloc((void **)ptr, std::max<size_t>(n, 1) * sizeof(**ptr)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(*ptr);
    return HPS_OK;
  };
  if (da(&B.ustage, (size_t)g.N * R) || da(&B.Rb, (size_t)g.N_int * R) || da(&B.KL, 6 * (size_t)g.N_int * R) ||
      da(&B.KE, 6 * (size_t)g.N_int * R) || da(&B.r, (size_t)g.N * R) || da(&B.g32, (size_t)g.N * R) ||
      da(&B.w32, (size_t)g.N_int * R))
    return HPS_ENOMEM;
  B.h32.assign(H->L + 1, nullptr);
  B.w332.assign(H->L, nullptr);
  for (int l = 0; l <= H->L; ++l) {
    const Level &lv = H->lev[l];
    if (da(&B.h32[l], (size_t)lv.nodes * lv.nb * R)) return HPS_ENOMEM;
    if (l < H->L && da(&B.w332[l], (size_t)lv.nodes * lv.n3 * R)) return HPS_ENOMEM;
  }
  B.partial_len = partial_floats(H, R);
  if (da(&B.partial32, std::max<size_t>(1, B.partial_len))) return HPS_ENOMEM;
  cudaMemset(B.r, 0, (size_t)g.N * R * sizeof(double));
  if (cudaDeviceSynchronize() != cudaSuccess) return HPS_ECUDA;
  B.Rmax = R;
  return HPS_OK;
}

int solve_batch(hps_handle *H, int R, const double *rhs, const double *f, double *u, int refine, cudaStream_t st) {
  if (R > H->batch.Rmax) return HPS_EINVAL;
  Combo c{};
  add_term_b(c, rhs, 1.0);
  return refined_solve(H, H->impl, H->batch.impl32, R, c, nullptr, rhs, f, u, refine, H->gamma_dt, st);
}

int ark_batch(hps_handle *H, int R, double *u, double dt, const hps_ark_terms *terms, int refine, const ArkTable &tb,
              cudaStream_t st) {
  Batch &B = H->batch;
  if (R > B.Rmax) return HPS_EINVAL;
  const GridDims &g = H->g;
  const int64_t ni = g.N_int * R, nbd = g.N_bd * R;
  const double *q = terms ? terms->q : nullptr;
  const double *f = terms ? terms->f : nullptr;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  const double gp0 = terms ? terms->g_param[0] : 0.0, gp1 = terms ? terms->g_param[1] : 0.0;
  // stage 1 (explicit): dt L u^n, dt (q_1 + g(u^n))
  Leaf64Args E = leaf64_args(H, kEval, R);
  E.u = u;
  E.out0 = B.KL;
  E.out1 = B.KE;
  E.q = q;
  E.dt = dt;
  E.g_kind = gk;
  E.gp0 = gp0;
  E.gp1 = gp1;
  if (int e = leaf64(H, E, st)) return e;
  for (int i = 1; i < 6; ++i) {
    Combo c{};
    add_term_b(c, u, 1.0);
    for (int j = 0; j < i; ++j) {
      add_term_b(c, B.KL + j * ni, tb.A[i][j]);
      add_term_b(c, B.KE + j * ni, tb.Ah[i][j]);
    }
    if (int e = refined_solve(H, H->impl, B.impl32, R, c, B.Rb, B.Rb, f ? f + i * nbd : nullptr, B.ustage, refine,
                              H->gamma_dt, st))
      return e;
    Leaf64Args P = leaf64_args(H, kEpilogue, R);
    P.u = B.ustage;
    P.Rb = B.Rb;
    P.out0 = B.KL + i * ni;
    P.out1 = B.KE + i * ni;
    P.q = q ? q + i * ni : nullptr;
    P.inv_gamma = 1.0 / tb.A[1][1];
    P.dt = dt;
    P.g_kind = gk;
    P.gp0 = gp0;
    P.gp1 = gp1;
    if (int e = leaf64(H, P, st)) return e;
  }
  // step close: ARK combination at interior points, shared-edge values from the identity
  // operator solve (refined against its residual: interior R - u and the flux jumps)
  Combo c{};
  add_term_b(c, u, 1.0);
  for (int j = 0; j < 6; ++j) {
    add_term_b(c, B.KL + j * ni, tb.b[j]);
    add_term_b(c, B.KE + j * ni, tb.b[j]);
  }
  return refined_solve(H, H->ident, B.ident32, R, c, B.Rb, B.Rb, f ? f + 5 * nbd : nullptr, u, refine, 0.0, st);
}

}  // namespace hps
