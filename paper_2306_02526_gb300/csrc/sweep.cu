// HPS solve sweep on the GPU (FP64): the repeated solve inside every implicit ARK stage.
//
//   leaf_up    (a1+a2)  R = linear combination of stage vectors at the interior points,
//                       w = A_ii^{-1} R, h = D_bi w            (particular solution, its fluxes)
//   merge_up   (a3)     w3 = X (h^b_3 - h^a_3),  h^t = [h^a_1 + T^a_13 w3 ; h^b_2 + T^b_23 w3]
//   merge_down (a4)     u3 = S^t u_b + w3                       (Alg. 1 with the body load)
//   leaf_down  (a5)     u_i = w + S u_b, fused ARK epilogue: dt L u_i = (u_i - R_i)/gamma and
//                       dt (q_i + g(u_i)) with g's derivatives by leaf-local differentiation
//
// Every apply is a matrix-vector product on a transposed (column-major) operator: one thread
// per output row, a warp reads 32 consecutive rows of a column, the vector sits in shared
// memory; levels with few rows split the columns over several CTAs and add the partial sums
// in a fixed order (deterministic).  Operators are per node (stride) or shared by a whole
// level (stride 0).
#include <algorithm>

#include "hps_internal.cuh"

namespace hps {

namespace {

// Flux h_e = (D_bi w)_e at leaf edge e (south, east, north, west blocks of m) of a field
// given at the interior points only (Sec. 2.1: d/dy on horizontal, d/dx on vertical edges).
__device__ __forceinline__ double flux_interior(int e, const double *W, const double *D1x, const double *D1y,
                                                int p, int m) {
  const int side = e / m, t = e % m;
  double s = 0.0;
  if (side == 0) {
    const double *d = D1y;
    for (int jj = 1; jj <= m; ++jj) s = fma(d[jj], W[(jj - 1) * m + t], s);
  } else if (side == 1) {
    const double *d = D1x + (p - 1) * p;
    for (int ii = 1; ii <= m; ++ii) s = fma(d[ii], W[t * m + ii - 1], s);
  } else if (side == 2) {
    const double *d = D1y + (p - 1) * p;
    for (int jj = 1; jj <= m; ++jj) s = fma(d[jj], W[(jj - 1) * m + t], s);
  } else {
    const double *d = D1x;
    for (int ii = 1; ii <= m; ++ii) s = fma(d[ii], W[t * m + ii - 1], s);
  }
  return s;
}

struct CoefView {
  const double *base;  // 5 x N_int or null
  int64_t N_int;
  double cst[5];
  __device__ __forceinline__ double get(int k, int64_t idx) const {
    return base ? base[k * N_int + idx] : cst[k];
  }
};

__device__ __forceinline__ double g_eval(int kind, double u, double ux, double uy, double p0, double p1) {
  switch (kind) {
    case HPS_G_ALLEN_CAHN: return p0 * (u - u * u * u);
    case HPS_G_FISHER: return p0 * u * (1.0 - u);
    case HPS_G_BURGERS: return -u * (p0 * ux + p1 * uy);
    default: return 0.0;
  }
}

// Full p x p local field U[j*p + i] of a leaf (corners 0): interior block + the four edges.
__device__ void load_leaf_field(const GridDims &g, const double *gvec, int ix, int iy, double *U) {
  const int p = g.p, m = g.m;
  const int64_t base = ((int64_t)iy * g.n1 + ix) * m * m;
  for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
    const int i = idx % p, j = idx / p;
    double v = 0.0;
    const bool ei = (i == 0 || i == p - 1), ej = (j == 0 || j == p - 1);
    if (!ei && !ej) v = gvec[base + (j - 1) * m + (i - 1)];
    else if (ei && !ej) v = gvec[vseg(g, ix + (i == 0 ? 0 : 1), iy, j - 1)];
    else if (!ei && ej) v = gvec[hseg(g, iy + (j == 0 ? 0 : 1), ix, i - 1)];
    U[idx] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Operators are stored transposed: entry (row r, column c) of node k's matrix is at
// A[k*str + c*ld + r], so one thread owns one output row and a warp reads 32 consecutive
// rows of a column (coalesced); each product needs one FMA and no reduction across lanes.

// Leaves per CTA for the leaf kernels: fill up to 512 threads with whole leaves.
__host__ __device__ inline int leaf_lpc(int q) { return q >= 512 ? 1 : (512 / q < 16 ? 512 / q : 16); }

__global__ void __launch_bounds__(512) k_leaf_up(GridDims g, int nleaf, const int *__restrict__ origin, Combo rhs,
                                                 double *__restrict__ Rsave, const double *__restrict__ AinvT,
                                                 int ldA, int64_t strA, int identity, const double *__restrict__ Dg,
                                                 double *__restrict__ wleaf, double *__restrict__ hleaf) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, lpc = leaf_lpc(q);
  double *D1x = sm, *D1y = sm + p * p, *Rs = sm + 2 * p * p, *Ws = Rs + lpc * q;
  const int k0 = blockIdx.x * lpc;
  const int nl = min(lpc, nleaf - k0);
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) sm[i] = Dg[i];
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
    const int lo = idx / q, r = idx % q, k = k0 + lo;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
    double v = 0.0;
    for (int t = 0; t < rhs.n; ++t) v = fma(rhs.coef[t], rhs.ptr[t][l0 + r], v);
    Rs[idx] = v;
    if (Rsave) Rsave[l0 + r] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
    const int lo = idx / q, r = idx % q;
    double acc;
    if (identity) {
      acc = Rs[idx];
    } else {
      const double *a = AinvT + (int64_t)(k0 + lo) * strA + r;
      const double *x = Rs + lo * q;
      acc = 0.0;
#pragma unroll 7
      for (int c = 0; c < q; ++c) acc = fma(__ldg(a + (int64_t)c * ldA), x[c], acc);
    }
    Ws[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) wleaf[(int64_t)k0 * q + idx] = Ws[idx];
  for (int idx = threadIdx.x; idx < nl * b; idx += blockDim.x) {
    const int lo = idx / b, e = idx % b;
    hleaf[(int64_t)k0 * b + idx] = flux_interior(e, Ws + lo * q, D1x, D1y, p, m);
  }
}

// Leaf apply by fast diagonalization (constant coefficients): W = (V_y (x) V_x) Lam
// (V_y^-1 (x) V_x^-1) R as four passes of m-point products along grid lines, 4 m^3 instead of
// m^4 multiply-adds per leaf.  fd holds [V_x, V_x^-1, V_y, V_y^-1, Lam], each m x mp; the x
// passes read their operator transposed (consecutive threads = consecutive output points).
__global__ void __launch_bounds__(512) k_leaf_up_fd(GridDims g, int nleaf, const int *__restrict__ origin, Combo rhs,
                                                    double *__restrict__ Rsave, const double *__restrict__ fd, int mp,
                                                    const double *__restrict__ Dg, double *__restrict__ wleaf,
                                                    double *__restrict__ hleaf) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, lpc = leaf_lpc(q), mm = m * m;
  double *D1x = sm, *D1y = sm + p * p, *Ms = sm + 2 * p * p, *Rs = Ms + 5 * mm, *Ts = Rs + lpc * q;
  const int k0 = blockIdx.x * lpc;
  const int nl = min(lpc, nleaf - k0);
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) sm[i] = Dg[i];
  for (int idx = threadIdx.x; idx < 5 * mm; idx += blockDim.x) {  // x operators transposed: [k][i]
    const int a = idx / mm, r = idx % mm, x = r / m, y = r % m;
    const bool tr = a == 0 || a == 1;
    Ms[idx] = tr ? fd[((size_t)a * m + y) * mp + x] : fd[((size_t)a * m + x) * mp + y];
  }
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
    const int lo = idx / q, r = idx % q, k = k0 + lo;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
    double v = 0.0;
    for (int t = 0; t < rhs.n; ++t) v = fma(rhs.coef[t], rhs.ptr[t][l0 + r], v);
    Rs[idx] = v;
    if (Rsave) Rsave[l0 + r] = v;
  }
  const double *VxT = Ms, *VxiT = Ms + mm, *Vy = Ms + 2 * mm, *Vyi = Ms + 3 * mm, *Lam = Ms + 4 * mm;
  auto pass_x = [&](const double *in, double *out, const double *MT) {  // out(j,i) = sum_k M(i,k) in(j,k)
    for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
      const int lo = idx / q, r = idx % q, j = r / m, i = r % m;
      const double *x = in + lo * q + j * m;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(MT[k * m + i], x[k], s);
      out[idx] = s;
    }
  };
  auto pass_y = [&](const double *in, double *out, const double *M, const double *lam) {  // out(j,i) = sum_k M(j,k) in(k,i)
    for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
      const int lo = idx / q, r = idx % q, j = r / m, i = r % m;
      const double *x = in + lo * q + i;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(M[j * m + k], x[k * m], s);
      out[idx] = lam ? s * lam[r] : s;
    }
  };
  __syncthreads();
  pass_x(Rs, Ts, VxiT);
  __syncthreads();
  pass_y(Ts, Rs, Vyi, Lam);
  __syncthreads();
  pass_y(Rs, Ts, Vy, nullptr);
  __syncthreads();
  pass_x(Ts, Rs, VxT);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) wleaf[(int64_t)k0 * q + idx] = Rs[idx];
  for (int idx = threadIdx.x; idx < nl * b; idx += blockDim.x) {
    const int lo = idx / b, e = idx % b;
    hleaf[(int64_t)k0 * b + idx] = flux_interior(e, Rs + lo * q, D1x, D1y, p, m);
  }
}

__global__ void __launch_bounds__(512) k_leaf_down(GridDims g, int nleaf, const int *__restrict__ origin,
                                                   const double *__restrict__ SlT, int ldS, int64_t strS,
                                                   int identity, const double *__restrict__ wleaf,
                                                   const double *__restrict__ gvec, double *__restrict__ out_int,
                                                   Epilogue ep, const double *__restrict__ Dg) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, pp = p * p, lpc = leaf_lpc(q);
  double *D1x = sm, *D1y = sm + pp, *U = sm + 2 * pp, *ubs = U + lpc * pp;
  const int k0 = blockIdx.x * lpc;
  const int nl = min(lpc, nleaf - k0);
  for (int i = threadIdx.x; i < 2 * pp; i += blockDim.x) sm[i] = Dg[i];
  for (int idx = threadIdx.x; idx < nl * b; idx += blockDim.x) {
    const int lo = idx / b, e = idx % b, k = k0 + lo;
    ubs[idx] = gvec[box_bd(g, origin[2 * k], origin[2 * k + 1], 1, 1, e)];
  }
  for (int idx = threadIdx.x; idx < nl * pp; idx += blockDim.x) U[idx] = 0.0;
  __syncthreads();
  // edges of every local field from u_b (south, east, north, west)
  for (int idx = threadIdx.x; idx < nl * b; idx += blockDim.x) {
    const int lo = idx / b, e = idx % b;
    const int side = e / m, t = e % m;
    const int li = side == 0 ? (t + 1) : side == 1 ? (t + 1) * p + (p - 1) : side == 2 ? (p - 1) * p + t + 1
                                                                               : (t + 1) * p;
    U[lo * pp + li] = ubs[idx];
  }
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
    const int lo = idx / q, r = idx % q;
    double acc = wleaf[(int64_t)k0 * q + idx];
    if (!identity) {
      const double *a = SlT + (int64_t)(k0 + lo) * strS + r;
      const double *x = ubs + lo * b;
#pragma unroll 8
      for (int e = 0; e < b; ++e) acc = fma(__ldg(a + (int64_t)e * ldS), x[e], acc);
    }
    U[lo * pp + (r / m + 1) * p + (r % m + 1)] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nl * q; idx += blockDim.x) {
    const int lo = idx / q, r = idx % q, k = k0 + lo;
    const int i = r % m + 1, j = r / m + 1;
    const double *Ul = U + lo * pp;
    const double u = Ul[j * p + i];
    const int64_t gi = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q + r;
    if (out_int) out_int[gi] = u;
    if (ep.KL) {
      ep.KL[gi] = (u - ep.Rsaved[gi]) * ep.inv_gamma;
      double ux = 0.0, uy = 0.0;
      if (ep.g_kind == HPS_G_BURGERS) {
        for (int kk = 0; kk < p; ++kk) {
          ux = fma(D1x[i * p + kk], Ul[j * p + kk], ux);
          uy = fma(D1y[j * p + kk], Ul[kk * p + i], uy);
        }
      }
      double e = g_eval(ep.g_kind, u, ux, uy, ep.gp0, ep.gp1);
      if (ep.q) e += ep.q[gi];
      ep.KE[gi] = ep.dt * e;
    }
  }
}

// ---- merge levels: batched transposed mat-vec with node packing and split-K ----------------
struct GemvPlan {
  int M, K, nodes;
  int npc;        // nodes per CTA (small M) ...
  int rows_cta;   // ... or a tile of rows of one node (large M)
  int row_tiles, node_groups;
  int ksplit, kchunk;
};

constexpr int kGemvThreads = 256;

GemvPlan plan_gemv(int M, int K, int nodes, int target_ctas) {
  const int sms = target_ctas;
  GemvPlan P;
  P.M = M;
  P.K = K;
  P.nodes = nodes;
  if (M <= kGemvThreads / 2) {
    P.npc = std::max(1, std::min(nodes, kGemvThreads / M));
    P.rows_cta = M;
    P.row_tiles = 1;
  } else {
    P.npc = 1;
    P.rows_cta = kGemvThreads;
    P.row_tiles = (M + kGemvThreads - 1) / kGemvThreads;
  }
  P.node_groups = (nodes + P.npc - 1) / P.npc;
  // the same column split as the persistent kernel's task plan, so both paths add in one order
  const int ctas = P.node_groups * P.row_tiles;
  const int target = sms;
  int ks = 1;
  if (ctas < target) ks = std::min({(target + ctas - 1) / ctas, std::max(1, K / 32), kMaxSplit});
  P.kchunk = (K + ks - 1) / ks;
  while (P.npc * P.kchunk > kPSmemDoubles) P.kchunk = (P.kchunk + 1) / 2;
  P.ksplit = (K + P.kchunk - 1) / P.kchunk;
  return P;
}

// x loaders
struct XDiff {  // d = h^b_3 - h^a_3 from the children's fluxes (+ the interface right-hand side)
  const double *hC;
  int nbc, j3a, j3b;
  const double *jump;  // global vector read at interface points, or null
  GridDims g;
  const int *origin;
  int a, c, split;
  __device__ double operator()(int k, int cc) const {
    double d = hC[(int64_t)(2 * k + 1) * nbc + j3b + cc] - hC[(int64_t)(2 * k) * nbc + j3a + cc];
    if (jump) d += jump[iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, cc)];
    return d;
  }
};
struct XVec {
  const double *v;
  int n;
  __device__ double operator()(int k, int c) const { return v[(int64_t)k * n + c]; }
};
struct XBoundary {  // u on the box boundary, gathered from the global vector
  GridDims g;
  const int *origin;
  int a, c;
  const double *gvec;
  __device__ double operator()(int k, int pos) const {
    return gvec[box_bd(g, origin[2 * k], origin[2 * k + 1], a, c, pos)];
  }
};
// epilogues
struct EStore {
  double *out;
  int n;
  __device__ void operator()(int k, int r, double v) const { out[(int64_t)k * n + r] = v; }
};
struct EFlux {  // h^t = [h^a_1 ; h^b_2] + Tcat w3
  const int *hsrc;
  const double *hC;
  int nbc, nb;
  double *h;
  __device__ void operator()(int k, int r, double v) const {
    h[(int64_t)k * nb + r] = hC[(int64_t)(2 * k) * nbc + hsrc[r]] + v;
  }
};
struct EScatter {  // u3 = S u_b + w3 onto the interface of the cut
  GridDims g;
  const int *origin;
  int a, c, split, n3;
  const double *w3;
  double *gvec;
  __device__ void operator()(int k, int r, double v) const {
    gvec[iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r)] = v + w3[(int64_t)k * n3 + r];
  }
};

template <class XL, class EP>
__global__ void __launch_bounds__(kGemvThreads) k_gemv_t(GemvPlan P, const double *__restrict__ AT, int ld,
                                                         int64_t str, XL xl, EP ep, double *__restrict__ partial) {
  extern __shared__ double xs[];
  const int ng = blockIdx.x / P.row_tiles, tile = blockIdx.x % P.row_tiles;
  const int node0 = ng * P.npc;
  const int nn = min(P.npc, P.nodes - node0);
  const int ks = blockIdx.y;
  const int c0 = ks * P.kchunk, klen = min(P.kchunk, P.K - c0);
  for (int idx = threadIdx.x; idx < nn * klen; idx += blockDim.x) {
    const int lo = idx / klen, c = idx % klen;
    xs[idx] = xl(node0 + lo, c0 + c);
  }
  __syncthreads();
  int lo, r;
  if (P.npc > 1) {
    lo = threadIdx.x / P.M;
    r = threadIdx.x % P.M;
  } else {
    lo = 0;
    r = tile * P.rows_cta + threadIdx.x;
  }
  if (lo >= nn || r >= P.M) return;
  const int k = node0 + lo;
  const double *a = AT + (int64_t)k * str + (int64_t)c0 * ld + r;
  const double *x = xs + lo * klen;
  double acc = 0.0;
#pragma unroll 8
  for (int c = 0; c < klen; ++c) acc = fma(__ldg(a + (int64_t)c * ld), x[c], acc);
  if (P.ksplit == 1) ep(k, r, acc);
  else partial[((int64_t)ks * P.nodes + k) * P.M + r] = acc;
}

// Deterministic split-K reduction: partial sums added in split order, then the epilogue.
template <class EP>
__global__ void k_gemv_reduce(GemvPlan P, const double *__restrict__ partial, EP ep) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)P.nodes * P.M) return;
  const int k = (int)(idx / P.M), r = (int)(idx % P.M);
  double acc = 0.0;
#pragma unroll 8
  for (int ks = 0; ks < P.ksplit; ++ks) acc += partial[((int64_t)ks * P.nodes + k) * P.M + r];
  ep(k, r, acc);
}

// dt L u and dt (q + g(u)) at the interior points of every leaf (explicit first stage).
__global__ void __launch_bounds__(256) k_leaf_eval(GridDims g, const int *__restrict__ origin,
                                                   const double *__restrict__ u, double *__restrict__ KL,
                                                   double *__restrict__ KE, const double *__restrict__ q,
                                                   double dt, int g_kind, double gp0, double gp1, CoefView cf,
                                                   const double *__restrict__ Dg) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, qq = m * m;
  double *D1x = sm, *D1y = sm + p * p, *Dxx = sm + 2 * p * p, *Dyy = sm + 3 * p * p, *U = sm + 4 * p * p;
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * qq;
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) sm[i] = Dg[i];
  load_leaf_field(g, u, ix, iy, U);
  __syncthreads();
  for (int r = threadIdx.x; r < qq; r += blockDim.x) {
    const int i = r % m + 1, j = r / m + 1;
    double ux = 0.0, uy = 0.0, uxx = 0.0, uyy = 0.0;
    for (int kk = 0; kk < p; ++kk) {
      const double vx = U[j * p + kk], vy = U[kk * p + i];
      ux = fma(D1x[i * p + kk], vx, ux);
      uxx = fma(Dxx[i * p + kk], vx, uxx);
      uy = fma(D1y[j * p + kk], vy, uy);
      uyy = fma(Dyy[j * p + kk], vy, uyy);
    }
    const int64_t gi = l0 + r;
    const double uu = U[j * p + i];
    const double Lu = cf.get(0, gi) * uxx + cf.get(1, gi) * uyy + cf.get(2, gi) * ux + cf.get(3, gi) * uy +
                      cf.get(4, gi) * uu;
    KL[gi] = dt * Lu;
    double e = g_eval(g_kind, uu, ux, uy, gp0, gp1);
    if (q) e += q[gi];
    KE[gi] = dt * e;
  }
}

__global__ void k_set_boundary(GridDims g, double *__restrict__ gvec, const double *__restrict__ f) {
  const int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= g.N_bd) return;
  const int64_t nv = (int64_t)g.n2 * g.m, nh = (int64_t)g.n1 * g.m;
  int64_t gi;
  if (kk < nv) gi = g.N_int + kk;
  else if (kk < 2 * nv) gi = g.N_int + (int64_t)g.n1 * nv + (kk - nv);
  else if (kk < 2 * nv + nh) gi = g.N_int + g.N_v + (kk - 2 * nv);
  else gi = g.N_int + g.N_v + (int64_t)g.n2 * nh + (kk - 2 * nv - nh);
  gvec[gi] = f ? f[kk] : 0.0;
}

template <class XL, class EP>
int launch_gemv(hps_handle *H, int slot, const GemvPlan &P, const double *AT, int ld, int64_t str, XL xl, EP ep,
                cudaStream_t st) {
  const size_t smem = (size_t)P.npc * P.kchunk * sizeof(double);
  if (int e_ = smem_optin((const void *)k_gemv_t<XL, EP>, smem)) return e_;
  if (P.ksplit > 1 && (size_t)P.ksplit * P.nodes * P.M > H->partial_len) return HPS_EINVAL;
  H->trace.begin(slot, st);
  dim3 grid(P.node_groups * P.row_tiles, P.ksplit);
  k_gemv_t<XL, EP><<<grid, kGemvThreads, smem, st>>>(P, AT, ld, str, xl, ep, H->partial);
  if (P.ksplit > 1) {
    const int64_t n = (int64_t)P.nodes * P.M;
    k_gemv_reduce<EP><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, H->partial, ep);
  }
  H->trace.end(slot, st);
  return HPS_OK;
}

constexpr int kThreads = 256;

}  // namespace

constexpr size_t kTracePairs = 16384;

void GraphEntry::destroy() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  for (auto &e : ev) cudaEventDestroy(e);
  ev.clear();
  ev_slot.clear();
  nev = 0;
  valid = seen = pending = false;
}

void drain_graph(hps_handle *H, GraphEntry &e) {
  if (!e.pending) return;
  for (int i = 0; i < e.nev; ++i) {
    float t = 0.f;
    cudaEventSynchronize(e.ev[2 * i + 1]);
    if (cudaEventElapsedTime(&t, e.ev[2 * i], e.ev[2 * i + 1]) == cudaSuccess) {
      H->trace.ms[e.ev_slot[i]] += t;
      ++H->trace.timed[e.ev_slot[i]];
    } else {
      cudaGetLastError();  // a failed timing query must not surface as a launch error later
    }
  }
  e.pending = false;
}

void Trace::begin(int slot, cudaStream_t st) {
  open_slot = -1;
  if (capturing) {  // recording a graph: count per replay, time with the graph's own events
    ++capturing->launches[slot];
    if ((mask & (1u << slot)) && capturing->nev < GraphEntry::kEventPairs) {
      // an external record becomes an event-record node that runs on every replay
      cudaEventRecordWithFlags(capturing->ev[2 * capturing->nev], st, cudaEventRecordExternal);
      open_slot = slot;
    }
    return;
  }
  ++launches[slot];
  if (!(mask & (1u << slot))) return;
  if (pool.empty()) {
    pool.resize(2 * kTracePairs);
    for (auto &e : pool) cudaEventCreate(&e);
    pair_slot.assign(kTracePairs, -1);
  }
  if (used == kTracePairs) drain();
  cudaEventRecord(pool[2 * used], st);
  open_slot = slot;
}

void Trace::end(int slot, cudaStream_t st) {
  if (open_slot != slot) return;
  if (capturing) {
    cudaEventRecordWithFlags(capturing->ev[2 * capturing->nev + 1], st, cudaEventRecordExternal);
    capturing->ev_slot[capturing->nev] = slot;
    ++capturing->nev;
    open_slot = -1;
    return;
  }
  cudaEventRecord(pool[2 * used + 1], st);
  pair_slot[used] = slot;
  ++used;
  open_slot = -1;
}

void Trace::drain() {
  for (size_t i = 0; i < used; ++i) {
    float t = 0.f;
    cudaEventSynchronize(pool[2 * i + 1]);
    if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
      ms[pair_slot[i]] += t;
      ++timed[pair_slot[i]];
    } else {
      cudaGetLastError();
    }
  }
  used = 0;
}

void Trace::release() {
  for (auto &e : pool) cudaEventDestroy(e);
  pool.clear();
  used = 0;
}

int set_boundary(hps_handle *H, double *gvec, const double *f, cudaStream_t st) {
  const int64_t n = H->g.N_bd;
  H->trace.begin(kSetBoundary, st);
  k_set_boundary<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(H->g, gvec, f);
  H->trace.end(kSetBoundary, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

int leaf_eval(hps_handle *H, const double *u, double *KL, double *KE, const double *q, double dt, int g_kind,
              double gp0, double gp1, cudaStream_t st) {
  const int p = H->p;
  CoefView cf;
  cf.base = H->d_coef;
  cf.N_int = H->g.N_int;
  for (int i = 0; i < 5; ++i) cf.cst[i] = H->cst[i];
  const hps::Level &lv = H->lev[H->L];
  const size_t smem = (size_t)5 * p * p * sizeof(double);
  H->trace.begin(kLeafEval, st);
  k_leaf_eval<<<lv.nodes, kThreads, smem, st>>>(H->g, lv.d_origin, u, KL, KE, q, dt, g_kind, gp0, gp1, cf, H->d_D);
  H->trace.end(kLeafEval, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

size_t partial_doubles(const hps_handle *H) {
  size_t mx = 0;
  for (int l = 0; l < H->L; ++l) {
    const Level &lv = H->lev[l];
    const int tgt = H->fp64_plan_target * H->num_sms;
    const GemvPlan P[3] = {plan_gemv(lv.n3, lv.n3, lv.nodes, tgt), plan_gemv(lv.nb, lv.n3, lv.nodes, tgt),
                           plan_gemv(lv.n3, lv.nb, lv.nodes, tgt)};
    for (const GemvPlan &p : P)
      if (p.ksplit > 1) mx = std::max(mx, (size_t)p.ksplit * p.nodes * p.M);
  }
  return mx;
}

int sweep(hps_handle *H, const OpSet &ops, const Combo &rhs, double *Rsave, double *gvec, double *out_interior,
          const Epilogue *ep, cudaStream_t st, const double *jump) {
  const int L = H->L, p = H->p, q = H->q, b = H->b;
  if (jump && H->persistent) return HPS_EINVAL;  // the persistent merge kernel has no interface input
  const Level &leaf = H->lev[L];
  const int lpc = leaf_lpc(q);
  const int lthreads = std::min(512, ((lpc * q + 31) / 32) * 32);
  const unsigned lgrid = (unsigned)((leaf.nodes + lpc - 1) / lpc);
  if (H->fd.on && H->batch.fast_diag && !ops.identity) {
    const size_t smem = (size_t)(2 * p * p + 5 * H->m * H->m + 2 * lpc * q) * sizeof(double);
    if (int e_ = smem_optin((const void *)k_leaf_up_fd, smem)) return e_;
    H->trace.begin(kLeafUp, st);
    k_leaf_up_fd<<<lgrid, lthreads, smem, st>>>(H->g, leaf.nodes, leaf.d_origin, rhs, Rsave, H->fd.d64, H->fd.mp,
                                                H->d_D, H->wleaf, H->h[L]);
    H->trace.end(kLeafUp, st);
  } else {
    const size_t smem = (size_t)(2 * p * p + 2 * lpc * q) * sizeof(double);
    H->trace.begin(kLeafUp, st);
    k_leaf_up<<<lgrid, lthreads, smem, st>>>(H->g, leaf.nodes, leaf.d_origin, rhs, Rsave, ops.Ainv, ops.ldA, ops.strA,
                                             ops.identity ? 1 : 0, H->d_D, H->wleaf, H->h[L]);
    H->trace.end(kLeafUp, st);
  }
  if (H->persistent) {
    if (int e = merge_persistent(H, ops, true, gvec, st)) return e;
    if (int e = merge_persistent(H, ops, false, gvec, st)) return e;
  }
  for (int l = L - 1; l >= 0 && !H->persistent; --l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const GemvPlan Pw = plan_gemv(lv.n3, lv.n3, lv.nodes, H->fp64_plan_target * H->num_sms);
    if (int e = launch_gemv(H, kMergeUpW3, Pw, mo.X, mo.ldX, mo.strX,
                            XDiff{H->h[l + 1], lv.nbc, lv.j3a, lv.j3b, jump, H->g, lv.d_origin, lv.a, lv.c, lv.split},
                            EStore{H->w3[l], lv.n3}, st))
      return e;
    if (l > 0) {
      const GemvPlan Ph = plan_gemv(lv.nb, lv.n3, lv.nodes, H->fp64_plan_target * H->num_sms);
      if (int e = launch_gemv(H, kMergeUpH, Ph, mo.Tcat, mo.ldT, mo.strT, XVec{H->w3[l], lv.n3},
                              EFlux{lv.d_hsrc, H->h[l + 1], lv.nbc, lv.nb, H->h[l]}, st))
        return e;
    }
  }
  for (int l = 0; l < L && !H->persistent; ++l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const GemvPlan Pd = plan_gemv(lv.n3, lv.nb, lv.nodes, H->fp64_plan_target * H->num_sms);
    if (int e = launch_gemv(H, kMergeDown, Pd, mo.S, mo.ldS, mo.strS, XBoundary{H->g, lv.d_origin, lv.a, lv.c, gvec},
                            EScatter{H->g, lv.d_origin, lv.a, lv.c, lv.split, lv.n3, H->w3[l], gvec}, st))
      return e;
  }
  {
    Epilogue none;
    const size_t smem = (size_t)(2 * p * p + lpc * (p * p + b)) * sizeof(double);
    H->trace.begin(kLeafDown, st);
    k_leaf_down<<<lgrid, lthreads, smem, st>>>(H->g, leaf.nodes, leaf.d_origin, ops.Sleaf, ops.ldSl, ops.strSl,
                                               ops.identity ? 1 : 0, H->wleaf, gvec, out_interior, ep ? *ep : none,
                                               H->d_D);
    H->trace.end(kLeafDown, st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // namespace hps
