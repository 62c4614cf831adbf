// HPS solve sweep on the GPU (FP64): the repeated solve inside every implicit ARK stage.
//
//   leaf_up    (a1+a2)  R = linear combination of stage vectors at the interior points,
//                       w = A_ii^{-1} R, h = D_bi w            (particular solution, its fluxes)
//   merge_up   (a3)     w3 = X (h^b_3 - h^a_3),  h^t = [h^a_1 + T^a_13 w3 ; h^b_2 + T^b_23 w3]
//   merge_down (a4)     u3 = S^t u_b + w3                       (Alg. 1 with the body load)
//   leaf_down  (a5)     u_i = w + S u_b, fused ARK epilogue: dt L u_i = (u_i - R_i)/gamma and
//                       dt (q_i + g(u_i)) with g's derivatives by leaf-local differentiation
//
// Every apply is a row-major matrix-vector product: a group of G lanes per row streams the
// row with coalesced loads, reduces by warp shuffles; the vector sits in shared memory.
// Operators are per node (stride) or shared by a whole level (stride 0).
#include "hps_internal.cuh"

namespace hps {

namespace {

template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// out(r, sum_c A[r*ld + c] * xs[c]) for rows r in [r0, r1).  Every thread of the block must
// call this (the row loop is uniform so that the shuffles see full warps).
template <int G, class Out>
__device__ __forceinline__ void block_gemv(const double *__restrict__ A, int ld, int K, const double *xs, int r0,
                                           int r1, Out out) {
  const int NG = blockDim.x / G;
  const int g = threadIdx.x / G, lg = threadIdx.x % G;
  for (int base = r0; base < r1; base += NG) {
    const int r = base + g;
    double acc = 0.0;
    if (r < r1) {
      const double *a = A + (int64_t)r * ld;
      for (int c = lg; c < K; c += G) acc = fma(__ldg(a + c), xs[c], acc);
    }
    acc = group_sum<G>(acc);
    if (r < r1 && lg == 0) out(r, acc);
  }
}

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
template <int G>
__global__ void __launch_bounds__(256) k_leaf_up(GridDims g, const int *__restrict__ origin, Combo rhs,
                                                 double *__restrict__ Rsave, const double *__restrict__ Ainv,
                                                 int ldA, int64_t strA, int identity, const double *__restrict__ Dg,
                                                 double *__restrict__ wleaf, double *__restrict__ hleaf) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m;
  double *D1x = sm, *D1y = sm + p * p, *Rs = sm + 2 * p * p, *Ws = Rs + q;
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) sm[i] = Dg[i];
  for (int r = threadIdx.x; r < q; r += blockDim.x) {
    double v = 0.0;
    for (int t = 0; t < rhs.n; ++t) v = fma(rhs.coef[t], rhs.ptr[t][l0 + r], v);
    Rs[r] = v;
    if (Rsave) Rsave[l0 + r] = v;
  }
  __syncthreads();
  if (identity) {
    for (int r = threadIdx.x; r < q; r += blockDim.x) Ws[r] = Rs[r];
  } else {
    block_gemv<G>(Ainv + k * strA, ldA, q, Rs, 0, q, [&](int r, double v) { Ws[r] = v; });
  }
  __syncthreads();
  for (int r = threadIdx.x; r < q; r += blockDim.x) wleaf[(int64_t)k * q + r] = Ws[r];
  for (int e = threadIdx.x; e < b; e += blockDim.x) hleaf[(int64_t)k * b + e] = flux_interior(e, Ws, D1x, D1y, p, m);
}

template <int G>
__global__ void __launch_bounds__(256) k_merge_up_w3(int n3, int nbc, int j3a, int j3b, int rpc,
                                                     const double *__restrict__ hC, const double *__restrict__ X,
                                                     int ldX, int64_t strX, double *__restrict__ w3) {
  extern __shared__ double ds[];
  const int k = blockIdx.y;
  const double *ha = hC + (int64_t)(2 * k) * nbc + j3a;
  const double *hb = hC + (int64_t)(2 * k + 1) * nbc + j3b;
  for (int c = threadIdx.x; c < n3; c += blockDim.x) ds[c] = hb[c] - ha[c];
  __syncthreads();
  const int r0 = blockIdx.x * rpc, r1 = min(n3, r0 + rpc);
  double *out = w3 + (int64_t)k * n3;
  block_gemv<G>(X + k * strX, ldX, n3, ds, r0, r1, [&](int r, double v) { out[r] = v; });
}

template <int G>
__global__ void __launch_bounds__(256) k_merge_up_h(int nb, int n3, int nbc, int rpc, const int *__restrict__ hsrc,
                                                    const double *__restrict__ hC, const double *__restrict__ Tcat,
                                                    int ldT, int64_t strT, const double *__restrict__ w3,
                                                    double *__restrict__ h) {
  extern __shared__ double ws[];
  const int k = blockIdx.y;
  for (int c = threadIdx.x; c < n3; c += blockDim.x) ws[c] = w3[(int64_t)k * n3 + c];
  __syncthreads();
  const int r0 = blockIdx.x * rpc, r1 = min(nb, r0 + rpc);
  const double *hk = hC + (int64_t)(2 * k) * nbc;
  double *out = h + (int64_t)k * nb;
  block_gemv<G>(Tcat + k * strT, ldT, n3, ws, r0, r1, [&](int r, double v) { out[r] = hk[hsrc[r]] + v; });
}

template <int G>
__global__ void __launch_bounds__(256) k_merge_down(GridDims g, const int *__restrict__ origin, int a, int c,
                                                    int split, int nb, int n3, int rpc, const double *__restrict__ S,
                                                    int ldS, int64_t strS, const double *__restrict__ w3,
                                                    double *__restrict__ gvec) {
  extern __shared__ double ub[];
  const int k = blockIdx.y;
  const int ix0 = origin[2 * k], iy0 = origin[2 * k + 1];
  for (int pos = threadIdx.x; pos < nb; pos += blockDim.x) ub[pos] = gvec[box_bd(g, ix0, iy0, a, c, pos)];
  __syncthreads();
  const int r0 = blockIdx.x * rpc, r1 = min(n3, r0 + rpc);
  const double *wk = w3 + (int64_t)k * n3;
  block_gemv<G>(S + k * strS, ldS, nb, ub, r0, r1,
                [&](int r, double v) { gvec[iface_bd(g, ix0, iy0, a, c, split, r)] = v + wk[r]; });
}

template <int G>
__global__ void __launch_bounds__(256) k_leaf_down(GridDims g, const int *__restrict__ origin,
                                                   const double *__restrict__ Sleaf, int ldS, int64_t strS,
                                                   int identity, const double *__restrict__ wleaf,
                                                   const double *__restrict__ gvec, double *__restrict__ out_int,
                                                   Epilogue ep, const double *__restrict__ Dg) {
  extern __shared__ double sm[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m;
  double *D1x = sm, *D1y = sm + p * p, *U = sm + 2 * p * p, *ubs = U + p * p;
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) sm[i] = Dg[i];
  for (int e = threadIdx.x; e < b; e += blockDim.x) ubs[e] = gvec[box_bd(g, ix, iy, 1, 1, e)];
  for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) U[idx] = 0.0;
  __syncthreads();
  // edges of the local field from u_b (south, east, north, west)
  for (int e = threadIdx.x; e < b; e += blockDim.x) {
    const int side = e / m, t = e % m;
    const int idx = side == 0 ? (t + 1) : side == 1 ? (t + 1) * p + (p - 1) : side == 2 ? (p - 1) * p + t + 1
                                                                                 : (t + 1) * p;
    U[idx] = ubs[e];
  }
  const double *wk = wleaf + (int64_t)k * q;
  if (identity) {
    for (int r = threadIdx.x; r < q; r += blockDim.x) U[(r / m + 1) * p + (r % m + 1)] = wk[r];
  } else {
    block_gemv<G>(Sleaf + k * strS, ldS, b, ubs, 0, q,
                  [&](int r, double v) { U[(r / m + 1) * p + (r % m + 1)] = wk[r] + v; });
  }
  __syncthreads();
  for (int r = threadIdx.x; r < q; r += blockDim.x) {
    const int i = r % m + 1, j = r / m + 1;
    const double u = U[j * p + i];
    if (out_int) out_int[l0 + r] = u;
    if (ep.KL) {
      ep.KL[l0 + r] = (u - ep.Rsaved[l0 + r]) * ep.inv_gamma;
      double ux = 0.0, uy = 0.0;
      if (ep.g_kind == HPS_G_BURGERS) {
        for (int kk = 0; kk < p; ++kk) {
          ux = fma(D1x[i * p + kk], U[j * p + kk], ux);
          uy = fma(D1y[j * p + kk], U[kk * p + i], uy);
        }
      }
      double e = g_eval(ep.g_kind, u, ux, uy, ep.gp0, ep.gp1);
      if (ep.q) e += ep.q[l0 + r];
      ep.KE[l0 + r] = ep.dt * e;
    }
  }
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

inline int pick_G(int K) { return K >= 64 ? 32 : (K >= 24 ? 16 : 8); }

#define HPS_DISPATCH_G(Gv, KERNEL, GRID, BLOCK, SMEM, ST, ...)                     \
  do {                                                                             \
    if ((Gv) == 32) KERNEL<32><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);            \
    else if ((Gv) == 16) KERNEL<16><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);       \
    else KERNEL<8><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);                        \
  } while (0)

template <class K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void set_smem_limits(size_t bytes) {
  static size_t done = 0;
  if (bytes <= done) return;
  allow_smem(k_merge_up_w3<32>, bytes); allow_smem(k_merge_up_w3<16>, bytes); allow_smem(k_merge_up_w3<8>, bytes);
  allow_smem(k_merge_up_h<32>, bytes); allow_smem(k_merge_up_h<16>, bytes); allow_smem(k_merge_up_h<8>, bytes);
  allow_smem(k_merge_down<32>, bytes); allow_smem(k_merge_down<16>, bytes); allow_smem(k_merge_down<8>, bytes);
  done = bytes;
}

constexpr int kThreads = 256;

}  // namespace

constexpr size_t kTracePairs = 16384;

void Trace::begin(int slot, cudaStream_t st) {
  ++launches[slot];
  open_slot = -1;
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

int sweep(hps_handle *H, const OpSet &ops, const Combo &rhs, double *Rsave, double *gvec, double *out_interior,
          const Epilogue *ep, cudaStream_t st) {
  const int L = H->L, p = H->p, q = H->q, b = H->b;
  size_t maxk = 0;
  for (int l = 0; l < L; ++l) maxk = std::max<size_t>(maxk, (size_t)std::max(H->lev[l].nb, H->lev[l].n3));
  set_smem_limits(maxk * sizeof(double));
  const Level &leaf = H->lev[L];
  {
    const size_t smem = (size_t)(2 * p * p + 2 * q) * sizeof(double);
    H->trace.begin(kLeafUp, st);
    HPS_DISPATCH_G(pick_G(q), k_leaf_up, leaf.nodes, kThreads, smem, st, H->g, leaf.d_origin, rhs, Rsave, ops.Ainv,
                   ops.ldA, ops.strA, ops.identity ? 1 : 0, H->d_D, H->wleaf, H->h[L]);
    H->trace.end(kLeafUp, st);
  }
  for (int l = L - 1; l >= 0; --l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const int G = pick_G(lv.n3);
    const int rpc = kThreads / G;
    dim3 gw((lv.n3 + rpc - 1) / rpc, lv.nodes);
    H->trace.begin(kMergeUpW3, st);
    HPS_DISPATCH_G(G, k_merge_up_w3, gw, kThreads, lv.n3 * sizeof(double), st, lv.n3, lv.nbc, lv.j3a, lv.j3b, rpc,
                   H->h[l + 1], mo.X, mo.ldX, mo.strX, H->w3[l]);
    H->trace.end(kMergeUpW3, st);
    if (l > 0) {
      dim3 gh((lv.nb + rpc - 1) / rpc, lv.nodes);
      H->trace.begin(kMergeUpH, st);
      HPS_DISPATCH_G(G, k_merge_up_h, gh, kThreads, lv.n3 * sizeof(double), st, lv.nb, lv.n3, lv.nbc, rpc, lv.d_hsrc,
                     H->h[l + 1], mo.Tcat, mo.ldT, mo.strT, H->w3[l], H->h[l]);
      H->trace.end(kMergeUpH, st);
    }
  }
  for (int l = 0; l < L; ++l) {
    const Level &lv = H->lev[l];
    const MergeOps &mo = ops.merge[l];
    const int G = pick_G(lv.nb);
    const int rpc = kThreads / G;
    dim3 gd((lv.n3 + rpc - 1) / rpc, lv.nodes);
    H->trace.begin(kMergeDown, st);
    HPS_DISPATCH_G(G, k_merge_down, gd, kThreads, lv.nb * sizeof(double), st, H->g, lv.d_origin, lv.a, lv.c, lv.split,
                   lv.nb, lv.n3, rpc, mo.S, mo.ldS, mo.strS, H->w3[l], gvec);
    H->trace.end(kMergeDown, st);
  }
  {
    Epilogue none;
    const size_t smem = (size_t)(3 * p * p + b) * sizeof(double);
    H->trace.begin(kLeafDown, st);
    HPS_DISPATCH_G(pick_G(b), k_leaf_down, leaf.nodes, kThreads, smem, st, H->g, leaf.d_origin, ops.Sleaf, ops.ldSl,
                   ops.strSl, ops.identity ? 1 : 0, H->wleaf, gvec, out_interior, ep ? *ep : none, H->d_D);
    H->trace.end(kLeafDown, st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // namespace hps
