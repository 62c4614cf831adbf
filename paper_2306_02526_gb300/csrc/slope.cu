// ARK step in slope form (Sec. 3.1, eq. slope0; with a nonlinear term eq. slope), FP64, one state,
// with the penalized interface conditions of Sec. 3.1 ("Penalization in the slope formulation").
//
// With kappa_i = dt k_i (the slopes times dt) the stage equations read
//   kappa_1 = dt L u^n + dt q_1                                   (explicit; edges: identity system)
//   (I - gamma dt L) kappa_i = dt L u^n + sum_{j<i} a_ij (dt L kappa_j) + dt q_i,   i = 2..6
//   u^{n+1} = u^n + sum_j b_j kappa_j                             (every point)
// dt L kappa_1 comes from leaf-local differentiation, dt L kappa_j (j >= 2) from the stage
// equation, (kappa_j - R_j) / gamma (the leaf solve's epilogue).  Every slope system has the
// interface right-hand side -(flux jump of u^n): since sum_j b_j = 1, u^{n+1} has no flux jump.
// Slope boundary data: dt u_t(t^n + c_i dt) from terms->f (the caller's u_t values), else 0.
//
// With g (a preset) the explicit slopes lambda_j = dt l_j join them (eq. slope):
//   lambda_1 = dt g(u^n),  lambda_i = dt g(U_i),  U_i = u^n + sum_{j<=i} a_ij kappa_j + sum_{j<i} ahat_ij lambda_j
//   (I - gamma dt L) kappa_i = dt L u^n + sum_{j<i} (a_ij dt L kappa_j + ahat_ij dt L lambda_j) + dt q_i
//   u^{n+1} = u^n + sum_j b_j (kappa_j + lambda_j)            (bhat = b for this tableau)
// each lambda_j a complete field: dt g at the interior points, shared edges from the identity-operator
// system (continuous flux), zero on the boundary (the paper gives slope boundary data with g only
// for time-independent Dirichlet data: terms->f must be NULL); dt L lambda_j by differentiation.
#include <cstring>

#include "hps_internal.cuh"

namespace hps {

namespace {

// boundary rows of the global vector gvec: scale * f (f in boundary order, see hps.h), or 0
__global__ void k_set_boundary_scaled(GridDims g, double *__restrict__ gvec, const double *__restrict__ f,
                                      double scale) {
  const int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= g.N_bd) return;
  const int64_t nv = (int64_t)g.n2 * g.m, nh = (int64_t)g.n1 * g.m;
  int64_t gi;
  if (kk < nv) gi = g.N_int + kk;
  else if (kk < 2 * nv) gi = g.N_int + (int64_t)g.n1 * nv + (kk - nv);
  else if (kk < 2 * nv + nh) gi = g.N_int + g.N_v + (kk - 2 * nv);
  else gi = g.N_int + g.N_v + (int64_t)g.n2 * nh + (kk - 2 * nv - nh);
  gvec[gi] = f ? scale * f[kk] : 0.0;
}

// out[i] = sum_t c.coef[t] c.ptr[t][i] for i < n (out may be one of the terms: same index)
__global__ void k_combine_all(int64_t n, Combo c, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = c.coef[0] == 1.0 ? c.ptr[0][i] : c.coef[0] * c.ptr[0][i];
  for (int t = 1; t < c.n; ++t) acc = fma(c.coef[t], c.ptr[t][i], acc);
  out[i] = acc;
}

inline unsigned nblocks(int64_t n) { return (unsigned)((n + 255) / 256); }

void add(Combo &c, const double *p, double coef) {
  if (coef == 0.0) return;
  c.ptr[c.n] = p;
  c.coef[c.n] = coef;
  ++c.n;
}

}  // namespace

int ark_slope(hps_handle *H, double *u, double dt, const hps_ark_terms *terms, const ArkTable &tb, cudaStream_t st) {
  const GridDims &g = H->g;
  const int64_t N = g.N, ni = g.N_int, nbd = g.N_bd;
  if (!H->d_proj) return HPS_EINVAL;  // a single leaf has no shared edges to project
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  const double gp0 = terms ? terms->g_param[0] : 0.0, gp1 = terms ? terms->g_param[1] : 0.0;
  const double *q = terms ? terms->q : nullptr, *f = terms ? terms->f : nullptr;
  if (gk != HPS_G_NONE && f) return HPS_EINVAL;  // with g: time-independent boundary data only
  if (!H->slope_k) {
    if (cudaMalloc(&H->slope_k, (7 * (size_t)N) * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(H->slope_k);
  }
  // with g: lambda_1..6 (N each), the stage value U (N), dt L lambda_1..6 (N_int each), scratch (N_int)
  if (gk != HPS_G_NONE && !H->slope_l) {
    if (cudaMalloc(&H->slope_l, (7 * (size_t)N + 7 * (size_t)ni) * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(H->slope_l);
  }
  double *kap = H->slope_k, *J = H->slope_k + 6 * N;  // kappa_1..6; interface right-hand side
  double *lam = H->slope_l, *U = lam ? lam + 6 * N : nullptr, *dLl = U ? U + N : nullptr, *scr = dLl ? dLl + 6 * ni : nullptr;
  const double(&A)[6][6] = tb.A;
  const double(&Ah)[6][6] = tb.Ah;
  const double(&b)[6] = tb.b;  // (the explicit weights equal the implicit ones for this tableau)
  const double gam = A[1][1];
  // interface right-hand side of every slope system: -(flux jump of u^n) (kept zero elsewhere)
  if (cudaMemsetAsync(J, 0, N * sizeof(double), st) != cudaSuccess) return HPS_ECUDA;
  if (int e = flux_jump_rhs(H, 1, u, J, st)) return e;
  // lambda_i = dt g(v) at the interior, shared edges by the identity-operator system (flux
  // continuous), zero on the boundary; dt L lambda_i into dLl_i
  auto explicit_slope = [&](const double *v, int i) -> int {
    double *li = lam + i * N;
    if (int e = leaf_eval(H, v, scr, li + 0, nullptr, dt, gk, gp0, gp1, st)) return e;  // KE slot: dt g(v)
    H->trace.begin(kSetBoundary, st);
    k_set_boundary_scaled<<<nblocks(nbd), 256, 0, st>>>(g, li, nullptr, dt);
    H->trace.end(kSetBoundary, st);
    if (cudaMemcpyAsync(scr, li, ni * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) return HPS_ECUDA;
    Combo c{};
    add(c, scr, 1.0);
    if (int e = edge_projection(H, 1, c, li, H->ustage, st, nullptr)) return e;
    return leaf_eval(H, li, dLl + i * ni, scr, nullptr, dt, HPS_G_NONE, 0.0, 0.0, st);
  };
  // dt L u^n into KL[0] (KE: dt q_1, unused)
  if (int e = leaf_eval(H, u, H->KL, H->KE, nullptr, dt, HPS_G_NONE, 0.0, 0.0, st)) return e;
  // kappa_1: interior dt (L u^n + q_1); boundary dt u_t; shared edges by the edge projection
  {
    H->trace.begin(kSetBoundary, st);
    k_set_boundary_scaled<<<nblocks(nbd), 256, 0, st>>>(g, kap, f, dt);
    H->trace.end(kSetBoundary, st);
    Combo c{};
    add(c, H->KL, 1.0);
    if (q) add(c, q, dt);
    if (int e = edge_projection(H, 1, c, kap, H->ustage, st, J)) return e;
    // dt L kappa_1 into KL[1]
    if (int e = leaf_eval(H, kap, H->KL + ni, H->KE, nullptr, dt, HPS_G_NONE, 0.0, 0.0, st)) return e;
  }
  if (gk != HPS_G_NONE)
    if (int e = explicit_slope(u, 0)) return e;
  for (int i = 1; i < 6; ++i) {
    double *ki = kap + i * N;
    H->trace.begin(kSetBoundary, st);
    k_set_boundary_scaled<<<nblocks(nbd), 256, 0, st>>>(g, ki, f ? f + i * nbd : nullptr, dt);
    H->trace.end(kSetBoundary, st);
    Combo c{};
    add(c, H->KL, 1.0);
    if (q) add(c, q + i * ni, dt);
    for (int j = 0; j < i; ++j) add(c, H->KL + (j + 1) * ni, A[i][j]);
    if (gk != HPS_G_NONE)
      for (int j = 0; j < i; ++j) add(c, dLl + j * ni, Ah[i][j]);
    Epilogue ep;  // dt L kappa_i = (kappa_i - R_i) / gamma into KL[i + 1] (the last one is not needed)
    ep.KL = i < 5 ? H->KL + (i + 1) * ni : nullptr;
    ep.KE = H->KE;
    ep.Rsaved = H->R;
    ep.inv_gamma = 1.0 / gam;
    ep.dt = dt;
    ep.g_kind = HPS_G_NONE;
    if (int e = sweep(H, H->impl, c, H->R, ki, ki, ep.KL ? &ep : nullptr, st, J)) return e;
    if (gk != HPS_G_NONE) {
      // the stage value U_i = u^n + sum_{j<=i} a_ij kappa_j + sum_{j<i} ahat_ij lambda_j at every point
      Combo cu{};
      add(cu, u, 1.0);
      for (int j = 0; j <= i; ++j) add(cu, kap + j * N, A[i][j]);
      for (int j = 0; j < i; ++j) add(cu, lam + j * N, Ah[i][j]);
      k_combine_all<<<nblocks(N), 256, 0, st>>>(N, cu, U);
      if (int e = explicit_slope(U, i)) return e;
    }
  }
  // u^{n+1} = u^n + sum_j b_j (kappa_j + lambda_j) at every point
  Combo c{};
  add(c, u, 1.0);
  for (int j = 0; j < 6; ++j) add(c, kap + j * N, b[j]);
  if (gk != HPS_G_NONE)
    for (int j = 0; j < 6; ++j) add(c, lam + j * N, b[j]);
  k_combine_all<<<nblocks(N), 256, 0, st>>>(N, c, u);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // namespace hps
