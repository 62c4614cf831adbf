// Fast diagonalization of the constant-coefficient leaf operator (Sec. 4.2: the leaf interior
// operator is a Kronecker sum L_ii = E (x) I + I (x) E of one-dimensional Chebyshev operators
// with real, distinct, negative eigenvalues).  With E_x = V_x Lam_x V_x^-1 (x lines) and
// E_y = V_y Lam_y V_y^-1 (y lines),
//   A_ii^-1 = (V_y (x) V_x) diag(1 / (c - gamma dt (lam_y,j + lam_x,i))) (V_y^-1 (x) V_x^-1),
// c = 1 - gamma dt a0: four m x m products per line instead of one q x q product (q = m^2).
// Host code only: the eigen-decompositions (Hessenberg reduction and shifted QR to a real Schur
// form, eigenvectors by back substitution) and the check of the factored inverse against the
// assembled A_ii; the applies are in batched.cu.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hps_internal.cuh"

namespace hps {

namespace {

// Real eigen-decomposition A = V diag(lam) V^-1 of a small dense matrix (row-major n x n)
// whose eigenvalues are real and distinct.  Returns false for a complex pair, a defective or
// ill-conditioned eigenvector matrix, or no convergence.
bool real_eigen(int n, const std::vector<double> &A, std::vector<double> &V, std::vector<double> &Vi,
                std::vector<double> &lam) {
  std::vector<double> H = A, Q(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  auto h = [&](int i, int j) -> double & { return H[i * n + j]; };
  auto q = [&](int i, int j) -> double & { return Q[i * n + j]; };
  // Householder reduction to upper Hessenberg form, H = Q^T A Q
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += h(i, k) * h(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (h(k + 1, k) > 0) alpha = -alpha;
    std::vector<double> v(n, 0.0);
    v[k + 1] = h(k + 1, k) - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = h(i, k);
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = 0; j < n; ++j) {  // H = (I - 2vv^T/vv) H
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * h(i, j);
      s *= 2.0 / vv;
      for (int i = k + 1; i < n; ++i) h(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {  // H = H (I - 2vv^T/vv), Q = Q (I - 2vv^T/vv)
      double s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += h(i, j) * v[j];
        t += q(i, j) * v[j];
      }
      s *= 2.0 / vv;
      t *= 2.0 / vv;
      for (int j = k + 1; j < n; ++j) {
        h(i, j) -= s * v[j];
        q(i, j) -= t * v[j];
      }
    }
  }
  // shifted QR iterations (Givens rotations) on the active block [lo, hi] until H is triangular
  const double eps = 1e-15;
  int hi = n - 1, iter = 0;
  while (hi > 0) {
    if (++iter > 100 * n) return false;
    int lo = hi;
    while (lo > 0 && std::fabs(h(lo, lo - 1)) > eps * (std::fabs(h(lo, lo)) + std::fabs(h(lo - 1, lo - 1)))) --lo;
    if (lo > 0) h(lo, lo - 1) = 0.0;
    if (lo == hi) {
      --hi;
      continue;
    }
    // Wilkinson shift from the trailing 2 x 2 block (a complex pair there means failure)
    const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    const double tr = 0.5 * (a - d), disc = tr * tr + b * c;
    if (disc < 0.0 && iter > 50 * n) return false;
    double mu = d;
    if (disc >= 0.0) {
      const double r = std::sqrt(disc);
      const double e1 = 0.5 * (a + d) + r, e2 = 0.5 * (a + d) - r;
      mu = std::fabs(e1 - d) < std::fabs(e2 - d) ? e1 : e2;
    }
    for (int i = lo; i <= hi; ++i) h(i, i) -= mu;
    std::vector<double> cs(n), sn(n);
    for (int k = lo; k < hi; ++k) {  // H = G^T H (rows k, k+1)
      const double x = h(k, k), y = h(k + 1, k), r = std::hypot(x, y);
      const double cc = r == 0.0 ? 1.0 : x / r, ss = r == 0.0 ? 0.0 : y / r;
      cs[k] = cc;
      sn[k] = ss;
      for (int j = k; j < n; ++j) {
        const double u = h(k, j), w = h(k + 1, j);
        h(k, j) = cc * u + ss * w;
        h(k + 1, j) = -ss * u + cc * w;
      }
    }
    for (int k = lo; k < hi; ++k) {  // H = H G, Q = Q G (columns k, k+1)
      const double cc = cs[k], ss = sn[k];
      for (int i = 0; i <= std::min(k + 2, hi); ++i) {
        const double u = h(i, k), w = h(i, k + 1);
        h(i, k) = cc * u + ss * w;
        h(i, k + 1) = -ss * u + cc * w;
      }
      for (int i = 0; i < n; ++i) {
        const double u = q(i, k), w = q(i, k + 1);
        q(i, k) = cc * u + ss * w;
        q(i, k + 1) = -ss * u + cc * w;
      }
    }
    for (int i = lo; i <= hi; ++i) h(i, i) += mu;
  }
  // eigenvectors of the triangular T = H by back substitution, then V = Q Y
  lam.assign(n, 0.0);
  for (int k = 0; k < n; ++k) lam[k] = h(k, k);
  std::vector<double> Y(n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    Y[k * n + k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1; j <= k; ++j) s += h(i, j) * Y[j * n + k];
      const double den = h(i, i) - lam[k];
      if (std::fabs(den) < 1e-12 * (std::fabs(lam[k]) + 1.0)) return false;  // repeated eigenvalue
      Y[i * n + k] = -s / den;
    }
  }
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += q(i, j) * Y[j * n + k];
      V[i * n + k] = s;
    }
  for (int k = 0; k < n; ++k) {  // unit columns
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += V[i * n + k] * V[i * n + k];
    s = std::sqrt(s);
    for (int i = 0; i < n; ++i) V[i * n + k] /= s;
  }
  // V^-1 by Gauss-Jordan with partial pivoting
  std::vector<double> G = V;
  Vi.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Vi[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(G[i * n + c]) > std::fabs(G[piv * n + c])) piv = i;
    if (std::fabs(G[piv * n + c]) < 1e-300) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(G[c * n + j], G[piv * n + j]);
      std::swap(Vi[c * n + j], Vi[piv * n + j]);
    }
    const double inv = 1.0 / G[c * n + c];
    for (int j = 0; j < n; ++j) {
      G[c * n + j] *= inv;
      Vi[c * n + j] *= inv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = G[i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        G[i * n + j] -= f * G[c * n + j];
        Vi[i * n + j] -= f * Vi[c * n + j];
      }
    }
  }
  // checks: A V = V Lam, conditioning of V
  double amax = 0.0, res = 0.0, vmax = 0.0, vimax = 0.0;
  for (double x : A) amax = std::max(amax, std::fabs(x));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += A[i * n + j] * V[j * n + k];
      res = std::max(res, std::fabs(s - lam[k] * V[i * n + k]));
      vmax = std::max(vmax, std::fabs(V[i * n + k]));
      vimax = std::max(vimax, std::fabs(Vi[i * n + k]));
    }
  return res <= 1e-11 * amax && n * vmax * vimax < 1e4;
}

}  // namespace

// The factored inverse [V_x, V_x^-1, V_y, V_y^-1, Lam] (each m x m, row-major) for constant
// coefficients cst = (a11, a22, a1, a2, a0) and gamma dt, with Dh = the scaled D1x, D1y, Dxx, Dyy
// (p x p each).  Returns false when a 1-D operator has no real, well-conditioned
// eigen-decomposition or the factored inverse misses A_ii; *max_err (if non-null) gets
// max |A_ii F e - e| over the unit vectors e checked (all of them when check_all).
bool fastdiag_factor(int p, const double *Dh, const double *cst, double gdt, bool check_all,
                     std::vector<double> (&F)[5], double *max_err) {
  const int m = p - 2, pp = p * p;
  std::vector<double> Ex(m * m), Ey(m * m);
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) {  // interior blocks of the 1-D operators (rows/cols 1..p-2)
      const int a = (i + 1) * p + (k + 1);
      Ex[i * m + k] = cst[0] * Dh[2 * pp + a] + cst[2] * Dh[a];
      Ey[i * m + k] = cst[1] * Dh[3 * pp + a] + cst[3] * Dh[pp + a];
    }
  std::vector<double> &Vx = F[0], &Vxi = F[1], &Vy = F[2], &Vyi = F[3], &Lam = F[4];
  std::vector<double> lx, ly;
  if (!real_eigen(m, Ex, Vx, Vxi, lx) || !real_eigen(m, Ey, Vy, Vyi, ly)) return false;
  const double c0 = 1.0 - gdt * cst[4];
  Lam.assign(m * m, 0.0);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      const double d = c0 - gdt * (ly[j] + lx[i]);
      if (std::fabs(d) < 1e-300) return false;
      Lam[j * m + i] = 1.0 / d;
    }
  // check: A_ii (F e) = e for unit vectors e, F the factored inverse
  const int q = m * m;
  double worst = 0.0;
  for (int t = 0; t < (check_all ? q : 3); ++t) {
    const int e = check_all ? t : (t * 97 + 13) % q;
    std::vector<double> x(q, 0.0), y(q, 0.0);
    x[e] = 1.0;
    auto line_x = [&](const std::vector<double> &M, std::vector<double> &v) {  // v(j, i) <- sum_k M(i,k) v(j,k)
      std::vector<double> o(q, 0.0);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
          double s = 0.0;
          for (int k = 0; k < m; ++k) s += M[i * m + k] * v[j * m + k];
          o[j * m + i] = s;
        }
      v = o;
    };
    auto line_y = [&](const std::vector<double> &M, std::vector<double> &v) {  // v(j, i) <- sum_k M(j,k) v(k,i)
      std::vector<double> o(q, 0.0);
      for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
          double s = 0.0;
          for (int k = 0; k < m; ++k) s += M[j * m + k] * v[k * m + i];
          o[j * m + i] = s;
        }
      v = o;
    };
    line_x(Vxi, x);
    line_y(Vyi, x);
    for (int k = 0; k < q; ++k) x[k] *= Lam[k];
    line_y(Vy, x);
    line_x(Vx, x);
    // y = A_ii x = c0 x - gdt (Ex along x + Ey along y)
    std::vector<double> ax = x, ay = x;
    line_x(Ex, ax);
    line_y(Ey, ay);
    for (int k = 0; k < q; ++k) {
      y[k] = c0 * x[k] - gdt * (ax[k] + ay[k]);
      worst = std::max(worst, std::fabs(y[k] - (k == e ? 1.0 : 0.0)));
    }
  }
  if (max_err) *max_err = worst;
  return worst <= 1e-12;
}

// Factors of A_ii^-1 for the handle's constant coefficients and gamma dt; leaves H->fd off when
// they do not exist or miss A_ii (fastdiag_factor).
int fastdiag_build(hps_handle *H, const std::vector<double> &Dh, cudaStream_t st) {
  H->fd = FastDiag{};
  if (!H->shared || H->gamma_dt == 0.0) return HPS_OK;
  const int m = H->m;
  std::vector<double> F[5];
  if (!fastdiag_factor(H->p, Dh.data(), H->cst, H->gamma_dt, false, F, nullptr)) return HPS_OK;
  // device copies: [Vx, Vx^-1, Vy, Vy^-1, Lam], each m x mp (rows padded to 4 for float4 loads);
  // the FP32 copy is followed by D1x, D1y (p x p each)
  const int mp = (m + 3) & ~3;
  std::vector<double> h64(5 * (size_t)m * mp, 0.0);
  for (int a = 0; a < 5; ++a)
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) h64[((size_t)a * m + i) * mp + k] = F[a][i * m + k];
  std::vector<float> h32(h64.begin(), h64.end());
  // the batched leaf apply also reads the scaled D1x, D1y in FP32 from here (after the factors)
  const size_t pp = (size_t)H->p * H->p;
  for (size_t i = 0; i < 2 * pp; ++i) h32.push_back((float)Dh[i]);
  if (cudaMalloc(&H->fd.d64, h64.size() * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(H->fd.d64);
  if (cudaMalloc(&H->fd.d32, h32.size() * sizeof(float)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(H->fd.d32);
  cudaMemcpyAsync(H->fd.d64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(H->fd.d32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;
  H->fd.on = true;
  H->fd.mp = mp;
  return HPS_OK;
}

}  // namespace hps
