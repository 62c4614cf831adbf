// HPS operator build on the GPU in FP64 (Sec. 2.1).
//
// Leaves (eq. ``discretize``, eq. ``leaf``): the augmented matrix [A_ii | I | A_ib] of
// A = I - gamma_dt L is reduced by Gauss-Jordan elimination with partial pivoting to
// [I | A_ii^{-1} | A_ii^{-1} A_ib]; then S = -A_ii^{-1} A_ib and T = D_bi S + D_bb.
// Merges (Sec. 2.1 merge formulas): [T^a_33 - T^b_33 | I | -T^a_31, T^b_32] is reduced the
// same way to [I | X | S^t]; T^t = diag(T^a_11, T^b_22) + [T^a_13; T^b_23] S^t by a batched
// FP64 GEMM.  One Gauss-Jordan step is two launches (pivot row, rank-1 elimination) over a
// batch of matrices held in global memory.
#include <algorithm>
#include <cmath>

#include "hps_internal.cuh"

namespace hps {

namespace {

constexpr int kT = 256;

inline int ld_pad(int n) { return (n + 1) & ~1; }  // even leading dimension: 16-byte rows

// ---- leaf assembly -----------------------------------------------------------------------
// Row r of [A_ii | I | A_ib] for interior node (i, j): A = I - gdt (a11 Dxx + a22 Dyy + a1 Dx + a2 Dy + a0).
__global__ void k_leaf_assemble(GridDims g, const int *__restrict__ origin, int k0, const double *__restrict__ coef,
                                int64_t N_int, double c0, double c1, double c2, double c3, double c4,
                                const double *__restrict__ Dg, double gdt, double *__restrict__ G, int ldG) {
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, W = 2 * q + b;
  const int k = k0 + blockIdx.x;
  double *Gk = G + (int64_t)blockIdx.x * q * ldG;
  const double *D1x = Dg, *D1y = Dg + p * p, *Dxx = Dg + 2 * p * p, *Dyy = Dg + 3 * p * p;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int64_t idx = threadIdx.x; idx < (int64_t)q * ldG; idx += blockDim.x) Gk[idx] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < q; r += blockDim.x) {
    const int i = r % m + 1, j = r / m + 1;
    double a11 = c0, a22 = c1, a1 = c2, a2 = c3, a0 = c4;
    if (coef) {
      a11 = coef[0 * N_int + l0 + r];
      a22 = coef[1 * N_int + l0 + r];
      a1 = coef[2 * N_int + l0 + r];
      a2 = coef[3 * N_int + l0 + r];
      a0 = coef[4 * N_int + l0 + r];
    }
    double *row = Gk + (int64_t)r * ldG;
    // x-direction couplings: nodes (kk, j)
    for (int kk = 0; kk < p; ++kk) {
      const double v = -gdt * (a11 * Dxx[i * p + kk] + a1 * D1x[i * p + kk]);
      int col;
      if (kk == 0) col = 2 * q + 3 * m + (j - 1);            // west edge
      else if (kk == p - 1) col = 2 * q + m + (j - 1);       // east edge
      else col = (j - 1) * m + (kk - 1);
      row[col] += v;
    }
    // y-direction couplings: nodes (i, kk)
    for (int kk = 0; kk < p; ++kk) {
      const double v = -gdt * (a22 * Dyy[j * p + kk] + a2 * D1y[j * p + kk]);
      int col;
      if (kk == 0) col = 2 * q + (i - 1);                    // south edge
      else if (kk == p - 1) col = 2 * q + 2 * m + (i - 1);   // north edge
      else col = (kk - 1) * m + (i - 1);
      row[col] += v;
    }
    row[r] += 1.0 - gdt * a0;
    row[q + r] = 1.0;
  }
  (void)W;
}

// ---- Gauss-Jordan with partial pivoting, one step = pivot kernel + elimination kernel ----
__global__ void k_gj_pivot(double *__restrict__ G, int ldG, int W, int n, int kstep, double *__restrict__ mult,
                           int *__restrict__ info) {
  __shared__ double sv[kT];
  __shared__ int si[kT];
  double *Gm = G + (int64_t)blockIdx.x * n * ldG;
  double *mu = mult + (int64_t)blockIdx.x * n;
  double best = -1.0;
  int bi = kstep;
  for (int r = kstep + threadIdx.x; r < n; r += blockDim.x) {
    const double v = fabs(Gm[(int64_t)r * ldG + kstep]);
    if (v > best) { best = v; bi = r; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const int oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int piv = si[0];
  double *rk = Gm + (int64_t)kstep * ldG;
  double *rp = Gm + (int64_t)piv * ldG;
  if (piv != kstep) {
    for (int c = kstep + threadIdx.x; c < W; c += blockDim.x) {
      const double t = rk[c];
      rk[c] = rp[c];
      rp[c] = t;
    }
  }
  __syncthreads();
  const double pv = rk[kstep];
  const bool bad = !(fabs(pv) > 0.0) || !isfinite(pv);
  if (bad && threadIdx.x == 0) atomicOr(info, 1);
  __syncthreads();
  for (int c = kstep + 1 + threadIdx.x; c < W; c += blockDim.x) rk[c] = bad ? 0.0 : rk[c] / pv;
  __syncthreads();
  if (threadIdx.x == 0) rk[kstep] = 1.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) mu[r] = (r == kstep) ? 0.0 : Gm[(int64_t)r * ldG + kstep];
}

// G[r][c] -= mult[r] * G[k][c] for r != k, c >= k.  Block: 32 columns x 8 row-lanes.
__global__ void k_gj_elim(double *__restrict__ G, int ldG, int W, int n, int kstep, const double *__restrict__ mult) {
  double *Gm = G + (int64_t)blockIdx.z * n * ldG;
  const double *mu = mult + (int64_t)blockIdx.z * n;
  const int c = kstep + blockIdx.x * 32 + threadIdx.x;
  if (c >= W) return;
  const double pk = Gm[(int64_t)kstep * ldG + c];
  for (int r = blockIdx.y * blockDim.y + threadIdx.y; r < n; r += gridDim.y * blockDim.y) {
    if (r == kstep) continue;
    const double f = mu[r];
    if (f != 0.0) Gm[(int64_t)r * ldG + c] -= f * pk;
  }
}

int gauss_jordan(double *G, int ldG, int W, int n, int batch, double *mult, int *info, cudaStream_t st) {
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<batch, kT, 0, st>>>(G, ldG, W, n, k, mult, info);
    const int cols = W - k;
    dim3 blk(32, 8);
    const int gy = std::max(1, std::min((n + 7) / 8, std::max(1, 2048 / std::max(1, batch))));
    dim3 grd((cols + 31) / 32, gy, batch);
    k_gj_elim<<<grd, blk, 0, st>>>(G, ldG, W, n, k, mult);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// ---- leaf extraction: A_ii^{-1}, S = -A_ii^{-1} A_ib, T = D_bi S + D_bb -------------------
__global__ void k_leaf_extract(int p, int k0, const double *__restrict__ G, int ldG, double *__restrict__ Ainv,
                               int ldA, int64_t strA, double *__restrict__ Sl, int ldS, int64_t strS,
                               double *__restrict__ T, int b_ld, const double *__restrict__ Dg) {
  const int m = p - 2, q = m * m, b = 4 * m;
  const int k = k0 + blockIdx.x;
  const double *Gk = G + (int64_t)blockIdx.x * q * ldG;
  double *Ak = Ainv + k * strA;
  double *Sk = Sl + k * strS;
  // stored transposed (column c of the operator is a contiguous run of its q rows)
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int c = idx / q, r = idx % q;
    Ak[(int64_t)c * ldA + r] = Gk[(int64_t)r * ldG + q + c];
  }
  for (int idx = threadIdx.x; idx < q * b; idx += blockDim.x) {
    const int c = idx / q, r = idx % q;
    Sk[(int64_t)c * ldS + r] = -Gk[(int64_t)r * ldG + 2 * q + c];
  }
  __syncthreads();
  const double *D1x = Dg, *D1y = Dg + p * p;
  double *Tk = T + (int64_t)k * b * b_ld;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int e = idx / b, e2 = idx % b;
    const int side = e / m, t = e % m;
    double s = 0.0;
    // D_bi S: flux at edge e of the interior field S[:, e2]
    if (side == 0 || side == 2) {
      const double *d = D1y + (side == 0 ? 0 : (p - 1) * p);
      for (int jj = 1; jj <= m; ++jj) s = fma(d[jj], Sk[(int64_t)e2 * ldS + (jj - 1) * m + t], s);
      // D_bb: the same column's two end points (south = t, north = 2m + t)
      if (e2 == t) s += d[0];
      if (e2 == 2 * m + t) s += d[p - 1];
    } else {
      const double *d = D1x + (side == 1 ? (p - 1) * p : 0);
      for (int ii = 1; ii <= m; ++ii) s = fma(d[ii], Sk[(int64_t)e2 * ldS + t * m + ii - 1], s);
      // west = 3m + t, east = m + t
      if (e2 == 3 * m + t) s += d[0];
      if (e2 == m + t) s += d[p - 1];
    }
    Tk[(int64_t)e * b_ld + e2] = s;
  }
}

// Identity operator on a leaf: S = 0, T = D_bb.
__global__ void k_leaf_T_ident(int p, double *__restrict__ T, int b_ld, const double *__restrict__ Dg) {
  const int m = p - 2, b = 4 * m;
  const double *D1x = Dg, *D1y = Dg + p * p;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int e = idx / b, e2 = idx % b;
    const int side = e / m, t = e % m;
    double s = 0.0;
    if (side == 0 || side == 2) {
      const double *d = D1y + (side == 0 ? 0 : (p - 1) * p);
      if (e2 == t) s += d[0];
      if (e2 == 2 * m + t) s += d[p - 1];
    } else {
      const double *d = D1x + (side == 1 ? (p - 1) * p : 0);
      if (e2 == 3 * m + t) s += d[0];
      if (e2 == m + t) s += d[p - 1];
    }
    T[(int64_t)e * b_ld + e2] = s;
  }
}

// ---- merge assembly ------------------------------------------------------------------------
// Node k (children 2k, 2k+1 of the child level; child T per node with stride strTc, or
// shared with stride 0): rows of [T^a_33 - T^b_33 | I | B] with B's column for parent
// boundary position kk = -T^a_3,pos (alpha) or +T^b_3,pos (beta), and Tcat[kk][c] = T^child[pos][3].
__global__ void k_merge_assemble(int k0, int n3, int nb, int nbc, int j3a, int j3b, const int *__restrict__ hsrc,
                                 const double *__restrict__ Tc, int ldTc, int64_t strTc, double *__restrict__ G,
                                 int ldG, double *__restrict__ Tcat, int ldT, int64_t strT) {
  const int k = k0 + blockIdx.x;
  const double *Ta = Tc + (int64_t)(2 * k) * strTc;
  const double *Tb = Tc + (int64_t)(2 * k + 1) * strTc;
  double *Gk = G + (int64_t)blockIdx.x * n3 * ldG;
  const int W = 2 * n3 + nb;
  for (int64_t idx = threadIdx.x; idx < (int64_t)n3 * W; idx += blockDim.x) {
    const int r = (int)(idx / W), c = (int)(idx % W);
    double v;
    if (c < n3) {
      v = Ta[(int64_t)(j3a + r) * ldTc + j3a + c] - Tb[(int64_t)(j3b + r) * ldTc + j3b + c];
    } else if (c < 2 * n3) {
      v = (c - n3 == r) ? 1.0 : 0.0;
    } else {
      const int kk = c - 2 * n3;
      const int src = hsrc[kk];
      const int ch = src / nbc, pos = src % nbc;
      v = ch == 0 ? -Ta[(int64_t)(j3a + r) * ldTc + pos] : Tb[(int64_t)(j3b + r) * ldTc + pos];
    }
    Gk[(int64_t)r * ldG + c] = v;
  }
  if (!Tcat) return;
  double *Tk = Tcat + k * strT;
  for (int64_t idx = threadIdx.x; idx < (int64_t)nb * n3; idx += blockDim.x) {  // stored transposed
    const int c = (int)(idx / nb), kk = (int)(idx % nb);
    const int src = hsrc[kk];
    const int ch = src / nbc, pos = src % nbc;
    Tk[(int64_t)c * ldT + kk] = ch == 0 ? Ta[(int64_t)pos * ldTc + j3a + c] : Tb[(int64_t)pos * ldTc + j3b + c];
  }
}

__global__ void k_merge_extract(int k0, int n3, int nb, const double *__restrict__ G, int ldG, double *__restrict__ X,
                                int ldX, int64_t strX, double *__restrict__ S, int ldS, int64_t strS) {
  const int k = k0 + blockIdx.x;
  const double *Gk = G + (int64_t)blockIdx.x * n3 * ldG;
  double *Xk = X + k * strX;
  double *Sk = S + k * strS;
  // stored transposed (column c contiguous over the n3 rows)
  for (int64_t idx = threadIdx.x; idx < (int64_t)n3 * n3; idx += blockDim.x) {
    const int c = (int)(idx / n3), r = (int)(idx % n3);
    Xk[(int64_t)c * ldX + r] = Gk[(int64_t)r * ldG + n3 + c];
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n3 * nb; idx += blockDim.x) {
    const int c = (int)(idx / n3), r = (int)(idx % n3);
    Sk[(int64_t)c * ldS + r] = Gk[(int64_t)r * ldG + 2 * n3 + c];
  }
}

// Parent T initialised to diag(T^a_11, T^b_22) in parent boundary order.
__global__ void k_merge_tdiag(int nb, int nbc, const int *__restrict__ hsrc, const double *__restrict__ Tc, int ldTc,
                              int64_t strTc, double *__restrict__ Tp, int ldTp, int64_t strTp) {
  const int k = blockIdx.y;
  const double *Ta = Tc + (int64_t)(2 * k) * strTc;
  const double *Tb = Tc + (int64_t)(2 * k + 1) * strTc;
  double *Tk = Tp + k * strTp;
  const int64_t total = (int64_t)nb * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / nb), c = (int)(idx % nb);
    const int sr = hsrc[r], sc = hsrc[c];
    const int chr = sr / nbc, chc = sc / nbc;
    double v = 0.0;
    if (chr == chc) v = (chr == 0 ? Ta : Tb)[(int64_t)(sr % nbc) * ldTc + (sc % nbc)];
    Tk[(int64_t)r * ldTp + c] = v;
  }
}

// C[z] += A[z] (M x K) * B[z] (K x N) in FP64; A(r,k) = A[r*sar + k*sak], B(k,c) = B[k*sbk + c*sbc],
// C row-major.  64x64 tile, 256 threads, 4x4 outputs each.
__global__ void __launch_bounds__(256) k_dgemm_acc(int M, int N, int K, const double *__restrict__ A, int64_t sar,
                                                   int64_t sak, int64_t strA, const double *__restrict__ B,
                                                   int64_t sbk, int64_t sbc, int64_t strB, double *__restrict__ C,
                                                   int ldc, int64_t strC) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const double *Az = A + blockIdx.z * strA;
  const double *Bz = B + blockIdx.z * strB;
  double *Cz = C + blockIdx.z * strC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int kb = 0; kb < K; kb += 16) {
    for (int idx = threadIdx.x; idx < 64 * 16; idx += 256) {
      // consecutive threads walk the unit-stride index of each operand
      int r, kk;
      if (sar == 1) { r = idx % 64; kk = idx / 64; } else { r = idx / 16; kk = idx % 16; }
      const int gr = row0 + r, gk = kb + kk;
      As[kk][r] = (gr < M && gk < K) ? Az[gr * sar + gk * sak] : 0.0;
      int kk2, cc;
      if (sbk == 1) { kk2 = idx % 16; cc = idx / 16; } else { kk2 = idx / 64; cc = idx % 64; }
      const int gk2 = kb + kk2, gc = col0 + cc;
      Bs[kk2][cc] = (gk2 < K && gc < N) ? Bz[gk2 * sbk + gc * sbc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c < N) Cz[(int64_t)r * ldc + c] += acc[i][j];
    }
  }
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  int alloc(size_t bytes) {
    if (p) { cudaFree(p); p = nullptr; }
    return cudaMalloc(&p, std::max<size_t>(bytes, 16)) == cudaSuccess ? HPS_OK : HPS_ENOMEM;
  }
  template <class T> T *as() { return static_cast<T *>(p); }
};

constexpr size_t kWorkBytes = size_t(1) << 30;  // Gauss-Jordan workspace per chunk

}  // namespace

// Builds ops (leaf + merge operators) for A = I - gamma_dt L, or for the identity.
int build_operators(hps_handle *H, OpSet &ops, double gamma_dt, bool identity, cudaStream_t st) {
  const int L = H->L, p = H->p, m = H->m, q = H->q, b = H->b;
  const bool shared = identity || H->shared;
  ops.identity = identity;
  ops.merge.assign(L, MergeOps());
  DevBuf info_buf;
  if (info_buf.alloc(sizeof(int))) return HPS_ENOMEM;
  int *info = info_buf.as<int>();
  cudaMemsetAsync(info, 0, sizeof(int), st);

  // child-level DtN maps T, per node or shared
  const int b_ld = ld_pad(b);
  const int nleaf_ops = shared ? 1 : H->lev[L].nodes;
  DevBuf Tchild;
  if (Tchild.alloc((size_t)nleaf_ops * b * b_ld * sizeof(double))) return HPS_ENOMEM;
  int64_t strTc = shared ? 0 : (int64_t)b * b_ld;
  int ldTc = b_ld;

  if (identity) {
    k_leaf_T_ident<<<1, kT, 0, st>>>(p, Tchild.as<double>(), b_ld, H->d_D);
  } else {
    ops.ldA = ld_pad(q);   // A_ii^{-1} stored transposed: q columns of ldA
    ops.ldSl = ld_pad(q);  // S stored transposed: b columns of ldSl
    ops.strA = shared ? 0 : (int64_t)q * ops.ldA;
    ops.strSl = shared ? 0 : (int64_t)b * ops.ldSl;
    const size_t na = (size_t)nleaf_ops * q * ops.ldA, ns = (size_t)nleaf_ops * b * ops.ldSl;
    if (cudaMalloc(&ops.Ainv, na * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(ops.Ainv);
    if (cudaMalloc(&ops.Sleaf, ns * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(ops.Sleaf);
    const int W = 2 * q + b, ldG = ld_pad(W);
    const size_t per = (size_t)q * ldG * sizeof(double);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)nleaf_ops, kWorkBytes / per, (size_t)32768}));
    DevBuf Gb, Mb;
    if (Gb.alloc(per * chunk) || Mb.alloc((size_t)chunk * q * sizeof(double))) return HPS_ENOMEM;
    for (int k0 = 0; k0 < nleaf_ops; k0 += chunk) {
      const int nc = std::min(chunk, nleaf_ops - k0);
      k_leaf_assemble<<<nc, kT, 0, st>>>(H->g, H->lev[L].d_origin, k0, H->d_coef, H->g.N_int, H->cst[0], H->cst[1],
                                         H->cst[2], H->cst[3], H->cst[4], H->d_D, gamma_dt, Gb.as<double>(), ldG);
      if (int e = gauss_jordan(Gb.as<double>(), ldG, W, q, nc, Mb.as<double>(), info, st)) return e;
      k_leaf_extract<<<nc, kT, 0, st>>>(p, k0, Gb.as<double>(), ldG, ops.Ainv, ops.ldA, ops.strA, ops.Sleaf,
                                        ops.ldSl, ops.strSl, Tchild.as<double>(), b_ld, H->d_D);
    }
  }
  if (cudaPeekAtLastError() != cudaSuccess) return HPS_ECUDA;

  for (int l = L - 1; l >= 0; --l) {
    const Level &lv = H->lev[l];
    MergeOps &mo = ops.merge[l];
    const int n3 = lv.n3, nb = lv.nb, nops = shared ? 1 : lv.nodes;
    // all three stored transposed: X^T (n3 x n3), S^T (nb x n3), Tcat^T (n3 x nb)
    mo.ldX = ld_pad(n3);
    mo.ldS = ld_pad(n3);
    mo.ldT = ld_pad(nb);
    mo.strX = shared ? 0 : (int64_t)n3 * mo.ldX;
    mo.strS = shared ? 0 : (int64_t)nb * mo.ldS;
    mo.strT = shared ? 0 : (int64_t)n3 * mo.ldT;
    if (cudaMalloc(&mo.X, (size_t)nops * n3 * mo.ldX * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(mo.X);
    if (cudaMalloc(&mo.S, (size_t)nops * nb * mo.ldS * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(mo.S);
    if (l > 0) {  // the root never forms h^t, so it keeps no Tcat
      if (cudaMalloc(&mo.Tcat, (size_t)nops * n3 * mo.ldT * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
      H->allocs.push_back(mo.Tcat);
    }
    const int W = 2 * n3 + nb, ldG = ld_pad(W);
    const size_t per = (size_t)n3 * ldG * sizeof(double);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)nops, kWorkBytes / per, (size_t)32768}));
    DevBuf Gb, Mb;
    if (Gb.alloc(per * chunk) || Mb.alloc((size_t)chunk * n3 * sizeof(double))) return HPS_ENOMEM;
    for (int k0 = 0; k0 < nops; k0 += chunk) {
      const int nc = std::min(chunk, nops - k0);
      k_merge_assemble<<<nc, kT, 0, st>>>(k0, n3, nb, lv.nbc, lv.j3a, lv.j3b, lv.d_hsrc, Tchild.as<double>(), ldTc,
                                          strTc, Gb.as<double>(), ldG, mo.Tcat, mo.ldT, mo.strT);
      if (int e = gauss_jordan(Gb.as<double>(), ldG, W, n3, nc, Mb.as<double>(), info, st)) return e;
      k_merge_extract<<<nc, kT, 0, st>>>(k0, n3, nb, Gb.as<double>(), ldG, mo.X, mo.ldX, mo.strX, mo.S, mo.ldS,
                                         mo.strS);
    }
    if (l > 0) {
      // T^t = diag(T^a_11, T^b_22) + Tcat S^t
      const int ldTp = ld_pad(nb);
      const int64_t strTp = shared ? 0 : (int64_t)nb * ldTp;
      DevBuf Tp;
      if (Tp.alloc((size_t)nops * nb * ldTp * sizeof(double))) return HPS_ENOMEM;
      const int64_t tot = (int64_t)nb * nb;
      dim3 gd((unsigned)std::min<int64_t>(4096, (tot + kT - 1) / kT), nops);
      k_merge_tdiag<<<gd, kT, 0, st>>>(nb, lv.nbc, lv.d_hsrc, Tchild.as<double>(), ldTc, strTc, Tp.as<double>(), ldTp,
                                       strTp);
      dim3 gg((nb + 63) / 64, (nb + 63) / 64, nops);
      // A = Tcat (nb x n3) from Tcat^T, B = S (n3 x nb) from S^T
      k_dgemm_acc<<<gg, 256, 0, st>>>(nb, nb, n3, mo.Tcat, 1, mo.ldT, mo.strT, mo.S, 1, mo.ldS, mo.strS,
                                      Tp.as<double>(), ldTp, strTp);
      if (cudaPeekAtLastError() != cudaSuccess) return HPS_ECUDA;
      std::swap(Tchild.p, Tp.p);
      ldTc = ldTp;
      strTc = strTp;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;  // before workspaces are freed
  }
  int hinfo = 0;
  cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;
  if (hinfo) return HPS_ESINGULAR;
  (void)m;
  return HPS_OK;
}

}  // namespace hps
