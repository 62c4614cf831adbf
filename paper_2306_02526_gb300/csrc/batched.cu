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
#include <cooperative_groups.h>
#include <cstdlib>
#include <utility>

#include "hps_internal.cuh"
#include "tc5.cuh"
#include <cuda_bf16.h>

namespace hps {

namespace {

constexpr int kBT = 256;
constexpr int kBSmemFloats = 8192;  // vector staging of the merge applies (32 KB)

__host__ __device__ inline int round4(int r) { return (r + 3) & ~3; }

}  // namespace

// FP32 <-> FP64 conversions on the integer pipe.  On this GPU the hardware conversions issue
// to the FP64 pipe (2 per SM per cycle, the rate of DFMA), which bounds the FP64 vector kernels;
// the IEEE-754 binary32 / binary64 layouts make the common cases a few integer operations.
// float -> double is exact: sign, exponent rebiased (+1023 - 127), mantissa shifted by 29;
// zeros are built directly, subnormal / infinite / NaN inputs take the hardware conversion.
__device__ __forceinline__ double f2d_int(float x) {
  const unsigned b = __float_as_uint(x), e = (b >> 23) & 0xffu, man = b & 0x7fffffu;
  if (e == 0xffu || (e == 0u && man != 0u)) return (double)x;
  const unsigned hi = (b & 0x80000000u) | (e == 0u ? 0u : ((e + 896u) << 20) | (man >> 3));
  return __hiloint2double((int)hi, (int)(man << 29));
}
// double -> float, rounded to nearest (ties to even): the top 23 of the 52 mantissa bits plus
// the rounding of the other 29 (a carry out of the mantissa increments the exponent, up to
// infinity, as IEEE rounding does); zeros directly; results below the normal float range,
// infinities and NaN take the hardware conversion.
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // binary32 biased exponent
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  if (e <= 0 || e >= 255) return (float)x;
  unsigned r = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) + ((unsigned)e << 23) + r);
}

// Self-check of the two conversions against the hardware ones over n bit patterns from a
// counter hash (all classes: zeros, subnormals, normals, infinities, NaN payloads) plus the
// float range edges; mismatches counted (NaN: any NaN result matches).
__global__ void k_conv_check(int64_t n, unsigned long long seed, unsigned long long *bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long z = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);  // splitmix64
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  double d = __longlong_as_double((long long)z);
  if ((i & 3) == 1) {  // doubles near the float range: exponent within +-40 of float's
    const unsigned long long ex = 896ull + (z >> 56) % 300ull - 20ull;
    d = __longlong_as_double((long long)((z & 0x800fffffffffffffull) | (ex << 52)));
  }
  if ((i & 3) == 2) {  // ties: the low 29 bits exactly half
    d = __longlong_as_double((long long)((z & ~0x1fffffffull) | 0x10000000ull));
  }
  const float fh = (float)d, fs = d2f_int(d);
  const bool okf = (fh != fh) ? (fs != fs) : __float_as_uint(fh) == __float_as_uint(fs);
  const float f = __uint_as_float((unsigned)z);
  const double dh = (double)f, ds = f2d_int(f);
  const bool okd = (dh != dh) ? (ds != ds) : __double_as_longlong(dh) == __double_as_longlong(ds);
  if (!okf || !okd) atomicAdd(bad, 1ull);
}

namespace {

// Where a sweep's FP32 result goes in the FP64 solution: u = v (assign) or u += v (a correction).
struct UOut {
  double *u;
  int assign;
};
__device__ __forceinline__ void u_out(const UOut &U, int64_t i, float v) {
  const double d = f2d_int(v);
  U.u[i] = U.assign ? d : U.u[i] + d;
}

// Stage epilogue of an implicit ARK stage (Eq. 2.3-2.4 split): from the solved stage value
// U_i (interior point o of an [N][R] vector) the implicit term is recovered from the stage
// equation U_i - gamma dt L U_i = Rb_i: the batched path keeps it as gamma dt L U_i = U_i - Rb_i
// (the stage combinations take A_ij / gamma, exact for gamma = 1/4); the explicit term is
// dt (q_i + g(U_i)).  Only g without derivatives (pointwise) takes this form.
struct StageEpi {
  int on;
  const double *Rb;     // [N_int][R] stage right-hand side
  double *KL, *KE;      // [N_int][R] outputs (KL: gamma dt L U_i; may be null)
  const double *q;      // [N_int][qld] (columns qoff ..) or null
  int qld, qoff, g_kind;
  double dt, dtg;       // dt, dt * g_param[0]
};
__device__ __forceinline__ void stage_epi_point(const StageEpi &E, int R, int64_t o, double uu) {
  double e;
  switch (E.g_kind) {
    case HPS_G_ALLEN_CAHN: e = E.dtg * (uu - uu * uu * uu); break;
    case HPS_G_FISHER: e = E.dtg * uu * (1.0 - uu); break;
    default: e = 0.0;
  }
  if (E.q) e = fma(E.dt, E.q[(o / R) * E.qld + E.qoff + o % R], e);
  if (E.KL) E.KL[o] = uu - E.Rb[o];
  E.KE[o] = e;
}

// u[u0 + idx] = (u[u0 + idx] +) val(idx, w[idx]) for idx < n (UOut semantics, exact float-to-double
// conversion), each thread loading w and u of U points before it stores any: a store to u may
// alias a later load of u, so a plain loop would wait out one load latency per point.
template <int U, class Val>
__device__ __forceinline__ void leaf_u_out(const UOut &uo, int64_t u0, const float *__restrict__ w, int n, Val val) {
  for (int base = threadIdx.x; base < n; base += U * blockDim.x) {
    float wv[U];
    double uv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < n) {
        wv[u] = w[idx];
        uv[u] = uo.assign ? 0.0 : uo.u[u0 + idx];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < n) {
        const double d = f2d_int(val(idx, wv[u]));
        uo.u[u0 + idx] = uo.assign ? d : uv[u] + d;
      }
    }
  }
}

// Block-wide loop over [0, n): every thread issues U independent loads before it uses any of
// them (a warp issues in order, so a load-then-store loop would wait out one load latency per
// element).
template <int U, class T, class Load, class Use>
__device__ __forceinline__ void block_gather(int n, Load ld, Use use) {
  for (int base = threadIdx.x; base < n; base += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < n) v[u] = ld(idx);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < n) use(idx, v[u]);
    }
  }
}

// The stage right-hand sides of all leaves at once (interior points are contiguous): FP64 sum
// to Rsave (if non-null) and its FP32 copy to r32, four entries per thread.
__global__ void k_b_combo(int64_t n, Combo rhs, double *__restrict__ Rsave, float *__restrict__ r32) {
  constexpr int U = 4;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x;
  double acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0.0;
  for (int t = 0; t < rhs.n; t += 2) {
    const bool two = t + 1 < rhs.n;
    const double *s0 = rhs.ptr[t], *s1 = two ? rhs.ptr[t + 1] : s0;
    const double c0 = rhs.coef[t], c1 = two ? rhs.coef[t + 1] : 0.0;
    double v0[U], v1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + (int64_t)u * blockDim.x;
      v0[u] = i < n ? s0[i] : 0.0;
      v1[u] = i < n ? s1[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = fma(c1, v1[u], fma(c0, v0[u], acc[u]));
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = base + (int64_t)u * blockDim.x;
    if (i < n) {
      if (Rsave) Rsave[i] = acc[u];
      r32[i] = d2f_int(acc[u]);
    }
  }
}

// 16-byte asynchronous global -> shared copies (cp.async): a CTA issues all copies of a tile,
// then waits once, so the tile costs one memory round trip instead of one per dependent load.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the previous kernel in the stream finishes; pdl_wait blocks until that kernel has
// completed and its memory operations are visible, so everything before it may only read data no
// kernel of the step writes (the operators).  pdl_trigger lets the next such kernel be scheduled
// once every CTA of this grid has started.  Both are no-ops without that launch attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The stage right-hand side of one leaf, sum_t coef_t ptr_t, over its nq = q*R contiguous
// entries from offset `off` (FP64): saved to Rsave if non-null and staged as FP32 at
// Rs[(f / R) * Rp + f % R]; U entries per thread and two terms per round of loads.
// (threads t0, t0 + nt, ... of the CTA take part; default: all of them)
template <int U>
__device__ __forceinline__ void stage_combo(const Combo &rhs, int64_t off, int nq, int R, int Rp,
                                            double *__restrict__ Rsave, float *Rs, int t0 = -1, int nt = 0) {
  // FP64 operations per point: one per term, none for a leading term with coefficient 1 (the
  // FP64 pipe bounds this loop on this GPU)
  const bool unit0 = rhs.n > 0 && rhs.coef[0] == 1.0;
  if (t0 < 0) {
    t0 = (int)threadIdx.x;
    nt = (int)blockDim.x;
  }
  for (int base = t0; base < nq; base += U * nt) {
    double acc[U];
    {
      const double *s0 = rhs.ptr[0] + off;
      const double c0 = rhs.n > 0 ? rhs.coef[0] : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * nt;
        const double v = idx < nq && rhs.n > 0 ? s0[idx] : 0.0;
        acc[u] = unit0 ? v : c0 * v;
      }
    }
    int t = 1;
    for (; t + 1 < rhs.n; t += 2) {
      const double *s0 = rhs.ptr[t] + off, *s1 = rhs.ptr[t + 1] + off;
      const double c0 = rhs.coef[t], c1 = rhs.coef[t + 1];
      double v0[U], v1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * nt;
        v0[u] = idx < nq ? s0[idx] : 0.0;
        v1[u] = idx < nq ? s1[idx] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = fma(c1, v1[u], fma(c0, v0[u], acc[u]));
    }
    if (t < rhs.n) {
      const double *s0 = rhs.ptr[t] + off;
      const double c0 = rhs.coef[t];
      double v0[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * nt;
        v0[u] = idx < nq ? s0[idx] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = fma(c0, v0[u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * nt;
      if (idx < nq) {
        if (Rsave) Rsave[off + idx] = acc[u];
        Rs[(idx / R) * Rp + idx % R] = d2f_int(acc[u]);
      }
    }
  }
}


// 4 columns (j0 .. j0+3) of the flux of edge point e: float4 reads of the interior field.
__device__ __forceinline__ float4 flux4(int e, int j0, int Rp, const float *W, const float *D1x, const float *D1y,
                                        int p, int m) {
  const int side = e / m, t = e - side * m;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  const float *d;
  int base, step;
  if (side == 0 || side == 2) {  // horizontal edge: d/dy along column t
    d = D1y + (side == 0 ? 0 : (p - 1) * p);
    base = t;
    step = m;
  } else {  // vertical edge: d/dx along row t
    d = D1x + (side == 1 ? (p - 1) * p : 0);
    base = t * m;
    step = 1;
  }
  for (int jj = 1; jj <= m; ++jj) {
    const float dv = d[jj];
    const float4 w = *reinterpret_cast<const float4 *>(W + (base + (jj - 1) * step) * Rp + j0);
    s.x = fmaf(dv, w.x, s.x);
    s.y = fmaf(dv, w.y, s.y);
    s.z = fmaf(dv, w.z, s.z);
    s.w = fmaf(dv, w.w, s.w);
  }
  return s;
}

// Outputs of a leaf apply from the interior field W [q][Rp] in shared memory: w32 (the field)
// and h32 (its fluxes on the b edge points), four columns per thread step.
__device__ __forceinline__ void leaf_up_out(int64_t k, int q, int b, int R, int Rp, const float *Ws, const float *D1x,
                                            const float *D1y, int p, int m, float *__restrict__ w32,
                                            float *__restrict__ h32, int t0, int nt) {
  const int Rq = Rp / 4;
  if (R == Rp) {
    float4 *wo = reinterpret_cast<float4 *>(w32 + k * q * R);
    for (int i = t0; i < q * Rq; i += nt) wo[i] = reinterpret_cast<const float4 *>(Ws)[i];
  } else {
    for (int idx = t0; idx < q * R; idx += nt) {
      const int r = idx / R, j = idx - r * R;
      w32[(k * q + r) * R + j] = Ws[r * Rp + j];
    }
  }
  for (int i = t0; i < b * Rq; i += nt) {
    const int e = i / Rq, j0 = 4 * (i - e * Rq);
    const float4 f = flux4(e, j0, Rp, Ws, D1x, D1y, p, m);
    float *o = h32 + (k * b + e) * R + j0;
    if (R == Rp) {
      *reinterpret_cast<float4 *>(o) = f;
    } else {
      const float fv[4] = {f.x, f.y, f.z, f.w};
      for (int t = 0; t < 4 && j0 + t < R; ++t) o[t] = fv[t];
    }
  }
}
__device__ __forceinline__ void leaf_up_out(int64_t k, int q, int b, int R, int Rp, const float *Ws, const float *D1x,
                                            const float *D1y, int p, int m, float *__restrict__ w32,
                                            float *__restrict__ h32) {
  leaf_up_out(k, q, b, R, Rp, Ws, D1x, D1y, p, m, w32, h32, (int)threadIdx.x, (int)blockDim.x);
}

// The boundary values of box (ix, iy, a x c) for R columns into ub [nb][Rp] (zero padding):
// the global index of each boundary position is computed once per four columns.
template <int U = 4>
__device__ __forceinline__ void gather_box(const GridDims &g, int ix, int iy, int a, int c, int nb, int R, int Rp,
                                           const float *__restrict__ src, float *ub) {
  const int Rq = Rp / 4;
  block_gather<U, float4>(
      nb * Rq,
      [&](int i) {
        const int pos = i / Rq, j0 = 4 * (i - pos * Rq);
        const float *p = src + box_bd(g, ix, iy, a, c, pos) * R + j0;
        return make_float4(p[0], j0 + 1 < R ? p[1] : 0.f, j0 + 2 < R ? p[2] : 0.f, j0 + 3 < R ? p[3] : 0.f);
      },
      [&](int i, float4 v) { reinterpret_cast<float4 *>(ub)[i] = v; });
}

// ---- leaf applies (FP32, R columns) ------------------------------------------------------
// Register tile per thread: 4 consecutive rows (one 16-byte operator load per column of the
// transposed operator) x TC columns of the right-hand sides (TC/4 16-byte shared loads).

template <int TC>
__device__ __forceinline__ void tile_fma(float (&acc)[4][TC], const float4 a, const float *x) {
  float xv[TC];
  if constexpr (TC % 4 == 0) {
#pragma unroll
    for (int t = 0; t < TC; t += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(x + t);
      xv[t] = v.x; xv[t + 1] = v.y; xv[t + 2] = v.z; xv[t + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int t = 0; t < TC; t += 2) {
      const float2 v = *reinterpret_cast<const float2 *>(x + t);
      xv[t] = v.x; xv[t + 1] = v.y;
    }
  }
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    acc[0][t] = fmaf(a.x, xv[t], acc[0][t]);
    acc[1][t] = fmaf(a.y, xv[t], acc[1][t]);
    acc[2][t] = fmaf(a.z, xv[t], acc[2][t]);
    acc[3][t] = fmaf(a.w, xv[t], acc[3][t]);
  }
}

// acc += A x over K columns of the transposed operator (4 rows per float4 load, column c at
// a + c ld) with U operator loads in flight per thread: the chain of dependent L2 round trips
// is K / U long instead of K.
template <int TC, int U>
__device__ __forceinline__ void stream_fma(float (&acc)[4][TC], const float *__restrict__ a, int64_t ld, int K,
                                           const float *x, int Rp) {
  int c = 0;
  for (; c + U <= K; c += U) {
    float4 av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) av[u] = __ldg(reinterpret_cast<const float4 *>(a + (int64_t)(c + u) * ld));
#pragma unroll
    for (int u = 0; u < U; ++u) tile_fma<TC>(acc, av[u], x + (c + u) * Rp);
  }
  for (; c < K; ++c) tile_fma<TC>(acc, __ldg(reinterpret_cast<const float4 *>(a + (int64_t)c * ld)), x + c * Rp);
}

// acc += A x with the operator tile in shared memory (4 rows per float4, column c at a + c lda)
template <int TC>
__device__ __forceinline__ void smem_fma(float (&acc)[4][TC], const float *a, int lda, int K, const float *x, int Rp) {
#pragma unroll 4
  for (int c = 0; c < K; ++c) tile_fma<TC>(acc, *reinterpret_cast<const float4 *>(a + c * lda), x + c * Rp);
}

template <int TC>
__global__ void __launch_bounds__(kBT) k_b_leaf_up(GridDims g, int R, const int *__restrict__ origin, Combo rhs,
                                                   double *__restrict__ Rsave, const float *__restrict__ r32,
                                                   const float *__restrict__ AinvT, int ldA, int64_t strA,
                                                   int identity, const double *__restrict__ Dg,
                                                   float *__restrict__ w32, float *__restrict__ h32) {
  extern __shared__ __align__(16) float smf[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, Rp = round4(R);
  float *D1x = smf, *D1y = smf + p * p, *Rs = smf + round4(2 * p * p), *Ws = Rs + q * Rp;
  const int k = blockIdx.x;
  const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) smf[i] = (float)Dg[i];
  if (r32 && Rp == R) {  // right-hand side formed by k_b_combo: one asynchronous copy
    for (int i = threadIdx.x; i < q * R / 4; i += blockDim.x) cp_async16(Rs + 4 * i, r32 + l0 * R + 4 * i);
    cp_async_wait_all();
  } else if (r32) {
    block_gather<8, float>(
        q * Rp,
        [&](int idx) {
          const int r = idx / Rp, j = idx % Rp;
          return j < R ? r32[(l0 + r) * R + j] : 0.f;
        },
        [&](int idx, float v) { Rs[idx] = v; });
  } else {
    if (Rp != R)  // padding columns
      for (int idx = threadIdx.x; idx < q * Rp; idx += blockDim.x) Rs[idx] = 0.f;
    __syncthreads();
    stage_combo<8>(rhs, l0 * R, q * R, R, Rp, Rsave, Rs);
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
      stream_fma<TC, 8>(acc, AinvT + (int64_t)k * strA + r0, ldA, q, Rs + j0, Rp);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (r0 + e < q)
#pragma unroll
        for (int t = 0; t < TC; ++t) Ws[(r0 + e) * Rp + j0 + t] = acc[e][t];
  }
  __syncthreads();
  leaf_up_out(k, q, b, R, Rp, Ws, D1x, D1y, p, m, w32, h32);
}

template <int TC>
__global__ void __launch_bounds__(kBT) k_b_leaf_down(GridDims g, int R, const int *__restrict__ origin,
                                                     const float *__restrict__ SlT, int ldS, int64_t strS, int identity,
                                                     int staged, const float *__restrict__ w32,
                                                     const float *__restrict__ g32, UOut uo) {
  extern __shared__ __align__(16) float ub[];  // [b][Rp], then (staged) the output tile [q][Rp]
  const int m = g.m, q = m * m, b = 4 * m, Rp = round4(R);
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  float *Os = ub + b * Rp;
  if (!identity) {
    gather_box<2>(g, ix, iy, 1, 1, b, R, Rp, g32, ub);
    __syncthreads();
    const int QQ = (q + 3) / 4, CG = Rp / TC;
    for (int it = threadIdx.x; it < QQ * CG; it += blockDim.x) {
      const int r0 = 4 * (it % QQ), j0 = TC * (it / QQ);
      float acc[4][TC];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
      stream_fma<TC, 8>(acc, SlT + (int64_t)k * strS + r0, ldS, b, ub + j0, Rp);
      if (staged) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (r0 + e < q)
#pragma unroll
            for (int t = 0; t < TC; t += 4)
              *reinterpret_cast<float4 *>(Os + (r0 + e) * Rp + j0 + t) =
                  make_float4(acc[e][t], acc[e][t + 1], acc[e][t + 2], acc[e][t + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (r0 + e < q)
#pragma unroll
            for (int t = 0; t < TC; ++t)
              if (j0 + t < R)
                u_out(uo, (l0 + r0 + e) * R + j0 + t, w32[((int64_t)k * q + r0 + e) * R + j0 + t] + acc[e][t]);
      }
    }
    if (!staged) return;
    __syncthreads();
  }
  // u_i = w + S u_b: the leaf's interior block is contiguous in both vectors
  leaf_u_out<4>(uo, l0 * R, w32 + (int64_t)k * q * R, q * R,
                [&](int idx, float w) { return w + (identity ? 0.f : Os[(idx / R) * Rp + idx % R]); });
}

// ---- leaf apply by fast diagonalization (constant coefficients) -----------------------------
// W = A_ii^-1 R = (V_y (x) V_x) Lam (V_y^-1 (x) V_x^-1) R as four passes of m x m products along
// grid lines (x lines: the m interior points of a row; y lines: of a column), 4 m^3 R
// multiply-adds per leaf instead of m^4 R.  Each thread forms 4 outputs x 4 columns per pass
// (an outer product of a float4 of the transposed line operator and a float4 of the field).

// x pass: out[(j, i)][c] = sum_k M(i, k) in[(j, k)][c] (times Lam(j, i) if lam); MT = M^T [k][mp]
__device__ __forceinline__ void fd_pass_x(const float *in, float *out, const float *MT, int m, int mp, int Rp,
                                          const float *lam) {
  const int IQ = mp / 4, Rq = Rp / 4;
  for (int it = threadIdx.x; it < m * IQ * Rq; it += blockDim.x) {
    const int c4 = it % Rq, t = it / Rq, iq = t % IQ, j = t / IQ;
    float4 acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float *inr = in + j * m * Rp + 4 * c4;
    for (int k = 0; k < m; ++k) {
      const float4 x = *reinterpret_cast<const float4 *>(inr + k * Rp);
      const float4 mv = *reinterpret_cast<const float4 *>(MT + k * mp + 4 * iq);
      const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a].x = fmaf(mm[a], x.x, acc[a].x);
        acc[a].y = fmaf(mm[a], x.y, acc[a].y);
        acc[a].z = fmaf(mm[a], x.z, acc[a].z);
        acc[a].w = fmaf(mm[a], x.w, acc[a].w);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * iq + a;
      if (i >= m) break;
      float4 v = acc[a];
      if (lam) {
        const float l = lam[j * mp + i];
        v.x *= l;
        v.y *= l;
        v.z *= l;
        v.w *= l;
      }
      *reinterpret_cast<float4 *>(out + (j * m + i) * Rp + 4 * c4) = v;
    }
  }
}

// y pass: out[(j, i)][c] = sum_k M(j, k) in[(k, i)][c] (times Lam(j, i) if lam)
__device__ __forceinline__ void fd_pass_y(const float *in, float *out, const float *MT, int m, int mp, int Rp,
                                          const float *lam) {
  const int JQ = mp / 4, Rq = Rp / 4;
  for (int it = threadIdx.x; it < m * JQ * Rq; it += blockDim.x) {
    const int c4 = it % Rq, t = it / Rq, jq = t % JQ, i = t / JQ;
    float4 acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float *inc = in + i * Rp + 4 * c4;
    for (int k = 0; k < m; ++k) {
      const float4 x = *reinterpret_cast<const float4 *>(inc + k * m * Rp);
      const float4 mv = *reinterpret_cast<const float4 *>(MT + k * mp + 4 * jq);
      const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a].x = fmaf(mm[a], x.x, acc[a].x);
        acc[a].y = fmaf(mm[a], x.y, acc[a].y);
        acc[a].z = fmaf(mm[a], x.z, acc[a].z);
        acc[a].w = fmaf(mm[a], x.w, acc[a].w);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int j = 4 * jq + a;
      if (j >= m) break;
      float4 v = acc[a];
      if (lam) {
        const float l = lam[j * mp + i];
        v.x *= l;
        v.y *= l;
        v.z *= l;
        v.w *= l;
      }
      *reinterpret_cast<float4 *>(out + (j * m + i) * Rp + 4 * c4) = v;
    }
  }
}

// One leaf per CTA: stage right-hand side (FP64 combination, saved if requested), the four
// passes between two shared-memory buffers, then w and the fluxes.  fd32 holds [V_x, V_x^-1,
// V_y, V_y^-1, Lam], each m x mp, then D1x, D1y (p x p each, read through L1: with 54.7 KB of
// shared memory and 64 registers four CTAs fit on an SM).
__global__ void __launch_bounds__(kBT, 4) k_b_leaf_up_fd(GridDims g, int R, const int *__restrict__ origin, Combo rhs,
                                                      double *__restrict__ Rsave, const float *__restrict__ fd32,
                                                      int mp, float *__restrict__ w32, float *__restrict__ h32) {
  extern __shared__ __align__(16) float sfd[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, Rp = round4(R), mm = m * mp;
  float *MT = sfd, *Lam = MT + 4 * mm;
  const float *D1x = fd32 + 5 * mm, *D1y = D1x + p * p;  // FP32 copies after the factors (L1-cached)
  float *Rs = Lam + mm, *Ts = Rs + q * Rp;
  const int k = blockIdx.x;
  const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
  for (int idx = threadIdx.x; idx < 4 * mm; idx += blockDim.x) {  // transposed line operators
    const int a = idx / mm, r = idx % mm, kk = r / mp, i = r % mp;
    MT[idx] = i < m ? fd32[((size_t)a * m + i) * mp + kk] : 0.f;
  }
  for (int idx = threadIdx.x; idx < mm; idx += blockDim.x) Lam[idx] = fd32[4 * (size_t)mm + idx];
  if (Rp != R)
    for (int idx = threadIdx.x; idx < q * Rp; idx += blockDim.x) Rs[idx] = 0.f;
  __syncthreads();
  stage_combo<8>(rhs, l0 * R, q * R, R, Rp, Rsave, Rs);
  __syncthreads();
  fd_pass_x(Rs, Ts, MT + 1 * mm, m, mp, Rp, nullptr);  // V_x^-1 along x
  __syncthreads();
  fd_pass_y(Ts, Rs, MT + 3 * mm, m, mp, Rp, Lam);      // V_y^-1 along y, then Lam
  __syncthreads();
  fd_pass_y(Rs, Ts, MT + 2 * mm, m, mp, Rp, nullptr);  // V_y along y
  __syncthreads();
  fd_pass_x(Ts, Rs, MT + 0 * mm, m, mp, Rp, nullptr);  // V_x along x
  __syncthreads();
  leaf_up_out(k, q, b, R, Rp, Rs, D1x, D1y, p, m, w32, h32);
}

// ---- leaf apply on the tensor cores: 3xTF32 warp MMA (m16n8k8) -----------------------------
// W = A_ii^{-1} R with the shared operator: each FP32 operand x is split into two TF32 numbers
// x = hi + lo (hi = x rounded to TF32, lo = x - hi rounded to TF32) and the product is formed as
// A_lo B_hi + A_hi B_lo + A_hi B_hi with FP32 accumulation (the dropped A_lo B_lo is below FP32
// rounding), i.e. FP32 accuracy at tensor-core rate.  The operator's hi / lo fragments are laid
// out once in lane order (k_frag_a); the right-hand side is split while it is staged.
// Fragment layouts of mma.m16n8k8 with .tf32 operands (g = lane / 4, t = lane % 4):
//   A 16x8 row-major: a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B 8x8:            b0 (k = t, n = g), b1 (k = t + 4, n = g)
//   C 16x8 FP32:      c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
constexpr int kTcMaxMT = 16;  // row tiles of 16 (q <= 256)
constexpr int kTcMaxNT = 4;   // column tiles of 8 (R <= 32)
__host__ __device__ inline int tc_rs(int Rp) { return Rp + (Rp % 16 == 0 ? 8 : 0); }

__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint4 &a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// hi / lo TF32 fragments of the q x q operator (stored transposed: A(r, c) at AT[c ld + r]),
// tile (mt, kt), lane l, register i at ((mt KT + kt) 32 + l) 4 + i; zero outside q x q.
__global__ void k_frag_a(const float *__restrict__ AT, int ld, int q, int MT, int KT, unsigned *__restrict__ hi,
                         unsigned *__restrict__ lo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)MT * KT * 128) return;
  const int i = (int)(idx % 4), lane = (int)(idx / 4 % 32);
  const int64_t tile = idx / 128;
  const int mt = (int)(tile / KT), kt = (int)(tile % KT);
  const int g = lane / 4, t = lane % 4;
  const int r = mt * 16 + g + (i & 1) * 8, c = kt * 8 + t + (i >> 1) * 4;
  const float v = (r < q && c < q) ? AT[(int64_t)c * ld + r] : 0.f;
  const unsigned h = tf32_rna(v);
  hi[idx] = h;
  lo[idx] = tf32_rna(v - __uint_as_float(h));
}

// One leaf per CTA (8 warps; warp w takes row tiles w, w + 8).  Shared memory: the right-hand
// side as TF32 hi / lo [KT*8][RS] (RS = 8 or 24 mod 32 keeps the B-fragment reads conflict-free), then
// W [q][Rp] in the hi buffer, and the differentiation rows for the fluxes.
template <int NT>
__global__ void __launch_bounds__(kBT) k_b_leaf_up_tc(GridDims g, int R, const int *__restrict__ origin, Combo rhs,
                                                      double *__restrict__ Rsave, const uint4 *__restrict__ Ahi,
                                                      const uint4 *__restrict__ Alo, int MT, int KT,
                                                      const double *__restrict__ Dg, float *__restrict__ w32,
                                                      float *__restrict__ h32) {
  extern __shared__ __align__(16) float smt[];
  const int p = g.p, m = g.m, q = m * m, b = 4 * m, Rp = NT * 8, RS = tc_rs(Rp);
  float *D1x = smt, *D1y = smt + p * p;
  unsigned *Bh = reinterpret_cast<unsigned *>(smt + round4(2 * p * p)), *Bl = Bh + KT * 8 * RS;
  float *Ws = reinterpret_cast<float *>(Bh);  // [q][Rp] after the products
  const int k = blockIdx.x;
  const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) smt[i] = (float)Dg[i];
  for (int i = threadIdx.x; i < (KT * 8 - q) * RS; i += blockDim.x) {  // padding rows of K
    Bh[q * RS + i] = 0u;
    Bl[q * RS + i] = 0u;
  }
  if (R != Rp)  // padding columns
    for (int i = threadIdx.x; i < q * RS; i += blockDim.x) {
      Bh[i] = 0u;
      Bl[i] = 0u;
    }
  __syncthreads();
  // stage right-hand side (FP64 combination, saved if requested), split into TF32 hi / lo
  constexpr int U = 8;
  const int nq = q * R;
  for (int base = threadIdx.x; base < nq; base += U * blockDim.x) {
    double acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0;
    for (int t = 0; t < rhs.n; t += 2) {
      const bool two = t + 1 < rhs.n;
      const double *s0 = rhs.ptr[t] + l0 * R, *s1 = two ? rhs.ptr[t + 1] + l0 * R : s0;
      const double c0 = rhs.coef[t], c1 = two ? rhs.coef[t + 1] : 0.0;
      double v0[U], v1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * blockDim.x;
        v0[u] = idx < nq ? s0[idx] : 0.0;
        v1[u] = idx < nq ? s1[idx] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = fma(c1, v1[u], fma(c0, v0[u], acc[u]));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < nq) {
        if (Rsave) Rsave[l0 * R + idx] = acc[u];
        const float v = d2f_int(acc[u]);
        const unsigned h = tf32_rna(v);
        const int o = (idx / R) * RS + idx % R;
        Bh[o] = h;
        Bl[o] = tf32_rna(v - __uint_as_float(h));
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, gq = lane / 4, tq = lane % 4;
  float acc[2][NT][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[s][n][e] = 0.f;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int mt = warp + 8 * s;
    if (mt >= MT) break;
    for (int kt = 0; kt < KT; ++kt) {
      const uint4 ah = __ldg(Ahi + ((int64_t)mt * KT + kt) * 32 + lane);
      const uint4 al = __ldg(Alo + ((int64_t)mt * KT + kt) * 32 + lane);
      const int r0 = (kt * 8 + tq) * RS + gq, r1 = r0 + 4 * RS;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const unsigned bh0 = Bh[r0 + 8 * n], bh1 = Bh[r1 + 8 * n], bl0 = Bl[r0 + 8 * n], bl1 = Bl[r1 + 8 * n];
        mma_tf32(acc[s][n], al, bh0, bh1);
        mma_tf32(acc[s][n], ah, bl0, bl1);
        mma_tf32(acc[s][n], ah, bh0, bh1);
      }
    }
  }
  __syncthreads();  // every warp is done with the staged right-hand side
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int mt = warp + 8 * s;
    if (mt >= MT) break;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int r = mt * 16 + gq, c = n * 8 + 2 * tq;
      if (r < q) {
        Ws[r * Rp + c] = acc[s][n][0];
        Ws[r * Rp + c + 1] = acc[s][n][1];
      }
      if (r + 8 < q) {
        Ws[(r + 8) * Rp + c] = acc[s][n][2];
        Ws[(r + 8) * Rp + c + 1] = acc[s][n][3];
      }
    }
  }
  __syncthreads();
  leaf_up_out(k, q, b, R, Rp, Ws, D1x, D1y, p, m, w32, h32);
}

// ---- leaf apply with per-node operators on the 5th-generation tensor cores -----------------
// W = A_ii^{-1} Rs on every leaf from the per-node FP32 operators split once, at reserve time,
// into TF32 hi and lo parts (A = Ah + Al exactly in FP32; both stored K-major, [leaf][hi|lo][row]
// [ldk]), as 3xTF32 products W ~ Ah Bh + Ah Bl + Al Bh (Rs = Bh + Bl) accumulated in FP32 in
// tensor memory: an M = 128 x N = RP accumulator per 128-row tile of the leaf, two accumulator
// sets so that one leaf's products run while the previous leaf's are read back.  Storing the
// split costs twice the operator bytes but leaves the operands exactly as the TMA writes them, so
// no thread touches them: the kernel streams HBM -> shared memory -> tensor cores.
// Persistent CTAs (one per SM) with three warp roles that meet only at mbarriers:
//   warp 0   TMA producer: per box the hi and lo boxes of 128 rows x 32 columns (128-byte swizzle;
//            rows and columns beyond q read as zeros) into one of kUmmaStages stages;
//   warp 1   MMA issuer: per box 4 K steps x 3 tcgen05.mma kind::tf32, committed to the stage's
//            "free" barrier, and per leaf to its accumulator set's barrier;
//   warps 2+ math: the leaf's right-hand side (FP32, formed in FP64 by the streaming combination
//            pass k_b_combo, which also saves the FP64 sum; prefetched into registers one leaf
//            ahead) into hi / lo operand tiles (two buffers, by leaf parity), and the epilogue of
//            the previous leaf (tcgen05.ld into shared memory over that leaf's operand tiles,
//            then w and its edge fluxes like every other leaf apply).
// Every wait is bounded: one that runs out raises the CTA's abort flag, the roles leave their
// loops, the copies and products still in flight are waited for, *err is set and the CTA returns.
constexpr int kUmmaStages = 3;
constexpr int kUmmaMathWarps = 8;
constexpr int kUmmaThreads = 64 + 32 * kUmmaMathWarps;
constexpr unsigned kUmmaBoxBytes = 128u * 32u * 4u;  // one box: 128 rows x 32 FP32
constexpr uint64_t kUmmaWaitNs = 2000000000ull;
constexpr int kUmmaPre = 8;  // float4 registers per math thread for the next leaf's right-hand side

__host__ __device__ inline int umma_kc(int q) { return (q + 31) / 32; }
__host__ __device__ inline int umma_mt(int q) { return (q + 127) / 128; }
// W staging row stride (floats): RP + 4 keeps the accumulator read-back from piling onto a bank
__host__ __device__ constexpr int umma_ldw(int RP) { return RP + 4; }
// barriers: full and free per stage; operand tiles ready; per accumulator set done and free;
// W staged, W read; drain
constexpr int kUmmaBars = 2 * kUmmaStages + 1 + 4 + 2 + 1;
// dynamic shared memory of k_b_leaf_up_umma<RP> (bytes, with the 1024-byte alignment slack)
inline size_t umma_smem_bytes(int p, int RP) {
  const int q = (p - 2) * (p - 2);
  return 1024 + (size_t)kUmmaStages * 2 * kUmmaBoxBytes + 2 * 2 * (size_t)umma_kc(q) * RP * 128 +
         (size_t)2 * p * p * 4 + kUmmaBars * 8 + 16;
}
// the leaf's q x R right-hand side block must fit the prefetch registers and be float4-aligned,
// W (q x ldw) must fit over one operand-tile buffer, and a 32-column operator box must not be
// wider than the operator (q >= 32, i.e. p >= 8)
inline bool umma_fits(int p, int R, int RP) {
  const int q = (p - 2) * (p - 2);
  return (q * R) % 4 == 0 && q * R <= 4 * kUmmaPre * 32 * kUmmaMathWarps && q >= 32 && q <= 256 &&
         (size_t)q * umma_ldw(RP) * 4 <= 2 * (size_t)umma_kc(q) * RP * 128 && umma_smem_bytes(p, RP) <= 232448;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc5::smem_u32(bar)) : "memory");
}
// Bounded wait that also gives up as soon as another role has raised the abort flag.
__device__ __forceinline__ bool umma_wait(uint64_t *bar, unsigned parity, volatile int *abort_flag) {
  if (tc5::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = tc5::global_ns();
  while (!tc5::mbar_try_wait(bar, parity)) {
    if (*abort_flag || tc5::global_ns() - t0 > kUmmaWaitNs) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
// RP/2 accumulator columns of the calling warp's 32 TMEM lanes
template <int NC>
__device__ __forceinline__ void tmem_ld_half(unsigned taddr, float *v) {
  if constexpr (NC == 16) {
    float t[16];
    tc5::tmem_ld16(taddr, t);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
  } else {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
  }
}
// One operand element of B (K index r, column n) as TF32 hi / lo at its swizzled position.
// (BF: the value rounded to BF16 at its position in the 64-per-line BF16 layout, no lo part)
template <int RP, bool BF>
__device__ __forceinline__ void umma_put_b(uint8_t *Bh, uint8_t *Bl, int r, int n, float v) {
  if constexpr (BF) {
    const int k = r & 63;
    const unsigned off = (unsigned)(r >> 6) * (RP * 128) + (unsigned)(n * 128 + ((((k >> 3) ^ (n & 7)) & 7) << 4) + (k & 7) * 2);
    *reinterpret_cast<__nv_bfloat16 *>(Bh + off) = __float2bfloat16_rn(v);
  } else {
    const float h = tc5::tf32_hi(v);
    const unsigned off = (unsigned)(r >> 5) * (RP * 128) + tc5::sw128_off(n, r & 31);
    *reinterpret_cast<float *>(Bh + off) = h;
    *reinterpret_cast<float *>(Bl + off) = v - h;
  }
}

template <int RP, bool BF>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_b_leaf_up_umma(GridDims g, int nodes, int R, const int *__restrict__ origin, const float *__restrict__ r32,
                     const __grid_constant__ CUtensorMap tmA, const double *__restrict__ Dg,
                     float *__restrict__ w32, float *__restrict__ h32, int *__restrict__ err) {
  namespace t5 = tc5;
  constexpr int kSet = 2 * RP;     // TMEM columns of one accumulator set (up to 2 row tiles)
  constexpr int kCols = 2 * kSet;  // two sets: 64 or 128 columns
  constexpr int NTM = 32 * kUmmaMathWarps, RQ = RP / 4, LDW = umma_ldw(RP);
  extern __shared__ uint8_t sm_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
  const int p = g.p, m = g.m, q = m * m, b = 4 * m;
  // BF (the BF16 trial): one BF16 product per K step of 16, 64 K values per 128-byte line
  constexpr int KL = BF ? 64 : 32;
  const int KC = (q + KL - 1) / KL, MT = umma_mt(q), KSTEPS = BF ? (q + 15) / 16 : (q + 7) / 8, NCH = MT * KC;
  const int BT = umma_kc(q) * RP * 128;                        // one operand-tile set (hi or lo)
  uint8_t *Stg = sm;                                           // stages: hi box, lo box
  uint8_t *Bbuf = sm + kUmmaStages * 2 * kUmmaBoxBytes;        // two buffers of (Bh, Bl)
  float *D1x = reinterpret_cast<float *>(Bbuf + 4 * BT), *D1y = D1x + p * p;
  uint64_t *bars = reinterpret_cast<uint64_t *>(D1y + p * p);
  uint64_t *full = bars, *sfree = full + kUmmaStages, *bready = sfree + kUmmaStages;
  uint64_t *accum = bready + 1, *tfree = accum + 2, *wsready = tfree + 2, *wsdone = wsready + 1;
  uint64_t *drain = wsdone + 1;
  unsigned *tslot = reinterpret_cast<unsigned *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kUmmaStages; ++s) {
      t5::mbar_init(&full[s], 1);
      t5::mbar_init(&sfree[s], 1);
    }
    t5::mbar_init(bready, NTM);
    for (int h = 0; h < 2; ++h) {
      t5::mbar_init(&accum[h], 1);
      t5::mbar_init(&tfree[h], NTM);
    }
    t5::mbar_init(wsready, NTM);
    t5::mbar_init(wsdone, NTM);
    t5::mbar_init(drain, 1);
    *abort_flag = 0;
    t5::fence_barrier_init();
    t5::tma_prefetch_desc(&tmA);
  }
  for (int i = tid; i < 2 * p * p; i += blockDim.x) D1x[i] = (float)Dg[i];
  if (warp == 1) t5::tmem_alloc(tslot, kCols);
  t5::tc_fence_before();
  __syncthreads();
  t5::tc_fence_after();
  const unsigned tmem = *tslot;
  // this CTA's leaves k = blockIdx.x + j gridDim.x; box c = j NCH + i, i = t KC + kc (row tile t,
  // column box kc), in stage c % kUmmaStages
  const int nl = (int)blockIdx.x < nodes ? (nodes - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = nl * NCH;
  int last_box[kUmmaStages];  // producer: last box loaded into each stage (-1: none)
  if (warp == 0 && lane == 0) {
    // ---------------- producer ----------------
    for (int s = 0; s < kUmmaStages; ++s) last_box[s] = -1;
    for (int c = 0; c < total; ++c) {
      const int j = c / NCH, i = c - j * NCH, s = c % kUmmaStages;
      const int k = (int)blockIdx.x + j * (int)gridDim.x;
      if (c >= kUmmaStages && !umma_wait(&sfree[s], (unsigned)((c - kUmmaStages) / kUmmaStages) & 1u, abort_flag))
        break;
      uint8_t *dst = Stg + s * 2 * kUmmaBoxBytes;
      if constexpr (BF) {  // one BF16 box of 128 rows x 64 columns
        t5::mbar_expect_tx(&full[s], kUmmaBoxBytes);
        t5::tma_load_3d(dst, &tmA, (i % KC) * 64, (i / KC) * 128, k, &full[s]);
      } else {
        t5::mbar_expect_tx(&full[s], 2 * kUmmaBoxBytes);
        t5::tma_load_3d(dst, &tmA, (i % KC) * 32, (i / KC) * 128, 2 * k, &full[s]);
        t5::tma_load_3d(dst + kUmmaBoxBytes, &tmA, (i % KC) * 32, (i / KC) * 128, 2 * k + 1, &full[s]);
      }
      last_box[s] = c;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const unsigned idesc = BF ? t5::idesc_bf16(128, RP) : t5::idesc_tf32(128, RP);
    for (int j = 0; j < nl; ++j) {
      const int hs = j & 1;
      if (j >= 2 && !umma_wait(&tfree[hs], (unsigned)((j - 2) >> 1) & 1u, abort_flag)) break;
      if (!umma_wait(bready, (unsigned)j & 1u, abort_flag)) break;
      t5::tc_fence_after();
      const uint8_t *Bh = Bbuf + hs * 2 * BT, *Bl = Bh + BT;
      bool ok = true;
      for (int i = 0; i < NCH; ++i) {
        const int c = j * NCH + i, s = c % kUmmaStages, t = i / KC, kc = i - t * KC;
        if (!umma_wait(&full[s], (unsigned)(c / kUmmaStages) & 1u, abort_flag)) {
          ok = false;
          break;
        }
        t5::tc_fence_after();
        const unsigned a_h = t5::smem_u32(Stg + s * 2 * kUmmaBoxBytes), a_l = a_h + kUmmaBoxBytes;
        const unsigned b_h = t5::smem_u32(Bh + kc * RP * 128), b_l = t5::smem_u32(Bl + kc * RP * 128);
        const unsigned d = tmem + (unsigned)(hs * kSet + t * RP);
        for (int ks = 0; ks < 4 && kc * 4 + ks < KSTEPS; ++ks) {
          const unsigned o = 32u * ks;  // 8 TF32 (16 BF16) values further along K in the 128-byte line
          if constexpr (BF) {
            t5::mma_bf16(d, t5::desc_sw128_kmajor(a_h + o), t5::desc_sw128_kmajor(b_h + o), idesc,
                         (kc > 0 || ks > 0) ? 1u : 0u);
          } else {
            t5::mma_tf32(d, t5::desc_sw128_kmajor(a_h + o), t5::desc_sw128_kmajor(b_h + o), idesc,
                         (kc > 0 || ks > 0) ? 1u : 0u);
            t5::mma_tf32(d, t5::desc_sw128_kmajor(a_h + o), t5::desc_sw128_kmajor(b_l + o), idesc, 1u);
            t5::mma_tf32(d, t5::desc_sw128_kmajor(a_l + o), t5::desc_sw128_kmajor(b_h + o), idesc, 1u);
          }
        }
        t5::mma_commit(&sfree[s]);
      }
      if (!ok) break;
      t5::mma_commit(&accum[hs]);
    }
    t5::mma_commit(drain);  // completes once every product this thread issued has completed
  } else if (warp >= 2) {
    // ---------------- math warps ----------------
    const int mt = tid - 64, mw = warp - 2;
    const int quarter = warp & 3, chalf = mw / 4;  // TMEM lanes 32 quarter .. +31, column half chalf
    const int nf4 = q * R / 4;
    float4 pre[kUmmaPre];  // the next leaf's right-hand side block (q x R FP32, contiguous)
    auto prefetch = [&](int jj) {
      const int k = (int)blockIdx.x + jj * (int)gridDim.x;
      const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
      const float4 *src = reinterpret_cast<const float4 *>(r32 + l0 * R);
#pragma unroll
      for (int u = 0; u < kUmmaPre; ++u) {
        const int e = mt + u * NTM;
        if (e < nf4) pre[u] = __ldg(src + e);
      }
    };
    // epilogue of leaf jj: accumulators -> W [q][LDW] over the leaf's operand tiles -> w, fluxes
    auto epilogue = [&](int jj) -> bool {
      const int hs = jj & 1, k = (int)blockIdx.x + jj * (int)gridDim.x;
      float *Ws = reinterpret_cast<float *>(Bbuf + hs * 2 * BT);
      bool ok = umma_wait(&accum[hs], (unsigned)(jj >> 1) & 1u, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) return false;
      t5::tc_fence_after();
      for (int t = 0; t < MT; ++t) {
        const int r = t * 128 + quarter * 32 + lane;
        const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(hs * kSet + t * RP + chalf * (RP / 2));
        float v[RP / 2];
        tmem_ld_half<RP / 2>(ta, v);
        if (r < q)
#pragma unroll
          for (int n = 0; n < RP / 2; n += 4)
            *reinterpret_cast<float4 *>(Ws + r * LDW + chalf * (RP / 2) + n) =
                make_float4(v[n], v[n + 1], v[n + 2], v[n + 3]);
      }
      t5::tc_fence_before();
      mbar_arrive(&tfree[hs]);  // this accumulator set may take the leaf after next
      mbar_arrive(wsready);
      ok = umma_wait(wsready, (unsigned)jj & 1u, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) return false;
      for (int i = mt; i < q * RQ; i += NTM) {  // w
        const int r = i / RQ, j0 = 4 * (i - r * RQ);
        const float4 v = *reinterpret_cast<const float4 *>(Ws + r * LDW + j0);
        float *o = w32 + ((int64_t)k * q + r) * R + j0;
        if (R == RP) {
          *reinterpret_cast<float4 *>(o) = v;
        } else {
          const float vv[4] = {v.x, v.y, v.z, v.w};
          for (int t = 0; t < 4 && j0 + t < R; ++t) o[t] = vv[t];
        }
      }
      for (int i = mt; i < b * RQ; i += NTM) {  // its fluxes on the b edge points
        const int e = i / RQ, j0 = 4 * (i - e * RQ);
        const float4 f = flux4(e, j0, LDW, Ws, D1x, D1y, p, m);
        float *o = h32 + ((int64_t)k * b + e) * R + j0;
        if (R == RP) {
          *reinterpret_cast<float4 *>(o) = f;
        } else {
          const float fv[4] = {f.x, f.y, f.z, f.w};
          for (int t = 0; t < 4 && j0 + t < R; ++t) o[t] = fv[t];
        }
      }
      mbar_arrive(wsdone);
      ok = umma_wait(wsdone, (unsigned)jj & 1u, abort_flag);  // W read: the region takes operand tiles
      return __all_sync(0xffffffffu, ok);
    };
    if (nl > 0) prefetch(0);
    bool run = true;
    for (int j = 0; j < nl; ++j) {
      // the leaf's right-hand side as hi / lo operand tiles in buffer j & 1 (N = RP lines, K = KC*32;
      // zero beyond q and R); the buffer's last use, leaf j - 2 and its epilogue, is over
      uint8_t *Bh = Bbuf + (j & 1) * 2 * BT, *Bl = Bh + BT;
#pragma unroll
      for (int u = 0; u < kUmmaPre; ++u) {
        const int e = mt + u * NTM;
        if (e < nf4) {
          const float vv[4] = {pre[u].x, pre[u].y, pre[u].z, pre[u].w};
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int f = 4 * e + cc, r = f / R;
            umma_put_b<RP, BF>(Bh, Bl, r, f - r * R, vv[cc]);
          }
        }
      }
      for (int idx = mt; idx < (KC * KL - q) * RP; idx += NTM)
        umma_put_b<RP, BF>(Bh, Bl, q + idx / RP, idx % RP, 0.f);
      if (R < RP)
        for (int idx = mt; idx < q * (RP - R); idx += NTM)
          umma_put_b<RP, BF>(Bh, Bl, idx / (RP - R), R + idx % (RP - R), 0.f);
      t5::fence_async_smem();
      mbar_arrive(bready);
      if (j + 1 < nl) prefetch(j + 1);
      if (j >= 1 && !epilogue(j - 1)) {
        run = false;
        break;
      }
    }
    if (run && nl > 0 && !*abort_flag) epilogue(nl - 1);
  }
  // wind down: every role has left its loop
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {  // copies still in flight (only a stage's last one can be)
    for (int s = 0; s < kUmmaStages; ++s)
      if (last_box[s] >= 0) t5::mbar_wait(&full[s], (unsigned)(last_box[s] / kUmmaStages) & 1u, kUmmaWaitNs);
    atomicExch(err, 1);
  }
  if (warp == 1 && lane == 0) t5::mbar_wait(drain, 0u, kUmmaWaitNs);  // products still running
  t5::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    t5::tc_fence_after();
    t5::tmem_dealloc(tmem, kCols);
  }
}

// Shared leaf operator, persistent CTAs: S_leaf^T is copied to shared memory once per CTA and
// every leaf the CTA takes is applied from there (a per-leaf CTA re-reads it from L1/L2).
template <int TC>
__global__ void __launch_bounds__(kBT) k_b_leaf_down_res(GridDims g, int nodes, int R, const int *__restrict__ origin,
                                                         const float *__restrict__ SlT, int ldS,
                                                         const float *__restrict__ w32, const float *__restrict__ g32,
                                                         UOut uo, StageEpi ep) {
  extern __shared__ __align__(16) float sres[];
  const int m = g.m, q = m * m, b = 4 * m, Rp = round4(R);
  float *Ss = sres, *ub = sres + (size_t)b * ldS, *Os = ub + b * Rp;  // [b][ldS], [b][Rp], [q][Rp]
  for (int i = threadIdx.x; i < b * ldS / 4; i += blockDim.x) cp_async16(Ss + 4 * i, SlT + 4 * i);
  cp_async_wait_all();
  const int QQ = (q + 3) / 4, CG = Rp / TC;
  for (int k = blockIdx.x; k < nodes; k += gridDim.x) {
    const int ix = origin[2 * k], iy = origin[2 * k + 1];
    const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
    __syncthreads();  // previous leaf done with ub; operator copy visible
    gather_box<2>(g, ix, iy, 1, 1, b, R, Rp, g32, ub);
    __syncthreads();
    for (int it = threadIdx.x; it < QQ * CG; it += blockDim.x) {
      // column groups fastest: the staged output rows are written without bank conflicts
      const int r0 = 4 * (it / CG), j0 = TC * (it % CG);
      float acc[4][TC];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
      smem_fma<TC>(acc, Ss + r0, ldS, b, ub + j0, Rp);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (r0 + e < q)
#pragma unroll
          for (int t = 0; t < TC; t += 4)
            *reinterpret_cast<float4 *>(Os + (r0 + e) * Rp + j0 + t) =
                make_float4(acc[e][t], acc[e][t + 1], acc[e][t + 2], acc[e][t + 3]);
    }
    __syncthreads();
    // u_i = w + S u_b: the leaf's interior block is contiguous in both vectors; the last sweep of
    // a stage solve also writes the stage epilogue from the finished value
    for (int idx = threadIdx.x; idx < q * R; idx += blockDim.x) {
      const int64_t o = l0 * R + idx;
      const float v = w32[(int64_t)k * q * R + idx] + Os[(idx / R) * Rp + idx % R];
      const double un = uo.assign ? (double)v : uo.u[o] + (double)v;
      uo.u[o] = un;
      if (ep.on) stage_epi_point(ep, R, o, un);
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
  if (R != 4)
    for (int idx = threadIdx.x; idx < q * 4; idx += blockDim.x) Rs[idx] = 0.f;
  __syncthreads();
  stage_combo<4>(rhs, l0 * R, q * R, R, 4, Rsave, Rs);
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
  leaf_up_out(k, q, b, R, 4, Ws, D1x, D1y, p, m, w32, h32);
}

__global__ void __launch_bounds__(kBT) k_b_leaf_down_narrow(GridDims g, int R, const int *__restrict__ origin,
                                                            const float *__restrict__ SlT, int ldS, int64_t strS,
                                                            int identity, const float *__restrict__ w32,
                                                            const float *__restrict__ g32, UOut uo) {
  extern __shared__ float smf[];
  const int m = g.m, q = m * m, b = 4 * m, QQ = (q + 3) / 4, KS = max(1, kBT / QQ);
  float *ub = smf, *part = smf + 4 * b;
  const int k = blockIdx.x;
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  gather_box(g, ix, iy, 1, 1, b, R, 4, g32, ub);
  __syncthreads();
  if (!identity) quad_apply_sliced(SlT + (int64_t)k * strS, ldS, b, ub, 4, QQ, KS, part);
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * R; idx += blockDim.x) {
    const int r = idx / R, j = idx % R;
    float s = w32[((int64_t)k * q + r) * R + j];
    if (!identity)
      for (int ks = 0; ks < KS; ++ks) s += part[(int64_t)ks * 16 * QQ + r * 4 + j];
    u_out(uo, (l0 + r) * R + j, s);
  }
}

// ---- streaming leaf applies for one to four columns (per-leaf operators) ------------------
// The per-leaf operators (A_ii^-1 for the particular solve, S for the interior solve) are read
// once per sweep and, leaf after leaf, lie contiguously in memory: one persistent CTA per SM
// streams its leaves' operators through a ring of shared-memory stages with 1-D bulk copies
// (cp.async.bulk, completion counted on an mbarrier per stage) issued by one producer thread,
// while 8 consumer warps apply each chunk of columns from shared memory.  The producer runs up to
// a ring ahead of the consumers, so the loads of the next leaf keep flowing through a leaf's
// right-hand side gather and output phases.  Every wait is bounded (a timeout sets the error word).
constexpr int kStreamConsumers = 256;                 // 8 consumer warps
constexpr int kStreamThreads = 32 + kStreamConsumers;  // + the producer warp
constexpr int kStreamMaxStages = 16;

struct StreamPlan {
  int nodes, M, K, ld;  // leaves, operator rows and columns, column stride (floats)
  int64_t str;          // floats from one leaf's operator to the next
  int C, NCH, S;        // columns per chunk, chunks per leaf, ring stages
  int QQ, KS;           // row quads, K slices of the consumer threads
  int hint;             // L2 evict-first hint on the operator copies
};

inline size_t stream_smem(const StreamPlan &P, int role_floats);
// cps: CTAs per SM (1 to 4), each with its own ring: while one CTA gathers a leaf's right-hand
// side or writes its outputs, the others keep streaming
inline StreamPlan stream_plan(int nodes, int M, int K, int ld, int64_t str, int cps = 2, int role_floats = 0,
                              int chunk_kb = 16) {
  StreamPlan P{};
  P.nodes = nodes;
  P.M = M;
  P.K = K;
  P.ld = ld;
  P.str = str;
  P.C = std::max(1, std::min(K, chunk_kb * 1024 / (ld * 4)));
  P.NCH = (K + P.C - 1) / P.C;
  P.QQ = (M + 3) / 4;
  P.KS = std::max(1, kStreamConsumers / P.QQ);
  P.hint = 1;
  P.S = 0;
  // per CTA: a cps-th of the SM's 228 KB less the 1 KB the hardware reserves for each resident CTA
  const size_t rest = stream_smem(P, role_floats), budget = (size_t)(228 * 1024) / std::max(1, cps) - 1024;
  if (budget > rest) P.S = (int)std::min<size_t>(kStreamMaxStages, (budget - rest) / ((size_t)P.C * ld * 4));
  return P;
}
// shared memory (bytes): ring, right-hand side xs [K][4], slice partials, output ys [4 QQ][4],
// the role's own floats, barriers and the abort flag
inline size_t stream_smem(const StreamPlan &P, int role_floats) {
  const size_t f = (size_t)P.S * P.C * P.ld + 4 * (size_t)P.K + (size_t)P.KS * 16 * P.QQ + 16 * (size_t)P.QQ +
                   round4(role_floats);
  return f * sizeof(float) + 2 * kStreamMaxStages * sizeof(uint64_t) + 16;
}
inline bool stream_fits(const StreamPlan &P, int role_floats) {
  return P.QQ <= kStreamConsumers && P.S >= 2 && (P.ld * 4) % 16 == 0 && (P.str * 4) % 16 == 0 &&
         stream_smem(P, role_floats) <= 227 * 1024;
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kStreamConsumers) : "memory"); }
// consumer barrier that also ORs a predicate over the consumer threads (a uniform decision)
__device__ __forceinline__ bool consumer_sync_or(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "n"(kStreamConsumers)
      : "memory");
  return r != 0;
}

// Particular solve: xs = the leaf's stage right-hand side, ys = A_ii^-1 xs -> w and its fluxes.
struct StreamUp {
  GridDims g;
  int R;
  const int *origin;
  Combo rhs;
  double *Rsave;
  const double *Dg;
  float *w32, *h32;
  static constexpr int kPre = 0, kEpi = 0;  // (no per-leaf register prefetch)
  __host__ __device__ int role_floats() const { return 2 * g.p * g.p; }
  __device__ void setup(float *rs, int t0, int nt) const {
    for (int i = t0; i < 2 * g.p * g.p; i += nt) rs[i] = (float)Dg[i];
  }
  __device__ void prologue(int k, float *xs, float *, int t0, int nt) const {
    const int q = g.m * g.m;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
    for (int i = t0; i < q * (4 - R); i += nt) xs[(i / (4 - R)) * 4 + R + i % (4 - R)] = 0.f;
    stage_combo<4>(rhs, l0 * R, q * R, R, 4, Rsave, xs, t0, nt);
  }
  __device__ void epilogue(int k, const float *ys, const float *rs, int t0, int nt) const {
    const int p = g.p, m = g.m;
    leaf_up_out(k, m * m, 4 * m, R, 4, ys, rs, rs + p * p, p, m, w32, h32, t0, nt);
  }
};

// Interior solve: xs = the leaf's boundary values, u_i = w + S xs.
struct StreamDown {
  GridDims g;
  int R;
  const int *origin;
  const float *w32, *g32;
  UOut uo;
  // pre: the next leaf's boundary values and this leaf's w (and u, when adding to it) are loaded
  // into registers before this leaf's products and stored after them (a second xs buffer in the
  // role's floats), so no per-leaf load latency stalls the stream
  bool pre;
  static constexpr int kPre = 2, kEpi = 2;  // registers per consumer thread (4 b <= 480 for p <= 32)
  __host__ __device__ int role_floats() const { return pre ? 16 * g.m : 0; }
  __device__ void setup(float *, int, int) const {}
  __device__ float bd_value(int ix, int iy, int i) const {
    const int pos = i >> 2, j = i & 3;
    return j < R ? g32[box_bd(g, ix, iy, 1, 1, pos) * R + j] : 0.f;
  }
  __device__ void pre_load(int k, float (&v)[kPre], int t0, int nt) const {
    const int b = 4 * g.m, ix = origin[2 * k], iy = origin[2 * k + 1];
#pragma unroll
    for (int s = 0; s < kPre; ++s) v[s] = t0 + s * nt < 4 * b ? bd_value(ix, iy, t0 + s * nt) : 0.f;
  }
  __device__ void pre_store(int k, const float (&v)[kPre], float *xs, int t0, int nt) const {
    const int b = 4 * g.m;
#pragma unroll
    for (int s = 0; s < kPre; ++s)
      if (t0 + s * nt < 4 * b) xs[t0 + s * nt] = v[s];
    for (int i = t0 + kPre * nt; i < 4 * b; i += nt) xs[i] = bd_value(origin[2 * k], origin[2 * k + 1], i);
  }
  __device__ void epi_load(int k, float (&w)[kEpi], double (&u0)[kEpi], int t0, int nt) const {
    const int q = g.m * g.m;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
#pragma unroll
    for (int s = 0; s < kEpi; ++s) {
      const int idx = t0 + s * nt;
      w[s] = idx < q * R ? w32[(int64_t)k * q * R + idx] : 0.f;
      u0[s] = idx < q * R && !uo.assign ? uo.u[l0 * R + idx] : 0.0;
    }
  }
  __device__ void epilogue_pre(int k, const float *ys, const float (&w)[kEpi], const double (&u0)[kEpi], int t0,
                               int nt) const {
    const int q = g.m * g.m;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
#pragma unroll
    for (int s = 0; s < kEpi; ++s) {
      const int idx = t0 + s * nt;
      if (idx < q * R) {
        const int r = idx / R, j = idx - r * R;
        const double d = f2d_int(w[s] + ys[r * 4 + j]);
        uo.u[l0 * R + idx] = uo.assign ? d : u0[s] + d;
      }
    }
    for (int idx = t0 + kEpi * nt; idx < q * R; idx += nt) {
      const int r = idx / R, j = idx - r * R;
      u_out(uo, l0 * R + idx, w32[(int64_t)k * q * R + idx] + ys[r * 4 + j]);
    }
  }
  // One column (R = 1): row r of S u_b is the sum of the K slices' partials (slice order, as the
  // kernel's own sum), taken straight into u_i = w + S u_b.
  __device__ void epilogue_sum(int k, const float *part, int KS, int kstride, const float (&w)[kEpi],
                               const double (&u0)[kEpi], int t0, int nt) const {
    const int q = g.m * g.m;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
#pragma unroll
    for (int s = 0; s < kEpi; ++s) {
      const int r = t0 + s * nt;
      if (r < q) {
        float v = 0.f;
        for (int k2 = 0; k2 < KS; ++k2) v += part[(size_t)k2 * kstride + 4 * r];
        const double d = f2d_int(w[s] + v);
        uo.u[l0 + r] = uo.assign ? d : u0[s] + d;
      }
    }
    for (int r = t0 + kEpi * nt; r < q; r += nt) {
      float v = 0.f;
      for (int k2 = 0; k2 < KS; ++k2) v += part[(size_t)k2 * kstride + 4 * r];
      u_out(uo, l0 + r, w32[(int64_t)k * q + r] + v);
    }
  }
  __device__ void prologue(int k, float *xs, float *, int t0, int nt) const {
    const int b = 4 * g.m, ix = origin[2 * k], iy = origin[2 * k + 1];
    for (int i = t0; i < b * 4; i += nt) {
      const int pos = i >> 2, j = i & 3;
      xs[i] = j < R ? g32[box_bd(g, ix, iy, 1, 1, pos) * R + j] : 0.f;
    }
  }
  __device__ void epilogue(int k, const float *ys, const float *, int t0, int nt) const {
    const int q = g.m * g.m;
    const int64_t l0 = ((int64_t)origin[2 * k + 1] * g.n1 + origin[2 * k]) * q;
    for (int idx = t0; idx < q * R; idx += nt) {
      const int r = idx / R, j = idx - r * R;
      u_out(uo, (l0 + r) * R + j, w32[((int64_t)k * q + r) * R + j] + ys[r * 4 + j]);
    }
  }
};

// RC: right-hand-side columns computed (1: one column, scalar right-hand side per operator column;
// 4: up to four columns padded to four)
template <class Role, int RC>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_b_leaf_stream(StreamPlan P, const float *__restrict__ A, Role role, int *__restrict__ err) {
  extern __shared__ __align__(16) float sms[];
  const int S = P.S, stage_f = P.C * P.ld;
  float *ring = sms, *xs = ring + (size_t)S * stage_f, *part = xs + 4 * P.K, *ys = part + (size_t)P.KS * 16 * P.QQ;
  float *rs = ys + 16 * P.QQ;
  uint64_t *full = reinterpret_cast<uint64_t *>(rs + round4(role.role_floats()));
  uint64_t *empty = full + kStreamMaxStages;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + kStreamMaxStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc5::mbar_init(&full[s], 1);
      tc5::mbar_init(&empty[s], kStreamConsumers / 32);
    }
    *abort_flag = 0;
    tc5::fence_barrier_init();
  }
  __syncthreads();
  const int nl = (int)blockIdx.x < P.nodes ? (P.nodes - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = nl * P.NCH;
  int last_box[kStreamMaxStages];  // producer: last chunk copied into each stage (-1: none)
  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      const uint64_t pol = tc5::policy_evict_first();
      for (int s = 0; s < kStreamMaxStages; ++s) last_box[s] = -1;
      for (int c = 0; c < total; ++c) {
        const int j = c / P.NCH, i = c - j * P.NCH, s = c % S;
        const int k = (int)blockIdx.x + j * (int)gridDim.x;
        if (c >= S && !umma_wait(&empty[s], (unsigned)((c - S) / S) & 1u, abort_flag)) break;
        const int cols = min(P.C, P.K - i * P.C);
        const unsigned bytes = (unsigned)(cols * P.ld * 4);
        const float *src = A + (int64_t)k * P.str + (int64_t)i * P.C * P.ld;
        tc5::mbar_expect_tx(&full[s], bytes);
        if (P.hint)
          tc5::bulk_load_hint(ring + (size_t)s * stage_f, src, bytes, &full[s], pol);
        else
          tc5::bulk_load(ring + (size_t)s * stage_f, src, bytes, &full[s]);
        last_box[s] = c;
      }
    }
  } else {
    // ---------------- consumers ----------------
    const int ct = tid - 32;
    role.setup(rs, ct, kStreamConsumers);
    const int rq = ct % P.QQ, ks = ct / P.QQ;
    const bool live = ks < P.KS;
    bool failed = false;
    constexpr bool kRegs = Role::kPre > 0;  // the role can carry per-leaf loads in registers
    float pv[kRegs ? Role::kPre : 1], wv[kRegs ? Role::kEpi : 1];
    double uv[kRegs ? Role::kEpi : 1];
    bool pre = false;
    if constexpr (kRegs) {
      pre = role.pre;
      if (pre && nl > 0) {
        role.pre_load((int)blockIdx.x, pv, ct, kStreamConsumers);
        role.pre_store((int)blockIdx.x, pv, xs, ct, kStreamConsumers);
      }
    }
    for (int j = 0; j < nl; ++j) {
      const int k = (int)blockIdx.x + j * (int)gridDim.x;
      float *xsj = xs;  // this leaf's right-hand side (alternating buffers with pre)
      if constexpr (kRegs) {
        if (pre) {
          xsj = (j & 1) ? rs : xs;
          role.epi_load(k, wv, uv, ct, kStreamConsumers);
          if (j + 1 < nl) role.pre_load(k + (int)gridDim.x, pv, ct, kStreamConsumers);
        } else {
          role.prologue(k, xs, rs, ct, kStreamConsumers);
        }
      } else {
        role.prologue(k, xs, rs, ct, kStreamConsumers);
      }
      // (with pre, a later leaf's right-hand side was stored before the previous leaf's last sync)
      if (!pre || j == 0) consumer_sync();
      float acc[4][RC];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int u = 0; u < RC; ++u) acc[e][u] = 0.f;
      for (int i = 0; i < P.NCH; ++i) {
        const int c = j * P.NCH + i, s = c % S;
        if (!failed && !umma_wait(&full[s], (unsigned)(c / S) & 1u, abort_flag)) failed = true;
        if (!failed && live) {
          const float *a = ring + (size_t)s * stage_f + 4 * rq;
          const float *x = xsj + 4 * i * P.C;
          const int cols = min(P.C, P.K - i * P.C);
          if constexpr (RC == 1) {
#pragma unroll 4
            for (int cc = ks; cc < cols; cc += P.KS) {
              const float4 av = *reinterpret_cast<const float4 *>(a + cc * P.ld);
              const float xv = x[4 * cc];
              acc[0][0] = fmaf(av.x, xv, acc[0][0]);
              acc[1][0] = fmaf(av.y, xv, acc[1][0]);
              acc[2][0] = fmaf(av.z, xv, acc[2][0]);
              acc[3][0] = fmaf(av.w, xv, acc[3][0]);
            }
          } else {
#pragma unroll 4
            for (int cc = ks; cc < cols; cc += P.KS)
              tile_fma<4>(acc, *reinterpret_cast<const float4 *>(a + cc * P.ld), x + 4 * cc);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      if (live) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          *reinterpret_cast<float4 *>(part + ((size_t)ks * 4 * P.QQ + 4 * rq + e) * 4) =
              RC == 1 ? make_float4(acc[e][0], 0.f, 0.f, 0.f)
                      : make_float4(acc[e][0], acc[e][RC > 1 ? 1 : 0], acc[e][RC > 2 ? 2 : 0], acc[e][RC > 3 ? 3 : 0]);
      }
      consumer_sync();
      if constexpr (kRegs && RC == 1) {
        if (pre) {  // one column: the slice sums go straight into the outputs (no ys pass)
          if (j + 1 < nl) role.pre_store(k + (int)gridDim.x, pv, ((j + 1) & 1) ? rs : xs, ct, kStreamConsumers);
          role.epilogue_sum(k, part, P.KS, 16 * P.QQ, wv, uv, ct, kStreamConsumers);
          if (consumer_sync_or(failed || *abort_flag)) break;
          continue;
        }
      }
      for (int idx = ct; idx < 16 * P.QQ; idx += kStreamConsumers) {  // slices in order: deterministic
        float v = 0.f;
        for (int k2 = 0; k2 < P.KS; ++k2) v += part[(size_t)k2 * 16 * P.QQ + idx];
        ys[idx] = v;
      }
      consumer_sync();
      if constexpr (kRegs) {
        if (pre) {  // the next leaf's right-hand side into the other buffer (read after the sync below)
          if (j + 1 < nl) role.pre_store(k + (int)gridDim.x, pv, ((j + 1) & 1) ? rs : xs, ct, kStreamConsumers);
          role.epilogue_pre(k, ys, wv, uv, ct, kStreamConsumers);
        } else {
          role.epilogue(k, ys, rs, ct, kStreamConsumers);
        }
      } else {
        role.epilogue(k, ys, rs, ct, kStreamConsumers);
      }
      if (consumer_sync_or(failed || *abort_flag)) break;  // uniform: every consumer leaves together
    }
  }
  // wind down: every role has left its loop
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort_flag) {  // copies still in flight (only a stage's last one can be)
    for (int s = 0; s < S; ++s)
      if (last_box[s] >= 0) tc5::mbar_wait(&full[s], (unsigned)(last_box[s] / S) & 1u, kUmmaWaitNs);
    atomicExch(err, 1);
  }
}

template <class Role>
int launch_stream(hps_handle *H, const StreamPlan &P, int cps, const float *A, const Role &role, cudaStream_t st) {
  const size_t smem = stream_smem(P, role.role_floats());
  auto kern = role.R == 1 ? k_b_leaf_stream<Role, 1> : k_b_leaf_stream<Role, 4>;
  if (int e_ = smem_optin((const void *)kern, smem)) return e_;
  kern<<<std::min(P.nodes, H->num_sms * cps), kStreamThreads, smem, st>>>(P, A, role, H->perr);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Launch with programmatic stream serialization when `pdl` (the kernel must call pdl_wait before
// it touches data of earlier kernels), else an ordinary launch.
template <class... KArgs, class... Args>
cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---- merge applies (FP32, R columns) -------------------------------------------------------
struct BPlan {
  int M, K, nodes, R, Rp, TC, MQ, CG;
  int npc, quads_cta, row_tiles, node_groups, ksplit, kchunk;
  int shared_op;  // operator shared by all nodes (stride 0)
  int trows;      // rows of the operator tile a CTA stages (multiple of 4)
};

constexpr int kBOpFloats = 16384;  // operator tile staged in shared memory (64 KB)

__host__ __device__ inline int b_tiles(const BPlan &P) { return P.shared_op ? 1 : P.npc; }
size_t b_smem_floats(const BPlan &P) {  // operator tile(s) + vector chunk
  return (size_t)b_tiles(P) * P.kchunk * P.trows + (size_t)P.npc * P.kchunk * P.Rp;
}

// Split-K plan of one level apply.  Tunables (handle options): the CTAs aimed at (target), the
// smallest K chunk of a split (kmin) and the most nodes one CTA takes (npc_max).
struct PlanTune {
  int kmin, npc_max, tc;  // tc: register-tile columns (8 or 4)
};

BPlan plan_b(int M, int K, int nodes, int R, int target, bool shared_op, PlanTune tune) {
  BPlan P;
  P.shared_op = shared_op ? 1 : 0;
  P.M = M;
  P.K = K;
  P.nodes = nodes;
  P.R = R;
  P.Rp = round4(R);
  P.TC = tune.tc == 2 ? 2 : P.Rp % 8 == 0 && tune.tc == 8 ? 8 : 4;
  P.MQ = (M + 3) / 4;
  P.CG = P.Rp / P.TC;
  const int per = P.MQ * P.CG;
  if (per <= kBT / 2) {
    P.npc = std::max(1, std::min({nodes, kBT / per, tune.npc_max}));
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
  if (base < target) ks = std::min({(target + base - 1) / base, std::max(1, K / tune.kmin), kMaxSplit});
  P.kchunk = (K + ks - 1) / ks;
  P.trows = P.npc > 1 ? 4 * P.MQ : 4 * std::min(P.quads_cta, P.MQ);
  while ((int64_t)P.npc * P.kchunk * P.Rp > kBSmemFloats ||
         (int64_t)b_tiles(P) * P.kchunk * P.trows > kBOpFloats)
    P.kchunk = (P.kchunk + 1) / 2;
  P.ksplit = (K + P.kchunk - 1) / P.kchunk;
  return P;
}

int plan_target(const hps_handle *H) { return H->batch.plan_target * H->num_sms; }
PlanTune plan_tune(const hps_handle *H, int slot) {  // slot: kMergeUpW3, kMergeUpH or kMergeDown
  const int i = slot == kMergeUpW3 ? 0 : slot == kMergeUpH ? 1 : 2;
  const int tc = H->batch.tile_cols_apply[i] ? H->batch.tile_cols_apply[i] : H->batch.plan_tile_cols;
  return PlanTune{H->batch.plan_kmin, H->batch.plan_npc_max, tc};
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
  __device__ float4 load4(int k, int cc, int j0) const {  // row addresses once per 4 columns
    const float *pb = hC + ((int64_t)(2 * k + 1) * nbc + j3b + cc) * R + j0;
    const float *pa = hC + ((int64_t)(2 * k) * nbc + j3a + cc) * R + j0;
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = j0 + t < R ? pb[t] - pa[t] : 0.f;
    if (jump) {
      const double *pj = jump + iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, cc) * R + j0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (j0 + t < R) v[t] += d2f_int(pj[t]);
    }
    return make_float4(v[0], v[1], v[2], v[3]);
  }
};
struct BXVec {
  const float *v;
  int n, R;
  __device__ float operator()(int k, int c, int j) const { return v[((int64_t)k * n + c) * R + j]; }
  __device__ float4 load4(int k, int c, int j0) const {
    const float *p = v + ((int64_t)k * n + c) * R + j0;
    return make_float4(p[0], j0 + 1 < R ? p[1] : 0.f, j0 + 2 < R ? p[2] : 0.f, j0 + 3 < R ? p[3] : 0.f);
  }
};
struct BXBd {
  GridDims g;
  const int *origin;
  int a, c, R;
  const float *gv;
  __device__ float operator()(int k, int pos, int j) const {
    return gv[box_bd(g, origin[2 * k], origin[2 * k + 1], a, c, pos) * R + j];
  }
  __device__ float4 load4(int k, int pos, int j0) const {
    const float *p = gv + box_bd(g, origin[2 * k], origin[2 * k + 1], a, c, pos) * R + j0;
    return make_float4(p[0], j0 + 1 < R ? p[1] : 0.f, j0 + 2 < R ? p[2] : 0.f, j0 + 3 < R ? p[3] : 0.f);
  }
};
struct BEStore {
  float *out;
  int n, R;
  __device__ void operator()(int k, int r, int j, float v) const { out[((int64_t)k * n + r) * R + j] = v; }
  template <int TC>
  __device__ void row(int k, int r, int j0, const float (&v)[TC]) const {
    float *o = out + ((int64_t)k * n + r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t)
      if (j0 + t < R) o[t] = v[t];
  }
  // unsplit applies: the additive part is loaded into the accumulators before the product
  // (its latency hides behind the arithmetic) and `store` writes the finished row
  template <int TC>
  __device__ void init(int, int, int, float (&a)[TC], double (&)[TC]) const {
#pragma unroll
    for (int t = 0; t < TC; ++t) a[t] = 0.f;
  }
  template <int TC>
  __device__ void store(int k, int r, int j0, const float (&v)[TC], const double (&)[TC]) const {
    row<TC>(k, r, j0, v);
  }
};
struct BEFlux {
  const int *hsrc;
  const float *hC;
  int nbc, nb, R;
  float *h;
  __device__ void operator()(int k, int r, int j, float v) const {
    h[((int64_t)k * nb + r) * R + j] = hC[((int64_t)(2 * k) * nbc + hsrc[r]) * R + j] + v;
  }
  template <int TC>
  __device__ void row(int k, int r, int j0, const float (&v)[TC]) const {
    const float *src = hC + ((int64_t)(2 * k) * nbc + hsrc[r]) * R + j0;
    float *o = h + ((int64_t)k * nb + r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t)
      if (j0 + t < R) o[t] = src[t] + v[t];
  }
  template <int TC>
  __device__ void init(int k, int r, int j0, float (&a)[TC], double (&)[TC]) const {
    const float *src = hC + ((int64_t)(2 * k) * nbc + hsrc[r]) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t) a[t] = j0 + t < R ? src[t] : 0.f;
  }
  template <int TC>
  __device__ void store(int k, int r, int j0, const float (&v)[TC], const double (&)[TC]) const {
    float *o = h + ((int64_t)k * nb + r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t)
      if (j0 + t < R) o[t] = v[t];
  }
};
struct BEScatter {  // interface values: FP32 for the levels below, and into the FP64 solution
  GridDims g;
  const int *origin;
  int a, c, split, n3, R;
  const float *w3;
  float *gv;
  UOut uo;
  __device__ void operator()(int k, int r, int j, float v) const {
    const int64_t i = iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r) * R + j;
    const float x = v + w3[((int64_t)k * n3 + r) * R + j];
    gv[i] = x;
    u_out(uo, i, x);
  }
  template <int TC>
  __device__ void row(int k, int r, int j0, const float (&v)[TC]) const {
    const int64_t i0 = iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r) * R + j0;
    const float *w = w3 + ((int64_t)k * n3 + r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t)
      if (j0 + t < R) {
        const float x = v[t] + w[t];
        gv[i0 + t] = x;
        u_out(uo, i0 + t, x);
      }
  }
  template <int TC>
  __device__ void init(int k, int r, int j0, float (&acc)[TC], double (&old)[TC]) const {
    const float *w = w3 + ((int64_t)k * n3 + r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t) acc[t] = j0 + t < R ? w[t] : 0.f;
    if (!uo.assign) {  // the correction adds to u: fetch the old values now
      const double *u0 = uo.u + iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r) * R + j0;
#pragma unroll
      for (int t = 0; t < TC; ++t) old[t] = j0 + t < R ? u0[t] : 0.0;
    }
  }
  template <int TC>
  __device__ void store(int k, int r, int j0, const float (&v)[TC], const double (&old)[TC]) const {
    const int64_t i0 = iface_bd(g, origin[2 * k], origin[2 * k + 1], a, c, split, r) * R + j0;
#pragma unroll
    for (int t = 0; t < TC; ++t)
      if (j0 + t < R) {
        gv[i0 + t] = v[t];
        uo.u[i0 + t] = uo.assign ? f2d_int(v[t]) : old[t] + f2d_int(v[t]);
      }
  }
};

// An operator range to prefetch into L2 (the next apply's operator; p null: none).  p is 16-byte
// aligned and bytes a multiple of 16 (a cudaMalloc'd operator of rows padded to 4 floats).
struct Pf {
  const char *p;
  int64_t bytes;
};

// This CTA's share of the prefetch (CTA `cta` of `nctas`): pieces of 32 KB, one per lane of the
// first warp at a time.
__device__ __forceinline__ void prefetch_share(const Pf &f, int64_t cta, int64_t nctas) {
  if (!f.p || threadIdx.x >= 32) return;
  const int64_t units = f.bytes >> 4, per = (units + nctas - 1) / nctas;
  const int64_t u0 = cta * per, u1 = min(units, u0 + per);
  constexpr int64_t kPiece = 2048;  // 16-byte units
  for (int64_t u = u0 + (int64_t)threadIdx.x * kPiece; u < u1; u += 32 * kPiece)
    tc5::bulk_prefetch_l2(f.p + (u << 4), (unsigned)(min(kPiece, u1 - u) << 4));
}

// The body of one CTA (block bx, K chunk by) of a merge apply; k_b_gemv runs it for its own grid,
// k_b_gemv_group for the blocks of many instances' applies in one launch.
template <int TC, class XL, class EP>
__device__ __forceinline__ void gemv_tile(const BPlan &P, const float *__restrict__ AT, int ld, int64_t str, XL xl, EP ep,
                                          float *__restrict__ partial, unsigned *__restrict__ tile_count, unsigned bx,
                                          unsigned by) {
  extern __shared__ __align__(16) float smb[];
  const int ng = bx / P.row_tiles, tile = bx % P.row_tiles;
  const int node0 = ng * P.npc, nn = min(P.npc, P.nodes - node0);
  const int ks = by, c0 = ks * P.kchunk, klen = min(P.kchunk, P.K - c0);
  const int Rp = P.Rp;
  // operator tile(s) [tile][klen][trows] by asynchronous copies, overlapping the vector staging
  const int trows = P.trows, rlo = P.npc > 1 ? 0 : 4 * tile * P.quads_cta;
  const int trow = min(trows, 4 * P.MQ - rlo);  // rows of this CTA's tile (ragged last tile)
  const int ntile = P.shared_op ? 1 : nn;
  float *As = smb, *xs = smb + (size_t)b_tiles(P) * P.kchunk * trows;
  {
    const int q4 = trow / 4, n16 = ntile * klen * q4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
      const int t = i / (klen * q4), rem = i % (klen * q4), c = rem / q4, qq = rem % q4;
      cp_async16(As + ((size_t)t * klen + c) * trows + 4 * qq,
                 AT + (int64_t)(node0 + t) * str + (int64_t)(c0 + c) * ld + rlo + 4 * qq);
    }
  }
  pdl_wait();  // (the operator tile is in flight; the vector is the previous kernel's output)
  {  // vector chunk [nn][klen][Rp], four columns per load (row addresses once per 4 columns)
    const int Rq = Rp / 4, n4 = nn * klen * Rq;
    const bool pow2 = (Rq & (Rq - 1)) == 0;
    const int sh = __ffs(Rq) - 1;
    block_gather<4, float4>(
        n4,
        [&](int t) {
          const int row = pow2 ? t >> sh : t / Rq, j0 = 4 * (pow2 ? t & (Rq - 1) : t % Rq);
          const int lo = row / klen, c = row - lo * klen;
          return xl.load4(node0 + lo, c0 + c, j0);
        },
        [&](int t, float4 v) { reinterpret_cast<float4 *>(xs)[t] = v; });
  }
  cp_async_wait_all();
  __syncthreads();
  // column groups fastest across the threads: a warp's epilogue loads and stores cover whole
  // row segments (coalesced); its operator reads are broadcasts of a few row quads
  int lo, rq, cg;
  if (P.npc > 1) {
    const int per = P.MQ * P.CG;
    lo = threadIdx.x / per;
    const int rem = threadIdx.x % per;
    rq = rem / P.CG;
    cg = rem % P.CG;
  } else {
    lo = 0;
    cg = threadIdx.x % P.CG;
    const int lq = threadIdx.x / P.CG;
    rq = lq < P.quads_cta ? tile * P.quads_cta + lq : P.MQ;  // past the tile: idle
  }
  const bool live = lo < nn && cg < P.CG && rq < P.MQ;
  const int r0 = 4 * rq, j0 = TC * cg;
  float acc[4][TC];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
  double aux[4][TC];
  if (live && P.ksplit == 1)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (r0 + e < P.M) ep.template init<TC>(node0 + lo, r0 + e, j0, acc[e], aux[e]);
  if (live)
    smem_fma<TC>(acc, As + (size_t)(P.shared_op ? 0 : lo) * klen * trows + (r0 - rlo), trows, klen,
                 xs + (int64_t)lo * klen * Rp + j0, Rp);
  pdl_trigger();  // the products are done: the next kernel may take the SMs this grid frees
  const int k = node0 + lo;
  if (live)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + e;
      if (r >= P.M) continue;
      if (P.ksplit == 1) {
        ep.template store<TC>(k, r, j0, acc[e], aux[e]);
      } else {
        float *dst = partial + (((int64_t)ks * P.nodes + k) * P.M + r) * Rp + j0;
#pragma unroll
        for (int t = 0; t < TC; t += 2)
          *reinterpret_cast<float2 *>(dst + t) = make_float2(acc[e][t], acc[e][t + 1]);
      }
    }
  if (P.ksplit == 1 || !tile_count) return;
  // split K, summed here: the CTA that finishes a tile last adds its ksplit partials in chunk
  // order (deterministic) and runs the epilogue; it also re-arms the tile's counter
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(tile_count + bx, 1u) == (unsigned)(P.ksplit - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int Rq = Rp / 4, rows = P.npc > 1 ? P.M : min(trow, P.M - rlo);
  const int64_t kstride = (int64_t)P.nodes * P.M * Rp;
  for (int i = threadIdx.x; i < nn * rows * Rq; i += blockDim.x) {
    const int q4 = i % Rq, row = i / Rq, l2 = row / rows, r = rlo + row - l2 * rows, j0q = 4 * q4;
    const float *src = partial + ((int64_t)(node0 + l2) * P.M + r) * Rp + j0q;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ks2 = 0; ks2 < P.ksplit; ++ks2) {
      const float4 x = __ldcg(reinterpret_cast<const float4 *>(src + ks2 * kstride));
      v[0] += x.x;
      v[1] += x.y;
      v[2] += x.z;
      v[3] += x.w;
    }
    ep.template row<4>(node0 + l2, r, j0q, v);
  }
  if (threadIdx.x == 0) tile_count[bx] = 0u;
}

template <int TC, class XL, class EP>
__global__ void __launch_bounds__(kBT) k_b_gemv(BPlan P, const float *__restrict__ AT, int ld, int64_t str, XL xl,
                                                EP ep, float *__restrict__ partial, unsigned *__restrict__ tile_count,
                                                Pf pf) {
  gemv_tile<TC>(P, AT, ld, str, xl, ep, partial, tile_count, blockIdx.x, blockIdx.y);
  prefetch_share(pf, blockIdx.x + (int64_t)blockIdx.y * gridDim.x, (int64_t)gridDim.x * gridDim.y);
}

// Sum of the split-K partials in chunk order, four columns per thread.
template <class EP>
__device__ __forceinline__ void reduce_row(const BPlan &P, const float *__restrict__ partial, EP ep, int i) {
  const int Rq = P.Rp / 4;
  if (i >= P.nodes * P.M * Rq) return;
  const int row = i / Rq, j0 = 4 * (i - row * Rq), k = row / P.M, r = row - k * P.M;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  const int64_t stride = (int64_t)P.nodes * P.M * P.Rp;
  const float *src = partial + (int64_t)row * P.Rp + j0;
#pragma unroll 8
  for (int ks = 0; ks < P.ksplit; ++ks) {
    const float4 x = *reinterpret_cast<const float4 *>(src + ks * stride);
    v[0] += x.x;
    v[1] += x.y;
    v[2] += x.z;
    v[3] += x.w;
  }
  ep.template row<4>(k, r, j0, v);
}

template <class EP>
__global__ void k_b_reduce(BPlan P, const float *__restrict__ partial, EP ep) {
  pdl_trigger();
  pdl_wait();
  reduce_row(P, partial, ep, (int)(blockIdx.x * blockDim.x + threadIdx.x));
}

template <class XL, class EP>
int launch_b(hps_handle *H, BatchWork &B, int slot, const BPlan &P, const float *AT, int ld, int64_t str, XL xl,
             EP ep, cudaStream_t st, Pf pf = Pf{}) {
  const size_t smem = b_smem_floats(P) * sizeof(float);
  if (P.ksplit > 1 && (size_t)P.ksplit * P.nodes * P.M * P.Rp > B.partial_len) return HPS_EINVAL;
  if (int e_ = smem_optin((const void *)k_b_gemv<8, XL, EP>, smem)) return e_;
  if (int e_ = smem_optin((const void *)k_b_gemv<4, XL, EP>, smem)) return e_;
  if (int e_ = smem_optin((const void *)k_b_gemv<2, XL, EP>, smem)) return e_;
  H->trace.begin(slot, st);
  const dim3 grid(P.node_groups * P.row_tiles, P.ksplit);
  // split-K sums: in the kernel (last CTA of a tile) unless the tiles are too many or too deep
  const bool in_kernel = P.ksplit <= H->batch.last_cta_max_split &&
                         (size_t)P.node_groups * P.row_tiles <= B.tile_count_len;
  unsigned *tc = in_kernel ? B.tile_count : nullptr;
  const bool pdl = H->batch.pdl;
  auto kern = P.TC == 8 ? k_b_gemv<8, XL, EP> : P.TC == 4 ? k_b_gemv<4, XL, EP> : k_b_gemv<2, XL, EP>;
  launch_k(pdl, kern, grid, dim3(kBT), smem, st, P, AT, ld, str, xl, ep, B.partial32, tc, pf);
  if (P.ksplit > 1 && !in_kernel) {
    const int64_t n = (int64_t)P.nodes * P.M * (P.Rp / 4);
    launch_k(pdl, k_b_reduce<EP>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, P,
             (const float *)B.partial32, ep);
  }
  H->trace.end(slot, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// ---- one merge apply of many instances in one launch ------------------------------------------
// The lockstep multi-instance step runs a tree level of every instance (levels counted from the
// leaves upward, from the root downward) as ONE launch per operator: the blocks of all instances'
// tiled applies in one grid, each block finding its instance in a prefix table of the kernel's
// parameter block and running the instance's own plan (k_b_gemv's body); split-K partial sums
// follow in one grouped reduction.
constexpr int kGroupMax = 64;

template <class XL, class EP>
struct GemvGroup {
  int n;
  int block0[kGroupMax + 1];  // first block of each instance's flattened grid
  int gx[kGroupMax];          // its grid's x extent (y: the K chunks)
  BPlan P[kGroupMax];
  const float *AT[kGroupMax];
  int ld[kGroupMax];
  int64_t str[kGroupMax];
  XL xl[kGroupMax];
  EP ep[kGroupMax];
  float *partial[kGroupMax];
};

// (kernel parameters may take up to 32764 bytes)
static_assert(sizeof(GemvGroup<BXDiff, BEStore>) <= 32000, "grouped w3 parameters");
static_assert(sizeof(GemvGroup<BXVec, BEFlux>) <= 32000, "grouped h parameters");
static_assert(sizeof(GemvGroup<BXBd, BEScatter>) <= 32000, "grouped down parameters");

__device__ __forceinline__ int group_of(const int *block0, int n, int b) {  // block0[i] <= b < block0[i + 1]
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (block0[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int TC, class XL, class EP>
__global__ void __launch_bounds__(kBT) k_b_gemv_group(const __grid_constant__ GemvGroup<XL, EP> G) {
  const int i = group_of(G.block0, G.n, (int)blockIdx.x), local = (int)blockIdx.x - G.block0[i];
  gemv_tile<TC>(G.P[i], G.AT[i], G.ld[i], G.str[i], G.xl[i], G.ep[i], G.partial[i], nullptr,
                (unsigned)(local % G.gx[i]), (unsigned)(local / G.gx[i]));
}

template <class EP>
struct ReduceGroup {
  int n;
  int block0[kGroupMax + 1];
  BPlan P[kGroupMax];
  const float *partial[kGroupMax];
  EP ep[kGroupMax];
};

template <class EP>
__global__ void k_b_reduce_group(const __grid_constant__ ReduceGroup<EP> G) {
  const int i = group_of(G.block0, G.n, (int)blockIdx.x);
  reduce_row(G.P[i], G.partial[i], G.ep[i], ((int)blockIdx.x - G.block0[i]) * (int)blockDim.x + (int)threadIdx.x);
}

// One instance's part of a grouped apply.
template <class XL, class EP>
struct GroupItem {
  hps_handle *H;
  BatchWork *B;
  int slot, M, K, nodes, R;
  const float *AT;
  int ld;
  int64_t str;
  XL xl;
  EP ep;
};

template <class XL, class EP>
int launch_group(std::vector<GroupItem<XL, EP>> &items, cudaStream_t st) {
  if (items.empty()) return HPS_OK;
  struct Planned {
    BPlan P;
    const GroupItem<XL, EP> *it;
  };
  std::vector<Planned> pl;
  pl.reserve(items.size());
  for (const auto &it : items) {
    const BPlan P = plan_b(it.M, it.K, it.nodes, it.R, plan_target(it.H), it.str == 0, plan_tune(it.H, it.slot));
    if (P.ksplit > 1 && (size_t)P.ksplit * P.nodes * P.M * P.Rp > it.B->partial_len) return HPS_EINVAL;
    pl.push_back({P, &it});
  }
  // instances with the same register-tile width share a launch (at most kGroupMax each)
  std::stable_sort(pl.begin(), pl.end(), [](const Planned &a, const Planned &b) { return a.P.TC > b.P.TC; });
  for (size_t g0 = 0; g0 < pl.size();) {
    size_t g1 = g0;
    while (g1 < pl.size() && g1 - g0 < (size_t)kGroupMax && pl[g1].P.TC == pl[g0].P.TC) ++g1;
    GemvGroup<XL, EP> G{};
    ReduceGroup<EP> Rg{};
    size_t smem = 0;
    int blocks = 0, rblocks = 0;
    for (size_t k = g0; k < g1; ++k) {
      const BPlan &P = pl[k].P;
      const GroupItem<XL, EP> &it = *pl[k].it;
      const int i = (int)(k - g0);
      G.block0[i] = blocks;
      G.gx[i] = P.node_groups * P.row_tiles;
      G.P[i] = P;
      G.AT[i] = it.AT;
      G.ld[i] = it.ld;
      G.str[i] = it.str;
      G.xl[i] = it.xl;
      G.ep[i] = it.ep;
      G.partial[i] = it.B->partial32;
      blocks += G.gx[i] * P.ksplit;
      smem = std::max(smem, b_smem_floats(P) * sizeof(float));
      if (P.ksplit > 1) {
        const int r = Rg.n++;
        Rg.block0[r] = rblocks;
        Rg.P[r] = P;
        Rg.partial[r] = it.B->partial32;
        Rg.ep[r] = it.ep;
        rblocks += (int)(((int64_t)P.nodes * P.M * (P.Rp / 4) + 255) / 256);
      }
    }
    G.n = (int)(g1 - g0);
    G.block0[G.n] = blocks;
    Rg.block0[Rg.n] = rblocks;
    const int TC = pl[g0].P.TC;
    auto kern = TC == 8 ? k_b_gemv_group<8, XL, EP> : TC == 4 ? k_b_gemv_group<4, XL, EP> : k_b_gemv_group<2, XL, EP>;
    if (int e_ = smem_optin((const void *)kern, smem)) return e_;
    kern<<<blocks, kBT, smem, st>>>(G);
    if (Rg.n > 0) k_b_reduce_group<EP><<<rblocks, 256, 0, st>>>(Rg);
    g0 = g1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// ---- merge applies with one column and per-node operators (the HBM-bound single-RHS sweep) ----
// y_k = A_k x_k for every node k of a level, A_k (M x K, stored transposed: column c at
// AT + k str + c ld) streamed straight from global memory: a thread owns a quad of 4 rows of one
// node (one 16-byte load per column), the kw warps of a quad group split K inside the CTA and add
// their partial sums through shared memory in warp order, and levels with too few quads for the
// GPU split K over CTAs as well (summed by k_b_reduce in chunk order).  No operator staging: each
// element is used once.
struct BPlan1 {
  int M, K, nodes, QN;   // rows, columns, nodes, row quads per node
  int kw, qcta;          // warps per quad group (in-CTA split of K), quads per CTA
  int ks, kchunk;        // split of K over CTAs
  int64_t quads;
};

BPlan1 plan_b1(int M, int K, int nodes, int target, int kw_max = 8) {
  BPlan1 P{};
  P.M = M;
  P.K = K;
  P.nodes = nodes;
  P.QN = (M + 3) / 4;
  P.quads = (int64_t)nodes * P.QN;
  P.kw = kw_max;
  while (P.kw > 1 && K / P.kw < 16) P.kw /= 2;  // at least 16 columns per warp
  P.qcta = 32 * (8 / P.kw);
  const int64_t gx = (P.quads + P.qcta - 1) / P.qcta;
  int ks = 1;
  if (gx < target) ks = (int)std::min<int64_t>({(target + gx - 1) / gx, std::max(1, K / (16 * P.kw)), kMaxSplit});
  P.kchunk = (K + ks - 1) / ks;
  P.ks = (K + P.kchunk - 1) / P.kchunk;
  return P;
}

// The vector entries a CTA needs (its nodes x its K range) are staged in shared memory once
// (every thread of a node would otherwise rebuild the same entry; the correction sweeps' interface
// right-hand side is an FP64 gather per entry).
__host__ __device__ inline int64_t b1_node_span(const BPlan1 &P) { return P.qcta / P.QN + 2; }

// ROLL: each operator register is reloaded as soon as its product is taken (a rolling window of
// kU loads in flight per thread); else the kU loads go out as a batch after the batch's products.
// Both add the columns in the same order (bit-identical results).
template <class XL, class EP, bool ROLL>
__global__ void __launch_bounds__(kBT) k_b_gemv1(BPlan1 P, const float *__restrict__ AT, int ld, int64_t str, XL xl,
                                                 EP ep, float *__restrict__ partial, unsigned *__restrict__ tile_count,
                                                 Pf pf) {
  __shared__ float4 red[kBT / 32][32];
  extern __shared__ float xs1[];  // [node - n0][c - c0]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / P.kw, wk = warp - grp * P.kw;
  const int64_t q0 = (int64_t)blockIdx.x * P.qcta, quad = q0 + grp * 32 + lane;
  const int ks = blockIdx.y, c0 = ks * P.kchunk, c1 = min(P.K, c0 + P.kchunk), klen = c1 - c0;
  const int n0 = (int)(q0 / P.QN), n1 = (int)(min(P.quads, q0 + P.qcta) - 1) / P.QN;  // nodes of this CTA
  const bool live = quad < P.quads;
  const int node = live ? (int)(quad / P.QN) : 0, r0 = live ? 4 * (int)(quad - (int64_t)node * P.QN) : 0;
  const float *a = AT + (int64_t)node * str + r0;
  const int step = P.kw;
  constexpr int kU = 8;  // operator loads in flight per thread
  float4 av[kU];
  int c = c0 + wk;
  // the first operator loads go out before the vector staging, so their latency overlaps it (and,
  // launched dependently, the previous kernel's tail)
  pdl_trigger();
#pragma unroll
  for (int u = 0; u < kU; ++u)
    if (live && c + u * step < c1) av[u] = __ldg(reinterpret_cast<const float4 *>(a + (int64_t)(c + u * step) * ld));
  prefetch_share(pf, blockIdx.x + (int64_t)blockIdx.y * gridDim.x, (int64_t)gridDim.x * gridDim.y);
  pdl_wait();
  for (int i = threadIdx.x; i < (n1 - n0 + 1) * klen; i += blockDim.x) {
    const int nn = i / klen, cc = i - nn * klen;
    xs1[i] = xl(n0 + nn, c0 + cc, 0);
  }
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (live && ROLL) {
    const float *x = xs1 + (int64_t)(node - n0) * klen - c0;
    for (; c < c1; c += kU * step) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int cu = c + u * step;
        if (cu < c1) {
          const float xv = x[cu];
          acc.x = fmaf(av[u].x, xv, acc.x);
          acc.y = fmaf(av[u].y, xv, acc.y);
          acc.z = fmaf(av[u].z, xv, acc.z);
          acc.w = fmaf(av[u].w, xv, acc.w);
          const int cn = cu + kU * step;
          if (cn < c1) av[u] = __ldg(reinterpret_cast<const float4 *>(a + (int64_t)cn * ld));
        }
      }
    }
  } else if (live) {
    const float *x = xs1 + (int64_t)(node - n0) * klen - c0;
    for (;;) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int cu = c + u * step;
        if (cu < c1) {
          const float xv = x[cu];
          acc.x = fmaf(av[u].x, xv, acc.x);
          acc.y = fmaf(av[u].y, xv, acc.y);
          acc.z = fmaf(av[u].z, xv, acc.z);
          acc.w = fmaf(av[u].w, xv, acc.w);
        }
      }
      c += kU * step;
      if (c >= c1) break;
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (c + u * step < c1) av[u] = __ldg(reinterpret_cast<const float4 *>(a + (int64_t)(c + u * step) * ld));
    }
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (wk == 0 && live) {
    float4 s = red[warp][lane];
    for (int w = 1; w < P.kw; ++w) {  // in warp order: deterministic
      const float4 t = red[warp + w][lane];
      s.x += t.x;
      s.y += t.y;
      s.z += t.z;
      s.w += t.w;
    }
    const float v[4] = {s.x, s.y, s.z, s.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + e;
      if (r >= P.M) continue;
      if (P.ks == 1) {
        const float vv[4] = {v[e], 0.f, 0.f, 0.f};
        ep.template row<4>(node, r, 0, vv);
      } else if (tile_count) {  // one float per (K chunk, node, row)
        partial[((int64_t)ks * P.nodes + node) * P.M + r] = v[e];
      } else {  // the k_b_reduce layout of a 4-column (padded) plan
        *reinterpret_cast<float4 *>(partial + (((int64_t)ks * P.nodes + node) * P.M + r) * 4) =
            make_float4(v[e], 0.f, 0.f, 0.f);
      }
    }
  }
  if (P.ks == 1 || !tile_count) return;
  // split K, summed here: the CTA of a quad block that finishes last adds the ks partials of its
  // rows in chunk order (deterministic), runs the epilogue and re-arms the block's counter
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(tile_count + blockIdx.x, 1u) == (unsigned)(P.ks - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < 4 * P.qcta; i += blockDim.x) {
    const int64_t qd = q0 + i / 4;
    if (qd >= P.quads) break;
    const int nd = (int)(qd / P.QN), r = 4 * (int)(qd - (int64_t)nd * P.QN) + (i & 3);
    if (r >= P.M) continue;
    const float *src = partial + (int64_t)nd * P.M + r;
    const int64_t kstride = (int64_t)P.nodes * P.M;
    float v = 0.f;
    for (int k2 = 0; k2 < P.ks; ++k2) v += __ldcg(src + k2 * kstride);
    const float vv[4] = {v, 0.f, 0.f, 0.f};
    ep.template row<4>(nd, r, 0, vv);
  }
  if (threadIdx.x == 0) tile_count[blockIdx.x] = 0u;
}

template <class XL, class EP>
int launch_b1(hps_handle *H, BatchWork &B, int slot, int M, int K, int nodes, const float *AT, int ld, int64_t str,
              XL xl, EP ep, cudaStream_t st, bool *done, Pf pf = Pf{}) {
  *done = false;
  const BPlan1 P = plan_b1(M, K, nodes, 4 * H->num_sms, H->batch.b1_kw);
  const int64_t gx = (P.quads + P.qcta - 1) / P.qcta;
  // split-K sums inside the kernel (last CTA of a quad block) where the counters reach
  unsigned *tc = H->batch.one_column_merge_sum && gx <= (int64_t)B.tile_count_len ? B.tile_count : nullptr;
  if (P.ks > 1 && (size_t)P.ks * nodes * M * (tc ? 1 : 4) > B.partial_len) return HPS_OK;  // the general path
  const size_t smem = (size_t)b1_node_span(P) * P.kchunk * sizeof(float);
  if (smem > 96 * 1024) return HPS_OK;
  auto kern = H->batch.b1_roll ? k_b_gemv1<XL, EP, true> : k_b_gemv1<XL, EP, false>;
  if (int e_ = smem_optin((const void *)kern, smem)) return e_;
  *done = true;
  H->trace.begin(slot, st);
  launch_k(H->batch.pdl, kern, dim3((unsigned)gx, (unsigned)P.ks), dim3(kBT), smem, st, P, AT, ld, str, xl,
           ep, B.partial32, tc, pf);
  if (P.ks > 1 && !tc) {
    BPlan R4{};
    R4.M = M;
    R4.K = K;
    R4.nodes = nodes;
    R4.R = 1;
    R4.Rp = 4;
    R4.ksplit = P.ks;
    const int64_t n = (int64_t)nodes * M;
    launch_k(H->batch.pdl, k_b_reduce<EP>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, R4,
             (const float *)B.partial32, ep);
  }
  H->trace.end(slot, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// ---- merge applies of the upper levels: split K inside the CTA and across a cluster ---------
// One CTA per (node, row tile) and cluster rank; 256 threads = S K-slices x Qc row quads x CG
// column groups, each thread a 4 x TC register tile over its slice of the CTA's K chunk.  The S
// slices are added in shared memory, the C CTAs of a cluster (its ranks: consecutive K chunks)
// through distributed shared memory, both in a fixed order (deterministic), and the epilogue
// runs where the sum is formed: no partial sums in global memory, no reduction launch.
struct BPlan2 {
  int M, K, nodes, R, Rp, TC, CG, MQ, S, Qc, RT, C, chunk, slice;
};

BPlan2 plan_b2(int M, int K, int nodes, int R) {
  BPlan2 P{};
  P.M = M;
  P.K = K;
  P.nodes = nodes;
  P.R = R;
  P.Rp = round4(R);
  P.TC = P.Rp % 8 == 0 ? 8 : 4;
  P.CG = P.Rp / P.TC;
  P.MQ = (M + 3) / 4;
  const int ks_total = std::max(1, (K + 31) / 32);  // about 32 operator columns per thread
  P.S = 1;
  while (P.S < 8 && P.S < ks_total && kBT / (2 * P.S * P.CG) >= 4) P.S *= 2;
  P.C = 1;
  while (P.C < 8 && P.S * P.C < ks_total) P.C *= 2;
  P.Qc = kBT / (P.S * P.CG);
  P.RT = (P.MQ + P.Qc - 1) / P.Qc;
  P.chunk = (K + P.C - 1) / P.C;
  P.slice = (P.chunk + P.S - 1) / P.S;
  return P;
}

size_t b2_smem(const BPlan2 &P) {  // x chunk + slice partials + CTA partial
  return ((size_t)P.chunk * P.Rp + (size_t)P.S * P.Qc * 4 * P.Rp + (size_t)P.Qc * 4 * P.Rp) * sizeof(float);
}

template <int TC, class XL, class EP>
__global__ void __launch_bounds__(kBT) k_b_gemv2(BPlan2 P, const float *__restrict__ AT, int ld, int64_t str, XL xl,
                                                 EP ep) {
  extern __shared__ float sm[];
  const int Rp = P.Rp, rows = P.Qc * 4;
  float *xs = sm, *red = xs + (size_t)P.chunk * Rp, *cta = red + (size_t)P.S * rows * Rp;
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  const int k = blockIdx.x / P.RT, rt = blockIdx.x % P.RT;
  const int crank = (int)cl.block_rank();  // cluster dims (1, C, 1): rank = blockIdx.y = K chunk
  const int c0 = crank * P.chunk, clen = max(0, min(P.chunk, P.K - c0));
  block_gather<8, float>(
      clen * Rp,
      [&](int idx) {
        const int c = idx / Rp, j = idx % Rp;
        return j < P.R ? xl(k, c0 + c, j) : 0.f;
      },
      [&](int idx, float v) { xs[idx] = v; });
  __syncthreads();
  const int qi = threadIdx.x % P.Qc, cg = (threadIdx.x / P.Qc) % P.CG, sl = threadIdx.x / (P.Qc * P.CG);
  const int r0 = 4 * (rt * P.Qc + qi), j0 = TC * cg;
  float acc[4][TC];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int t = 0; t < TC; ++t) acc[e][t] = 0.f;
  const bool live = sl < P.S;  // 256 need not be a multiple of S Qc CG
  const int s0 = min(clen, sl * P.slice), s1 = min(clen, s0 + P.slice);
  if (live && r0 < P.M && s1 > s0)
    stream_fma<TC, 8>(acc, AT + (int64_t)k * str + (int64_t)(c0 + s0) * ld + r0, ld, s1 - s0, xs + s0 * Rp + j0, Rp);
  if (live) {
    float *mine = red + ((size_t)sl * rows + 4 * qi) * Rp + j0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int t = 0; t < TC; t += 4)
        *reinterpret_cast<float4 *>(mine + e * Rp + t) =
            make_float4(acc[e][t], acc[e][t + 1], acc[e][t + 2], acc[e][t + 3]);
  }
  __syncthreads();
  // slices -> CTA partial (fixed order)
  for (int idx = threadIdx.x; idx < rows * Rp; idx += blockDim.x) {
    float v = 0.f;
    for (int s2 = 0; s2 < P.S; ++s2) v += red[(size_t)s2 * rows * Rp + idx];
    if (P.C == 1) {
      const int r = 4 * rt * P.Qc + idx / Rp, j = idx % Rp;
      if (r < P.M && j < P.R) ep(k, r, j, v);
    } else {
      cta[idx] = v;
    }
  }
  if (P.C == 1) return;
  cl.sync();
  // this rank adds rows [crank * rows / C, (crank + 1) * rows / C) of the C CTA partials
  const int ra = crank * rows / P.C, rb = (crank + 1) * rows / P.C;
  for (int idx = ra * Rp + threadIdx.x; idx < rb * Rp; idx += blockDim.x) {
    float v = 0.f;
    for (int q2 = 0; q2 < P.C; ++q2) v += cl.map_shared_rank(cta, q2)[idx];
    const int r = 4 * rt * P.Qc + idx / Rp, j = idx % Rp;
    if (r < P.M && j < P.R) ep(k, r, j, v);
  }
  cl.sync();  // keep this CTA's partial alive until every rank has read it
}

constexpr size_t kB2MaxSmem = 160 * 1024;

// ---- the lowest merge levels of the upward sweep fused per subtree --------------------------
// One CTA per (subtree rooted at level lb, group of up to 8 columns) runs levels lb + D - 1 (the
// deepest) up to lb: per level, d = h^b_3 - h^a_3 (+ interface right-hand side) of each of the
// subtree's nodes, w3 = X d (written to global memory: the downward sweep needs it) and
// h = [h^a_1; h^b_2] + Tcat w3.  The children's h of the deepest level come from the leaf
// kernel; the h of the levels inside the subtree stay in shared memory, and the top level's h goes
// to global memory for the levels above.  Sums over K run in order (one output per thread), so the
// result differs from the per-level kernels' in the order of FP32 rounding only.
constexpr int kSubMaxLevels = 6;
constexpr int kSubCols = 8;

struct SubLevel {
  float *w3;               // [node][n3][R]
  const float *X, *T;      // transposed operators (column c at + c ld), per node at + k str
  int ldX, ldT;
  int64_t strX, strT;
  const int *hsrc;         // [nb]: parent boundary position -> child * nbc + position
  const int *origin;       // [node][2]
  int nbc, nb, n3, j3a, j3b, a, c, split;
};
struct SubUp {
  int lb, D, R;
  const float *hleaf;      // h of the level below the deepest fused one: [node][nbc][R]
  float *htop;             // h of level lb: [node][nb][R] (null when lb is the root)
  const double *jump;      // interface right-hand side ([N][R] FP64) or null
  GridDims g;
  SubLevel lv[kSubMaxLevels];  // lv[i]: level lb + i
};

// shared memory: two h buffers (the first takes the staged children's h of the deepest level,
// then the two alternate between levels) and the d / w3 pair of one level
inline size_t sub_buf_floats(const SubUp &P) {
  size_t hmax = (size_t)(2 << (P.D - 1)) * P.lv[P.D - 1].nbc * kSubCols;  // staged children
  for (int i = 0; i < P.D; ++i) hmax = std::max(hmax, (size_t)(1 << i) * P.lv[i].nb * kSubCols);
  return hmax;
}
inline size_t sub_dbuf_floats(const SubUp &P) {
  size_t dmax = 0;
  for (int i = 0; i < P.D; ++i) dmax = std::max(dmax, (size_t)(1 << i) * P.lv[i].n3 * kSubCols);
  return dmax;
}
inline size_t sub_smem_floats(const SubUp &P) { return 2 * sub_buf_floats(P) + 2 * sub_dbuf_floats(P); }

__global__ void __launch_bounds__(kBT) k_b_up_sub(SubUp P, int hmax, int dmax) {
  extern __shared__ __align__(16) float smu[];
  float *buf0 = smu, *buf1 = smu + hmax, *ds = smu + 2 * hmax, *ws = ds + dmax;
  const int s = blockIdx.x, j0 = blockIdx.y * kSubCols, RC = min(kSubCols, P.R - j0);
  // the children's h of the deepest fused level: 2^D nodes from node s 2^D of the level below
  {
    const int nbc = P.lv[P.D - 1].nbc, nch = 2 << (P.D - 1);
    const int64_t c0 = (int64_t)s * nch;
    block_gather<8, float>(
        nch * nbc * kSubCols,
        [&](int idx) {
          const int jj = idx % kSubCols, row = idx / kSubCols;  // row = child * nbc + position
          return jj < RC ? P.hleaf[(c0 * nbc + row) * P.R + j0 + jj] : 0.f;
        },
        [&](int idx, float v) { buf0[idx] = v; });
  }
  __syncthreads();
  const float *hin = buf0;
  for (int i = P.D - 1; i >= 0; --i) {
    const SubLevel &L = P.lv[i];
    const int nn = 1 << i, k0 = s << i, n3 = L.n3, nb = L.nb, nbc = L.nbc;
    // d of the nn nodes: [kk][cc][jj]
    for (int idx = threadIdx.x; idx < nn * n3 * kSubCols; idx += blockDim.x) {
      const int jj = idx % kSubCols, rest = idx / kSubCols, cc = rest % n3, kk = rest / n3;
      float v = hin[((2 * kk + 1) * nbc + L.j3b + cc) * kSubCols + jj] - hin[((2 * kk) * nbc + L.j3a + cc) * kSubCols + jj];
      if (P.jump && jj < RC) {
        const int k = k0 + kk;
        v += d2f_int(P.jump[iface_bd(P.g, L.origin[2 * k], L.origin[2 * k + 1], L.a, L.c, L.split, cc) * P.R + j0 + jj]);
      }
      ds[idx] = v;
    }
    __syncthreads();
    // w3 = X d, to shared memory and to global memory
    for (int idx = threadIdx.x; idx < nn * n3 * kSubCols; idx += blockDim.x) {
      const int jj = idx % kSubCols, rest = idx / kSubCols, r = rest % n3, kk = rest / n3;
      const int k = k0 + kk;
      const float *x = L.X + (int64_t)k * L.strX + r;
      const float *d = ds + kk * n3 * kSubCols + jj;
      float acc = 0.f;
#pragma unroll 4
      for (int c2 = 0; c2 < n3; ++c2) acc = fmaf(__ldg(x + (int64_t)c2 * L.ldX), d[c2 * kSubCols], acc);
      ws[idx] = acc;
      if (jj < RC) L.w3[((int64_t)k * n3 + r) * P.R + j0 + jj] = acc;
    }
    __syncthreads();
    // h = [h^a_1; h^b_2] + Tcat w3 into the other buffer (the top level: global memory)
    const bool top = i == 0;
    float *hout = hin == buf0 ? buf1 : buf0;
    if (!top || P.htop) {
      for (int idx = threadIdx.x; idx < nn * nb * kSubCols; idx += blockDim.x) {
        const int jj = idx % kSubCols, rest = idx / kSubCols, r = rest % nb, kk = rest / nb;
        const int k = k0 + kk, src = __ldg(L.hsrc + r);  // child * nbc + position, child 0 or 1
        float acc = hin[((2 * kk) * nbc + src) * kSubCols + jj];
        const float *t = L.T + (int64_t)k * L.strT + r;
        const float *w = ws + kk * n3 * kSubCols + jj;
#pragma unroll 4
        for (int c2 = 0; c2 < n3; ++c2) acc = fmaf(__ldg(t + (int64_t)c2 * L.ldT), w[c2 * kSubCols], acc);
        if (top) {
          if (jj < RC) P.htop[((int64_t)k * nb + r) * P.R + j0 + jj] = acc;
        } else {
          hout[idx] = acc;
        }
      }
    }
    hin = hout;
    __syncthreads();
  }
}

// One merge apply of a level: the cluster split-K kernel, or (handle option, or when its K chunk
// does not fit in shared memory) the split-K kernel with partial sums in global memory.
template <class XL, class EP>
int launch_b2(hps_handle *H, BatchWork &B, int slot, int M, int K, int nodes, int R, const float *AT, int ld,
              int64_t str, XL xl, EP ep, cudaStream_t st, Pf pf = Pf{}) {
  // per-node operators, one column: streaming applies (the small interface solves w3 = X d of the
  // lower levels stay on the tiled kernel, which measured faster there)
  if (R == 1 && str != 0 && H->batch.one_column_merge && !(slot == kMergeUpW3 && M < 128)) {
    bool done = false;
    if (int e = launch_b1(H, B, slot, M, K, nodes, AT, ld, str, xl, ep, st, &done, pf)) return e;
    if (done) return HPS_OK;
  }
  const BPlan2 P = plan_b2(M, K, nodes, R);
  const size_t smem = b2_smem(P);
  if (!H->batch.gemv2 || smem > kB2MaxSmem)
    return launch_b(H, B, slot, plan_b(M, K, nodes, R, plan_target(H), str == 0, plan_tune(H, slot)), AT, ld, str,
                    xl, ep, st, pf);
  auto kern = P.TC == 8 ? k_b_gemv2<8, XL, EP> : k_b_gemv2<4, XL, EP>;
  if (int e_ = smem_optin((const void *)kern, smem)) return e_;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(P.RT * nodes), (unsigned)P.C, 1);
  cfg.blockDim = dim3(kBT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = (unsigned)P.C;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  H->trace.begin(slot, st);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P, AT, ld, str, xl, ep);
  H->trace.end(slot, st);
  return e == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// ---- merges of the lower tree levels as one dataflow kernel per direction ------------------
// On the lower levels a node's merge is far smaller than a kernel launch.  There, one grid of
// resident CTAs takes node tasks in ticket order (upward: deepest level first; downward: top
// level first) and a task waits only for its own inputs: upward the two children, downward the
// parent (per-node flags, release/acquire).  Tickets are taken by running CTAs in an order in
// which every dependency holds a smaller ticket, so every awaited task is already running.
// Each wait is bounded by a time limit; on expiry the handle's error word is set (hps_status
// reports HPS_ETIMEOUT) and the CTA stops taking tasks.
constexpr int kFlowMaxLevels = 12;

struct FlowLevel {
  int nodes, n3, nb, nbc, j3a, j3b, a, c, split, level;
  const int *origin, *hsrc;
  const float *X, *T, *S;
  int ldX, ldT, ldS;
  int64_t strX, strT, strS;
  float *w3, *h;
  const float *hC;  // h of the child level
  int flag0;        // first node flag of this level
};

struct FlowArgs {
  int nlev, R, Rp, ntasks;
  GridDims g;
  FlowLevel lv[kFlowMaxLevels];  // index t = level - (top flow level)
  int seg_t[kFlowMaxLevels], seg0[kFlowMaxLevels + 1];  // ticket segments: level index, first ticket
  unsigned *sync;  // [0]: ticket counter, [1 ..]: node flags
  int *err;
  const double *jump;
  float *g32;
  UOut uo;
  unsigned long long limit_ns;
};

__device__ __forceinline__ unsigned long long flow_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned flow_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// thread 0: wait (bounded) until every flag in f[0..n) is set; false on timeout or error
__device__ bool flow_wait(const unsigned *f, int n, int *err, unsigned long long limit_ns) {
  unsigned long long t0 = 0;
  for (int i = 0; i < n; ++i) {
    while (!flow_acquire(f + i)) {
      if (flow_acquire(reinterpret_cast<const unsigned *>(err))) return false;
      if (t0 == 0) t0 = flow_ns();
      else if (flow_ns() - t0 > limit_ns) {
        atomicOr(err, 1);
        return false;
      }
      __nanosleep(32);
    }
  }
  return true;
}

// acc[0..3] = sum_c A(r, c) x[c][0..3]: A stored transposed (A(r, c) at a[c * ld]), x in shared
// memory with row stride Rp
__device__ __forceinline__ void flow_dot(float4 &acc, const float *__restrict__ a, int ld, int K, const float *x,
                                         int Rp) {
#pragma unroll 8
  for (int c = 0; c < K; ++c) {
    const float av = __ldg(a + (int64_t)c * ld);
    const float4 xv = *reinterpret_cast<const float4 *>(x + c * Rp);
    acc.x = fmaf(av, xv.x, acc.x);
    acc.y = fmaf(av, xv.y, acc.y);
    acc.z = fmaf(av, xv.z, acc.z);
    acc.w = fmaf(av, xv.w, acc.w);
  }
}

__device__ __forceinline__ bool flow_task(const FlowArgs &A, int &t, int &k) {
  __shared__ int s_ticket;
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = (int)atomicAdd(A.sync, 1u);
  __syncthreads();
  const int tk = s_ticket;
  if (tk >= A.ntasks) return false;
  int s = 0;
  while (tk >= A.seg0[s + 1]) ++s;
  t = A.seg_t[s];
  k = tk - A.seg0[s];
  return true;
}

__device__ __forceinline__ bool flow_wait_block(const FlowArgs &A, const unsigned *f, int n) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = flow_wait(f, n, A.err, A.limit_ns);
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void flow_done(const FlowArgs &A, const FlowLevel &L, int k) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(A.sync + 1 + L.flag0 + k, 1u);
  }
}

__global__ void __launch_bounds__(kBT) k_b_flow_up(FlowArgs A) {
  extern __shared__ float sm[];
  const int R = A.R, Rp = A.Rp, CQ = Rp / 4;
  int t, k;
  while (flow_task(A, t, k)) {
    const FlowLevel &L = A.lv[t];
    if (t + 1 < A.nlev && !flow_wait_block(A, A.sync + 1 + A.lv[t + 1].flag0 + 2 * k, 2)) return;
    // both children's h (contiguous: nodes 2k, 2k+1) in one asynchronous copy; every later read
    // of this task is from shared memory
    const int nch = 2 * L.nbc * R;
    float *Hs = sm, *D = sm + round4(nch), *Ws = D + L.n3 * Rp;
    {
      const float *src = L.hC + (int64_t)(2 * k) * L.nbc * R;
      if (R % 4 == 0)
        for (int i = threadIdx.x; i < nch / 4; i += blockDim.x) cp_async16(Hs + 4 * i, src + 4 * i);
      else
        for (int i = threadIdx.x; i < nch; i += blockDim.x) Hs[i] = src[i];
      cp_async_wait_all();
    }
    __syncthreads();
    // d = h^b_3 - h^a_3 (+ the interface right-hand side)
    block_gather<4, float4>(
        L.n3 * CQ,
        [&](int i) {
          const int cc = i / CQ, j0 = 4 * (i - cc * CQ);
          const float *pb = Hs + (L.nbc + L.j3b + cc) * R + j0, *pa = Hs + (L.j3a + cc) * R + j0;
          float v[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) v[t] = j0 + t < R ? pb[t] - pa[t] : 0.f;
          if (A.jump) {
            const double *pj =
                A.jump + iface_bd(A.g, L.origin[2 * k], L.origin[2 * k + 1], L.a, L.c, L.split, cc) * R + j0;
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (j0 + t < R) v[t] += (float)pj[t];
          }
          return make_float4(v[0], v[1], v[2], v[3]);
        },
        [&](int i, float4 v) { reinterpret_cast<float4 *>(D)[i] = v; });
    __syncthreads();
    // w3 = X d
    for (int it = threadIdx.x; it < L.n3 * CQ; it += blockDim.x) {
      const int r = it % L.n3, j0 = 4 * (it / L.n3);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      flow_dot(acc, L.X + (int64_t)k * L.strX + r, L.ldX, L.n3, D + j0, Rp);
      *reinterpret_cast<float4 *>(Ws + r * Rp + j0) = acc;
      float *w = L.w3 + ((int64_t)k * L.n3 + r) * R + j0;
      if (j0 + 0 < R) w[0] = acc.x;
      if (j0 + 1 < R) w[1] = acc.y;
      if (j0 + 2 < R) w[2] = acc.z;
      if (j0 + 3 < R) w[3] = acc.w;
    }
    __syncthreads();
    // h of the parent = [h^a_1; h^b_2] + Tcat w3 (none at the root of the tree)
    if (L.level > 0) {
      for (int it = threadIdx.x; it < L.nb * CQ; it += blockDim.x) {
        const int r = it % L.nb, j0 = 4 * (it / L.nb);
        const float *hc = Hs + L.hsrc[r] * R + j0;  // hsrc = child * nbc + position
        float4 acc = make_float4(j0 < R ? hc[0] : 0.f, j0 + 1 < R ? hc[1] : 0.f, j0 + 2 < R ? hc[2] : 0.f,
                                 j0 + 3 < R ? hc[3] : 0.f);
        flow_dot(acc, L.T + (int64_t)k * L.strT + r, L.ldT, L.n3, Ws + j0, Rp);
        float *h = L.h + ((int64_t)k * L.nb + r) * R + j0;
        if (j0 + 0 < R) h[0] = acc.x;
        if (j0 + 1 < R) h[1] = acc.y;
        if (j0 + 2 < R) h[2] = acc.z;
        if (j0 + 3 < R) h[3] = acc.w;
      }
    }
    flow_done(A, L, k);
  }
}

__global__ void __launch_bounds__(kBT) k_b_flow_down(FlowArgs A) {
  extern __shared__ float sm[];
  const int R = A.R, Rp = A.Rp, CQ = Rp / 4;
  int t, k;
  while (flow_task(A, t, k)) {
    const FlowLevel &L = A.lv[t];
    if (t > 0 && !flow_wait_block(A, A.sync + 1 + A.lv[t - 1].flag0 + k / 2, 1)) return;
    float *Ub = sm, *W3 = sm + L.nb * Rp;
    const int ox = L.origin[2 * k], oy = L.origin[2 * k + 1];
    {  // this node's w3 rows (contiguous) by asynchronous copies, overlapping the boundary gather
      const float *src = L.w3 + (int64_t)k * L.n3 * R;
      if (R % 4 == 0)
        for (int i = threadIdx.x; i < L.n3 * R / 4; i += blockDim.x) cp_async16(W3 + 4 * i, src + 4 * i);
      else
        for (int i = threadIdx.x; i < L.n3 * R; i += blockDim.x) W3[i] = src[i];
    }
    gather_box(A.g, ox, oy, L.a, L.c, L.nb, R, Rp, A.g32, Ub);
    cp_async_wait_all();
    __syncthreads();
    // u3 = S u_b + w3, scattered to the interface points
    for (int it = threadIdx.x; it < L.n3 * CQ; it += blockDim.x) {
      const int r = it % L.n3, j0 = 4 * (it / L.n3);
      const float *w = W3 + r * R + j0;
      float4 acc = make_float4(j0 < R ? w[0] : 0.f, j0 + 1 < R ? w[1] : 0.f, j0 + 2 < R ? w[2] : 0.f,
                               j0 + 3 < R ? w[3] : 0.f);
      flow_dot(acc, L.S + (int64_t)k * L.strS + r, L.ldS, L.nb, Ub + j0, Rp);
      const int64_t i0 = iface_bd(A.g, ox, oy, L.a, L.c, L.split, r) * R + j0;
      float *o = A.g32 + i0;
      const float v4[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (j0 + t < R) {
          o[t] = v4[t];
          u_out(A.uo, i0 + t, v4[t]);
        }
    }
    flow_done(A, L, k);
  }
}

// ---- FP64 leaf kernels: residual, stage epilogue, explicit first stage ---------------------
enum { kResid = 0, kEpilogue = 1, kEval = 2 };

struct Leaf64Args {
  int mode, R;
  const double *u;      // [N][R]
  const double *Rb;     // [N_int][R] stage right-hand side (kResid, kEpilogue)
  double *out0, *out1;  // kResid: r; kEpilogue / kEval: KL, KE
  const double *q;      // [N_int][qld] (columns qoff ..) or null
  int qld, qoff;
  const double *coef;   // 5 x N_int or null (constants in cst)
  double cst[5];
  int64_t N_int;
  double gdt, dtL, dt;  // dtL: scale of L u in kEval (gamma dt in the batched ARK step)
  int g_kind;
  double gp0, gp1;
  int need_d1, need_d2;  // first / second derivatives needed (zero terms are skipped)
  // fold: the even-odd kernel takes the mode's scale (gamma dt or dt) times the constant
  // coefficients into its half matrices (s1x, s1y: first, s2x, s2y: second derivatives, s0:
  // the zeroth-order term), so its line sums are the scaled terms of L u
  int fold, has_s0;
  int rc;  // even-odd kernel: columns per pass
  double s1x, s1y, s2x, s2y, s0;
  double *flux_r;  // kResid, even-odd kernel: the leaf adds its side fluxes into r at shared edges
};

__global__ void __launch_bounds__(kBT) k_b_leaf64(GridDims g, int nodes, const int *__restrict__ origin,
                                                  Leaf64Args A, const double *__restrict__ Dg) {
  extern __shared__ double sd[];
  const int p = g.p, m = g.m, q = m * m, pp = p * p, R = A.R;
  const int Rc = max(1, min(R, 4096 / pp));
  double *D1x = sd, *D1y = sd + pp, *Dxx = sd + 2 * pp, *Dyy = sd + 3 * pp, *U = sd + 4 * pp;  // U [pp][Rc]
  for (int i = threadIdx.x; i < 4 * pp; i += blockDim.x) sd[i] = Dg[i];
  for (int k = blockIdx.x; k < nodes; k += gridDim.x) {  // one leaf per CTA, or a persistent grid
  const int ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int j0 = 0; j0 < R; j0 += Rc) {
    const int rc = min(Rc, R - j0);
    __syncthreads();
    block_gather<4, double>(
        pp * rc,
        [&](int idx) {
          const int node = idx / rc, jj = idx % rc;
          const int i = node % p, j = node / p;
          const bool ei = (i == 0 || i == p - 1), ej = (j == 0 || j == p - 1);
          int64_t gi = -1;
          if (!ei && !ej) gi = l0 + (j - 1) * m + (i - 1);
          else if (ei && !ej) gi = vseg(g, ix + (i == 0 ? 0 : 1), iy, j - 1);
          else if (!ei && ej) gi = hseg(g, iy + (j == 0 ? 0 : 1), ix, i - 1);
          return gi >= 0 ? A.u[gi * R + j0 + jj] : 0.0;
        },
        [&](int idx, double v) { U[(idx / rc) * Rc + idx % rc] = v; });
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
        if (A.q) e += A.q[gi * A.qld + A.qoff + col];
        A.out0[o] = A.mode == kEval ? A.dtL * Lu : uu - A.Rb[o];
        A.out1[o] = A.dt * e;
      }
    }
  }
  }
}

// Output of one interior point for the FP64 leaf modes; terms of L with zero constant
// coefficients are skipped (A.need_*).
__device__ __forceinline__ void leaf64_out(const Leaf64Args &A, int64_t gi, int col, double uu, double ux, double uy,
                                           double uxx, double uyy) {
  const int64_t o = gi * A.R + col;
  if (A.fold) {  // the derivative terms arrive scaled: their sum is gamma dt L u (kResid) or dt L u (kEval)
    double Ls = 0.0;
    if (A.need_d2) Ls = uxx + uyy;
    if (A.need_d1) Ls += ux + uy;
    if (A.has_s0) Ls = fma(A.s0, uu, Ls);
    if (A.mode == kResid) {
      A.out0[o] = (A.Rb[o] - uu) + Ls;
    } else {
      double e;
      switch (A.g_kind) {
        case HPS_G_ALLEN_CAHN: e = A.gp0 * (uu - uu * uu * uu); break;
        case HPS_G_FISHER: e = A.gp0 * uu * (1.0 - uu); break;
        default: e = 0.0;
      }
      if (A.q) e += A.q[gi * A.qld + A.qoff + col];
      A.out0[o] = Ls;
      A.out1[o] = A.dt * e;
    }
    return;
  }
  double Lu = 0.0;
  if (A.mode != kEpilogue) {
    if (A.coef) {
      Lu = A.coef[gi] * uxx + A.coef[A.N_int + gi] * uyy + A.coef[2 * A.N_int + gi] * ux +
           A.coef[3 * A.N_int + gi] * uy + A.coef[4 * A.N_int + gi] * uu;
    } else {
      if (A.need_d2) Lu = fma(A.cst[1], uyy, A.cst[0] * uxx);
      if (A.need_d1) Lu = fma(A.cst[3], uy, fma(A.cst[2], ux, Lu));
      if (A.cst[4] != 0.0) Lu = fma(A.cst[4], uu, Lu);
    }
  }
  if (A.mode == kResid) {
    A.out0[o] = fma(A.gdt, Lu, A.Rb[o] - uu);
  } else {
    double e;
    switch (A.g_kind) {
      case HPS_G_ALLEN_CAHN: e = A.gp0 * (uu - uu * uu * uu); break;
      case HPS_G_FISHER: e = A.gp0 * uu * (1.0 - uu); break;
      case HPS_G_BURGERS: e = -uu * (A.gp0 * ux + A.gp1 * uy); break;
      default: e = 0.0;
    }
    if (A.q) e += A.q[gi * A.qld + A.qoff + col];
    A.out0[o] = A.mode == kEval ? A.dtL * Lu : uu - A.Rb[o];
    A.out1[o] = A.dt * e;
  }
}

// The FP64 leaf modes for even p by the even-odd decomposition of the differentiation
// matrices (Solomonoff 1992): a Chebyshev matrix D is centro-symmetric (second derivative) or
// centro-antisymmetric (first derivative), so on the symmetric and antisymmetric parts of a
// grid line, E_k = U_k + U_{p-1-k} and O_k = U_k - U_{p-1-k} (k < p/2), the rows i and p-1-i
// of D U are e +- o (resp. +-(e -+ o)) with e = sum_k A_ik E_k, o = sum_k B_ik O_k,
// A = (D_ik + D_i,p-1-k)/2 and B = (D_ik - D_i,p-1-k)/2: p/2 instead of p multiply-adds per
// output.  The FP64 pipe bounds these kernels on this GPU, so the flop count is the runtime.
// One thread takes the four mirror images (i, j), (p-1-i, j), (i, p-1-j), (p-1-i, p-1-j).
__global__ void __launch_bounds__(kBT, 3) k_b_leaf64_eo(GridDims g, int nodes, const int *__restrict__ origin,
                                                     Leaf64Args A, const double *__restrict__ Dg) {
  extern __shared__ double sd[];
  const int p = g.p, m = g.m, q = m * m, pp = p * p, h = p / 2, hh = h * h, R = A.R;
  const int Rc = A.rc;  // columns per pass
  double *Hm = sd, *F0 = sd + 8 * hh, *U = F0 + 4 * h;  // half matrices; unscaled row 0 of the D1 halves; U [pp][Rc]
  double *Ex = U + pp * Rc, *Ox = Ex + m * h * Rc, *Ey = Ox + m * h * Rc, *Oy = Ey + m * h * Rc;  // [m][h][Rc]
  for (int i = threadIdx.x; i < 8 * hh; i += blockDim.x) {
    double v = Dg[4 * pp + i];
    if (A.fold) {
      const int mtx = i / (2 * hh);  // D1x, D1y, Dxx, Dyy halves in this order
      v *= mtx == 0 ? A.s1x : mtx == 1 ? A.s1y : mtx == 2 ? A.s2x : A.s2y;
    }
    Hm[i] = v;
  }
  for (int i = threadIdx.x; i < 4 * h; i += blockDim.x) F0[i] = Dg[4 * pp + (i / h) * hh + i % h];
  const double *A1x = Hm, *B1x = Hm + hh, *A1y = Hm + 2 * hh, *B1y = Hm + 3 * hh;
  const double *Axx = Hm + 4 * hh, *Bxx = Hm + 5 * hh, *Ayy = Hm + 6 * hh, *Byy = Hm + 7 * hh;
  for (int k = blockIdx.x; k < nodes; k += gridDim.x) {
    const int ix = origin[2 * k], iy = origin[2 * k + 1];
    const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
    for (int j0 = 0; j0 < R; j0 += Rc) {
      const int rc = min(Rc, R - j0);
      __syncthreads();
      block_gather<4, double>(
          pp * rc,
          [&](int idx) {
            const int node = idx / rc, jj = idx % rc;
            const int i = node % p, j = node / p;
            const bool ei = (i == 0 || i == p - 1), ej = (j == 0 || j == p - 1);
            int64_t gi = -1;
            if (!ei && !ej) gi = l0 + (j - 1) * m + (i - 1);
            else if (ei && !ej) gi = vseg(g, ix + (i == 0 ? 0 : 1), iy, j - 1);
            else if (!ei && ej) gi = hseg(g, iy + (j == 0 ? 0 : 1), ix, i - 1);
            return gi >= 0 ? A.u[gi * R + j0 + jj] : 0.0;
          },
          [&](int idx, double v) { U[(idx / rc) * Rc + idx % rc] = v; });
      __syncthreads();
      if (A.need_d1 || A.need_d2 || A.flux_r) {
        // symmetric / antisymmetric parts of the interior rows (x lines) and columns (y lines)
        for (int idx = threadIdx.x; idx < m * h * rc; idx += blockDim.x) {
          const int jj = idx % rc, t = idx / rc, kk = t % h, r = t / h + 1, o = t * Rc + jj;
          const double a = U[(r * p + kk) * Rc + jj], b = U[(r * p + p - 1 - kk) * Rc + jj];
          Ex[o] = a + b;
          Ox[o] = a - b;
          const double c = U[(kk * p + r) * Rc + jj], d = U[((p - 1 - kk) * p + r) * Rc + jj];
          Ey[o] = c + d;
          Oy[o] = c - d;
        }
        __syncthreads();
      }
      for (int idx = threadIdx.x; idx < (h - 1) * (h - 1) * rc; idx += blockDim.x) {
        const int jj = idx % rc, t = idx / rc, a = t % (h - 1) + 1, b = t / (h - 1) + 1;
        const int ai = p - 1 - a, bj = p - 1 - b;
        // points 0: (a, b)  1: (ai, b)  2: (a, bj)  3: (ai, bj)
        double xx[4] = {0.0, 0.0, 0.0, 0.0}, yy[4] = {0.0, 0.0, 0.0, 0.0};
        double x1[4] = {0.0, 0.0, 0.0, 0.0}, y1[4] = {0.0, 0.0, 0.0, 0.0};
        const double *exb = Ex + (b - 1) * h * Rc + jj, *oxb = Ox + (b - 1) * h * Rc + jj;
        const double *exj = Ex + (bj - 1) * h * Rc + jj, *oxj = Ox + (bj - 1) * h * Rc + jj;
        const double *eya = Ey + (a - 1) * h * Rc + jj, *oya = Oy + (a - 1) * h * Rc + jj;
        const double *eyi = Ey + (ai - 1) * h * Rc + jj, *oyi = Oy + (ai - 1) * h * Rc + jj;
        if (A.need_d2) {
          double e0 = 0.0, o0 = 0.0, e1 = 0.0, o1 = 0.0;
          for (int kk = 0; kk < h; ++kk) {
            const double ca = Axx[a * h + kk], cb = Bxx[a * h + kk];
            e0 = fma(ca, exb[kk * Rc], e0);
            o0 = fma(cb, oxb[kk * Rc], o0);
            e1 = fma(ca, exj[kk * Rc], e1);
            o1 = fma(cb, oxj[kk * Rc], o1);
          }
          xx[0] = e0 + o0; xx[1] = e0 - o0; xx[2] = e1 + o1; xx[3] = e1 - o1;
          e0 = o0 = e1 = o1 = 0.0;
          for (int kk = 0; kk < h; ++kk) {
            const double ca = Ayy[b * h + kk], cb = Byy[b * h + kk];
            e0 = fma(ca, eya[kk * Rc], e0);
            o0 = fma(cb, oya[kk * Rc], o0);
            e1 = fma(ca, eyi[kk * Rc], e1);
            o1 = fma(cb, oyi[kk * Rc], o1);
          }
          yy[0] = e0 + o0; yy[2] = e0 - o0; yy[1] = e1 + o1; yy[3] = e1 - o1;
        }
        if (A.need_d1) {
          double e0 = 0.0, o0 = 0.0, e1 = 0.0, o1 = 0.0;
          for (int kk = 0; kk < h; ++kk) {
            const double ca = A1x[a * h + kk], cb = B1x[a * h + kk];
            e0 = fma(ca, exb[kk * Rc], e0);
            o0 = fma(cb, oxb[kk * Rc], o0);
            e1 = fma(ca, exj[kk * Rc], e1);
            o1 = fma(cb, oxj[kk * Rc], o1);
          }
          x1[0] = e0 + o0; x1[1] = o0 - e0; x1[2] = e1 + o1; x1[3] = o1 - e1;
          e0 = o0 = e1 = o1 = 0.0;
          for (int kk = 0; kk < h; ++kk) {
            const double ca = A1y[b * h + kk], cb = B1y[b * h + kk];
            e0 = fma(ca, eya[kk * Rc], e0);
            o0 = fma(cb, oya[kk * Rc], o0);
            e1 = fma(ca, eyi[kk * Rc], e1);
            o1 = fma(cb, oyi[kk * Rc], o1);
          }
          y1[0] = e0 + o0; y1[2] = o0 - e0; y1[1] = e1 + o1; y1[3] = o1 - e1;
        }
#pragma unroll
        for (int pt = 0; pt < 4; ++pt) {
          const int i = (pt & 1) ? ai : a, j = (pt & 2) ? bj : b;
          leaf64_out(A, l0 + (j - 1) * m + (i - 1), j0 + jj, U[(j * p + i) * Rc + jj], x1[pt], y1[pt], xx[pt], yy[pt]);
        }
      }
      if (A.flux_r) {
        // Flux jumps at the shared edges (the interface conditions of the collocation system):
        // the normal derivatives on this leaf's four sides are row 0 / row p-1 of D1 on the
        // boundary lines, e + o and o - e from row 0 of the halves (D1 is centro-antisymmetric).
        // r at a shared edge is the second leaf's (east / north) row-0 flux minus the first
        // leaf's row-(p-1) flux; each leaf adds its signed term into r, zeroed beforehand: a sum
        // of two terms onto zero, the same whichever leaf comes first.
        for (int idx = threadIdx.x; idx < 2 * m * rc; idx += blockDim.x) {
          const int jj = idx % rc, t = idx / rc, r = t % m + 1, dir = t / m;
          const double *E = (dir ? Ey : Ex) + (r - 1) * h * Rc + jj, *O = (dir ? Oy : Ox) + (r - 1) * h * Rc + jj;
          const double *a0 = F0 + 2 * dir * h, *b0 = a0 + h;
          double e = 0.0, o = 0.0;
          for (int kk = 0; kk < h; ++kk) {
            e = fma(a0[kk], E[kk * Rc], e);
            o = fma(b0[kk], O[kk * Rc], o);
          }
          const int col = j0 + jj;
          if (dir == 0) {
            if (ix > 0) atomicAdd(A.flux_r + vseg(g, ix, iy, r - 1) * R + col, e + o);
            if (ix + 1 < g.n1) atomicAdd(A.flux_r + vseg(g, ix + 1, iy, r - 1) * R + col, -(o - e));
          } else {
            if (iy > 0) atomicAdd(A.flux_r + hseg(g, iy, ix, r - 1) * R + col, e + o);
            if (iy + 1 < g.n2) atomicAdd(A.flux_r + hseg(g, iy + 1, ix, r - 1) * R + col, -(o - e));
          }
        }
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
  const StageEpi E{1, A.Rb, A.out0, A.out1, A.q, A.qld, A.qoff, A.g_kind, A.dt, A.dt * A.gp0};
  stage_epi_point(E, A.R, o, uu);
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
#pragma unroll 4
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
#pragma unroll 4
    for (int k = 0; k < p; ++k) {
      const int64_t is = k == 0 ? hseg(g, L - 1, ix, in - 1) : k == p - 1 ? gi : ls + (k - 1) * m + (in - 1);
      const int64_t inn = k == 0 ? gi : k == p - 1 ? hseg(g, L + 1, ix, in - 1) : ln + (k - 1) * m + (in - 1);
      fa = fma(D1y[(p - 1) * p + k], u[is * R + col], fa);
      fb = fma(D1y[k], u[inn * R + col], fb);
    }
  }
  r[gi * R + col] = -(fa - fb);
}


// Step close by the edge projection (the identity-operator system of Sec. 3.1.1 solved
// directly).  With the interior values fixed, flux continuity at a shared-edge point involves
// only the grid line through it normal to the edge: the two leaves' interior points on that line
// and the edge values at the line's three leaf boundaries.  So on a uniform leaf grid the
// shared-edge values of one grid line (leaf row iy and node j for vertical edges, leaf column ix
// and node i for horizontal ones) solve a tridiagonal system
//   lo v_{L-1} + d v_L + up v_{L+1} = F0_E - Fl_W,  L = 1 .. n-1,  v_0 and v_n boundary data,
// lo = D1[p-1][0], d = D1[p-1][p-1] - D1[0][0], up = -D1[0][p-1], F0_E / Fl_W the east (north)
// leaf's row-0 and the west (south) leaf's row-(p-1) derivative sums over their interior points.
//
// k_b_close_leaf: one CTA per leaf; interior values = the combination `c` (written into u),
// then the leaf adds +F0 into the right-hand side of its west / south edge and -Fl into that of
// its east / north edge (rhs zeroed beforehand; two terms onto zero, so the order of the two
// leaves does not change the sum).
constexpr int kCloseRc = 16;
__global__ void __launch_bounds__(kBT) k_b_close_leaf(GridDims g, const int *__restrict__ origin, int R, Combo c,
                                                     double *__restrict__ u, double *__restrict__ rhs,
                                                     const double *__restrict__ Dg) {
  extern __shared__ double scl[];
  const int p = g.p, m = g.m, q = m * m, Rc = min(R, kCloseRc);
  double *Dr = scl, *Us = scl + 4 * p;  // rows 0 and p-1 of D1x, then of D1y; Us [q][Rc]
  for (int i = threadIdx.x; i < 4 * p; i += blockDim.x) {
    const int mtx = i / (2 * p), row = (i / p) % 2 ? p - 1 : 0;
    Dr[i] = Dg[mtx * p * p + row * p + i % p];
  }
  const int k = blockIdx.x, ix = origin[2 * k], iy = origin[2 * k + 1];
  const int64_t l0 = ((int64_t)iy * g.n1 + ix) * q;
  for (int j0 = 0; j0 < R; j0 += Rc) {
    const int rc = min(Rc, R - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < q * rc; idx += blockDim.x) {
      const int pt = idx / rc, jj = idx % rc;
      const int64_t o = (l0 + pt) * R + j0 + jj;
      double acc = 0.0;
      int t = 0;
      if (c.n > 0 && c.coef[0] == 1.0) {  // a leading unit term costs no FP64 operation
        acc = c.ptr[0][o];
        t = 1;
      }
      for (; t < c.n; ++t) acc = fma(c.coef[t], c.ptr[t][o], acc);
      u[o] = acc;
      Us[pt * Rc + jj] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * m * rc; idx += blockDim.x) {
      const int jj = idx % rc, t = idx / rc, r = t % m, dir = t / m;
      const double *d0 = Dr + 2 * dir * p, *dl = d0 + p;
      double f0 = 0.0, fl = 0.0;
      for (int kk = 1; kk <= m; ++kk) {  // x line j = r + 1 (dir 0) or y line i = r + 1 (dir 1)
        const double v = Us[(dir ? (kk - 1) * m + r : r * m + kk - 1) * Rc + jj];
        f0 = fma(d0[kk], v, f0);
        fl = fma(dl[kk], v, fl);
      }
      const int col = j0 + jj;
      if (dir == 0) {
        if (ix > 0) atomicAdd(rhs + vseg(g, ix, iy, r) * R + col, f0);
        if (ix + 1 < g.n1) atomicAdd(rhs + vseg(g, ix + 1, iy, r) * R + col, -fl);
      } else {
        if (iy > 0) atomicAdd(rhs + hseg(g, iy, ix, r) * R + col, f0);
        if (iy + 1 < g.n2) atomicAdd(rhs + hseg(g, iy + 1, ix, r) * R + col, -fl);
      }
    }
  }
}

// k_b_edge_tridiag: one thread per grid line of shared edges and column; forward elimination
// with the host's Thomas factors (w_L, 1/b_L) into rhs, back substitution into u.
__global__ void k_b_edge_tridiag(GridDims g, int R, double *__restrict__ rhs, double *__restrict__ u,
                                 const double *__restrict__ proj, double lox, double upx, double loy, double upy,
                                 const double *__restrict__ J) {
  const int64_t nvl = (int64_t)g.n2 * g.m, nhl = (int64_t)g.n1 * g.m;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (nvl + nhl) * R) return;
  const int col = (int)(idx % R);
  int64_t s = idx / R;
  const bool vert = s < nvl;
  if (!vert) s -= nvl;
  const int n = vert ? g.n1 : g.n2;  // lines 0 .. n; shared ones 1 .. n-1
  if (n < 2) return;
  const int a = (int)(s / g.m), node = (int)(s % g.m);  // leaf row (vertical) or column, node
  const double *w = vert ? proj : proj + 2 * (g.n1 - 1), *ib = w + (n - 1);
  const double lo = vert ? lox : loy, up = vert ? upx : upy;
  auto at = [&](int L) { return (vert ? vseg(g, L, a, node) : hseg(g, L, a, node)) * R + col; };
  const double v0 = u[at(0)], vn = u[at(n)];
  // blocks of kTB lines: the loads of a block are issued before its recurrence steps
  constexpr int kTB = 8;
  double rp = 0.0;
  for (int L0 = 1; L0 < n; L0 += kTB) {
    double r[kTB];
#pragma unroll
    for (int t = 0; t < kTB; ++t)
      if (L0 + t < n) r[t] = J ? rhs[at(L0 + t)] + J[at(L0 + t)] : rhs[at(L0 + t)];
#pragma unroll
    for (int t = 0; t < kTB; ++t) {
      const int L = L0 + t;
      if (L < n) {
        double x = r[t];
        if (L == 1) x -= lo * v0;
        if (L == n - 1) x -= up * vn;
        rp = L == 1 ? x : fma(-w[L - 1], rp, x);
        rhs[at(L)] = rp;
      }
    }
  }
  double v = 0.0;
  for (int L1 = n - 1; L1 >= 1; L1 -= kTB) {
    double r[kTB];
#pragma unroll
    for (int t = 0; t < kTB; ++t)
      if (L1 - t >= 1) r[t] = rhs[at(L1 - t)];
#pragma unroll
    for (int t = 0; t < kTB; ++t) {
      const int L = L1 - t;
      if (L >= 1) {
        v = L == n - 1 ? r[t] * ib[L - 1] : (r[t] - up * v) * ib[L - 1];
        u[at(L)] = v;
      }
    }
  }
}

// f: [N_bd][fld], this call's columns from foff; u (if non-null) gets the FP64 values
__global__ void k_b_set_boundary32(GridDims g, int R, float *__restrict__ g32, const double *__restrict__ f, int fld,
                                   int foff, double *__restrict__ u) {
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
  const double v = f ? f[kk * fld + foff + j] : 0.0;
  g32[gi * R + j] = d2f_int(v);
  if (u) u[gi * R + j] = v;
}


inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// y += a x (n entries)
__global__ void k_b_axpy(int64_t n, double a, const double *__restrict__ x, double *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}
// out[kk R + j] = a f[kk fld + foff + j] for the boundary points kk < n_bd (a scaled copy of one
// stage of boundary data in the [N_bd][R] layout)
__global__ void k_b_scale_bd(int64_t n_bd, int R, double a, const double *__restrict__ f, int fld, int foff,
                             double *__restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_bd * R) return;
  const int64_t kk = idx / R;
  const int j = (int)(idx % R);
  out[idx] = a * f[kk * fld + foff + j];
}
// out[i] = sum_t c.coef[t] c.ptr[t][i], i < n (out may be a term: same index)
__global__ void k_b_combine_all(int64_t n, Combo c, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = c.coef[0] == 1.0 ? c.ptr[0][i] : c.coef[0] * c.ptr[0][i];
  for (int t = 1; t < c.n; ++t) acc = fma(c.coef[t], c.ptr[t][i], acc);
  out[i] = acc;
}

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

// TF32 split of the per-node leaf operators for the tensor-core leaf apply, K-major:
// dst[node][0][r][c] = hi and dst[node][1][r][c] = lo of (float) A(r, c), A(r, c) at c ld + r of
// the transposed FP64 operator; hi keeps the top 10 mantissa bits (exactly TF32), lo = value - hi.
__global__ void k_kmajor_split(const double *__restrict__ src, int ld64, int64_t str64, int q, int64_t nops,
                               float *__restrict__ dst, int ldk) {
  const int64_t per = (int64_t)q * ldk, total = nops * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / per, rem = i % per;
    const int r = (int)(rem / ldk), c = (int)(rem % ldk);
    const float v = c < q ? (float)src[node * str64 + (int64_t)c * ld64 + r] : 0.f;
    const float h = tc5::tf32_hi(v);
    dst[node * 2 * per + rem] = h;
    dst[node * 2 * per + per + rem] = v - h;
  }
}

// BF16 copy of the per-node leaf operators for the BF16 trial, K-major: dst[node][r][c] (row stride
// ldk, a multiple of 8) = A(r, c) rounded to BF16.
__global__ void k_kmajor_bf16(const double *__restrict__ src, int ld64, int64_t str64, int q, int64_t nops,
                              __nv_bfloat16 *__restrict__ dst, int ldk) {
  const int64_t per = (int64_t)q * ldk, total = nops * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / per, rem = i % per;
    const int r = (int)(rem / ldk), c = (int)(rem % ldk);
    dst[i] = __float2bfloat16_rn(c < q ? (float)src[node * str64 + (int64_t)c * ld64 + r] : 0.f);
  }
}

// Tensor map of the split K-major leaf operators: 3-D (column, row, 2 leaf + part) FP32, boxes of
// 32 columns x 128 rows x 1 in the 128-byte swizzle; out-of-range rows and columns read as zeros.
int umma_map(hps_handle *H) {
  Batch &Bt = H->batch;
  using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult qr{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn)
    return HPS_ECUDA;
  const int q = H->q;
  const cuuint64_t dims[3] = {(cuuint64_t)q, (cuuint64_t)q, 2 * (cuuint64_t)H->lev[H->L].nodes};
  const cuuint64_t strides[2] = {(cuuint64_t)Bt.ainv_ldk * 4, (cuuint64_t)q * Bt.ainv_ldk * 4};
  const cuuint32_t box[3] = {32, 128, 1}, estr[3] = {1, 1, 1};
  CUtensorMap map;
  if (reinterpret_cast<EncodeFn>(fn)(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Bt.ainv_k, dims, strides, box, estr,
                                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HPS_ECUDA;
  static_assert(sizeof(map) == sizeof(Bt.ainv_map), "tensor map size");
  memcpy(Bt.ainv_map, &map, sizeof map);
  return HPS_OK;
}

// The BF16 copy of the per-node leaf operators and its tensor map (boxes of 64 columns x 128 rows),
// made when the BF16 trial is switched on.
int umma_bf16_reserve(hps_handle *H) {
  Batch &Bt = H->batch;
  if (Bt.ainv_bf) return HPS_OK;
  const int q = H->q;
  if (H->shared || !H->impl.Ainv || !H->impl.strA || q < 64 || q > 256) return HPS_EINVAL;
  using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult qr{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn)
    return HPS_ECUDA;
  cudaDeviceSynchronize();
  const int64_t nops = H->lev[H->L].nodes;
  const int ldk = (q + 7) & ~7;
  __nv_bfloat16 *p = nullptr;
  if (cudaMalloc(&p, (size_t)nops * q * ldk * sizeof(__nv_bfloat16)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(p);
  k_kmajor_bf16<<<4 * H->num_sms, 256>>>(H->impl.Ainv, H->impl.ldA, H->impl.strA, q, nops, p, ldk);
  const cuuint64_t dims[3] = {(cuuint64_t)q, (cuuint64_t)q, (cuuint64_t)nops};
  const cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)q * ldk * 2};
  const cuuint32_t box[3] = {64, 128, 1}, estr[3] = {1, 1, 1};
  CUtensorMap map;
  if (reinterpret_cast<EncodeFn>(fn)(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p, dims, strides, box, estr,
                                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HPS_ECUDA;
  memcpy(Bt.ainv_map_bf, &map, sizeof map);
  Bt.ainv_bf = p;
  return cudaDeviceSynchronize() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// The bytes of an FP32 operator set of `nodes` nodes with `cols` columns (as convert_op lays it out).
Pf op_range(const Op32 &o, int cols, int nodes) {
  if (!o.p) return Pf{};
  return Pf{reinterpret_cast<const char *>(o.p), (o.str ? (int64_t)nodes : 1) * cols * (int64_t)o.ld * (int64_t)sizeof(float)};
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

// Split-K scratch for calls with up to Rmax columns (the plan depends on the column count).
size_t partial_floats(hps_handle *H, int Rmax) {
  size_t mx = 0;
  for (int R = 1; R <= Rmax; ++R)
  for (int l = 0; l < H->L; ++l) {
    const Level &lv = H->lev[l];
    for (int sh = 0; sh < 2; ++sh) {  // the identity operators are shared even when the others are not
      const BPlan P[3] = {plan_b(lv.n3, lv.n3, lv.nodes, R, plan_target(H), sh, plan_tune(H, kMergeUpW3)),
                          plan_b(lv.nb, lv.n3, lv.nodes, R, plan_target(H), sh, plan_tune(H, kMergeUpH)),
                          plan_b(lv.n3, lv.nb, lv.nodes, R, plan_target(H), sh, plan_tune(H, kMergeDown))};
      for (const BPlan &pl : P)
        if (pl.ksplit > 1) mx = std::max(mx, (size_t)pl.ksplit * pl.nodes * pl.M * pl.Rp);
    }
  }
  return mx;
}

inline int m_of(const hps_handle *H) { return H->m; }

int flow_launch(hps_handle *H, BatchWork &B, const FlowArgs &FA, bool up, size_t smem, int nflags, cudaStream_t st) {
  if ((size_t)nflags + 1 > B.flow_len) return HPS_EINVAL;
  auto kern = up ? k_b_flow_up : k_b_flow_down;
  if (int e_ = smem_optin((const void *)kern, smem)) return e_;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, smem) != cudaSuccess || per_sm < 1)
    return HPS_ECUDA;
  const int grid = std::min(FA.ntasks, per_sm * H->num_sms);
  cudaMemsetAsync(B.flow_sync, 0, ((size_t)nflags + 1) * sizeof(unsigned), st);
  H->trace.begin(up ? kMergeUpFused : kMergeDownFused, st);
  kern<<<grid, kBT, smem, st>>>(FA);
  H->trace.end(up ? kMergeUpFused : kMergeDownFused, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Parts of a sweep (a sweep runs them in this order; the lockstep multi-instance step runs the
// leaf parts per instance and the merges of all instances as grouped launches in between).
enum : unsigned { kSweepLeafUp = 1, kSweepMerges = 2, kSweepLeafDown = 4, kSweepAll = 7 };

// One FP32 sweep on R columns: leaf applies, merges up (with an optional FP64 interface
// right-hand side), merges down into g32 (whose outer boundary the caller has set), leaf solves.
int sweep32(hps_handle *H, BatchWork &B, const OpSet &ops, const OpSet32 &o32, int R, const Combo &rhs,
            double *Rsave, const double *jump, UOut uo, bool allow_tc, cudaStream_t st, const StageEpi &ep,
            bool &epi_done, unsigned parts = kSweepAll) {
  const int L = H->L, p = H->p, q = H->q, b = H->b, Rp = round4(R);
  const Level &leaf = H->lev[L];
  const bool tc8 = Rp % 8 == 0;
  const bool narrow = Rp == 4 && !H->shared;  // streaming per-leaf operators, one column group
  const int QQ = (q + 3) / 4, KS = std::max(1, kBT / QQ);
  if (parts & kSweepLeafUp) {
    int cps = H->batch.stream_leaf;  // CTAs per SM: fewer where the rings of that many do not fit
    StreamPlan SPu{};
    for (; cps > 0; --cps) {
      SPu = stream_plan(leaf.nodes, q, q, o32.Ainv.ld, o32.Ainv.str, cps, 2 * p * p, H->batch.stream_chunk_kb);
      if (stream_fits(SPu, 2 * p * p)) break;
    }
    const bool stream_up = narrow && cps > 0 && !ops.identity && o32.Ainv.p;
    if (stream_up) {
      H->trace.begin(kLeafUp, st);
      if (int e = launch_stream(H, SPu, cps, o32.Ainv.p,
                                StreamUp{H->g, R, leaf.d_origin, rhs, Rsave, H->d_D, B.w32, B.h32[L]}, st))
        return e;
      H->trace.end(kLeafUp, st);
    } else if (narrow) {
      const size_t smem = (size_t)(round4(2 * p * p) + 8 * q + KS * 16 * QQ) * sizeof(float);
      if (int e_ = smem_optin((const void *)k_b_leaf_up_narrow, smem)) return e_;
      H->trace.begin(kLeafUp, st);
      k_b_leaf_up_narrow<<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, o32.Ainv.p, o32.Ainv.ld,
                                                        o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
      H->trace.end(kLeafUp, st);
    } else if (H->fd.on && H->batch.fast_diag && !ops.identity) {
      const int mp = H->fd.mp;
      const size_t smem = (size_t)(5 * m_of(H) * mp + 2 * q * Rp) * sizeof(float);
      if (int e_ = smem_optin((const void *)k_b_leaf_up_fd, smem)) return e_;
      H->trace.begin(kLeafUp, st);
      k_b_leaf_up_fd<<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, H->fd.d32, mp, B.w32,
                                                    B.h32[L]);
      H->trace.end(kLeafUp, st);
    } else if (allow_tc && H->batch.afrag_hi && H->batch.tensor_leaf && H->shared && !ops.identity && Rp % 8 == 0 &&
               Rp / 8 <= kTcMaxNT &&
               !H->batch.leaf_split) {
      const int MT = (q + 15) / 16, KT = (q + 7) / 8, NT = Rp / 8;
      const size_t smem = (size_t)(round4(2 * p * p) + 2 * KT * 8 * tc_rs(Rp)) * sizeof(float);
      auto kern = NT == 4 ? k_b_leaf_up_tc<4> : NT == 3 ? k_b_leaf_up_tc<3> : NT == 2 ? k_b_leaf_up_tc<2>
                                                                                     : k_b_leaf_up_tc<1>;
      if (int e_ = smem_optin((const void *)kern, smem)) return e_;
      H->trace.begin(kLeafUp, st);
      kern<<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, reinterpret_cast<const uint4 *>(H->batch.afrag_hi),
                                          reinterpret_cast<const uint4 *>(H->batch.afrag_lo), MT, KT, H->d_D, B.w32,
                                          B.h32[L]);
      H->trace.end(kLeafUp, st);
    } else if (allow_tc && H->batch.umma_leaf == 3 && H->batch.ainv_bf && !H->shared && !ops.identity &&
               (Rp == 16 || Rp == 32) && umma_fits(p, R, Rp)) {
      // BF16 trial: the first sweep's leaf applies as one BF16 product on the tensor cores
      const size_t smem = umma_smem_bytes(p, Rp);
      auto kern = Rp == 32 ? k_b_leaf_up_umma<32, true> : k_b_leaf_up_umma<16, true>;
      if (int e_ = smem_optin((const void *)kern, smem)) return e_;
      CUtensorMap map;
      memcpy(&map, H->batch.ainv_map_bf, sizeof map);
      H->trace.begin(kLeafUp, st);
      const int64_t n = H->g.N_int * R;
      k_b_combo<<<(unsigned)((n + 4 * 256 - 1) / (4 * 256)), 256, 0, st>>>(n, rhs, Rsave, B.r32);
      kern<<<std::min(leaf.nodes, H->num_sms), kUmmaThreads, smem, st>>>(H->g, leaf.nodes, R, leaf.d_origin, B.r32,
                                                                        map, H->d_D, B.w32, B.h32[L], H->perr);
      H->trace.end(kLeafUp, st);
    } else if ((allow_tc || H->batch.umma_leaf == 2) && (H->batch.umma_leaf == 1 || H->batch.umma_leaf == 2) &&
               H->batch.ainv_k && !H->shared && !ops.identity &&
               (Rp == 16 || Rp == 32) && umma_fits(p, R, Rp)) {
      // per-node leaf operators on the tcgen05 tensor cores (3xTF32), persistent CTAs, after the
      // stage right-hand side as its own streaming pass (FP64 sum saved, FP32 copy for the products)
      const size_t smem = umma_smem_bytes(p, Rp);
      auto kern = Rp == 32 ? k_b_leaf_up_umma<32, false> : k_b_leaf_up_umma<16, false>;
      if (int e_ = smem_optin((const void *)kern, smem)) return e_;
      CUtensorMap map;
      memcpy(&map, H->batch.ainv_map, sizeof map);
      H->trace.begin(kLeafUp, st);
      const int64_t n = H->g.N_int * R;
      k_b_combo<<<(unsigned)((n + 4 * 256 - 1) / (4 * 256)), 256, 0, st>>>(n, rhs, Rsave, B.r32);
      kern<<<std::min(leaf.nodes, H->num_sms), kUmmaThreads, smem, st>>>(H->g, leaf.nodes, R, leaf.d_origin, B.r32,
                                                                        map, H->d_D, B.w32, B.h32[L], H->perr);
      H->trace.end(kLeafUp, st);
    } else {
      const size_t smem = (size_t)(round4(2 * p * p) + 2 * q * Rp) * sizeof(float);
      if (int e_ = smem_optin((const void *)k_b_leaf_up<8>, smem)) return e_;
      if (int e_ = smem_optin((const void *)k_b_leaf_up<4>, smem)) return e_;
      H->trace.begin(kLeafUp, st);
      const float *r32 = nullptr;
      if (H->batch.leaf_split) {  // stage right-hand side as its own streaming pass
        const int64_t n = H->g.N_int * R;
        k_b_combo<<<(unsigned)((n + 4 * 256 - 1) / (4 * 256)), 256, 0, st>>>(n, rhs, Rsave, B.r32);
        r32 = B.r32;
      }
      if (tc8)
        k_b_leaf_up<8><<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, r32, o32.Ainv.p, o32.Ainv.ld,
                                                      o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
      else
        k_b_leaf_up<4><<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, rhs, Rsave, r32, o32.Ainv.p, o32.Ainv.ld,
                                                      o32.Ainv.str, ops.identity ? 1 : 0, H->d_D, B.w32, B.h32[L]);
      H->trace.end(kLeafUp, st);
    }
  }
  if (parts & kSweepMerges) {
    // lower levels (small nodes): one dataflow kernel per direction (levels lr .. L-1)
    int lr = L;
    while (lr > 0 && L - lr < std::min(kFlowMaxLevels, H->batch.flow_levels) &&
           H->lev[lr - 1].n3 <= H->batch.flow_n3_max && (int64_t)H->lev[lr - 1].nb * Rp <= 16384)
      --lr;
    const int nflow = L - lr;
    FlowArgs FA{};
    size_t smem_up = 0, smem_down = 0;
    int nflags = 0;
    if (nflow > 0) {
      FA.nlev = nflow;
      FA.R = R;
      FA.Rp = Rp;
      FA.g = H->g;
      int n3max = 0, nbmax = 0;
      for (int t = 0; t < nflow; ++t) {
        const int l = lr + t;
        const Level &lv = H->lev[l];
        FlowLevel &F = FA.lv[t];
        F.nodes = lv.nodes;
        F.n3 = lv.n3;
        F.nb = lv.nb;
        F.nbc = lv.nbc;
        F.j3a = lv.j3a;
        F.j3b = lv.j3b;
        F.a = lv.a;
        F.c = lv.c;
        F.split = lv.split;
        F.level = l;
        F.origin = lv.d_origin;
        F.hsrc = lv.d_hsrc;
        F.X = o32.X[l].p;
        F.ldX = o32.X[l].ld;
        F.strX = o32.X[l].str;
        F.T = o32.Tcat[l].p;
        F.ldT = o32.Tcat[l].ld;
        F.strT = o32.Tcat[l].str;
        F.S = o32.S[l].p;
        F.ldS = o32.S[l].ld;
        F.strS = o32.S[l].str;
        F.w3 = B.w332[l];
        F.h = B.h32[l];
        F.hC = B.h32[l + 1];
        F.flag0 = nflags;
        nflags += lv.nodes;
        n3max = std::max(n3max, lv.n3);
        nbmax = std::max(nbmax, lv.nb);
      }
      FA.ntasks = nflags;
      FA.sync = B.flow_sync;
      FA.err = H->perr;
      FA.jump = jump;
      FA.g32 = B.g32;
      FA.uo = uo;
      FA.limit_ns = 2000000000ull;
      int nbcmax = 0;
      for (int t = 0; t < nflow; ++t) nbcmax = std::max(nbcmax, FA.lv[t].nbc);
      smem_up = ((size_t)round4(2 * nbcmax * R) + 2 * (size_t)n3max * Rp) * sizeof(float);
      smem_down = ((size_t)nbmax * Rp + (size_t)n3max * R) * sizeof(float);
      // upward ticket order: deepest level first
      for (int s2 = 0, t = nflow - 1; t >= 0; --t, ++s2) {
        FA.seg_t[s2] = t;
        FA.seg0[s2] = s2 == 0 ? 0 : FA.seg0[s2 - 1] + FA.lv[FA.seg_t[s2 - 1]].nodes;
      }
      FA.seg0[nflow] = nflags;
      if (int e = flow_launch(H, B, FA, true, smem_up, nflags, st)) return e;
    }
    // the lowest levels fused per subtree (option): levels [lb, lr)
    int lup = lr;
    if (H->batch.sub_levels > 0 && nflow == 0) {
      const int D = std::min({H->batch.sub_levels, lr, kSubMaxLevels});
      const int lb = lr - D;
      const int cg = (R + kSubCols - 1) / kSubCols;
      if (D >= 2) {
        SubUp P{};
        P.lb = lb;
        P.D = D;
        P.R = R;
        P.hleaf = B.h32[lr];
        P.htop = lb > 0 ? B.h32[lb] : nullptr;
        P.jump = jump;
        P.g = H->g;
        for (int i = 0; i < D; ++i) {
          const int l = lb + i;
          const Level &lv = H->lev[l];
          SubLevel &S = P.lv[i];
          S.w3 = B.w332[l];
          S.X = o32.X[l].p;
          S.ldX = o32.X[l].ld;
          S.strX = o32.X[l].str;
          S.T = o32.Tcat[l].p;
          S.ldT = o32.Tcat[l].ld;
          S.strT = o32.Tcat[l].str;
          S.hsrc = lv.d_hsrc;
          S.origin = lv.d_origin;
          S.nbc = lv.nbc;
          S.nb = lv.nb;
          S.n3 = lv.n3;
          S.j3a = lv.j3a;
          S.j3b = lv.j3b;
          S.a = lv.a;
          S.c = lv.c;
          S.split = lv.split;
        }
        const size_t smem = sub_smem_floats(P) * sizeof(float);
        if (smem <= 96 * 1024) {
          if (int e_ = smem_optin((const void *)k_b_up_sub, smem)) return e_;
          H->trace.begin(kMergeUpW3, st);
          k_b_up_sub<<<dim3((unsigned)H->lev[lb].nodes, (unsigned)cg), kBT, smem, st>>>(P, (int)sub_buf_floats(P),
                                                                                      (int)sub_dbuf_floats(P));
          H->trace.end(kMergeUpW3, st);
          if (cudaPeekAtLastError() != cudaSuccess) return HPS_ECUDA;
          lup = lb;
        }
      }
    }
    // (option) each apply prefetches the operator of the apply after it into L2
    const bool pfn = H->batch.prefetch_next && !H->shared;
    auto opS = [&](int l) { return pfn && l < lr ? op_range(o32.S[l], H->lev[l].nb, H->lev[l].nodes) : Pf{}; };
    for (int l = lup - 1; l >= 0; --l) {
      const Level &lv = H->lev[l];
      const Pf nw3 = !pfn ? Pf{} : l > 0 ? op_range(o32.Tcat[l], lv.n3, lv.nodes) : opS(0);
      if (int e = launch_b2(H, B, kMergeUpW3, lv.n3, lv.n3, lv.nodes, R, o32.X[l].p, o32.X[l].ld, o32.X[l].str,
                            BXDiff{B.h32[l + 1], lv.nbc, lv.j3a, lv.j3b, R, jump, H->g, lv.d_origin, lv.a, lv.c, lv.split},
                            BEStore{B.w332[l], lv.n3, R}, st, nw3))
        return e;
      if (l > 0) {
        const Pf nh = pfn ? op_range(o32.X[l - 1], H->lev[l - 1].n3, H->lev[l - 1].nodes) : Pf{};
        if (int e = launch_b2(H, B, kMergeUpH, lv.nb, lv.n3, lv.nodes, R, o32.Tcat[l].p, o32.Tcat[l].ld, o32.Tcat[l].str,
                              BXVec{B.w332[l], lv.n3, R}, BEFlux{lv.d_hsrc, B.h32[l + 1], lv.nbc, lv.nb, R, B.h32[l]}, st,
                              nh))
          return e;
      }
    }
    for (int l = 0; l < lr; ++l) {
      const Level &lv = H->lev[l];
      if (int e = launch_b2(H, B, kMergeDown, lv.n3, lv.nb, lv.nodes, R, o32.S[l].p, o32.S[l].ld, o32.S[l].str,
                            BXBd{H->g, lv.d_origin, lv.a, lv.c, R, B.g32},
                            BEScatter{H->g, lv.d_origin, lv.a, lv.c, lv.split, lv.n3, R, B.w332[l], B.g32, uo}, st,
                            opS(l + 1)))
        return e;
    }
    if (nflow > 0) {
      // downward ticket order: top flow level first
      for (int t = 0; t < nflow; ++t) {
        FA.seg_t[t] = t;
        FA.seg0[t] = t == 0 ? 0 : FA.seg0[t - 1] + FA.lv[t - 1].nodes;
      }
      FA.seg0[nflow] = nflags;
      if (int e = flow_launch(H, B, FA, false, smem_down, nflags, st)) return e;
    }
  }
  if (parts & kSweepLeafDown) {
    H->trace.begin(kLeafDown, st);
    int cpd = H->batch.stream_leaf;
    StreamPlan SPd{};
    const bool spre = H->batch.stream_prefetch;
    const int down_floats = spre ? 4 * b : 0;  // (StreamDown::role_floats)
    for (; cpd > 0; --cpd) {
      SPd = stream_plan(leaf.nodes, q, b, o32.Sleaf.ld, o32.Sleaf.str, cpd, down_floats, H->batch.stream_chunk_kb);
      if (stream_fits(SPd, down_floats)) break;
    }
    const bool stream_down = narrow && cpd > 0 && !ops.identity && o32.Sleaf.p;
    if (stream_down) {
      if (int e = launch_stream(H, SPd, cpd, o32.Sleaf.p, StreamDown{H->g, R, leaf.d_origin, B.w32, B.g32, uo, spre}, st))
        return e;
    } else if (narrow)
      k_b_leaf_down_narrow<<<leaf.nodes, kBT, (size_t)(4 * b + KS * 16 * QQ) * sizeof(float), st>>>(
          H->g, R, leaf.d_origin, o32.Sleaf.p, o32.Sleaf.ld, o32.Sleaf.str, ops.identity ? 1 : 0, B.w32, B.g32, uo);
    else if (H->shared && !ops.identity && (size_t)(b * o32.Sleaf.ld + (b + q) * Rp) * sizeof(float) <= 110 * 1024) {
      const size_t smem = (size_t)(b * o32.Sleaf.ld + (b + q) * Rp) * sizeof(float);
      const bool t8 = tc8;
      auto kern = t8 ? k_b_leaf_down_res<8> : k_b_leaf_down_res<4>;
      if (int e_ = smem_optin((const void *)kern, smem)) return e_;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, smem) != cudaSuccess || per_sm < 1)
        return HPS_ECUDA;
      kern<<<std::min(leaf.nodes, per_sm * H->num_sms), kBT, smem, st>>>(H->g, leaf.nodes, R, leaf.d_origin,
                                                                        o32.Sleaf.p, o32.Sleaf.ld, B.w32, B.g32, uo, ep);
      epi_done = ep.on != 0;
    } else {
      const int staged = (size_t)(b + q) * Rp * sizeof(float) <= 96 * 1024;  // coalesced output through smem
      const size_t smem = (size_t)(staged ? b + q : b) * Rp * sizeof(float);
      auto kern = tc8 ? k_b_leaf_down<8> : k_b_leaf_down<4>;
      if (int e_ = smem_optin((const void *)kern, smem)) return e_;
      kern<<<leaf.nodes, kBT, smem, st>>>(H->g, R, leaf.d_origin, o32.Sleaf.p, o32.Sleaf.ld, o32.Sleaf.str,
                                          ops.identity ? 1 : 0, staged, B.w32, B.g32, uo);
    }
    H->trace.end(kLeafDown, st);
  }
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

// FP64 leaf pass of mode A.mode.  A.flux_r (kResid) asks the even-odd kernel for the shared-edge
// flux jumps as well; flux_done tells whether it took them (else the caller runs k_b_jump).
int leaf64(hps_handle *H, Leaf64Args A, cudaStream_t st, bool *flux_done = nullptr) {
  if (flux_done) *flux_done = false;
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
    A.flux_r = nullptr;
    H->trace.begin(slot, st);
    k_b_pointwise<<<blocks(n), 256, 0, st>>>(n, A);
    H->trace.end(slot, st);
    return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
  }
  const int p = H->p, pp = p * p;
  const Level &leaf = H->lev[H->L];
  const int per_sm = H->batch.fp64_ctas_per_sm;
  const int grid = per_sm > 0 ? std::min(leaf.nodes, per_sm * H->num_sms) : leaf.nodes;
  if (p % 2 == 0 && H->batch.even_odd) {
    const int h = p / 2, m = H->m;
    int Rc = std::max(1, std::min(A.R, H->batch.eo_cols));
    auto eo_smem = [&](int rc) { return (size_t)(8 * h * h + 4 * h + pp * rc + 4 * m * h * rc) * sizeof(double); };
    while (Rc > 1 && eo_smem(Rc) > 227 * 1024) Rc = (Rc + 1) / 2;
    A.rc = Rc;
    const size_t smem = eo_smem(Rc);
    // constant coefficients: scales folded into the half matrices (not for a g that needs the
    // plain first derivatives)
    if (!nodal && A.mode != kEpilogue && !(A.mode == kEval && A.g_kind == HPS_G_BURGERS) && H->batch.fold_scale) {
      const double sc = A.mode == kResid ? A.gdt : A.dtL;
      A.fold = 1;
      A.s1x = sc * H->cst[2];
      A.s1y = sc * H->cst[3];
      A.s2x = sc * H->cst[0];
      A.s2y = sc * H->cst[1];
      A.s0 = sc * H->cst[4];
      A.has_s0 = A.s0 != 0.0;
    }
    const bool flux = A.flux_r && A.mode == kResid && H->batch.fuse_jump;
    if (flux) {
      const GridDims &g = H->g;
      if (cudaMemsetAsync(A.flux_r + g.N_int * A.R, 0, (size_t)(g.N - g.N_int) * A.R * sizeof(double), st) !=
          cudaSuccess)
        return HPS_ECUDA;
      if (flux_done) *flux_done = true;
    } else {
      A.flux_r = nullptr;
    }
    if (int e_ = smem_optin((const void *)k_b_leaf64_eo, smem)) return e_;
    H->trace.begin(slot, st);
    // (every loop of the kernel strides by blockDim: fewer threads per CTA, more CTAs per SM; with
    // one column a pass keeps at most (p/2 - 1)^2 threads busy, and 128-thread CTAs measured 24 %
    // faster than 256-thread ones on 128 x 128 leaves, p = 16, while with 4 or 32 columns 256 is best)
    const int eo_threads = H->batch.eo_threads > 0 ? H->batch.eo_threads : Rc == 1 ? 128 : kBT;
    k_b_leaf64_eo<<<grid, eo_threads, smem, st>>>(H->g, leaf.nodes, leaf.d_origin, A, H->d_D);
    H->trace.end(slot, st);
    return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
  }
  const int Rc = std::max(1, std::min(A.R, 4096 / pp));
  const size_t smem = (size_t)(4 * pp + pp * Rc) * sizeof(double);
  A.flux_r = nullptr;
  if (int e_ = smem_optin((const void *)k_b_leaf64, smem)) return e_;
  H->trace.begin(slot, st);
  k_b_leaf64<<<grid, kBT, smem, st>>>(H->g, leaf.nodes, leaf.d_origin, A, H->d_D);
  H->trace.end(slot, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Residual of the stage system for u (FP64) into B.r: interior rows (gdt = the operator's
// gamma dt; 0 for the identity) and shared-edge flux jumps.
int residual(hps_handle *H, BatchWork &B, int R, const double *u, const double *Rb, double gdt, cudaStream_t st) {
  Leaf64Args A = leaf64_args(H, kResid, R);
  A.u = u;
  A.Rb = Rb;
  A.out0 = B.r;
  A.gdt = gdt;
  A.flux_r = B.r;
  bool flux_done = false;
  if (int e = leaf64(H, A, st, &flux_done)) return e;
  const int64_t npts = ((int64_t)(H->g.n1 - 1) * H->g.n2 + (int64_t)(H->g.n2 - 1) * H->g.n1) * H->m;
  if (npts > 0 && !flux_done) {
    H->trace.begin(kJump, st);
    k_b_jump<<<blocks(npts * R), 256, 0, st>>>(H->g, R, u, B.r, H->d_D);
    H->trace.end(kJump, st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// J (or null): interface right-hand side, A_if u = J instead of 0 (added to each line's
// right-hand side in the tridiagonal kernel, after the two leaves' flux sums).
int edge_projection_impl(hps_handle *H, int R, const Combo &c, double *u, double *rhs, cudaStream_t st,
                         const double *J = nullptr) {
  const GridDims &g = H->g;
  const Level &leaf = H->lev[H->L];
  if (cudaMemsetAsync(rhs + g.N_int * R, 0, (size_t)(g.N - g.N_int) * R * sizeof(double), st) != cudaSuccess)
    return HPS_ECUDA;
  const size_t smem = (size_t)(4 * H->p + H->q * std::min(R, kCloseRc)) * sizeof(double);  // <= 116 KB (p <= 32)
  if (int e_ = smem_optin((const void *)k_b_close_leaf, smem)) return e_;
  H->trace.begin(kClose, st);
  k_b_close_leaf<<<leaf.nodes, kBT, smem, st>>>(g, leaf.d_origin, R, c, u, rhs, H->d_D);
  const int64_t nsys = ((int64_t)g.n2 * g.m + (int64_t)g.n1 * g.m) * R;
  k_b_edge_tridiag<<<blocks(nsys, 128), 128, 0, st>>>(g, R, rhs, u, H->d_proj, H->proj_lo[0], H->proj_up[0],
                                                       H->proj_lo[1], H->proj_up[1], J);
  H->trace.end(kClose, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Boundary data of one group: f is [N_bd][fld] with the group's columns from foff.
struct BdView {
  const double *f;
  int ld, off;
};

// Solve A u = [rhs (given by combination `c`, saved to Rsave if non-null); 0; f] with refinement.
// The last sweep writes the stage epilogue `ep` too where its leaf kernel can (epi_done).
// J (or null, [N][R] FP64): the interface rows' right-hand side (flux jump of u equal to J instead
// of 0), taken by the first sweep and added to the shared-edge rows of every residual.
int refined_solve(hps_handle *H, BatchWork &B, const OpSet &ops, const OpSet32 &o32, int R, const Combo &c,
                  double *Rsave, const double *Rb, BdView f, double *u, int refine, double gdt, cudaStream_t st,
                  const StageEpi &ep, bool &epi_done, const double *J = nullptr) {
  const StageEpi none{};
  epi_done = false;
  const GridDims &g = H->g;
  H->trace.begin(kSetBoundary, st);
  k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, B.g32, f.f, f.ld, f.off, u);
  H->trace.end(kSetBoundary, st);
  // the sweeps write their FP32 results straight into u (interior points from the leaf solve,
  // shared-edge points from the merges; the outer boundary is f, set above)
  // the first sweep may take the 3xTF32 tensor-core leaf apply (its rounding is slightly coarser
  // than FP32 and biased); corrections use the FP32 FMA path, so the refined result keeps FP32
  // times FP32 accuracy
  if (int e = sweep32(H, B, ops, o32, R, c, Rsave, J, UOut{u, 1}, true, st, refine == 0 ? ep : none,
                      epi_done))
    return e;
  for (int it = 0; it < refine; ++it) {
    if (int e = residual(H, B, R, u, Rb, gdt, st)) return e;
    if (J) {  // interface rows: J - (flux jump of u)
      const int64_t n0 = g.N_int * (int64_t)R, n1 = g.N * (int64_t)R;
      H->trace.begin(kJump, st);
      k_b_axpy<<<blocks(n1 - n0), 256, 0, st>>>(n1 - n0, 1.0, J + n0, B.r + n0);
      H->trace.end(kJump, st);
    }
    H->trace.begin(kSetBoundary, st);
    k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, B.g32, nullptr, 0, 0, nullptr);
    H->trace.end(kSetBoundary, st);
    Combo cr{};
    cr.n = 1;
    cr.ptr[0] = B.r;
    cr.coef[0] = 1.0;
    if (int e = sweep32(H, B, ops, o32, R, cr, nullptr, B.r, UOut{u, 0}, false, st, it == refine - 1 ? ep : none,
                        epi_done))
      return e;
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

void add_term_b(Combo &c, const double *p, double coef) {
  if (coef == 0.0) return;
  c.ptr[c.n] = p;
  c.coef[c.n] = coef;
  ++c.n;
}

// dst[i*ldd + offd + j] = src[i*lds + offs + j] for i < rows, j < cols (column subsets of
// RHS-fastest vectors)
__global__ void k_cols(const double *__restrict__ src, int lds, int offs, double *__restrict__ dst, int ldd,
                       int offd, int64_t rows, int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx / cols;
  const int j = (int)(idx % cols);
  dst[i * ldd + offd + j] = src[i * lds + offs + j];
}

// Columns of group gi for a call with R columns: [c0, c0 + n).  Groups take multiples of 4
// columns (the FP32 applies work on column quads), the last one the rest; n may be 0.
void group_cols(int R, int G, int gi, int &c0, int &n) {
  const int per = round4((R + G - 1) / G);
  c0 = std::min(R, gi * per);
  n = std::min(R, c0 + per) - c0;
}

// One ARK step of one group: u is [N][R] (the group's own buffer or the caller's), q / f are
// stage-major with leading dimensions qld / fld and the group's columns from qoff / foff.
int ark_group(hps_handle *H, BatchWork &B, int R, double *u, double dt, const hps_ark_terms *terms, int qld, int qoff,
              int fld, int foff, int refine, const ArkTable &tb, cudaStream_t st, cudaEvent_t after_first = nullptr) {
  const GridDims &g = H->g;
  const int64_t ni = g.N_int * R;
  const double *q = terms ? terms->q : nullptr;
  const double *f = terms ? terms->f : nullptr;
  const int64_t qstage = g.N_int * (int64_t)qld, fstage = g.N_bd * (int64_t)fld;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  const double gp0 = terms ? terms->g_param[0] : 0.0, gp1 = terms ? terms->g_param[1] : 0.0;
  // stage 1 (explicit): gamma dt L u^n, dt (q_1 + g(u^n)); the implicit terms are kept times
  // gamma (KL_j = gamma dt L U_j) and their coefficients divided by it
  const double gam = tb.A[1][1];
  Leaf64Args E = leaf64_args(H, kEval, R);
  E.u = u;
  E.out0 = B.KL;
  E.out1 = B.KE;
  E.q = q;
  E.qld = qld;
  E.qoff = qoff;
  E.dt = dt;
  E.dtL = gam * dt;
  E.g_kind = gk;
  E.gp0 = gp0;
  E.gp1 = gp1;
  if (int e = leaf64(H, E, st)) return e;
  if (after_first) cudaEventRecord(after_first, st);
  bool sa_close = H->batch.sa_close;
  for (int j = 0; j < 6; ++j) sa_close = sa_close && tb.A[5][j] == tb.b[j];
  for (int i = 1; i < 6; ++i) {
    Combo c{};
    add_term_b(c, u, 1.0);
    for (int j = 0; j < i; ++j) {
      add_term_b(c, B.KL + j * ni, tb.A[i][j] / gam);
      add_term_b(c, B.KE + j * ni, tb.Ah[i][j]);
    }
    const BdView fv{f ? f + i * fstage : nullptr, fld, foff};
    const double *qi = q ? q + i * qstage : nullptr;
    // a pointwise g lets the last leaf kernel of the solve write the epilogue
    const bool fuse = H->batch.fuse_epilogue && gk != HPS_G_BURGERS;
    // the last stage's dt L U_6 is not needed by a stiffly accurate close
    double *kl = sa_close && i == 5 ? nullptr : B.KL + i * ni;
    const StageEpi ep{fuse ? 1 : 0, B.Rb, kl, B.KE + i * ni, qi, qld, qoff, gk, dt, dt * gp0};
    bool done = false;
    if (int e = refined_solve(H, B, H->impl, H->batch.impl32, R, c, B.Rb, B.Rb, fv, B.ustage, refine, H->gamma_dt,
                              st, ep, done))
      return e;
    if (done) continue;
    Leaf64Args P = leaf64_args(H, kEpilogue, R);
    P.u = B.ustage;
    P.Rb = B.Rb;
    P.out0 = B.KL + i * ni;
    P.out1 = B.KE + i * ni;
    P.q = qi;
    P.qld = qld;
    P.qoff = qoff;
    P.dt = dt;
    P.g_kind = gk;
    P.gp0 = gp0;
    P.gp1 = gp1;
    if (int e = leaf64(H, P, st)) return e;
  }
  // step close: ARK combination at interior points, shared-edge values from the identity
  // operator solve (refined against its residual: interior R - u and the flux jumps)
  Combo c{};
  if (sa_close) {
    // stiffly accurate implicit table (b = last row of A) and dt L U_6 taken from the stage
    // equation: u + sum_j b_j dt L U_j = U_6 - sum_j Ah_6j dt (q_j + g(U_j)), so the close needs
    // U_6 and the explicit terms only
    add_term_b(c, B.ustage, 1.0);
    for (int j = 0; j < 6; ++j) add_term_b(c, B.KE + j * ni, tb.b[j] - tb.Ah[5][j]);
  } else {
    add_term_b(c, u, 1.0);
    for (int j = 0; j < 6; ++j) {
      add_term_b(c, B.KL + j * ni, tb.b[j] / gam);
      add_term_b(c, B.KE + j * ni, tb.b[j]);
    }
  }
  const BdView fv{f ? f + 5 * fstage : nullptr, fld, foff};
  if (H->batch.edge_projection && H->d_proj) {
    H->trace.begin(kSetBoundary, st);
    k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, B.g32, fv.f, fv.ld, fv.off, u);
    H->trace.end(kSetBoundary, st);
    return edge_projection_impl(H, R, c, u, B.r, st);
  }
  bool done = false;
  return refined_solve(H, B, H->ident, H->batch.ident32, R, c, B.Rb, B.Rb, fv, u, refine, 0.0, st, StageEpi{}, done);
}

// ---- many instances in lockstep: one launch per tree level and operator for all of them -------
// Instance state of a lockstep step: its handle, work buffers and stream, and the arguments of
// the sweep in progress (the leaf parts read them on the instance's stream, the grouped merges on
// the main stream).
struct LsInst {
  hps_handle *H;
  BatchWork *B;
  int R;
  double *u;
  const hps_ark_terms *terms;
  cudaStream_t st;
  cudaEvent_t ev;
  Combo rhs;
  double *Rsave;
  const double *jump;
  UOut uo;
  StageEpi ep, ep_cur;
  bool epi_done;
  bool sa_close;
};

// The merges of one sweep of every instance: level L_i - 1 - s of instance i at upward step s (w3
// for all, then h), level s at downward step s, each step one grouped launch per operator.
int merges_lockstep(std::vector<LsInst> &I, cudaStream_t st) {
  int maxL = 0;
  for (const LsInst &x : I) maxL = std::max(maxL, x.H->L);
  for (int s = 0; s < maxL; ++s) {
    std::vector<GroupItem<BXDiff, BEStore>> w3;
    std::vector<GroupItem<BXVec, BEFlux>> hh;
    for (LsInst &x : I) {
      const int l = x.H->L - 1 - s;
      if (l < 0) continue;
      hps_handle *H = x.H;
      BatchWork &B = *x.B;
      const Level &lv = H->lev[l];
      const OpSet32 &o32 = H->batch.impl32;
      w3.push_back({H, &B, kMergeUpW3, lv.n3, lv.n3, lv.nodes, x.R, o32.X[l].p, o32.X[l].ld, o32.X[l].str,
                    BXDiff{B.h32[l + 1], lv.nbc, lv.j3a, lv.j3b, x.R, x.jump, H->g, lv.d_origin, lv.a, lv.c, lv.split},
                    BEStore{B.w332[l], lv.n3, x.R}});
      if (l > 0)
        hh.push_back({H, &B, kMergeUpH, lv.nb, lv.n3, lv.nodes, x.R, o32.Tcat[l].p, o32.Tcat[l].ld, o32.Tcat[l].str,
                      BXVec{B.w332[l], lv.n3, x.R}, BEFlux{lv.d_hsrc, B.h32[l + 1], lv.nbc, lv.nb, x.R, B.h32[l]}});
    }
    if (int e = launch_group(w3, st)) return e;
    if (int e = launch_group(hh, st)) return e;
  }
  for (int s = 0; s < maxL; ++s) {
    std::vector<GroupItem<BXBd, BEScatter>> dn;
    for (LsInst &x : I) {
      if (s >= x.H->L) continue;
      hps_handle *H = x.H;
      BatchWork &B = *x.B;
      const Level &lv = H->lev[s];
      const OpSet32 &o32 = H->batch.impl32;
      dn.push_back({H, &B, kMergeDown, lv.n3, lv.nb, lv.nodes, x.R, o32.S[s].p, o32.S[s].ld, o32.S[s].str,
                    BXBd{H->g, lv.d_origin, lv.a, lv.c, x.R, B.g32},
                    BEScatter{H->g, lv.d_origin, lv.a, lv.c, lv.split, lv.n3, x.R, B.w332[s], B.g32, x.uo}});
    }
    if (int e = launch_group(dn, st)) return e;
  }
  return HPS_OK;
}

// One FP32 sweep of every instance: leaf parts on the instances' streams, merges grouped on `st`.
int sweep_lockstep(std::vector<LsInst> &I, bool allow_tc, cudaStream_t st, cudaEvent_t evm) {
  for (LsInst &x : I) {
    if (int e = sweep32(x.H, *x.B, x.H->impl, x.H->batch.impl32, x.R, x.rhs, x.Rsave, x.jump, x.uo, allow_tc, x.st,
                        x.ep_cur, x.epi_done, kSweepLeafUp))
      return e;
    if (cudaEventRecord(x.ev, x.st) != cudaSuccess || cudaStreamWaitEvent(st, x.ev, 0) != cudaSuccess) return HPS_ECUDA;
  }
  if (int e = merges_lockstep(I, st)) return e;
  if (cudaEventRecord(evm, st) != cudaSuccess) return HPS_ECUDA;
  for (LsInst &x : I) {
    if (cudaStreamWaitEvent(x.st, evm, 0) != cudaSuccess) return HPS_ECUDA;
    if (int e = sweep32(x.H, *x.B, x.H->impl, x.H->batch.impl32, x.R, x.rhs, x.Rsave, x.jump, x.uo, allow_tc, x.st,
                        x.ep_cur, x.epi_done, kSweepLeafDown))
      return e;
  }
  return HPS_OK;
}

// The batched ARK step (ark_group) of every instance in lockstep: the same stages and refinement
// sweeps, each sweep through sweep_lockstep; the explicit evaluations, residuals, epilogues and the
// close per instance on its own stream.
int ark_lockstep(std::vector<LsInst> &I, double dt, int refine, const ArkTable &tb, cudaStream_t st, cudaEvent_t evm) {
  const double gam = tb.A[1][1];
  const StageEpi none{};
  for (LsInst &x : I) {  // stage 1: gamma dt L u^n, dt (q_1 + g(u^n))
    const hps_ark_terms *t = x.terms;
    Leaf64Args E = leaf64_args(x.H, kEval, x.R);
    E.u = x.u;
    E.out0 = x.B->KL;
    E.out1 = x.B->KE;
    E.q = t ? t->q : nullptr;
    E.qld = x.R;
    E.qoff = 0;
    E.dt = dt;
    E.dtL = gam * dt;
    E.g_kind = t ? t->g_kind : HPS_G_NONE;
    E.gp0 = t ? t->g_param[0] : 0.0;
    E.gp1 = t ? t->g_param[1] : 0.0;
    if (int e = leaf64(x.H, E, x.st)) return e;
    x.sa_close = x.H->batch.sa_close;
    for (int j = 0; j < 6; ++j) x.sa_close = x.sa_close && tb.A[5][j] == tb.b[j];
  }
  for (int i = 1; i < 6; ++i) {
    for (LsInst &x : I) {  // the stage's right-hand side, boundary data, epilogue
      const hps_ark_terms *t = x.terms;
      BatchWork &B = *x.B;
      const int64_t ni = x.H->g.N_int * x.R;
      Combo c{};
      add_term_b(c, x.u, 1.0);
      for (int j = 0; j < i; ++j) {
        add_term_b(c, B.KL + j * ni, tb.A[i][j] / gam);
        add_term_b(c, B.KE + j * ni, tb.Ah[i][j]);
      }
      const int gk = t ? t->g_kind : HPS_G_NONE;
      const double *qi = t && t->q ? t->q + i * ni : nullptr;
      const bool fuse = x.H->batch.fuse_epilogue && gk != HPS_G_BURGERS;
      double *kl = x.sa_close && i == 5 ? nullptr : B.KL + i * ni;
      x.ep = StageEpi{fuse ? 1 : 0, B.Rb, kl, B.KE + i * ni, qi, x.R, 0, gk, dt, dt * (t ? t->g_param[0] : 0.0)};
      const GridDims &g = x.H->g;
      const double *fi = t && t->f ? t->f + i * g.N_bd * (int64_t)x.R : nullptr;
      k_b_set_boundary32<<<blocks(g.N_bd * x.R), 256, 0, x.st>>>(g, x.R, B.g32, fi, x.R, 0, B.ustage);
      x.rhs = c;
      x.Rsave = B.Rb;
      x.jump = nullptr;
      x.uo = UOut{B.ustage, 1};
      x.ep_cur = refine == 0 ? x.ep : none;
      x.epi_done = false;
    }
    if (int e = sweep_lockstep(I, true, st, evm)) return e;
    for (int it = 0; it < refine; ++it) {
      for (LsInst &x : I) {  // the residual of the stage system, the correction's right-hand side
        BatchWork &B = *x.B;
        if (int e = residual(x.H, B, x.R, B.ustage, B.Rb, x.H->gamma_dt, x.st)) return e;
        k_b_set_boundary32<<<blocks(x.H->g.N_bd * x.R), 256, 0, x.st>>>(x.H->g, x.R, B.g32, nullptr, 0, 0, nullptr);
        Combo cr{};
        cr.n = 1;
        cr.ptr[0] = B.r;
        cr.coef[0] = 1.0;
        x.rhs = cr;
        x.Rsave = nullptr;
        x.jump = B.r;
        x.uo = UOut{B.ustage, 0};
        x.ep_cur = it == refine - 1 ? x.ep : none;
      }
      if (int e = sweep_lockstep(I, false, st, evm)) return e;
    }
    for (LsInst &x : I) {  // the stage epilogue where the last leaf kernel could not write it
      if (x.epi_done) continue;
      const hps_ark_terms *t = x.terms;
      BatchWork &B = *x.B;
      const int64_t ni = x.H->g.N_int * x.R;
      Leaf64Args P = leaf64_args(x.H, kEpilogue, x.R);
      P.u = B.ustage;
      P.Rb = B.Rb;
      P.out0 = B.KL + i * ni;
      P.out1 = B.KE + i * ni;
      P.q = t && t->q ? t->q + i * ni : nullptr;
      P.qld = x.R;
      P.qoff = 0;
      P.dt = dt;
      P.g_kind = t ? t->g_kind : HPS_G_NONE;
      P.gp0 = t ? t->g_param[0] : 0.0;
      P.gp1 = t ? t->g_param[1] : 0.0;
      if (int e = leaf64(x.H, P, x.st)) return e;
    }
  }
  for (LsInst &x : I) {  // the step close of each instance
    const hps_ark_terms *t = x.terms;
    BatchWork &B = *x.B;
    const int64_t ni = x.H->g.N_int * x.R;
    Combo c{};
    if (x.sa_close) {
      add_term_b(c, B.ustage, 1.0);
      for (int j = 0; j < 6; ++j) add_term_b(c, B.KE + j * ni, tb.b[j] - tb.Ah[5][j]);
    } else {
      add_term_b(c, x.u, 1.0);
      for (int j = 0; j < 6; ++j) {
        add_term_b(c, B.KL + j * ni, tb.b[j] / gam);
        add_term_b(c, B.KE + j * ni, tb.b[j]);
      }
    }
    const GridDims &g = x.H->g;
    const BdView fv{t && t->f ? t->f + 5 * g.N_bd * (int64_t)x.R : nullptr, x.R, 0};
    if (x.H->batch.edge_projection && x.H->d_proj) {
      k_b_set_boundary32<<<blocks(g.N_bd * x.R), 256, 0, x.st>>>(g, x.R, B.g32, fv.f, fv.ld, fv.off, x.u);
      if (int e = edge_projection_impl(x.H, x.R, c, x.u, B.r, x.st)) return e;
    } else {
      bool done = false;
      if (int e = refined_solve(x.H, B, x.H->ident, x.H->batch.ident32, x.R, c, B.Rb, B.Rb, fv, x.u, refine, 0.0,
                                x.st, StageEpi{}, done))
        return e;
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// One ARK step in slope form (Sec. 3.1, eq. slope0, g = 0) of one group, mixed precision: the
// slopes times dt, kappa_j = dt k_j ([N][R] each, in W.slope), solve
//   kappa_1 = dt L u^n + dt q_1                                     (explicit; edges: identity system)
//   (I - gamma dt L) kappa_i = dt L u^n + sum_{j<i} a_ij dt L kappa_j + dt q_i,   i = 2..6
// by FP32 sweeps with `refine` FP64 refinement sweeps each, and u^{n+1} = u^n + sum_j b_j kappa_j
// at every point.  Every slope system's interface rows carry J = -(flux jump of u^n) (the
// penalization of Sec. 3.1).  Implicit terms are kept times gamma (KL_0 = gamma dt L u^n, KL_j =
// gamma dt L kappa_j) with their coefficients divided by it, as in ark_group.  Slope boundary data:
// dt times the caller's u_t values (f, [6][N_bd][fld] from foff), else 0.  With a preset g
// (eq. slope, time-independent boundary data: f must be null) the explicit slopes lambda_j = dt
// g(U_j) join them as complete fields (interior g, shared edges from the identity-operator
// system, zero boundary; W.slope_g), U_i = u^n + sum_{j<=i} a_ij kappa_j + sum_{j<i} ahat_ij
// lambda_j, their gamma dt L lambda_j enter every slope system with ahat_ij / gamma, and
// u^{n+1} = u^n + sum_j b_j (kappa_j + lambda_j).
// (q enters the stage combinations, whose terms are [N_int][R] vectors: qld = R, qoff = 0)
int slope_group(hps_handle *H, BatchWork &W, int R, double *u, double dt, const hps_ark_terms *terms, int qld,
                int qoff, int fld, int foff, int refine, const ArkTable &tb, cudaStream_t st) {
  if (qld != R || qoff != 0) return HPS_EINVAL;
  const GridDims &g = H->g;
  const int64_t N = g.N, ni = g.N_int * R, nR = N * R;
  const double *q = terms ? terms->q : nullptr;
  const double *f = terms ? terms->f : nullptr;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  const double gp0 = terms ? terms->g_param[0] : 0.0, gp1 = terms ? terms->g_param[1] : 0.0;
  if (gk != HPS_G_NONE && (f || !W.slope_g)) return HPS_EINVAL;
  double *lam = W.slope_g, *Ust = lam ? lam + 6 * nR : nullptr, *dLl = Ust ? Ust + nR : nullptr;
  const int64_t qstage = g.N_int * (int64_t)qld, fstage = g.N_bd * (int64_t)fld;
  const double gam = tb.A[1][1];
  double *kap = W.slope, *J = W.slope + 6 * nR, *fs = J + nR;
  // interface right-hand side of every slope system: -(flux jump of u^n) (zero elsewhere)
  if (cudaMemsetAsync(J, 0, nR * sizeof(double), st) != cudaSuccess) return HPS_ECUDA;
  if (int e = flux_jump_rhs(H, R, u, J, st)) return e;
  // gamma dt L u^n (KL_0) and dt L kappa_1 (KL_1) by leaf-local differentiation; dt q into KE
  auto eval = [&](const double *v, double *kl) -> int {
    Leaf64Args E = leaf64_args(H, kEval, R);
    E.u = v;
    E.out0 = kl;
    E.out1 = W.KE;  // (not used)
    E.dt = dt;
    E.dtL = gam * dt;
    E.g_kind = HPS_G_NONE;
    return leaf64(H, E, st);
  };
  auto bd = [&](int i) -> BdView {  // dt u_t(t + c_i dt) on the boundary, or 0
    if (!f) return BdView{nullptr, 0, 0};
    H->trace.begin(kSetBoundary, st);
    k_b_scale_bd<<<blocks(g.N_bd * R), 256, 0, st>>>(g.N_bd, R, dt, f + i * fstage, fld, foff, fs);
    H->trace.end(kSetBoundary, st);
    return BdView{fs, R, 0};
  };
  // lambda_i = dt g(v): interior by the leaf evaluation, zero boundary, shared edges from the
  // identity-operator system; gamma dt L lambda_i into dLl_i
  auto explicit_slope = [&](const double *v, int i) -> int {
    double *li = lam + i * nR, *scr = W.KE + ni;
    Leaf64Args E = leaf64_args(H, kEval, R);
    E.u = v;
    E.out0 = W.KE;  // (gamma dt L v: not used)
    E.out1 = li;    // dt g(v) at the interior points
    E.dt = dt;
    E.dtL = gam * dt;
    E.g_kind = gk;
    E.gp0 = gp0;
    E.gp1 = gp1;
    if (int e = leaf64(H, E, st)) return e;
    H->trace.begin(kSetBoundary, st);
    k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, W.g32, nullptr, 0, 0, li);
    H->trace.end(kSetBoundary, st);
    if (cudaMemcpyAsync(scr, li, ni * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) return HPS_ECUDA;
    Combo c{};
    add_term_b(c, scr, 1.0);
    if (int e = edge_projection_impl(H, R, c, li, W.r, st, nullptr)) return e;
    return eval(li, dLl + i * ni);
  };
  if (int e = eval(u, W.KL)) return e;
  {  // kappa_1: interior dt (L u^n + q_1), boundary dt u_t, shared edges by the edge projection with J
    const BdView fv = bd(0);
    H->trace.begin(kSetBoundary, st);
    k_b_set_boundary32<<<blocks(g.N_bd * R), 256, 0, st>>>(g, R, W.g32, fv.f, fv.ld, fv.off, kap);
    H->trace.end(kSetBoundary, st);
    Combo c{};
    add_term_b(c, W.KL, 1.0 / gam);
    if (q) add_term_b(c, q, dt);
    if (int e = edge_projection_impl(H, R, c, kap, W.r, st, J)) return e;
    if (int e = eval(kap, W.KL + ni)) return e;
  }
  if (gk != HPS_G_NONE)
    if (int e = explicit_slope(u, 0)) return e;
  for (int i = 1; i < 6; ++i) {
    double *ki = kap + i * nR;
    Combo c{};
    add_term_b(c, W.KL, 1.0 / gam);
    if (q) add_term_b(c, q + i * qstage, dt);
    for (int j = 0; j < i; ++j) add_term_b(c, W.KL + (j + 1) * ni, tb.A[i][j] / gam);
    if (gk != HPS_G_NONE)
      for (int j = 0; j < i; ++j) add_term_b(c, dLl + j * ni, tb.Ah[i][j] / gam);
    // the epilogue keeps gamma dt L kappa_i = kappa_i - R_i (the last one is not needed)
    double *kl = i < 5 ? W.KL + (i + 1) * ni : nullptr;
    const StageEpi ep{H->batch.fuse_epilogue ? 1 : 0, W.Rb, kl, W.KE, nullptr, R, 0, HPS_G_NONE, dt, 0.0};
    bool done = false;
    if (int e = refined_solve(H, W, H->impl, H->batch.impl32, R, c, W.Rb, W.Rb, bd(i), ki, refine, H->gamma_dt, st,
                              ep, done, J))
      return e;
    if (!done && kl) {
      Leaf64Args P = leaf64_args(H, kEpilogue, R);
      P.u = ki;
      P.Rb = W.Rb;
      P.out0 = kl;
      P.out1 = W.KE;
      P.dt = dt;
      P.g_kind = HPS_G_NONE;
      if (int e = leaf64(H, P, st)) return e;
    }
    if (gk != HPS_G_NONE) {  // U_i at every point, then lambda_i
      Combo cu{};
      add_term_b(cu, u, 1.0);
      for (int j = 0; j <= i; ++j) add_term_b(cu, kap + j * nR, tb.A[i][j]);
      for (int j = 0; j < i; ++j) add_term_b(cu, lam + j * nR, tb.Ah[i][j]);
      H->trace.begin(kFinish, st);
      k_b_combine_all<<<blocks(nR), 256, 0, st>>>(nR, cu, Ust);
      H->trace.end(kFinish, st);
      if (int e = explicit_slope(Ust, i)) return e;
    }
  }
  // u^{n+1} = u^n + sum_j b_j (kappa_j + lambda_j) at every point (bhat = b for this tableau)
  Combo c{};
  add_term_b(c, u, 1.0);
  for (int j = 0; j < 6; ++j) add_term_b(c, kap + j * nR, tb.b[j]);
  if (gk != HPS_G_NONE)
    for (int j = 0; j < 6; ++j) add_term_b(c, lam + j * nR, tb.b[j]);
  H->trace.begin(kFinish, st);
  k_b_combine_all<<<blocks(nR), 256, 0, st>>>(nR, c, u);
  H->trace.end(kFinish, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Run `body(group, c0, n, stream)` for every non-empty group: inline on `st` with one group,
// else forked onto the groups' streams and joined back into `st` (capturable).
template <class F>
int for_groups(hps_handle *H, int R, cudaStream_t st, F body) {
  Batch &Bt = H->batch;
  if (Bt.groups == 1) return body(Bt.work[0], 0, R, st);
  if (cudaEventRecord(Bt.fork, st) != cudaSuccess) return HPS_ECUDA;
  int err = HPS_OK;
  for (int gi = 0; gi < Bt.groups; ++gi) {
    int c0, n;
    group_cols(R, Bt.groups, gi, c0, n);
    if (n == 0) continue;
    BatchWork &W = Bt.work[gi];
    cudaStreamWaitEvent(W.stream, Bt.fork, 0);
    if (err == HPS_OK) err = body(W, c0, n, W.stream);
    cudaEventRecord(W.done, W.stream);
    cudaStreamWaitEvent(st, W.done, 0);
  }
  if (err == HPS_OK && cudaPeekAtLastError() != cudaSuccess) err = HPS_ECUDA;
  return err;
}

}  // namespace

void batch_release(hps_handle *H) {
  Batch &Bt = H->batch;
  for (BatchWork &W : Bt.work) {
    if (W.stream) cudaStreamDestroy(W.stream);
    if (W.done) cudaEventDestroy(W.done);
    if (W.first) cudaEventDestroy(W.first);
    W.stream = nullptr;
    W.done = nullptr;
    W.first = nullptr;
  }
  if (Bt.fork) cudaEventDestroy(Bt.fork);
  Bt.fork = nullptr;
}

int edge_projection(hps_handle *H, int R, const Combo &c, double *u, double *rhs, cudaStream_t st, const double *J) {
  return edge_projection_impl(H, R, c, u, rhs, st, J);
}

int flux_jump_rhs(hps_handle *H, int R, const double *u, double *r, cudaStream_t st) {
  const int64_t npts = ((int64_t)(H->g.n1 - 1) * H->g.n2 + (int64_t)(H->g.n2 - 1) * H->g.n1) * H->m;
  if (npts == 0) return HPS_OK;
  H->trace.begin(kJump, st);
  k_b_jump<<<blocks(npts * R), 256, 0, st>>>(H->g, R, u, r, H->d_D);
  H->trace.end(kJump, st);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

int batch_reserve(hps_handle *H, int R, int groups) {
  Batch &Bt = H->batch;
  if (R <= 0 || R > 64 || groups < 1 || groups > 8) return HPS_EINVAL;
  if (R <= Bt.Rmax && groups == Bt.groups) return HPS_OK;
  cudaDeviceSynchronize();
  if (Bt.impl32.X.empty()) {  // FP32 operator copies (once)
    if (int e = convert_opset(H, H->impl, Bt.impl32, H->shared)) return e;
    if (int e = convert_opset(H, H->ident, Bt.ident32, true)) return e;
    const int q = H->q, MT = (q + 15) / 16, KT = (q + 7) / 8;
    if (H->shared && MT <= kTcMaxMT && Bt.impl32.Ainv.p) {  // TF32 hi / lo fragments of the leaf operator
      const size_t n = (size_t)MT * KT * 128;
      if (cudaMalloc(&Bt.afrag_hi, n * sizeof(unsigned)) != cudaSuccess ||
          cudaMalloc(&Bt.afrag_lo, n * sizeof(unsigned)) != cudaSuccess)
        return HPS_ENOMEM;
      H->allocs.push_back(Bt.afrag_hi);
      H->allocs.push_back(Bt.afrag_lo);
      k_frag_a<<<blocks((int64_t)n), 256>>>(Bt.impl32.Ainv.p, Bt.impl32.Ainv.ld, q, MT, KT, Bt.afrag_hi, Bt.afrag_lo);
    }
    if (!H->shared && H->impl.Ainv && H->impl.strA && q >= 32 && q <= 256 && umma_smem_bytes(H->p, 16) <= 232448) {
      // TF32 hi / lo split of the per-node leaf operators, K-major, and its tensor map (tensor-core leaf apply)
      const int64_t nops = H->lev[H->L].nodes;
      Bt.ainv_ldk = round4(q);
      if (cudaMalloc(&Bt.ainv_k, 2 * (size_t)nops * q * Bt.ainv_ldk * sizeof(float)) != cudaSuccess)
        return HPS_ENOMEM;
      H->allocs.push_back(Bt.ainv_k);
      k_kmajor_split<<<4 * H->num_sms, 256>>>(H->impl.Ainv, H->impl.ldA, H->impl.strA, q, nops, Bt.ainv_k,
                                              Bt.ainv_ldk);
      if (int e = umma_map(H)) return e;
    }
  }
  // (re)allocate the work vectors; old ones stay in the handle's list until hps_free
  const GridDims &g = H->g;
  auto da = [&](auto **ptr, size_t n) -> int {
    if (cudaMalloc((void **)ptr, std::max<size_t>(n, 1) * sizeof(**ptr)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(*ptr);
    return HPS_OK;
  };
  batch_release(H);
  Bt.work.assign(groups, BatchWork{});
  Bt.groups = groups;
  Bt.Rmax = 0;
  if (groups > 1 && cudaEventCreateWithFlags(&Bt.fork, cudaEventDisableTiming) != cudaSuccess) return HPS_ECUDA;
  for (int gi = 0; gi < groups; ++gi) {
    int c0, Rg;
    group_cols(R, groups, gi, c0, Rg);
    BatchWork &W = Bt.work[gi];
    if (Rg == 0) continue;
    if (groups > 1) {
      if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&W.done, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&W.first, cudaEventDisableTiming) != cudaSuccess)
        return HPS_ECUDA;
      if (da(&W.u, (size_t)g.N * Rg)) return HPS_ENOMEM;
    }
    if (da(&W.ustage, (size_t)g.N * Rg) || da(&W.Rb, (size_t)g.N_int * Rg) || da(&W.KL, 6 * (size_t)g.N_int * Rg) ||
        da(&W.KE, 6 * (size_t)g.N_int * Rg) || da(&W.r, (size_t)g.N * Rg) || da(&W.g32, (size_t)g.N * Rg) ||
        da(&W.w32, (size_t)g.N_int * Rg) || da(&W.r32, (size_t)g.N_int * Rg))
      return HPS_ENOMEM;
    W.h32.assign(H->L + 1, nullptr);
    W.w332.assign(H->L, nullptr);
    for (int l = 0; l <= H->L; ++l) {
      const Level &lv = H->lev[l];
      if (da(&W.h32[l], (size_t)lv.nodes * lv.nb * Rg)) return HPS_ENOMEM;
      if (l < H->L && da(&W.w332[l], (size_t)lv.nodes * lv.n3 * Rg)) return HPS_ENOMEM;
    }
    W.tile_count_len = 65536;
    if (da(&W.tile_count, W.tile_count_len)) return HPS_ENOMEM;
    cudaMemset(W.tile_count, 0, W.tile_count_len * sizeof(unsigned));
    W.flow_len = 1;
    for (const Level &lv : H->lev) W.flow_len += lv.nodes;
    if (da(&W.flow_sync, W.flow_len)) return HPS_ENOMEM;
    W.partial_len = partial_floats(H, Rg);
    if (da(&W.partial32, std::max<size_t>(1, W.partial_len))) return HPS_ENOMEM;
    cudaMemset(W.r, 0, (size_t)g.N * Rg * sizeof(double));
    W.Rmax = Rg;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return HPS_ECUDA;
  Bt.Rmax = R;
  return HPS_OK;
}

int batch_option(hps_handle *H, int opt, const int *set, int *get) {
  Batch &Bt = H->batch;
  int *field = nullptr;
  bool *flag = nullptr;
  switch (opt) {
    case HPS_OPT_TENSOR_LEAF: flag = &Bt.tensor_leaf; break;
    case HPS_OPT_UMMA_LEAF: field = &Bt.umma_leaf; break;
    case HPS_OPT_ONE_COLUMN_MERGE: flag = &Bt.one_column_merge; break;
    case HPS_OPT_ONE_COLUMN_SUM: flag = &Bt.one_column_merge_sum; break;
    case HPS_OPT_STREAM_LEAF: field = &Bt.stream_leaf; break;
    case HPS_OPT_STREAM_CHUNK_KB: field = &Bt.stream_chunk_kb; break;
    case HPS_OPT_SUB_LEVELS: field = &Bt.sub_levels; break;
    case HPS_OPT_PDL: flag = &Bt.pdl; break;
    case HPS_OPT_EO_THREADS: field = &Bt.eo_threads; break;
    case HPS_OPT_PREFETCH_NEXT: flag = &Bt.prefetch_next; break;
    case HPS_OPT_B1_ROLL: flag = &Bt.b1_roll; break;
    case HPS_OPT_STREAM_PREFETCH: flag = &Bt.stream_prefetch; break;
    case HPS_OPT_B1_KW: field = &Bt.b1_kw; break;
    case HPS_OPT_EVEN_ODD: flag = &Bt.even_odd; break;
    case HPS_OPT_FLOW_LEVELS: field = &Bt.flow_levels; break;
    case HPS_OPT_FLOW_N3_MAX: field = &Bt.flow_n3_max; break;
    case HPS_OPT_CLUSTER_SPLITK: flag = &Bt.gemv2; break;
    case HPS_OPT_PLAN_TARGET: field = &Bt.plan_target; break;
    case HPS_OPT_PLAN_KMIN: field = &Bt.plan_kmin; break;
    case HPS_OPT_PLAN_NPC_MAX: field = &Bt.plan_npc_max; break;
    case HPS_OPT_SPLIT_RHS: flag = &Bt.leaf_split; break;
    case HPS_OPT_FP64_CTAS_PER_SM: field = &Bt.fp64_ctas_per_sm; break;
    case HPS_OPT_GROUP_OFFSET: flag = &Bt.offset_groups; break;
    case HPS_OPT_LAST_CTA_SUM: field = &Bt.last_cta_max_split; break;
    case HPS_OPT_FAST_DIAG: flag = &Bt.fast_diag; break;
    case HPS_OPT_PLAN_TILE_COLS: field = &Bt.plan_tile_cols; break;
    case HPS_OPT_FUSE_EPILOGUE: flag = &Bt.fuse_epilogue; break;
    case HPS_OPT_FUSE_JUMP: flag = &Bt.fuse_jump; break;
    case HPS_OPT_FOLD_SCALE: flag = &Bt.fold_scale; break;
    case HPS_OPT_SA_CLOSE: flag = &Bt.sa_close; break;
    case HPS_OPT_EDGE_PROJECTION: flag = &Bt.edge_projection; break;
    case HPS_OPT_EO_COLS: field = &Bt.eo_cols; break;
    case HPS_OPT_TILE_COLS_W3: field = &Bt.tile_cols_apply[0]; break;
    case HPS_OPT_TILE_COLS_H: field = &Bt.tile_cols_apply[1]; break;
    case HPS_OPT_TILE_COLS_DOWN: field = &Bt.tile_cols_apply[2]; break;
    case HPS_OPT_FP64_PLAN_TARGET: field = &H->fp64_plan_target; break;
    default: return HPS_EINVAL;
  }
  if (get) *get = field ? *field : (*flag ? 1 : 0);
  if (!set) return HPS_OK;
  const int v = *set;
  const bool per_apply = opt == HPS_OPT_TILE_COLS_W3 || opt == HPS_OPT_TILE_COLS_H || opt == HPS_OPT_TILE_COLS_DOWN;
  const bool plan = opt == HPS_OPT_PLAN_TARGET || opt == HPS_OPT_PLAN_KMIN || opt == HPS_OPT_PLAN_NPC_MAX ||
                    opt == HPS_OPT_PLAN_TILE_COLS || per_apply;
  if (opt == HPS_OPT_PLAN_TILE_COLS && *set != 2 && *set != 4 && *set != 8) return HPS_EINVAL;
  if (per_apply && *set != 0 && *set != 2 && *set != 4 && *set != 8) return HPS_EINVAL;
  if (v < 0 || (plan && !per_apply && v < 1) || (opt == HPS_OPT_FLOW_LEVELS && v > kFlowMaxLevels)) return HPS_EINVAL;
  if (opt == HPS_OPT_EO_COLS && (v < 1 || v > 32)) return HPS_EINVAL;
  if (opt == HPS_OPT_UMMA_LEAF && v > 3) return HPS_EINVAL;
  if (opt == HPS_OPT_STREAM_LEAF && v > 4) return HPS_EINVAL;
  if (opt == HPS_OPT_STREAM_CHUNK_KB && (v < 2 || v > 64)) return HPS_EINVAL;
  if (opt == HPS_OPT_SUB_LEVELS && v > kSubMaxLevels) return HPS_EINVAL;
  if (opt == HPS_OPT_EO_THREADS && (v % 32 != 0 || v > kBT)) return HPS_EINVAL;
  if (opt == HPS_OPT_B1_KW && v != 1 && v != 2 && v != 4 && v != 8) return HPS_EINVAL;
  if (opt == HPS_OPT_UMMA_LEAF && v == 3)
    if (int e = umma_bf16_reserve(H)) return e;
  if (opt == HPS_OPT_FP64_PLAN_TARGET) {  // FP64 split plans: not while the persistent kernel holds tasks
    if (v < 1 || v > 8 || H->persistent) return HPS_EINVAL;
    H->fp64_plan_target = v;
    const size_t need = partial_doubles(H);
    if (need > H->partial_len) {
      cudaDeviceSynchronize();
      double *p = nullptr;
      if (cudaMalloc(&p, need * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
      H->allocs.push_back(p);
      H->partial = p;
      H->partial_len = need;
    }
    return HPS_OK;
  }
  if (field) *field = v;
  else *flag = v != 0;
  if (plan) {  // split-K scratch for the new plans
    cudaDeviceSynchronize();
    for (BatchWork &W : Bt.work) {
      if (W.Rmax == 0) continue;
      const size_t need = partial_floats(H, W.Rmax);
      if (need > W.partial_len) {
        float *p = nullptr;
        if (cudaMalloc(&p, need * sizeof(float)) != cudaSuccess) return HPS_ENOMEM;
        H->allocs.push_back(p);
        W.partial32 = p;
        W.partial_len = need;
      }
    }
  }
  return HPS_OK;
}

namespace {
__global__ void k_tune_fill(double *x, int64_t n) {  // deterministic right-hand side in [-0.1, 0.1]
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.1 * sin(0.37 * (double)(i % 100003) + 0.001 * (double)(i / 100003));
}
}  // namespace

int batch_autotune(hps_handle *H, int R, int refine, cudaStream_t st, hps_tune_result *res, int max_res, int *n_res) {
  Batch &Bt = H->batch;
  if (R <= 0 || R > Bt.Rmax || refine < 0 || refine > 8) return HPS_EINVAL;
  const GridDims &g = H->g;
  double *rhs = nullptr, *f = nullptr, *u = nullptr;
  auto cleanup = [&](int e) {
    cudaDeviceSynchronize();
    cudaFree(rhs);
    cudaFree(f);
    cudaFree(u);
    return e;
  };
  if (cudaMalloc(&rhs, (size_t)g.N_int * R * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&f, (size_t)g.N_bd * R * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&u, (size_t)g.N * R * sizeof(double)) != cudaSuccess)
    return cleanup(HPS_ENOMEM);
  k_tune_fill<<<blocks(g.N_int * R), 256, 0, st>>>(rhs, g.N_int * R);
  cudaMemsetAsync(f, 0, (size_t)g.N_bd * R * sizeof(double), st);
  struct Cand { int tile, flow, target, kmin; };
  std::vector<Cand> cands;
  for (int tile : {2, 8})
    for (int flow : {0, 3})
      for (const auto &tk : {std::pair<int, int>{2, 32}, std::pair<int, int>{4, 16}})
        cands.push_back({tile, flow, tk.first, tk.second});
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int nres = 0, ibest = -1;
  for (size_t i = 0; i < cands.size(); ++i) {
    const Cand &c = cands[i];
    const int vals[4] = {c.tile, c.flow, c.target, c.kmin};
    const int opts[4] = {HPS_OPT_PLAN_TILE_COLS, HPS_OPT_FLOW_LEVELS, HPS_OPT_PLAN_TARGET, HPS_OPT_PLAN_KMIN};
    int e = HPS_OK;
    for (int k = 0; k < 4 && e == HPS_OK; ++k) e = batch_option(H, opts[k], &vals[k], nullptr);
    for (int w = 0; w < 2 && e == HPS_OK; ++w) e = solve_batch(H, R, rhs, f, u, refine, st);
    cudaEventRecord(e0, st);
    for (int w = 0; w < 3 && e == HPS_OK; ++w) e = solve_batch(H, R, rhs, f, u, refine, st);
    cudaEventRecord(e1, st);
    if (e != HPS_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cleanup(e != HPS_OK ? e : HPS_ECUDA);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    if (res && nres < max_res) res[nres] = hps_tune_result{c.tile, c.flow, c.target, c.kmin, ms};
    if (res && nres < max_res) ++nres;
    if (ms < best) {
      best = ms;
      ibest = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const Cand &c = cands[ibest];
  const int vals[4] = {c.tile, c.flow, c.target, c.kmin};
  const int opts[4] = {HPS_OPT_PLAN_TILE_COLS, HPS_OPT_FLOW_LEVELS, HPS_OPT_PLAN_TARGET, HPS_OPT_PLAN_KMIN};
  for (int k = 0; k < 4; ++k) batch_option(H, opts[k], &vals[k], nullptr);
  if (n_res) *n_res = nres;
  return cleanup(HPS_OK);
}

int solve_batch(hps_handle *H, int R, const double *rhs, const double *f, double *u, int refine, cudaStream_t st) {
  if (R > H->batch.Rmax) return HPS_EINVAL;
  const GridDims &g = H->g;
  const bool grouped = H->batch.groups > 1;
  return for_groups(H, R, st, [&](BatchWork &W, int c0, int n, cudaStream_t s) -> int {
    const double *rb = rhs;
    double *uu = u;
    if (grouped) {  // the group's columns of rhs into its Rb buffer, u assembled in W.u
      H->trace.begin(kFinish, s);
      k_cols<<<blocks(g.N_int * n), 256, 0, s>>>(rhs, R, c0, W.Rb, n, 0, g.N_int, n);
      H->trace.end(kFinish, s);
      rb = W.Rb;
      uu = W.u;
    }
    Combo c{};
    add_term_b(c, rb, 1.0);
    bool done = false;
    if (int e = refined_solve(H, W, H->impl, H->batch.impl32, n, c, nullptr, rb, BdView{f, R, c0}, uu, refine,
                              H->gamma_dt, s, StageEpi{}, done))
      return e;
    if (grouped) {
      H->trace.begin(kFinish, s);
      k_cols<<<blocks(g.N * n), 256, 0, s>>>(W.u, n, 0, u, R, c0, g.N, n);
      H->trace.end(kFinish, s);
    }
    return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
  });
}

int ark_batch(hps_handle *H, int R, double *u, double dt, const hps_ark_terms *terms, int refine, const ArkTable &tb,
              cudaStream_t st) {
  if (R > H->batch.Rmax) return HPS_EINVAL;
  const GridDims &g = H->g;
  const bool grouped = H->batch.groups > 1;
  BatchWork *prev = nullptr;
  return for_groups(H, R, st, [&](BatchWork &W, int c0, int n, cudaStream_t s) -> int {
    double *uu = u;
    if (grouped) {
      // offset the groups by one phase: this group starts when the previous one has finished its
      // explicit first stage (FP64-bound), so FP64 and FP32 phases of different groups overlap
      if (prev && H->batch.offset_groups) cudaStreamWaitEvent(s, prev->first, 0);
      H->trace.begin(kFinish, s);
      k_cols<<<blocks(g.N * n), 256, 0, s>>>(u, R, c0, W.u, n, 0, g.N, n);
      H->trace.end(kFinish, s);
      uu = W.u;
    }
    if (int e = ark_group(H, W, n, uu, dt, terms, R, c0, R, c0, refine, tb, s, grouped ? W.first : nullptr)) return e;
    prev = &W;
    if (grouped) {
      H->trace.begin(kFinish, s);
      k_cols<<<blocks(g.N * n), 256, 0, s>>>(W.u, n, 0, u, R, c0, g.N, n);
      H->trace.end(kFinish, s);
    }
    return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
  });
}

// Many instances' batched ARK steps in lockstep (hps_multi with lockstep on): the instances'
// streams `sts` are forked from `st` by the caller and joined back by it; evs: one event per
// instance, evm: one for `st`.
int ark_batch_lockstep(hps_handle *const *h, int n, double *const *u, const int *R, const hps_ark_terms *terms,
                       double dt, int refine, const ArkTable &tb, cudaStream_t st, const cudaStream_t *sts,
                       const cudaEvent_t *evs, cudaEvent_t evm) {
  std::vector<LsInst> I(n);
  for (int i = 0; i < n; ++i) {
    hps_handle *H = h[i];
    if (R[i] > H->batch.Rmax || H->batch.groups != 1) return HPS_EINVAL;
    if (std::fabs(0.25 * dt - H->gamma_dt) > 1e-12 * H->gamma_dt) return HPS_EDT;
    const hps_ark_terms *t = terms ? &terms[i] : nullptr;
    if (t && (t->g_kind < HPS_G_NONE || t->g_kind > HPS_G_BURGERS)) return HPS_EINVAL;
    LsInst &x = I[i];
    x.H = H;
    x.B = &H->batch.work[0];
    x.R = R[i];
    x.u = u[i];
    x.terms = t;
    x.st = sts[i];
    x.ev = evs[i];
  }
  return ark_lockstep(I, dt, refine, tb, st, evm);
}

// Batched slope-form step (one column group; the first call allocates the slopes, 7 N + N_bd
// doubles per column).
int ark_slope_batch(hps_handle *H, int R, double *u, double dt, const hps_ark_terms *terms, int refine,
                    const ArkTable &tb, cudaStream_t st) {
  if (R > H->batch.Rmax || H->batch.groups != 1 || !H->d_proj) return HPS_EINVAL;
  BatchWork &W = H->batch.work[0];
  const size_t need = (7 * (size_t)H->g.N + (size_t)H->g.N_bd) * H->batch.Rmax;
  if (W.slope_len < need) {
    if (W.slope) return HPS_EINVAL;  // reserved for fewer columns: hps_batch_reserve frees and resets it
    if (cudaMalloc(&W.slope, need * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(W.slope);
    W.slope_len = need;
  }
  if (terms && terms->g_kind != HPS_G_NONE && !W.slope_g) {  // explicit slopes, a stage value, their L
    const size_t ng = (7 * (size_t)H->g.N + 6 * (size_t)H->g.N_int) * H->batch.Rmax;
    if (cudaMalloc(&W.slope_g, ng * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
    H->allocs.push_back(W.slope_g);
  }
  return slope_group(H, W, R, u, dt, terms, R, 0, R, 0, refine, tb, st);
}

}  // namespace hps

extern "C" int hps_selftest_conversions(int64_t n, uint64_t seed, hps_stream_t stream, int64_t *mismatches) {
  if (n < 1 || !mismatches) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *bad = nullptr;
  if (cudaMalloc(&bad, sizeof(unsigned long long)) != cudaSuccess) return HPS_ENOMEM;
  unsigned long long h = 0;
  int e = HPS_OK;
  if (cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st) != cudaSuccess) e = HPS_ECUDA;
  if (e == HPS_OK) {
    hps::k_conv_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, (unsigned long long)seed, bad);
    if (cudaPeekAtLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      e = HPS_ECUDA;
  }
  cudaFree(bad);
  *mismatches = (int64_t)h;
  return e;
}
