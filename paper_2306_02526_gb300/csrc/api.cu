// C ABI of libhps.so (include/hps.h): tree set-up, handle life cycle, hps_solve and ark_step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <unordered_map>

#include "hps_internal.cuh"

using hps::GridDims;
using hps::Level;
using hps::OpSet;

namespace {

bool is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

int check_tree(const hps_tree *t, int p) {
  if (!t) return HPS_EINVAL;
  if (!is_pow2(t->n1) || !is_pow2(t->n2) || (int64_t)t->n1 * t->n2 > 65536) return HPS_EINVAL;
  if (p < 4 || p > hps::kMaxP) return HPS_EINVAL;
  if (!(t->x1 > t->x0) || !(t->y1 > t->y0) || !std::isfinite(t->x1 - t->x0) || !std::isfinite(t->y1 - t->y0))
    return HPS_EINVAL;
  return HPS_OK;
}

GridDims dims(const hps_tree *t, int p) {
  GridDims g;
  g.n1 = t->n1;
  g.n2 = t->n2;
  g.p = p;
  g.m = p - 2;
  g.N_int = (int64_t)g.n1 * g.n2 * g.m * g.m;
  g.N_v = (int64_t)(g.n1 + 1) * g.n2 * g.m;
  g.N_h = (int64_t)(g.n2 + 1) * g.n1 * g.m;
  g.N = g.N_int + g.N_v + g.N_h;
  g.N_bd = 2LL * g.m * (g.n1 + g.n2);
  return g;
}

// Uniform binary tree (Sec. 2.1, boxes halved across the longer side; ties cut by a vertical line).
std::vector<Level> make_levels(const GridDims &g) {
  std::vector<Level> lev;
  Level root;
  root.nodes = 1;
  root.a = g.n1;
  root.c = g.n2;
  root.origin = {0, 0};
  lev.push_back(root);
  for (;;) {
    Level &cur = lev.back();
    cur.nb = 2 * (cur.a + cur.c) * g.m;
    if (cur.a == 1 && cur.c == 1) {
      cur.split = -1;
      break;
    }
    cur.split = cur.a >= cur.c ? 0 : 1;
    Level nxt;
    nxt.nodes = cur.nodes * 2;
    nxt.a = cur.split == 0 ? cur.a / 2 : cur.a;
    nxt.c = cur.split == 0 ? cur.c : cur.c / 2;
    nxt.origin.resize(2 * nxt.nodes);
    for (int k = 0; k < cur.nodes; ++k) {
      const int ix0 = cur.origin[2 * k], iy0 = cur.origin[2 * k + 1];
      nxt.origin[4 * k + 0] = ix0;
      nxt.origin[4 * k + 1] = iy0;
      nxt.origin[4 * k + 2] = cur.split == 0 ? ix0 + nxt.a : ix0;
      nxt.origin[4 * k + 3] = cur.split == 0 ? iy0 : iy0 + nxt.c;
    }
    cur.n3 = (cur.split == 0 ? cur.c : cur.a) * g.m;
    cur.nbc = 2 * (nxt.a + nxt.c) * g.m;
    lev.push_back(nxt);
  }
  // index maps of every merge level, from the boxes of node 0 (all nodes of a level are translates)
  for (size_t l = 0; l + 1 < lev.size(); ++l) {
    Level &cur = lev[l];
    const Level &ch = lev[l + 1];
    std::unordered_map<int64_t, int> pa, pb;
    for (int pos = 0; pos < cur.nbc; ++pos) {
      pa[hps::box_bd(g, ch.origin[0], ch.origin[1], ch.a, ch.c, pos)] = pos;
      pb[hps::box_bd(g, ch.origin[2], ch.origin[3], ch.a, ch.c, pos)] = pos;
    }
    cur.hsrc.resize(cur.nb);
    for (int pos = 0; pos < cur.nb; ++pos) {
      const int64_t gi = hps::box_bd(g, cur.origin[0], cur.origin[1], cur.a, cur.c, pos);
      auto ia = pa.find(gi);
      cur.hsrc[pos] = ia != pa.end() ? ia->second : cur.nbc + pb.at(gi);
    }
    const int64_t g0 = hps::iface_bd(g, cur.origin[0], cur.origin[1], cur.a, cur.c, cur.split, 0);
    cur.j3a = pa.at(g0);
    cur.j3b = pb.at(g0);
    for (int r = 0; r < cur.n3; ++r) {  // the interface is contiguous in both children
      const int64_t gi = hps::iface_bd(g, cur.origin[0], cur.origin[1], cur.a, cur.c, cur.split, r);
      if (pa.at(gi) != cur.j3a + r || pb.at(gi) != cur.j3b + r) throw std::bad_alloc();
    }
    // child boundary position -> parent boundary position, or nb + interface position
    cur.cmap.assign(2 * cur.nbc, -1);
    for (int pos = 0; pos < cur.nb; ++pos) cur.cmap[cur.hsrc[pos]] = pos;
    for (int r = 0; r < cur.n3; ++r) {
      cur.cmap[cur.j3a + r] = cur.nb + r;
      cur.cmap[cur.nbc + cur.j3b + r] = cur.nb + r;
    }
    for (int v : cur.cmap)
      if (v < 0) throw std::bad_alloc();
  }
  return lev;
}

// Chebyshev differentiation on ascending nodes xi_k = -cos(k pi/(p-1)): the closed form
// D_ij = (c_i/c_j)(-1)^{i+j}/(x_i - x_j), c_0 = c_N = 2, diagonal by the negative row sum.
std::vector<double> cheb_D(int p) {
  const int N = p - 1;
  std::vector<double> x(p), D((size_t)p * p, 0.0);
  for (int k = 0; k < p; ++k) x[k] = -std::cos(M_PI * k / N);
  for (int i = 0; i < p; ++i) {
    double s = 0.0;
    for (int j = 0; j < p; ++j) {
      if (i == j) continue;
      const double ci = (i == 0 || i == N) ? 2.0 : 1.0, cj = (j == 0 || j == N) ? 2.0 : 1.0;
      const double sg = ((i + j) % 2) ? -1.0 : 1.0;
      // x_i - x_j = 2 sin((i+j) pi/(2N)) sin((i-j) pi/(2N)) for ascending nodes
      const double dx = 2.0 * std::sin(M_PI * (i + j) / (2.0 * N)) * std::sin(M_PI * (i - j) / (2.0 * N));
      const double v = (ci / cj) * sg / dx;
      D[(size_t)i * p + j] = v;
      s += v;
    }
    D[(size_t)i * p + i] = -s;
  }
  return D;
}

template <class T>
int dalloc(hps_handle *H, T **ptr, size_t count) {
  if (cudaMalloc((void **)ptr, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(*ptr);
  return HPS_OK;
}

// D1x, D1y (Chebyshev differentiation scaled to leaves of width hx, hy), Dxx = D1x^2, Dyy = D1y^2
std::vector<double> scaled_D(int p, double hx, double hy) {
  const std::vector<double> D = cheb_D(p);
  std::vector<double> Dh((size_t)4 * p * p);
  const double sx = 2.0 / hx, sy = 2.0 / hy;
  for (int i = 0; i < p * p; ++i) {
    Dh[i] = sx * D[i];
    Dh[p * p + i] = sy * D[i];
  }
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      double sxx = 0.0, syy = 0.0;
      for (int k = 0; k < p; ++k) {
        sxx += Dh[i * p + k] * Dh[k * p + j];
        syy += Dh[p * p + i * p + k] * Dh[p * p + k * p + j];
      }
      Dh[2 * p * p + i * p + j] = sxx;
      Dh[3 * p * p + i * p + j] = syy;
    }
  return Dh;
}

size_t opset_bytes(const std::vector<Level> &lev, int q, int b, bool shared, bool identity) {
  auto pad = [](int n) { return (size_t)((n + 1) & ~1); };
  size_t s = 0;
  const int L = (int)lev.size() - 1;
  if (!identity) s += (shared ? 1 : lev[L].nodes) * (size_t)(q + b) * pad(q);
  for (int l = 0; l < L; ++l) {
    const size_t nops = shared ? 1 : lev[l].nodes;
    s += nops * ((size_t)lev[l].n3 * pad(lev[l].n3) + (size_t)lev[l].nb * pad(lev[l].n3) +
                 (l > 0 ? (size_t)lev[l].n3 * pad(lev[l].nb) : 0));
  }
  return s * sizeof(double);
}

size_t work_bytes(const GridDims &g, const std::vector<Level> &lev) {
  size_t s = (size_t)g.N + (size_t)g.N_int * (1 + 6 + 6 + 1);
  for (size_t l = 0; l < lev.size(); ++l) s += (size_t)lev[l].nodes * (lev[l].nb + lev[l].n3);
  return s * sizeof(double);
}

// ARK4(3)6L[2]SA (Table ``tbl:butcher``): implicit A (row 6 = b), explicit A-hat, b-hat = b.
struct Tableau {
  double A[6][6], Ah[6][6], b[6], c[6];
  Tableau() {
    std::memset(this, 0, sizeof(*this));
    c[0] = 0.0; c[1] = 1.0 / 2; c[2] = 83.0 / 250; c[3] = 31.0 / 50; c[4] = 17.0 / 20; c[5] = 1.0;
    b[0] = 82889.0 / 524892; b[1] = 0.0; b[2] = 15625.0 / 83664; b[3] = 69875.0 / 102672;
    b[4] = -2260.0 / 8211; b[5] = 1.0 / 4;
    A[1][0] = 1.0 / 4;
    A[2][0] = 8611.0 / 62500; A[2][1] = -1743.0 / 31250;
    A[3][0] = 5012029.0 / 34652500; A[3][1] = -654441.0 / 2922500; A[3][2] = 174375.0 / 388108;
    A[4][0] = 15267082809.0 / 155376265600; A[4][1] = -71443401.0 / 120774400;
    A[4][2] = 730878875.0 / 902184768; A[4][3] = 2285395.0 / 8070912;
    for (int j = 0; j < 6; ++j) A[5][j] = b[j];
    for (int i = 1; i < 6; ++i) A[i][i] = 1.0 / 4;
    Ah[1][0] = 1.0 / 2;
    Ah[2][0] = 13861.0 / 62500; Ah[2][1] = 6889.0 / 62500;
    Ah[3][0] = -116923316275.0 / 2393684061468; Ah[3][1] = -2731218467317.0 / 15368042101831;
    Ah[3][2] = 9408046702089.0 / 11113171139209;
    Ah[4][0] = -451086348788.0 / 2902428689909; Ah[4][1] = -2682348792572.0 / 7519795681897;
    Ah[4][2] = 12662868775082.0 / 11960479115383; Ah[4][3] = 3355817975965.0 / 11060851509271;
    Ah[5][0] = 647845179188.0 / 3216320057751; Ah[5][1] = 73281519250.0 / 8382639484533;
    Ah[5][2] = 552539513391.0 / 3454668386233; Ah[5][3] = 3354512671639.0 / 8306763924573;
    Ah[5][4] = 4040.0 / 17871;
  }
};

const Tableau &tableau() {
  static const Tableau t;
  return t;
}

void add_term(hps::Combo &c, const double *p, double coef) {
  if (coef == 0.0) return;
  c.ptr[c.n] = p;
  c.coef[c.n] = coef;
  ++c.n;
}

}  // namespace

extern "C" {

int hps_sizes(const hps_tree *tree, int p, int64_t *N, int64_t *N_int, int64_t *N_bd) {
  if (int e = check_tree(tree, p)) return e;
  const GridDims g = dims(tree, p);
  if (N) *N = g.N;
  if (N_int) *N_int = g.N_int;
  if (N_bd) *N_bd = g.N_bd;
  return HPS_OK;
}

int hps_coords(const hps_tree *tree, int p, double *x, double *y) {
  if (int e = check_tree(tree, p)) return e;
  if (!x || !y) return HPS_EINVAL;
  const GridDims g = dims(tree, p);
  const double hx = (tree->x1 - tree->x0) / g.n1, hy = (tree->y1 - tree->y0) / g.n2;
  std::vector<double> xi(p);
  for (int k = 0; k < p; ++k) xi[k] = -std::cos(M_PI * k / (p - 1));
  const int m = g.m;
  for (int iy = 0; iy < g.n2; ++iy)
    for (int ix = 0; ix < g.n1; ++ix) {
      const int64_t base = ((int64_t)iy * g.n1 + ix) * m * m;
      for (int j = 1; j <= m; ++j)
        for (int i = 1; i <= m; ++i) {
          x[base + (j - 1) * m + (i - 1)] = tree->x0 + hx * (ix + 0.5 * (1.0 + xi[i]));
          y[base + (j - 1) * m + (i - 1)] = tree->y0 + hy * (iy + 0.5 * (1.0 + xi[j]));
        }
    }
  for (int L = 0; L <= g.n1; ++L)
    for (int iy = 0; iy < g.n2; ++iy)
      for (int j = 1; j <= m; ++j) {
        const int64_t gi = hps::vseg(g, L, iy, j - 1);
        x[gi] = tree->x0 + hx * L;
        y[gi] = tree->y0 + hy * (iy + 0.5 * (1.0 + xi[j]));
      }
  for (int L = 0; L <= g.n2; ++L)
    for (int ix = 0; ix < g.n1; ++ix)
      for (int i = 1; i <= m; ++i) {
        const int64_t gi = hps::hseg(g, L, ix, i - 1);
        x[gi] = tree->x0 + hx * (ix + 0.5 * (1.0 + xi[i]));
        y[gi] = tree->y0 + hy * L;
      }
  return HPS_OK;
}

int hps_boundary_index(const hps_tree *tree, int p, int64_t *idx) {
  if (int e = check_tree(tree, p)) return e;
  if (!idx) return HPS_EINVAL;
  const GridDims g = dims(tree, p);
  int64_t k = 0;
  for (int L : {0, g.n1})
    for (int iy = 0; iy < g.n2; ++iy)
      for (int j = 0; j < g.m; ++j) idx[k++] = hps::vseg(g, L, iy, j);
  for (int L : {0, g.n2})
    for (int ix = 0; ix < g.n1; ++ix)
      for (int i = 0; i < g.m; ++i) idx[k++] = hps::hseg(g, L, ix, i);
  return HPS_OK;
}

size_t hps_bytes(const hps_tree *tree, int p, int coeff_kind, int flags) {
  if (check_tree(tree, p)) return 0;
  if (coeff_kind != HPS_COEF_CONST && coeff_kind != HPS_COEF_NODAL) return 0;
  const GridDims g = dims(tree, p);
  std::vector<Level> lev;
  try {
    lev = make_levels(g);
  } catch (...) {
    return 0;
  }
  const int q = g.m * g.m, b = 4 * g.m;
  const bool shared = coeff_kind == HPS_COEF_CONST && !(flags & HPS_FLAG_PER_NODE);
  size_t s = opset_bytes(lev, q, b, shared, false) + opset_bytes(lev, q, b, true, true) + work_bytes(g, lev);
  if (coeff_kind == HPS_COEF_NODAL) s += 5 * (size_t)g.N_int * sizeof(double);
  s += (4 * (size_t)p * p + 2 * (size_t)p * p) * sizeof(double);  // D matrices and their even-odd halves
  s += 2 * (size_t)(g.n1 - 1 + g.n2 - 1) * sizeof(double);         // edge-projection factors
  for (const Level &lv : lev) s += (2 * (size_t)lv.nodes + lv.hsrc.size() + lv.cmap.size()) * sizeof(int);
  return s;
}

void hps_free(hps_handle *H) {
  if (!H) return;
  cudaDeviceSynchronize();
  H->trace.release();
  H->g_ark.destroy();
  H->g_solve.destroy();
  H->g_ark_b.destroy();
  H->g_solve_b.destroy();
  if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
  hps::batch_release(H);
  for (void *p : H->allocs) cudaFree(p);
  delete H;
}

int hps_build(const hps_tree *tree, int p, const hps_coeffs *coeffs, double gamma_dt, int flags, hps_stream_t stream,
              hps_handle **out) {
  if (!out) return HPS_EINVAL;
  *out = nullptr;
  if (int e = check_tree(tree, p)) return e;
  if (!coeffs || (coeffs->kind != HPS_COEF_CONST && coeffs->kind != HPS_COEF_NODAL)) return HPS_EINVAL;
  if (coeffs->kind == HPS_COEF_NODAL &&
      (!coeffs->a11 || !coeffs->a22 || !coeffs->a1 || !coeffs->a2 || !coeffs->a0))
    return HPS_EINVAL;
  if (!(gamma_dt >= 0.0) || !std::isfinite(gamma_dt)) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  hps_handle *H = new (std::nothrow) hps_handle();
  if (!H) return HPS_ENOMEM;
  auto fail = [&](int e) {
    hps_free(H);
    return e;
  };
  H->tree = *tree;
  H->g = dims(tree, p);
  H->p = p;
  H->m = p - 2;
  H->q = H->m * H->m;
  H->b = 4 * H->m;
  H->hx = (tree->x1 - tree->x0) / tree->n1;
  H->hy = (tree->y1 - tree->y0) / tree->n2;
  H->gamma_dt = gamma_dt;
  H->coef_kind = coeffs->kind;
  H->shared = coeffs->kind == HPS_COEF_CONST && !(flags & HPS_FLAG_PER_NODE);
  const double cst[5] = {coeffs->c_a11, coeffs->c_a22, coeffs->c_a1, coeffs->c_a2, coeffs->c_a0};
  for (int i = 0; i < 5; ++i) H->cst[i] = coeffs->kind == HPS_COEF_CONST ? cst[i] : 0.0;
  try {
    H->lev = make_levels(H->g);
  } catch (...) {
    return fail(HPS_EINVAL);
  }
  H->L = (int)H->lev.size() - 1;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(HPS_ECUDA);
  }
  for (const Level &lv : H->lev)
    if (lv.nb > hps::kMaxBd || lv.n3 > hps::kMaxBd) return fail(HPS_EINVAL);
  // tree tables
  for (Level &lv : H->lev) {
    if (dalloc(H, &lv.d_origin, lv.origin.size())) return fail(HPS_ENOMEM);
    cudaMemcpyAsync(lv.d_origin, lv.origin.data(), lv.origin.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (!lv.hsrc.empty()) {
      if (dalloc(H, &lv.d_hsrc, lv.hsrc.size())) return fail(HPS_ENOMEM);
      cudaMemcpyAsync(lv.d_hsrc, lv.hsrc.data(), lv.hsrc.size() * sizeof(int), cudaMemcpyHostToDevice, st);
      if (dalloc(H, &lv.d_cmap, lv.cmap.size())) return fail(HPS_ENOMEM);
      cudaMemcpyAsync(lv.d_cmap, lv.cmap.data(), lv.cmap.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    }
  }
  // differentiation matrices D1x, D1y, Dxx = D1x^2, Dyy = D1y^2 on this leaf size
  {
    std::vector<double> Dh = scaled_D(p, H->hx, H->hy);
    {  // Thomas factors of the edge-projection systems (one per grid line of shared edges)
      std::vector<double> pr;
      for (int dir = 0; dir < 2; ++dir) {
        const double *D1 = Dh.data() + (size_t)dir * p * p;
        const int n = (dir ? H->g.n2 : H->g.n1) - 1;
        const double lo = D1[(p - 1) * p], d = D1[(p - 1) * p + p - 1] - D1[0], up = -D1[p - 1];
        H->proj_lo[dir] = lo;
        H->proj_up[dir] = up;
        std::vector<double> w(n, 0.0), ib(n);
        double b = d;
        for (int L = 0; L < n; ++L) {
          if (L > 0) {
            w[L] = lo / b;
            b = d - w[L] * up;
          }
          if (!(std::fabs(b) > 0.0)) return fail(HPS_EINVAL);
          ib[L] = 1.0 / b;
        }
        pr.insert(pr.end(), w.begin(), w.end());
        pr.insert(pr.end(), ib.begin(), ib.end());
      }
      if (!pr.empty()) {
        if (dalloc(H, &H->d_proj, pr.size())) return fail(HPS_ENOMEM);
        cudaMemcpyAsync(H->d_proj, pr.data(), pr.size() * sizeof(double), cudaMemcpyHostToDevice, st);
      }
    }
    if (p % 2 == 0) {  // even-odd halves of D1x, D1y, Dxx, Dyy: A = (D_ik + D_i,p-1-k) / 2, B = (D_ik - D_i,p-1-k) / 2
      const int h = p / 2;
      for (int mtx = 0; mtx < 4; ++mtx) {
        const double *Mx = Dh.data() + (size_t)mtx * p * p;
        std::vector<double> Ah((size_t)h * h), Bh((size_t)h * h);
        for (int i = 0; i < h; ++i)
          for (int k = 0; k < h; ++k) {
            Ah[i * h + k] = 0.5 * (Mx[i * p + k] + Mx[i * p + p - 1 - k]);
            Bh[i * h + k] = 0.5 * (Mx[i * p + k] - Mx[i * p + p - 1 - k]);
          }
        Dh.insert(Dh.end(), Ah.begin(), Ah.end());
        Dh.insert(Dh.end(), Bh.begin(), Bh.end());
      }
    }
    if (dalloc(H, &H->d_D, Dh.size())) return fail(HPS_ENOMEM);
    cudaMemcpyAsync(H->d_D, Dh.data(), Dh.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(HPS_ECUDA);
    if (int e = hps::fastdiag_build(H, Dh, st)) return fail(e);
  }
  if (coeffs->kind == HPS_COEF_NODAL) {
    const int64_t n = H->g.N_int;
    if (dalloc(H, &H->d_coef, 5 * (size_t)n)) return fail(HPS_ENOMEM);
    const double *src[5] = {coeffs->a11, coeffs->a22, coeffs->a1, coeffs->a2, coeffs->a0};
    for (int i = 0; i < 5; ++i)
      if (cudaMemcpyAsync(H->d_coef + i * n, src[i], n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(HPS_ECUDA);
  }
  if (int e = hps::build_operators(H, H->impl, gamma_dt, false, st)) return fail(e);
  if (int e = hps::build_operators(H, H->ident, 0.0, true, st)) return fail(e);
  // persistent merge kernel: task lists (operator data, shared by clones)
  if (int e = hps::build_tasks(H, H->impl)) return fail(e);
  if (int e = hps::build_tasks(H, H->ident)) return fail(e);
  if (int e = hps::alloc_work(H, st)) return fail(e);
  *out = H;
  return HPS_OK;
}

}  // extern "C"

namespace hps {

int smem_optin(const void *kernel, size_t bytes) {
  // the 48 KB default covers dynamic AND static shared memory: opt in well below it, so that a
  // kernel with a few static bytes (a flag, a counter) and 48 KB of dynamic memory still launches
  if (bytes <= 32 * 1024) return HPS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HPS_ECUDA;
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t &have = done[{kernel, dev}];
  if (bytes <= have) return HPS_OK;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ECUDA;
  }
  have = bytes;
  return HPS_OK;
}

// The per-call work buffers of a handle (everything a solve writes besides the caller's vectors).
int alloc_work(hps_handle *H, cudaStream_t st) {
  const GridDims &g = H->g;
  if (dalloc(H, &H->ustage, g.N) || dalloc(H, &H->R, g.N_int) || dalloc(H, &H->KL, 6 * (size_t)g.N_int) ||
      dalloc(H, &H->KE, 6 * (size_t)g.N_int) || dalloc(H, &H->wleaf, g.N_int))
    return HPS_ENOMEM;
  H->h.assign(H->L + 1, nullptr);
  H->w3.assign(H->L, nullptr);
  for (int l = 0; l <= H->L; ++l) {
    const Level &lv = H->lev[l];
    if (dalloc(H, &H->h[l], (size_t)lv.nodes * lv.nb)) return HPS_ENOMEM;
    if (l < H->L && dalloc(H, &H->w3[l], (size_t)lv.nodes * lv.n3)) return HPS_ENOMEM;
  }
  H->partial_len = partial_doubles(H);
  if (H->partial_len && dalloc(H, &H->partial, H->partial_len)) return HPS_ENOMEM;
  if (dalloc(H, &H->ppartial, std::max<size_t>(1, H->ppartial_len)) ||
      dalloc(H, &H->pcounters, std::max<size_t>(1, H->pcounter_len)) || dalloc(H, &H->pbar, 2) ||
      dalloc(H, &H->perr, 1))
    return HPS_ENOMEM;
  cudaMemsetAsync(H->pcounters, 0, std::max<size_t>(1, H->pcounter_len) * sizeof(unsigned), st);
  cudaMemsetAsync(H->pbar, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(H->perr, 0, sizeof(int), st);
  cudaMemsetAsync(H->ustage, 0, g.N * sizeof(double), st);
  return cudaStreamSynchronize(st) == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// A handle that shares base's operators (read only) and owns new work buffers, so that
// several states can be advanced concurrently with one factorization.  base must outlive it.
int clone_handle(const hps_handle *base, cudaStream_t st, hps_handle **out) {
  if (!base || !out) return HPS_EINVAL;
  hps_handle *H = new (std::nothrow) hps_handle();
  if (!H) return HPS_ENOMEM;
  H->tree = base->tree;
  H->g = base->g;
  H->p = base->p;
  H->m = base->m;
  H->q = base->q;
  H->b = base->b;
  H->L = base->L;
  H->hx = base->hx;
  H->hy = base->hy;
  H->gamma_dt = base->gamma_dt;
  H->shared = base->shared;
  H->coef_kind = base->coef_kind;
  for (int i = 0; i < 5; ++i) H->cst[i] = base->cst[i];
  H->d_coef = base->d_coef;
  H->d_D = base->d_D;
  H->fd = base->fd;
  H->d_proj = base->d_proj;
  for (int d = 0; d < 2; ++d) {
    H->proj_lo[d] = base->proj_lo[d];
    H->proj_up[d] = base->proj_up[d];
  }
  H->lev = base->lev;
  H->impl = base->impl;
  H->ident = base->ident;
  H->num_sms = base->num_sms;
  H->persistent = base->persistent;
  H->pgrid = base->pgrid;
  H->ppartial_len = base->ppartial_len;
  H->pcounter_len = base->pcounter_len;
  if (int e = alloc_work(H, st)) {
    hps_free(H);
    return e;
  }
  *out = H;
  return HPS_OK;
}

// Device bytes of the operators (both sets) and of one handle's work buffers.
int bytes_split(const hps_tree *tree, int p, int coeff_kind, int flags, size_t *ops, size_t *work) {
  if (check_tree(tree, p)) return HPS_EINVAL;
  const GridDims g = dims(tree, p);
  std::vector<Level> lev;
  try {
    lev = make_levels(g);
  } catch (...) {
    return HPS_EINVAL;
  }
  const int q = g.m * g.m, b = 4 * g.m;
  const bool shared = coeff_kind == HPS_COEF_CONST && !(flags & HPS_FLAG_PER_NODE);
  *ops = opset_bytes(lev, q, b, shared, false) + opset_bytes(lev, q, b, true, true) +
         (coeff_kind == HPS_COEF_NODAL ? 5 * (size_t)g.N_int * sizeof(double) : 0) + 4 * (size_t)p * p * sizeof(double);
  *work = work_bytes(g, lev);
  return HPS_OK;
}

// The ARK table of the implicit and explicit tableaus (Table 1), for the batched steps.
ArkTable ark_table() {
  ArkTable t;
  const Tableau &tb = tableau();
  std::memcpy(t.A, tb.A, sizeof(t.A));
  std::memcpy(t.Ah, tb.Ah, sizeof(t.Ah));
  std::memcpy(t.b, tb.b, sizeof(t.b));
  return t;
}

}  // namespace hps

namespace {

uint64_t bits(double v) {
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  return b;
}

int graph_launch(hps_handle *H, hps::GraphEntry &E, cudaStream_t st) {
  hps::drain_graph(H, E);  // the graph's timing events are reused by every replay
  if (cudaGraphLaunch(E.exec, st) != cudaSuccess) return HPS_ECUDA;
  for (int s = 0; s < hps::kNumSlots; ++s) H->trace.launches[s] += E.launches[s];
  E.pending = E.nev > 0;
  return HPS_OK;
}

// Run `enqueue` eagerly, or replay / record it as a CUDA graph (hps_set_graph).  The first
// call with a key runs eagerly (kernels get loaded, attributes set); the second records the
// sequence on an internal stream and replays it on `st`; later equal calls only replay.
template <class F>
int run_graphed(hps_handle *H, hps::GraphEntry &E, const uint64_t (&key)[hps::GraphEntry::kKey], F enqueue,
                cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!H->graph_mode || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return enqueue(st);
  const bool same = std::memcmp(E.key, key, sizeof(E.key)) == 0;
  if (E.valid && same) return graph_launch(H, E, st);
  if (!(E.seen && same)) {
    hps::drain_graph(H, E);
    E.destroy();
    std::memcpy(E.key, key, sizeof(E.key));
    E.seen = true;
    return enqueue(st);
  }
  if (!H->cap_stream && cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return HPS_ECUDA;
  if (H->trace.mask && E.ev.empty()) {
    E.ev.resize(2 * hps::GraphEntry::kEventPairs);
    for (auto &ev : E.ev) cudaEventCreate(&ev);
    E.ev_slot.assign(hps::GraphEntry::kEventPairs, -1);
  }
  for (auto &n : E.launches) n = 0;
  E.nev = 0;
  H->trace.capturing = &E;
  cudaGraph_t g = nullptr;
  int e = HPS_OK;
  if (cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) e = HPS_ECUDA;
  if (e == HPS_OK) {
    e = enqueue(H->cap_stream);
    if (cudaStreamEndCapture(H->cap_stream, &g) != cudaSuccess && e == HPS_OK) e = HPS_ECUDA;
  }
  H->trace.capturing = nullptr;
  if (e == HPS_OK && cudaGraphInstantiate(&E.exec, g, 0) != cudaSuccess) e = HPS_ECUDA;
  if (g) cudaGraphDestroy(g);
  if (e != HPS_OK) {
    E.destroy();
    cudaGetLastError();
    return e;
  }
  E.valid = true;
  return graph_launch(H, E, st);
}

int solve_enqueue(hps_handle *H, const double *rhs, const double *f, double *u, cudaStream_t st) {
  if (int e = hps::set_boundary(H, u, f, st)) return e;
  hps::Combo c{};
  add_term(c, rhs, 1.0);
  return hps::sweep(H, H->impl, c, nullptr, u, u, nullptr, st);
}

// KE += dt G: the caller's g (HPS_G_USER) added to a stage's explicit term
__global__ void k_add_user_g(int64_t n, double *__restrict__ KE, double dt, const double *__restrict__ G) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    KE[i] = fma(dt, G[i], KE[i]);
}

// g(u_j) by the caller's hook into H->gbuf (ordered on st), then KE_j += dt g(u_j)
int user_g_term(hps_handle *H, const hps_ark_terms *terms, const double *uj, double *KE, double dt, cudaStream_t st) {
  if (int e = terms->g_fn(terms->g_user, uj, H->gbuf, (hps_stream_t)st)) return e;
  const int64_t n = H->g.N_int;
  k_add_user_g<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, KE, dt, H->gbuf);
  return cudaPeekAtLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

int ark_enqueue(hps_handle *H, double *u, double dt, const hps_ark_terms *terms, cudaStream_t st) {
  const Tableau &tb = tableau();
  const bool user_g = terms && terms->g_kind == HPS_G_USER;
  // the kernels evaluate the presets; the caller's g is added after them
  const int gk = terms && !user_g ? terms->g_kind : HPS_G_NONE;
  const int64_t ni = H->g.N_int, nbd = H->g.N_bd;
  const double *q = terms ? terms->q : nullptr;
  const double *f = terms ? terms->f : nullptr;
  const double gp0 = terms ? terms->g_param[0] : 0.0, gp1 = terms ? terms->g_param[1] : 0.0;
  // stage 1 (explicit): dt L u^n and dt (q_1 + g(u^n))
  if (int e = hps::leaf_eval(H, u, H->KL, H->KE, q, dt, gk, gp0, gp1, st)) return e;
  if (user_g)
    if (int e = user_g_term(H, terms, u, H->KE, dt, st)) return e;
  for (int i = 1; i < 6; ++i) {
    hps::Combo c{};
    add_term(c, u, 1.0);
    for (int j = 0; j < i; ++j) {
      add_term(c, H->KL + j * ni, tb.A[i][j]);
      add_term(c, H->KE + j * ni, tb.Ah[i][j]);
    }
    if (int e = hps::set_boundary(H, H->ustage, f ? f + i * nbd : nullptr, st)) return e;
    hps::Epilogue ep;
    ep.KL = H->KL + i * ni;
    ep.KE = H->KE + i * ni;
    ep.Rsaved = H->R;
    ep.q = q ? q + i * ni : nullptr;
    ep.inv_gamma = 1.0 / tb.A[1][1];
    ep.dt = dt;
    ep.g_kind = gk;
    ep.gp0 = gp0;
    ep.gp1 = gp1;
    // (with the caller's g the stage value is completed in ustage -- interior points too -- for the hook)
    if (int e = hps::sweep(H, H->impl, c, H->R, H->ustage, user_g ? H->ustage : nullptr, &ep, st)) return e;
    if (user_g)
      if (int e = user_g_term(H, terms, H->ustage, H->KE + i * ni, dt, st)) return e;
  }
  // step close: ARK combination at interior points, shared-edge values from the identity-operator
  // system (flux continuity), by the edge projection or by an identity-operator sweep
  // (the stage sweeps leave the interior of ustage unwritten: the epilogue takes the stage
  // values in the leaf kernel, so the close keeps the full 13-term combination)
  hps::Combo c{};
  add_term(c, u, 1.0);
  for (int j = 0; j < 6; ++j) {
    add_term(c, H->KL + j * ni, tb.b[j]);
    add_term(c, H->KE + j * ni, tb.b[j]);
  }
  if (int e = hps::set_boundary(H, u, f ? f + 5 * nbd : nullptr, st)) return e;
  // (the projection's edge right-hand side goes into the edge range of ustage, free here)
  if (H->batch.edge_projection && H->d_proj) return hps::edge_projection(H, 1, c, u, H->ustage, st);
  return hps::sweep(H, H->ident, c, nullptr, u, u, nullptr, st);
}

}  // namespace

extern "C" {

int hps_solve(hps_handle *H, const double *rhs, const double *f, double *u, hps_stream_t stream) {
  if (!H || !rhs || !u) return HPS_EINVAL;
  const uint64_t key[hps::GraphEntry::kKey] = {(uint64_t)rhs, (uint64_t)f, (uint64_t)u, 0, 0, 0, 0, 0};
  return run_graphed(H, H->g_solve, key, [&](cudaStream_t s) { return solve_enqueue(H, rhs, f, u, s); },
                     (cudaStream_t)stream);
}

int hps_set_persistent(hps_handle *H, int enable) {
  if (!H) return HPS_EINVAL;
  cudaDeviceSynchronize();
  hps::drain_graph(H, H->g_ark);
  hps::drain_graph(H, H->g_solve);
  H->g_ark.destroy();  // recorded graphs hold the other kernel sequence
  H->g_solve.destroy();
  H->g_ark_b.destroy();
  H->g_solve_b.destroy();
  H->persistent = enable != 0;
  return HPS_OK;
}

int hps_status(hps_handle *H, hps_stream_t stream) {
  if (!H) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, H->perr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HPS_ECUDA;
  if (!herr) return HPS_OK;
  // a timed-out barrier leaves its counters behind: reset them for the next call
  cudaMemsetAsync(H->pcounters, 0, std::max<size_t>(1, H->pcounter_len) * sizeof(unsigned), st);
  cudaMemsetAsync(H->pbar, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(H->perr, 0, sizeof(int), st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPS_ECUDA;
  return HPS_ETIMEOUT;
}

int hps_trace_tasks(hps_handle *H, int enable, int upward, double *us, int max_tasks) {
  if (!H) return HPS_EINVAL;
  if (!H->pstamps && dalloc(H, &H->pstamps, 128)) return HPS_ENOMEM;
  if (enable >= 0) {
    cudaDeviceSynchronize();
    if (H->stamp_tasks != (enable != 0)) {  // recorded graphs carry the other kernel arguments
      H->g_ark.destroy();
      H->g_solve.destroy();
    }
    H->stamp_tasks = enable != 0;
    return HPS_OK;
  }
  const OpSet &ops = H->impl;
  const int n = upward ? ops.n_up : ops.n_down;
  unsigned long long st[65];
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(st, H->pstamps + (upward ? 0 : 64), (n + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return HPS_ECUDA;
  for (int t = 0; t < n && t < max_tasks; ++t) us[t] = 1e-3 * (double)(st[t + 1] - st[t]);
  return n;
}

int hps_selftest_barrier_timeout(hps_handle *H, hps_stream_t stream) {
  if (!H) return HPS_EINVAL;
  return hps::selftest_barrier(H, (cudaStream_t)stream);
}

int hps_set_graph(hps_handle *H, int enable) {
  if (!H) return HPS_EINVAL;
  cudaDeviceSynchronize();
  hps::drain_graph(H, H->g_ark);
  hps::drain_graph(H, H->g_solve);
  H->g_ark.destroy();
  H->g_solve.destroy();
  H->g_ark_b.destroy();
  H->g_solve_b.destroy();
  H->graph_mode = enable != 0;
  return HPS_OK;
}

int hps_ark_abscissae(double *c) {
  if (!c) return HPS_EINVAL;
  for (int i = 0; i < 6; ++i) c[i] = tableau().c[i];
  return HPS_OK;
}

int ark_step(hps_handle *H, double *u, double t, double dt, const hps_ark_terms *terms, hps_stream_t stream) {
  if (!H || !u || !(dt > 0.0) || !std::isfinite(t)) return HPS_EINVAL;
  if (std::fabs(0.25 * dt - H->gamma_dt) > 1e-12 * H->gamma_dt) return HPS_EDT;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  if (gk < HPS_G_NONE || gk > HPS_G_USER || (gk == HPS_G_USER && !terms->g_fn)) return HPS_EINVAL;
  if (gk == HPS_G_USER && !H->gbuf && dalloc(H, &H->gbuf, (size_t)H->g.N_int)) return HPS_ENOMEM;
  // (the hook and its argument stand in the key where a preset's parameters would)
  const bool user = gk == HPS_G_USER;
  const uint64_t key[hps::GraphEntry::kKey] = {
      (uint64_t)u, (uint64_t)(terms ? terms->q : nullptr), (uint64_t)(terms ? terms->f : nullptr), (uint64_t)gk,
      user ? (uint64_t)terms->g_fn : bits(terms ? terms->g_param[0] : 0.0),
      user ? (uint64_t)terms->g_user : bits(terms ? terms->g_param[1] : 0.0), bits(dt), 1};
  return run_graphed(H, H->g_ark, key, [&](cudaStream_t s) { return ark_enqueue(H, u, dt, terms, s); },
                     (cudaStream_t)stream);
}

int ark_slope_step(hps_handle *H, double *u, double t, double dt, const hps_ark_terms *terms, hps_stream_t stream) {
  if (!H || !u || !(dt > 0.0) || !std::isfinite(t)) return HPS_EINVAL;
  if (std::fabs(0.25 * dt - H->gamma_dt) > 1e-12 * H->gamma_dt) return HPS_EDT;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  if (gk < HPS_G_NONE || gk > HPS_G_BURGERS || H->persistent) return HPS_EINVAL;
  hps::ArkTable tab;
  const Tableau &tb = tableau();
  std::memcpy(tab.A, tb.A, sizeof(tab.A));
  std::memcpy(tab.Ah, tb.Ah, sizeof(tab.Ah));
  std::memcpy(tab.b, tb.b, sizeof(tab.b));
  return hps::ark_slope(H, u, dt, terms, tab, (cudaStream_t)stream);
}

int ark_slope_step_batch(hps_handle *H, int R, double *u, double t, double dt, const hps_ark_terms *terms, int refine,
                         hps_stream_t stream) {
  if (!H || !u || !(dt > 0.0) || !std::isfinite(t) || R <= 0 || R > H->batch.Rmax || refine < 0 || refine > 8)
    return HPS_EINVAL;
  if (std::fabs(0.25 * dt - H->gamma_dt) > 1e-12 * H->gamma_dt) return HPS_EDT;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  if (gk < HPS_G_NONE || gk > HPS_G_BURGERS || (gk != HPS_G_NONE && terms->f)) return HPS_EINVAL;
  hps::ArkTable tab;
  const Tableau &tb = tableau();
  std::memcpy(tab.A, tb.A, sizeof(tab.A));
  std::memcpy(tab.Ah, tb.Ah, sizeof(tab.Ah));
  std::memcpy(tab.b, tb.b, sizeof(tab.b));
  const uint64_t key[hps::GraphEntry::kKey] = {
      (uint64_t)u, (uint64_t)(terms ? terms->q : nullptr), (uint64_t)(terms ? terms->f : nullptr),
      (uint64_t)gk | ((uint64_t)R << 8) | ((uint64_t)refine << 24), bits(terms ? terms->g_param[0] : 0.0),
      bits(terms ? terms->g_param[1] : 0.0), bits(dt), 4};
  return run_graphed(H, H->g_ark_b, key,
                     [&](cudaStream_t s) { return hps::ark_slope_batch(H, R, u, dt, terms, refine, tab, s); },
                     (cudaStream_t)stream);
}

// Device buffer of at least n doubles for the host-buffer steps (kept by the handle).
static int host_stage(hps_handle *H, size_t n) {
  if (H->host_stage_len >= n) return HPS_OK;
  if (H->host_stage) {
    cudaDeviceSynchronize();  // the old buffer may still be read by queued work
    cudaFree(H->host_stage);
    H->allocs.erase(std::remove(H->allocs.begin(), H->allocs.end(), (void *)H->host_stage), H->allocs.end());
    H->host_stage = nullptr;
    H->host_stage_len = 0;
  }
  if (cudaMalloc(&H->host_stage, n * sizeof(double)) != cudaSuccess) return HPS_ENOMEM;
  H->allocs.push_back(H->host_stage);
  H->host_stage_len = n;
  return HPS_OK;
}

int ark_step_host(hps_handle *H, double *u_host, double t, double dt, const hps_ark_terms *terms,
                  hps_stream_t stream) {
  if (!H || !u_host) return HPS_EINVAL;
  const size_t n = (size_t)H->g.N;
  if (int e = host_stage(H, n)) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(H->host_stage, u_host, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HPS_ECUDA;
  if (int e = ark_step(H, H->host_stage, t, dt, terms, stream)) return e;
  return cudaMemcpyAsync(u_host, H->host_stage, n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess
             ? HPS_OK
             : HPS_ECUDA;
}

int ark_step_batch_host(hps_handle *H, int R, double *u_host, double t, double dt, const hps_ark_terms *terms,
                        int refine, hps_stream_t stream) {
  if (!H || !u_host || R <= 0 || R > H->batch.Rmax) return HPS_EINVAL;
  const size_t n = (size_t)H->g.N * R;
  if (int e = host_stage(H, (size_t)H->g.N * H->batch.Rmax)) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(H->host_stage, u_host, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HPS_ECUDA;
  if (int e = ark_step_batch(H, R, H->host_stage, t, dt, terms, refine, stream)) return e;
  return cudaMemcpyAsync(u_host, H->host_stage, n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess
             ? HPS_OK
             : HPS_ECUDA;
}

int hps_batch_reserve_groups(hps_handle *H, int R, int groups) {
  if (!H) return HPS_EINVAL;
  if (groups != H->batch.groups) {  // recorded graphs hold the old groups' buffers and streams
    hps::drain_graph(H, H->g_ark_b);
    hps::drain_graph(H, H->g_solve_b);
    H->g_ark_b.destroy();
    H->g_solve_b.destroy();
  }
  return hps::batch_reserve(H, R, groups);
}

static void drop_batch_graphs(hps_handle *H) {  // (the step-close options reach the FP64 step too)
  hps::drain_graph(H, H->g_ark_b);
  hps::drain_graph(H, H->g_solve_b);
  hps::drain_graph(H, H->g_ark);
  hps::drain_graph(H, H->g_solve);
  H->g_ark_b.destroy();
  H->g_solve_b.destroy();
  H->g_ark.destroy();
  H->g_solve.destroy();
}

int hps_fastdiag_check(int p, const double *coef, double gamma_dt, double hx, double hy, double *max_err) {
  if (p < 4 || p > 32 || !coef || !(gamma_dt > 0.0) || !(hx > 0.0) || !(hy > 0.0)) return HPS_EINVAL;
  const std::vector<double> Dh = scaled_D(p, hx, hy);
  std::vector<double> F[5];
  double err = 0.0;
  const bool ok = hps::fastdiag_factor(p, Dh.data(), coef, gamma_dt, true, F, &err);
  if (max_err) *max_err = err;
  return ok ? HPS_OK : HPS_EINVAL;
}

int hps_batch_set_option(hps_handle *H, int opt, int value) {
  if (!H) return HPS_EINVAL;
  drop_batch_graphs(H);
  return hps::batch_option(H, opt, &value, nullptr);
}

int hps_batch_get_option(hps_handle *H, int opt, int *value) {
  if (!H || !value) return HPS_EINVAL;
  return hps::batch_option(H, opt, nullptr, value);
}

int hps_batch_autotune(hps_handle *H, int R, int refine, hps_stream_t stream, hps_tune_result *results,
                       int max_results, int *n_results) {
  if (!H || max_results < 0) return HPS_EINVAL;
  drop_batch_graphs(H);
  const bool graph = H->graph_mode;
  H->graph_mode = false;  // time the kernels, not graph recording
  const int e = hps::batch_autotune(H, R, refine, (cudaStream_t)stream, results, max_results, n_results);
  H->graph_mode = graph;
  drop_batch_graphs(H);
  return e;
}

int hps_batch_reserve(hps_handle *H, int R) {
  if (!H) return HPS_EINVAL;
  return hps_batch_reserve_groups(H, R, H->batch.groups);
}

int hps_solve_batch(hps_handle *H, int R, const double *rhs, const double *f, double *u, int refine,
                    hps_stream_t stream) {
  if (!H || !rhs || !u || R <= 0 || R > H->batch.Rmax || refine < 0 || refine > 8) return HPS_EINVAL;
  const uint64_t key[hps::GraphEntry::kKey] = {(uint64_t)rhs, (uint64_t)f, (uint64_t)u, (uint64_t)R,
                                               (uint64_t)refine, 0, 0, 2};
  return run_graphed(H, H->g_solve_b, key,
                     [&](cudaStream_t s) { return hps::solve_batch(H, R, rhs, f, u, refine, s); },
                     (cudaStream_t)stream);
}

int ark_step_batch(hps_handle *H, int R, double *u, double t, double dt, const hps_ark_terms *terms, int refine,
                   hps_stream_t stream) {
  if (!H || !u || !(dt > 0.0) || !std::isfinite(t) || R <= 0 || R > H->batch.Rmax || refine < 0 || refine > 8)
    return HPS_EINVAL;
  if (std::fabs(0.25 * dt - H->gamma_dt) > 1e-12 * H->gamma_dt) return HPS_EDT;
  const int gk = terms ? terms->g_kind : HPS_G_NONE;
  if (gk < HPS_G_NONE || gk > HPS_G_BURGERS) return HPS_EINVAL;  // (no HPS_G_USER on the batched path)
  hps::ArkTable tab;
  const Tableau &tb = tableau();
  std::memcpy(tab.A, tb.A, sizeof(tab.A));
  std::memcpy(tab.Ah, tb.Ah, sizeof(tab.Ah));
  std::memcpy(tab.b, tb.b, sizeof(tab.b));
  const uint64_t key[hps::GraphEntry::kKey] = {
      (uint64_t)u, (uint64_t)(terms ? terms->q : nullptr), (uint64_t)(terms ? terms->f : nullptr),
      (uint64_t)gk | ((uint64_t)R << 8) | ((uint64_t)refine << 24), bits(terms ? terms->g_param[0] : 0.0),
      bits(terms ? terms->g_param[1] : 0.0), bits(dt), 3};
  return run_graphed(H, H->g_ark_b, key,
                     [&](cudaStream_t s) { return hps::ark_batch(H, R, u, dt, terms, refine, tab, s); },
                     (cudaStream_t)stream);
}

int hps_trace_enable(hps_handle *H, unsigned mask) {
  if (!H) return HPS_EINVAL;
  H->trace.drain();
  hps::drain_graph(H, H->g_ark);
  hps::drain_graph(H, H->g_solve);
  hps::drain_graph(H, H->g_ark_b);
  hps::drain_graph(H, H->g_solve_b);
  if (mask != H->trace.mask) {  // recorded graphs carry the old timing events
    H->g_ark.destroy();
    H->g_solve.destroy();
    H->g_ark_b.destroy();
    H->g_solve_b.destroy();
  }
  H->trace.mask = mask;
  for (int i = 0; i < hps::kNumSlots; ++i) {
    H->trace.launches[i] = 0;
    H->trace.timed[i] = 0;
    H->trace.ms[i] = 0.0;
  }
  return HPS_OK;
}

int hps_trace_read(hps_handle *H, int kernel, int64_t *launches, int64_t *timed, double *total_ms) {
  if (!H || kernel < 0 || kernel >= hps::kNumSlots) return HPS_EINVAL;
  H->trace.drain();
  hps::drain_graph(H, H->g_ark);
  hps::drain_graph(H, H->g_solve);
  hps::drain_graph(H, H->g_ark_b);
  hps::drain_graph(H, H->g_solve_b);
  if (launches) *launches = H->trace.launches[kernel];
  if (timed) *timed = H->trace.timed[kernel];
  if (total_ms) *total_ms = H->trace.ms[kernel];
  return HPS_OK;
}

const char *hps_strerror(int code) {
  switch (code) {
    case HPS_OK: return "ok";
    case HPS_EINVAL: return "invalid argument";
    case HPS_ENOMEM: return "device allocation failed";
    case HPS_ESINGULAR: return "zero or non-finite pivot in the operator build";
    case HPS_ETIMEOUT: return "bounded device wait expired";
    case HPS_ECUDA: return "CUDA error";
    case HPS_EDT: return "gamma*dt differs from the value the handle was built for";
    case HPS_ESCRATCH: return "problem too large for the static work array of hps_solve_static";
    default: return "unknown error";
  }
}

}  // extern "C"
