/*
 * hps.h -- C ABI of libhps.so: the HPS direct solver inside the implicit stages of an
 * additive Runge-Kutta (ESDIRK + ERK) step, on one GB300 GPU (sm_103a).
 *
 * Method: Chen, Appelo, Babb, Martinsson, "Fast and high-order approximation of parabolic
 * equations using hierarchical direct solvers and implicit Runge-Kutta methods".
 * Problem (eq. ``general``):  u_t = L u + q + g(u) on a rectangle, u = f on its boundary,
 *   L u = a11 u_xx + a22 u_yy + a1 u_x + a2 u_y + a0 u    (eq. ``operatorA`` with c12 = 0).
 *
 * Discretization (Sec. 2.1): n1 x n2 equal leaves (n1, n2 powers of two), p x p Chebyshev
 * nodes per leaf, leaf corners dropped, shared edge nodes stored once:
 *   N = (p-2)(p n1 n2 + n1 + n2) unknowns, m = p-2, N_int = n1 n2 m^2, N_bd = 2 m (n1 + n2).
 * Global vector order (every array named "global" below uses it):
 *   [0, N_int)        leaf interiors: leaf l = iy*n1 + ix, node (i, j) in 1..m (i along x)
 *                     at l*m*m + (j-1)*m + (i-1);
 *   then N_v = (n1+1) n2 m vertical-edge nodes: x-line L (0..n1), leaf row iy, node j:
 *                     N_int + (L*n2 + iy)*m + (j-1);
 *   then N_h = (n2+1) n1 m horizontal-edge nodes: y-line L (0..n2), leaf column ix, node i:
 *                     N_int + N_v + (L*n1 + ix)*m + (i-1).
 * A leaf's local node (i, j), 0 <= i, j < p, sits at
 *   x = x0 + hx*(ix + (1 + xi_i)/2),  y = y0 + hy*(iy + (1 + xi_j)/2),  xi_k = -cos(k pi/(p-1)).
 * "Interior order" = the first N_int entries.  "Boundary order" = the N_bd entries of the
 * outer boundary in ascending global index (hps_boundary_index lists them).
 *
 * Ownership: every vector argument is caller-owned DEVICE memory unless marked "host";
 * the handle owns its operators and work buffers (allocated by hps_build, released by
 * hps_free).  All GPU work is enqueued on the given stream (NULL = legacy default stream);
 * functions return after enqueueing.  A handle's work buffers are shared by its calls:
 * calls on the same handle must be ordered on one stream.
 * Errors: every int-returning function returns HPS_OK (0) or a negative HPS_E* code.
 */
#ifndef HPS_H
#define HPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_handle hps_handle;
typedef struct CUstream_st *hps_stream_t; /* identical to cudaStream_t */

enum {
  HPS_OK = 0,
  HPS_EINVAL = -1,    /* bad argument: tree not a power of two, p out of [4, 32], NULL pointer ... */
  HPS_ENOMEM = -2,    /* device allocation failed */
  HPS_ESINGULAR = -3, /* zero or non-finite pivot in a Gauss-Jordan elimination of the build */
  HPS_ETIMEOUT = -4,  /* a bounded device-side wait expired */
  HPS_ECUDA = -5,     /* a CUDA runtime call or kernel launch failed */
  HPS_EDT = -6,       /* ark_step: gamma*dt differs from the gamma_dt the handle was built for */
  HPS_ESCRATCH = -7   /* hps_solve_static: the problem's work vectors exceed the static array */
};

/* Domain [x0,x1] x [y0,y1] cut into n1 x n2 equal leaves; n1, n2 powers of two, n1*n2 <= 65536,
 * and every box boundary at most 24576 points (2 (n1 + n2)(p - 2) <= 24576).
 * Sec. 2.1 halves the domain repeatedly; a box is cut across its longer side (in leaves),
 * a tie is cut by a vertical line. */
typedef struct hps_tree {
  int n1, n2;
  double x0, x1, y0, y1;
} hps_tree;

enum { HPS_COEF_CONST = 0, HPS_COEF_NODAL = 1 };

/* Coefficients of L (eq. ``operatorA`` with c12 = 0, signs as in u_t = L u).
 * CONST: the c_* scalars are used.  NODAL: a11..a0 are device arrays of N_int doubles in
 * interior order (values at the interior nodes, the only rows where L is collocated);
 * hps_build copies them. */
typedef struct hps_coeffs {
  int kind;
  double c_a11, c_a22, c_a1, c_a2, c_a0;
  const double *a11, *a22, *a1, *a2, *a0;
} hps_coeffs;

/* hps_build flags */
enum {
  HPS_FLAG_PER_NODE = 1 /* keep one operator per tree node even for CONST coefficients
                           (default for CONST: one operator per tree level, shared) */
};

/* Sizes of the discretization (Sec. 2.1 point count).  Host outputs; any may be NULL. */
int hps_sizes(const hps_tree *tree, int p, int64_t *N, int64_t *N_int, int64_t *N_bd);

/* Coordinates of all N global points into host arrays x[N], y[N]. */
int hps_coords(const hps_tree *tree, int p, double *x, double *y);

/* Global indices of the N_bd outer-boundary points, ascending, into host idx[N_bd]. */
int hps_boundary_index(const hps_tree *tree, int p, int64_t *idx);

/* Device bytes a handle for this discretization holds (operators + work buffers), for
 * admission control.  coeff_kind: HPS_COEF_CONST or HPS_COEF_NODAL. Returns 0 on bad input. */
size_t hps_bytes(const hps_tree *tree, int p, int coeff_kind, int flags);

/* Build the HPS solution operators of A = I - gamma_dt L (Sec. 2.1: leaf S = -A_ii^{-1} A_ib,
 * T = D S (eq. ``leaf``); merges X = (T^a_33 - T^b_33)^{-1}, S^t = X[-T^a_31 | T^b_32],
 * T^t = diag(T^a_11, T^b_22) + [T^a_13; T^b_23] S^t), in FP64 on the GPU, plus the operators
 * of the identity on the same tree (the "explicit equation" of Sec. 3.1.1, used to close
 * an ARK step).  gamma_dt >= 0.  Synchronizes `stream` before returning (the build is
 * one-off).  On success *out receives a new handle. */
int hps_build(const hps_tree *tree, int p, const hps_coeffs *coeffs, double gamma_dt, int flags,
              hps_stream_t stream, hps_handle **out);

/* One HPS solve (upward body-load sweep, then Alg. 1 downward sweep) of the collocation
 * system of eq. ``sparse_A``: (I - gamma_dt L) u = rhs at interior points, flux continuity
 * across shared edges, u = f on the outer boundary.
 *   rhs: N_int (interior order);  f: N_bd (boundary order) or NULL for f = 0;
 *   u:   N (global order), written completely.  rhs/f must not alias u. */
int hps_solve(hps_handle *h, const double *rhs, const double *f, double *u, hps_stream_t stream);

/* hps_solve without device allocation, for callers that cannot call cudaMalloc when they
 * solve: a fixed memory budget set at start-up, a real-time loop, or an allocator that is
 * unavailable on the solving thread.  (The paper has no counterpart; this is a library
 * service.)  Same arguments, same kernels and same result as hps_solve; the per-call work
 * vectors (leaf particular solutions, fluxes, interface corrections, split-column partial
 * sums of the top tree levels) are placed in one
 * static device array of 2,097,152 doubles (16 MiB) compiled into libhps.so, which every
 * GPU that loads the library holds until the process exits.  The operators still come from
 * the handle.  Problems whose work vectors need more than that array -- N_int plus the
 * per-level flux and interface vectors and the partial sums, each rounded up to 256
 * bytes -- are rejected with
 * HPS_ESCRATCH (a 64 x 64 leaf grid with p = 16 fits; 128 x 128 with p = 16 does not).
 * The first call on a device looks up the array's device address with the device current
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share
 * the one array and it keeps the last call's contents (every entry a call reads it writes
 * first, except the few counters of the merge kernel, which each call clears): calls that
 * overlap on the GPU -- on different streams or different handles -- race and must be
 * serialized by the caller.  With hps_set_persistent on, a bounded wait that runs out in this
 * call is recorded in the handle's error word as for hps_solve (hps_status reports it). */
int hps_solve_static(hps_handle *h, const double *rhs, const double *f, double *u, hps_stream_t stream);

/* Nonlinear term presets g(u) (Sec. 1: at most first derivatives), evaluated at interior
 * points; derivatives by leaf-local Chebyshev differentiation. */
enum {
  HPS_G_NONE = 0,
  HPS_G_ALLEN_CAHN = 1, /* g = k0 (u - u^3) */
  HPS_G_FISHER = 2,     /* g = k0 u (1 - u) */
  HPS_G_BURGERS = 3,    /* g = -u (k0 u_x + k1 u_y) */
  HPS_G_USER = 4        /* g from the caller's hook hps_ark_terms.g_fn (ark_step, ark_step_host) */
};

/* A caller-supplied g (g_kind = HPS_G_USER).  For the value u_j of every stage (device, N doubles
 * in global order, complete: interior points, shared edges, boundary) the library calls
 * g_fn(g_user, u_j, g_out, stream) while it enqueues the step; the hook fills g_out (device, N_int
 * doubles) with g(u_j) at the interior points by work of its own ordered on `stream` (its kernels
 * or copies), and the step adds dt g_out to the stage's explicit term.  In graph mode the step,
 * the hook's work included, is recorded on the second call with the same arguments and then
 * replayed without calling the hook, so the hook must enqueue the same work at every call: g = g(u)
 * (Sec. 1), no explicit time dependence.  Returns 0, or an error code that the step returns. */
typedef int (*hps_g_fn)(void *user, const double *u, double *g_out, hps_stream_t stream);

/* Explicit terms of one ARK step.  Stage times t_j = t + c_j dt, j = 1..6 (hps_ark_abscissae).
 *   q: device, 6 * N_int doubles, q(t_j) at interior points, stage-major; NULL means q = 0.
 *   f: device, 6 * N_bd doubles, f(t_j) in boundary order, stage-major; NULL means f = 0.
 *      Entry j = 1 is not read (the first stage is u^n itself); entry 6 (c_6 = 1) is also
 *      the boundary value of u^{n+1}. */
typedef struct hps_ark_terms {
  const double *q;
  const double *f;
  int g_kind;
  double g_param[2];
  hps_g_fn g_fn;  /* g_kind == HPS_G_USER: the hook (else unused) */
  void *g_user;   /* passed to g_fn */
} hps_ark_terms;

/* Abscissae c_1..c_6 of ARK4(3)6L[2]SA (host output, 6 doubles); gamma = 1/4. */
int hps_ark_abscissae(double *c);

/* One ARK4(3)6L[2]SA step of eq. ``stage2`` in place on u (global order, N doubles):
 * u_1 = u^n; for i = 2..6 one hps_solve of (I - dt gamma L) u_i = u^n + dt sum_j a_ij L u_j
 * + dt sum_j ahat_ij (q_j + g_j) with u_i = f(t_i) on the boundary; L u^n by leaf-local
 * differentiation, dt L u_j = (u_j - R_j)/gamma for j >= 2; then
 * u^{n+1} = u^n + dt sum_j b_j L u_j + dt sum_j bhat_j (q_j + g_j) at interior points,
 * f(t + dt) on the boundary and shared-edge values from the identity-operator system (flux
 * continuity with those interior values), solved directly as one tridiagonal system per grid
 * line of shared edges (HPS_OPT_EDGE_PROJECTION, default) or by an identity-operator sweep.
 * The handle must have been built with gamma_dt == dt/4 (else HPS_EDT).  No allocation,
 * no host synchronization: the call can be captured in a CUDA graph. */
int ark_step(hps_handle *h, double *u, double t, double dt, const hps_ark_terms *terms,
             hps_stream_t stream);

/* Merge-level execution.  enable != 0: the upward merges of all levels run in one
 * cooperative kernel whose CTAs stay resident and pass a grid-wide barrier between tasks,
 * and likewise the downward merges; every barrier wait is bounded (2 s), and a wait that
 * runs out sets the handle's error word (read it with hps_status).  enable == 0 (default):
 * one launch per level and operator (plus a reduction launch where a level splits its
 * columns).  Both give bit-identical results. */
int hps_set_persistent(hps_handle *h, int enable);

/* Synchronizes `stream` and reports a bounded device-side wait that ran out since the last
 * call (HPS_ETIMEOUT; the handle's barrier state is reset so that later calls work), else
 * HPS_OK.  Results of the sweep that timed out are not valid. */
int hps_status(hps_handle *h, hps_stream_t stream);

/* Per-task timing of the persistent merge kernel (tracing; no effect on results).
 * enable = 1 / 0: start / stop stamping (the first CTA reads the GPU global timer at the start
 * of every task); enable = -1: synchronize the device and write into us[] the durations, in
 * microseconds, of the tasks of the last upward (upward != 0) or downward launch of the
 * implicit operator set, and return their number (upward: per level from the leaves up,
 * w3 then h; downward: per level from the root down). */
int hps_trace_tasks(hps_handle *h, int enable, int upward, double *us, int max_tasks);

/* Self-test of the bounded wait: runs the persistent merge kernel with a barrier that one
 * more CTA than exists must reach and a 1 ms limit, so the wait must run out.  Returns
 * HPS_ETIMEOUT when the kernel gave up and returned as designed (the handle stays usable),
 * HPS_OK if the barrier completed (a fault in the barrier), or an error code. */
int hps_selftest_barrier_timeout(hps_handle *h, hps_stream_t stream);

/* Self-test of the integer-pipe FP32 <-> FP64 conversions the batched kernels use in place of
 * the hardware conversions (which issue to the FP64 pipe on this GPU): n bit patterns from a
 * counter hash seeded by `seed` (zeros, subnormals, normals, infinities, NaN; doubles near the
 * float range; rounding ties), each converted both ways by both methods.  *mismatches (host)
 * receives the number of patterns whose results differ (any NaN matches any NaN).  Synchronous
 * on `stream`; allocates 8 bytes of device memory.  HPS_EINVAL for n < 1 or a null output. */
int hps_selftest_conversions(int64_t n, uint64_t seed, hps_stream_t stream, int64_t *mismatches);

/* Graph replay.  With enable != 0, ark_step and hps_solve record their kernel sequence
 * (about 380 launches per ARK step at 64 x 64 leaves) into a CUDA graph and replay it, so
 * the launch cost is paid once: the first call with a given set of pointers and arguments
 * (u, q, f, g, dt for ark_step; rhs, f, u for hps_solve) runs eagerly, the second records
 * the graph on an internal stream and replays it on the caller's stream, later equal calls
 * only replay; any change of those arguments starts over.  t is not part of the key (it
 * enters only through the q and f arrays).  Results are identical to eager calls.  Calls
 * made while the caller's stream is itself being captured always run eagerly.  Default: off. */
int hps_set_graph(hps_handle *h, int enable);

/* Kernels of the solve path, for launch counting and timing. */
enum {
  HPS_K_LEAF_UP = 0,     /* a1+a2: stage right-hand side, w = A_ii^{-1} R, h = D_bi w   */
  HPS_K_MERGE_UP_W3 = 1, /* a3: w3 = X (h^b_3 - h^a_3)                                  */
  HPS_K_MERGE_UP_H = 2,  /* a3: h^t = [h^a_1 ; h^b_2] + [T^a_13 ; T^b_23] w3              */
  HPS_K_MERGE_DOWN = 3,  /* a4: u3 = S^t u_b + w3                                       */
  HPS_K_LEAF_DOWN = 4,   /* a5: u_i = w + S u_b and the fused ARK stage epilogue          */
  HPS_K_LEAF_EVAL = 5,   /* explicit first stage: dt L u^n, dt (q + g(u^n))               */
  HPS_K_SET_BOUNDARY = 6, /* Dirichlet data onto the outer boundary                       */
  HPS_K_MERGE_UP_ALL = 7,  /* a3, all levels in one persistent kernel (hps_set_persistent);
                              batched path: the lower levels as one dataflow kernel             */
  HPS_K_MERGE_DOWN_ALL = 8, /* a4, likewise                                                    */
  HPS_K_RESIDUAL = 9,       /* batched path: FP64 collocation residual at interior points     */
  HPS_K_JUMP = 10,          /* batched path: FP64 flux-jump residual at shared edge points      */
  HPS_K_FINISH = 11,        /* batched path: FP32 sweep result into the FP64 vector; column
                              group copies                                                    */
  HPS_K_CLOSE = 12          /* step close by the edge projection: interior combination with the
                              leaves' flux sums, then one tridiagonal solve per grid line      */
};

/* Tracing (no effect on results).  Every launch of the solve path is counted per kernel;
 * kernels whose bit (1 << HPS_K_*) is set in `mask` are also bracketed by CUDA events
 * recorded on the launch stream.  hps_trace_enable resets all counters; mask 0 stops the
 * event timing.  In graph mode (hps_set_graph) the events are part of the recorded graph
 * and each replay's times are read before the next replay, which then waits for the
 * previous one to finish.  Do not enable event timing while capturing a CUDA graph yourself. */
int hps_trace_enable(hps_handle *h, unsigned mask);

/* Counters of one kernel since the last hps_trace_enable: launches, launches timed and
 * their summed device time in ms.  Synchronizes on the recorded events.  Host outputs,
 * any may be NULL. */
int hps_trace_read(hps_handle *h, int kernel, int64_t *launches, int64_t *timed, double *total_ms);

/* ---- Batched mixed precision (R right-hand sides, FP32 applies, FP64 refinement) ----------
 * Vectors with R columns are stored RHS-fastest: entry (point i, column j) at i*R + j, with
 * the point order of the single-column vector.  Each implicit solve A u = b is done as
 * u = S32(b), then `refine` times: r = b - A u in FP64 (the collocated rows of eq. ``sparse_A``:
 * interior R - (u - gamma dt L u) by leaf-local differentiation, shared-edge flux jumps), u +=
 * S32(r), where S32 is the HPS sweep with FP32 operators, FP32 work vectors and FP32
 * accumulation (the FP64 sweep is not used).  Measured on 64 x 64 leaves, p = 16, 32 states
 * of u_t = 0.01 Lap u + u - u^3 after 60 steps: relative max-norm distance to the FP64 path
 * 2e-12 with refine = 1, 6e-13 with refine = 2; without refinement about 1e-6. */

/* Convert the operators to FP32 (once) and allocate the R-column work buffers (R <= 64);
 * must precede the batched calls with this R.  Synchronizes the device. */
int hps_batch_reserve(hps_handle *h, int R);

/* hps_batch_reserve with the columns of every later batched call split into `groups` (1..8)
 * column groups of multiples of 4 columns, each run on its own internal stream, forked from
 * and joined back into the caller's stream (also inside a recorded graph).  Groups overlap one
 * group's FP64 residual kernels with another group's FP32 sweeps.  Results agree with the
 * ungrouped call to rounding (the split of the FP32 merge sums depends on the column count).
 * The default is one group; hps_batch_reserve keeps the handle's current count. */
int hps_batch_reserve_groups(hps_handle *h, int R, int groups);

/* R solves of hps_solve at once.  rhs: N_int x R; f: N_bd x R or NULL; u: N x R (written);
 * refine: 0..8 refinement sweeps. */
int hps_solve_batch(hps_handle *h, int R, const double *rhs, const double *f, double *u, int refine,
                    hps_stream_t stream);

/* ark_step on R states at once (u: N x R in place; terms->q: 6 x N_int x R, terms->f:
 * 6 x N_bd x R, both stage-major, or NULL; g a preset, HPS_G_USER is rejected with HPS_EINVAL).  Each implicit stage uses `refine` FP64 refinement
 * sweeps; the step close solves its identity-operator system directly (HPS_OPT_EDGE_PROJECTION)
 * or, with that option off, by a sweep with `refine` refinement sweeps. */
int ark_step_batch(hps_handle *h, int R, double *u, double t, double dt, const hps_ark_terms *terms, int refine,
                   hps_stream_t stream);

/* One ARK4(3)6L[2]SA step in slope form (Sec. 3.1, eq. slope0; eq. slope with g), FP64, on u (N, in
 * place): slopes k_1 = L u^n + q_1 (explicit; its shared-edge values from the identity-operator
 * system), (I - gamma dt L) k_i = L u^n + dt sum_{j<i} a_ij L k_j + q_i (one HPS solve each),
 * u^{n+1} = u^n + dt sum_j b_j k_j at every point.  Every slope system's interface rows carry
 * -1/dt times the flux jump of u^n (the penalization of Sec. 3.1), so u^{n+1} has no flux jump.
 * terms->q: 6 x N_int stage sources or NULL; terms->f: 6 x N_bd slope boundary data, i.e. u_t at
 * t + c_i dt on the boundary, or NULL for zero (time-independent Dirichlet data).  With a preset g
 * (terms->g_kind, eq. slope) explicit slopes l_i = g(U_i) join the k_i (U_i = u^n + dt sum_{j<=i}
 * a_ij k_j + dt sum_{j<i} ahat_ij l_j at every point), dt sum_j ahat_ij L l_j enters every slope
 * system and u^{n+1} = u^n + dt sum_j b_j (k_j + l_j); each l_i takes g at the interior points, its
 * shared-edge values from the identity-operator system and zero boundary values, so only
 * time-independent Dirichlet data are accepted (terms->f must be NULL, else HPS_EINVAL).
 * HPS_G_USER is rejected.  Needs at least two leaves and the per-level merge kernels (not
 * hps_set_persistent); the first call allocates 7 N doubles of work memory (with g 7 N + 7 N_int
 * more). */
int ark_slope_step(hps_handle *h, double *u, double t, double dt, const hps_ark_terms *terms, hps_stream_t stream);

/* ark_slope_step on R states at once in mixed precision (u: N x R in place; terms->q: 6 x N_int x R
 * stage sources, terms->f: 6 x N_bd x R slope boundary data (u_t), both stage-major, or NULL;
 * g_kind HPS_G_NONE or a preset, as for ark_slope_step: with g terms->f must be NULL and the first
 * such call allocates (7 N + 6 N_int) x Rmax doubles more): every slope system by FP32 sweeps with `refine` FP64 refinement sweeps
 * against its collocation residual, interface rows included (their right-hand side is the
 * penalization's -(flux jump of u^n), carried by the first sweep and by every residual).  Needs
 * hps_batch_reserve(R) with one column group, at least two leaves; the first call allocates
 * (7 N + N_bd) x Rmax doubles of slopes.  Agrees with ark_slope_step column by column to the
 * mixed-precision tolerance (1e-10 with refine = 2 on the tested problems; one sweep leaves about
 * 1e-10 relative to a state whose flux jumps have decayed). */
int ark_slope_step_batch(hps_handle *h, int R, double *u, double t, double dt, const hps_ark_terms *terms, int refine,
                         hps_stream_t stream);

/* ark_step / ark_step_batch on states held in HOST memory: u_host (N, resp. N x R doubles,
 * page-locked for asynchronous copies) is copied into a device buffer the handle keeps, stepped
 * and copied back, all in order on `stream`; terms are device pointers as above.  The first call
 * allocates the device buffer (N x Rmax doubles for the batched form, Rmax from
 * hps_batch_reserve); u_host holds the new states once `stream` has reached the end of the call. */
int ark_step_host(hps_handle *h, double *u_host, double t, double dt, const hps_ark_terms *terms,
                  hps_stream_t stream);
int ark_step_batch_host(hps_handle *h, int R, double *u_host, double t, double dt, const hps_ark_terms *terms,
                        int refine, hps_stream_t stream);

/* ---- Many instances ------------------------------------------------------------------------
 * n independent instances (handles with their own trees, p and coefficients, each reserved with
 * hps_batch_reserve for its column count) advanced together: one call runs every instance's
 * batched mixed-precision ARK step (ark_step_batch) on an internal stream forked from `stream`
 * and joined back into it, so the per-level kernels of different instances share the GPU.  With
 * hps_multi_set_graph(m, 1) the whole multi-instance step is recorded into one CUDA graph on the
 * second call with equal arguments (every instance a branch) and replayed: one graph launch per
 * step for all instances (the instances' own graph replay is switched off).  u[i]: device state of
 * instance i, N_i x R[i] RHS-fastest; terms: n entries (or NULL: no q, f, g); dt must match every
 * handle's gamma_dt (dt = 4 gamma_dt).  The handles must outlive the object and must not be used
 * on other streams while a step runs.  The instances' launches run concurrently inside one graph.
 * hps_multi_set_lockstep(m, 1) (every handle with one column group; HPS_EINVAL otherwise) fuses
 * the instances' merges instead: each FP32 sweep runs every instance's leaf part on its stream,
 * then one launch per tree level and merge operator for all instances together (upward levels
 * counted from each tree's leaves, downward from the roots), then the leaf parts again; the
 * residuals, epilogues and step close stay per instance.  Same results to the batched path's
 * tolerance (the FP32 sums of a merge split differently). */
typedef struct hps_multi hps_multi;
int hps_multi_create(hps_handle *const *handles, int n, hps_multi **out);
int hps_multi_set_graph(hps_multi *m, int enable);
int hps_multi_set_lockstep(hps_multi *m, int enable);
int hps_multi_ark_step(hps_multi *m, double *const *u, const int *R, const hps_ark_terms *terms, double dt, int refine,
                       hps_stream_t stream);
void hps_multi_free(hps_multi *m);

/* ---- Kernel variants and their autotuner --------------------------------------------------
 * Options select among kernel variants (all compute the same result to the path's tolerance:
 * 1e-10 for the batched mixed-precision path, 1e-12 for FP64).  Most belong to the batched path;
 * HPS_OPT_EDGE_PROJECTION and HPS_OPT_FP64_PLAN_TARGET also reach ark_step / hps_solve.  Setting
 * one drops the recorded graphs of the batched and FP64 calls and, for the split-K plan options
 * (HPS_OPT_FP64_PLAN_TARGET included), re-sizes the split-K scratch (synchronizes the device). */
enum {
  HPS_OPT_TENSOR_LEAF = 0,      /* 1: first sweep of a solve applies the shared leaf operator by
                                   3xTF32 warp MMA on the tensor cores (default 1)                */
  HPS_OPT_EVEN_ODD = 1,         /* 1: FP64 leaf kernels by the even-odd decomposition (default 1) */
  HPS_OPT_FLOW_LEVELS = 2,      /* lowest merge levels run as one dataflow kernel (default 0)     */
  HPS_OPT_FLOW_N3_MAX = 3,      /* ... levels whose interface has at most this many points (32)  */
  HPS_OPT_CLUSTER_SPLITK = 4,   /* 1: upper merge levels split K over a thread-block cluster and
                                   add the parts in distributed shared memory (default 0)        */
  HPS_OPT_PLAN_TARGET = 5,      /* split-K plans: CTAs per SM aimed at (default 2)                */
  HPS_OPT_PLAN_KMIN = 6,        /* split-K plans: smallest K chunk (default 32)                   */
  HPS_OPT_PLAN_NPC_MAX = 7,     /* split-K plans: most tree nodes per CTA (default unlimited)     */
  HPS_OPT_SPLIT_RHS = 8,        /* 1: stage right-hand side as its own pass (default 0)           */
  HPS_OPT_FP64_CTAS_PER_SM = 9, /* FP64 leaf kernels: persistent CTAs per SM, 0: one CTA per leaf  */
  HPS_OPT_GROUP_OFFSET = 10,    /* 1: column groups of an ARK step start one phase apart (1)     */
  HPS_OPT_LAST_CTA_SUM = 11,    /* split-K merge applies with at most this many chunks are summed
                                   by the last CTA of each tile, deeper ones by a reduction
                                   kernel (default 0: always the reduction kernel)                */
  HPS_OPT_FAST_DIAG = 12,       /* 1: constant-coefficient leaf solves by fast diagonalization
                                   (when the handle's 1-D operators have a real, well-conditioned
                                   eigen-decomposition; default 1)                                */
  HPS_OPT_PLAN_TILE_COLS = 13,  /* merge applies: columns per thread register tile, 8, 4 or 2 (2:
                                   more threads per level, the chain is latency-bound)            */
  HPS_OPT_FUSE_EPILOGUE = 14,   /* 1: the stage epilogue of a pointwise g (dt L U_i from the stage
                                   equation, dt (q_i + g(U_i))) is written by the last leaf kernel
                                   of the stage solve instead of its own pass (default 1)          */
  HPS_OPT_FUSE_JUMP = 15,       /* 1: the FP64 residual's flux jumps at shared edges come from the
                                   even-odd leaf kernel (side fluxes added into r) (default 1)     */
  HPS_OPT_FOLD_SCALE = 16,      /* 1: constant coefficients times gamma dt (or dt) folded into the
                                   even-odd half matrices (default 1)                              */
  HPS_OPT_SA_CLOSE = 17,        /* 1: the step close of the batched ARK step combines the last stage
                                   value and the explicit terms (b = last row of the implicit
                                   table), 7 instead of 13 terms (default 1)                       */
  HPS_OPT_EDGE_PROJECTION = 18, /* 1: the step close (batched and FP64 ARK steps; the identity
                                   operator of Sec. 3.1.1) solves for the
                                   shared-edge values directly: flux continuity with the given
                                   interior values is one tridiagonal system per grid line of
                                   shared edges (uniform leaves), in FP64; 0: identity-operator
                                   HPS solve with refinement (default 1)                          */
  HPS_OPT_EO_COLS = 19,         /* even-odd FP64 leaf kernels: columns per pass (default 12; shared
                                   memory grows with it)                                          */
  HPS_OPT_TILE_COLS_W3 = 20,    /* register-tile columns of the w3 applies (2, 4, 8; 0: PLAN_TILE_COLS) */
  HPS_OPT_TILE_COLS_H = 21,     /* ... of the h applies                                              */
  HPS_OPT_TILE_COLS_DOWN = 22,  /* ... of the u3 (downward) applies                                  */
  HPS_OPT_FP64_PLAN_TARGET = 23, /* FP64 path (hps_solve, ark_step): merge applies split their columns
                                   until this many CTAs per SM (1..8, default 3; not while the
                                   persistent merge kernel is on)                                  */
  HPS_OPT_UMMA_LEAF = 24,       /* 1: the first sweep of a solve applies PER-NODE leaf operators (variable
                                   coefficients, 32 <= q <= 256, 16 or 32 columns) on the 5th-generation
                                   tensor cores: tcgen05.mma kind::tf32 with 3xTF32 products and the
                                   accumulator in tensor memory, operator boxes streamed by TMA
                                   (default 1); 2: every sweep, the refinement sweeps included;
                                   3: BF16 trial -- the first sweep's leaf applies as ONE BF16
                                   product (kind::f16, BF16 operator copy made when set; q >= 64),
                                   refinement sweeps FP32 FFMA; 0: FP32 FFMA                        */
  HPS_OPT_ONE_COLUMN_MERGE = 25, /* 1: merge applies with ONE column and per-node operators stream the
                                   operator without shared-memory staging, K split over the warps
                                   of a CTA (default 1; 0: the general tiled applies)              */
  HPS_OPT_ONE_COLUMN_SUM = 26,   /* 1: their split-K partial sums added by the CTA that finishes a
                                   row block last, in chunk order (default 1; 0: a reduction
                                   launch)                                                          */
  HPS_OPT_STREAM_LEAF = 27,      /* c = 1..4: with one to four columns, the per-leaf operators of the
                                   leaf applies streamed through shared memory by 1-D bulk copies,
                                   c persistent CTAs per SM, fewer where c rings do not fit in shared
                                   memory (default 3; 0: one CTA per leaf)                          */
  HPS_OPT_STREAM_CHUNK_KB = 28,  /* their copies: whole operator columns of about this many KB
                                   (2..64, default 24)                                              */
  HPS_OPT_SUB_LEVELS = 29,       /* D = 2..6: the lowest D merge levels of every upward sweep in one
                                   launch, one CTA per (subtree, 8 columns), the h of the levels
                                   inside a subtree kept in shared memory (0: one launch per level
                                   and operator; default 0)                                         */
  HPS_OPT_PDL = 30,              /* 1: the merge applies and their split-K sums launched as
                                   programmatic dependents (griddepcontrol): each starts its
                                   operator loads while the kernel before it finishes and waits for
                                   its results in the kernel (0: ordinary launches)                */
  HPS_OPT_EO_THREADS = 31,       /* threads per CTA of the FP64 even-odd leaf kernel (residual,
                                   evaluation): 32..256 in steps of 32; 0 (default): 128 with one
                                   column per pass, else 256                                        */
  HPS_OPT_PREFETCH_NEXT = 32,    /* 1: each merge apply of an FP32 sweep prefetches the operator
                                   of the apply after it into L2 (bulk prefetch), so that the
                                   chain of dependent level applies finds it there (0: off)        */
  HPS_OPT_B1_ROLL = 33,          /* 1: the one-column merge applies reload each operator register as
                                   soon as its product is taken (a rolling window of loads in
                                   flight); 0: batches of loads, each waited for whole            */
  HPS_OPT_B1_KW = 34,            /* most warps that split K inside a CTA of the one-column merge
                                   applies (1, 2, 4 or 8; fewer: longer contiguous operator rows per
                                   CTA)                                                          */
  HPS_OPT_STREAM_PREFETCH = 35,  /* 1 (default): the streaming downward leaf apply loads the next
                                   leaf's boundary values and this leaf's w into registers while it
                                   takes this leaf's products, and with one column sums the K slices
                                   straight into u (two consumer barriers per leaf instead of four);
                                   0: loads and sums per leaf in separate phases                   */
  HPS_OPT_COUNT = 36
};
int hps_batch_set_option(hps_handle *h, int opt, int value);

/* Host-only check of the fast diagonalization for constant coefficients coef = (a11, a22, a1,
 * a2, a0), gamma dt and leaf widths hx, hy (Sec. 4.2: the leaf interior operator is a Kronecker
 * sum of 1-D Chebyshev operators): factors A_ii^-1 = (V_y (x) V_x) Lam (V_y^-1 (x) V_x^-1) and
 * reports *max_err = max over all unit vectors e of |A_ii F e - e|.  HPS_OK when the factors
 * exist and max_err <= 1e-12 (then hps_build uses them), HPS_EINVAL when a 1-D operator has no
 * real, well-conditioned eigen-decomposition.  Needs no GPU. */
int hps_fastdiag_check(int p, const double *coef, double gamma_dt, double hx, double hy, double *max_err);
int hps_batch_get_option(hps_handle *h, int opt, int *value);

/* One configuration tried by hps_batch_autotune and its time. */
typedef struct hps_tune_result {
  int tile_cols, flow_levels, plan_target, plan_kmin;
  float ms; /* device time of one hps_solve_batch with this configuration (mean of 3) */
} hps_tune_result;

/* Times hps_solve_batch (R columns, `refine` sweeps, synthetic right-hand sides) under each
 * candidate configuration (merge tile columns x dataflow levels x split-K plan) of the options
 * above on this handle's own operators, keeps the fastest and reports every candidate in `results` (up to max_results, count in *n_results;
 * either may be NULL).  Needs hps_batch_reserve(R) first; allocates and frees its own test
 * vectors; synchronizes the device. */
int hps_batch_autotune(hps_handle *h, int R, int refine, hps_stream_t stream, hps_tune_result *results,
                       int max_results, int *n_results);

/* ---- Serving: a continuous-batching request loop for time-stepping jobs -------------------
 * Jobs arrive at given times; the loop admits a waiting job (in arrival order) as soon as an
 * active slot is free and the device-memory budget holds its factorization -- unless one of an
 * identical operator (tree, p, coefficients, dt) is resident, which is then shared -- plus its
 * work buffers and state.  Every active job advances one ark_step at a time (graph replay) on
 * its own CUDA stream with up to two steps queued, so steps of different jobs overlap on the
 * GPU and newly admitted jobs join while others run.  A finished job copies its state to
 * u_out and releases its memory; factorizations without users stay cached until the budget
 * needs their memory.  Results are the same whether a job runs alone or in a mix (the same
 * kernels on the same data; no reduction order depends on other jobs). */
typedef struct hps_server hps_server;

/* Sources and boundary data of a served job's next step (eq. stage2: q and f at the stage times
 * t_j = t + c_j dt, c_j from hps_ark_abscissae): the callback fills q (device, 6 x N_int doubles,
 * stage-major, q(t_j) at the interior points in global interior order) and f (device, 6 x N_bd
 * doubles, stage-major, f(t_j) in boundary order; entry 6, c_6 = 1, is also the boundary value of
 * u^{n+1}) for the step that starts at t.  Every write must be ordered on `stream` (kernels or
 * asynchronous copies enqueued there): the server enqueues the step after the callback returns,
 * and the next fill of the same buffers only after that step.  It runs on the thread of
 * hps_server_run and returns 0, or an error code that ends the job (its status). */
typedef int (*hps_terms_fn)(void *user, double t, double dt, double *q, double *f, hps_stream_t stream);

typedef struct hps_job_desc {
  hps_tree tree;
  int p;
  double c_a11, c_a22, c_a1, c_a2, c_a0; /* constant coefficients of L (when a11 .. a0 are all NULL) */
  double dt, t0;                          /* step and start time (gamma dt = dt / 4) */
  int steps;
  int g_kind;                             /* HPS_G_* preset */
  double g_param[2];
  const double *u0;                       /* host, N doubles; valid until hps_server_run returns */
  double *u_out;                          /* host, N doubles, written when the job finishes */
  double arrival_s;                       /* seconds after hps_server_run starts */
  /* Nodal coefficients: host arrays of N_int values at the interior points (global interior
   * order), NULL for a coefficient that is zero; when any is non-NULL they replace c_a11 .. c_a0.
   * Valid until hps_server_run returns.  Jobs whose arrays hold the same values (compared entry
   * by entry) share one factorization. */
  const double *a11, *a22, *a1, *a2, *a0;
  hps_terms_fn terms;                     /* NULL: q = 0 and f = 0 */
  void *terms_user;                       /* passed to terms */
} hps_job_desc;

typedef struct hps_job_stats {
  int state;             /* 0 waiting, 1 active, 2 done, 3 rejected */
  int status;            /* HPS_OK or the error that ended it (HPS_ENOMEM: larger than the budget) */
  double arrival_s, admit_s, finish_s;
  int steps_done;
  int shared_operators;  /* 1 if it used a factorization built for an earlier job */
  size_t work_bytes;
  double step_ms_mean, step_ms_p50, step_ms_p99; /* device time of its steps (CUDA events) */
  int evictions;         /* times it was checkpointed to host memory and queued again */
} hps_job_stats;

typedef struct hps_server_stats {
  int jobs_done, jobs_rejected;
  double makespan_s;         /* wall time of hps_server_run */
  double dof_stages_per_s;   /* sum over jobs of N x 5 x steps, divided by the makespan */
  int64_t steps;
  double step_ms_p50, step_ms_p99;
  int max_concurrent;
  size_t peak_bytes;
  int factorizations_built, factorizations_shared;
  int batches_formed;        /* batching on: batches created */
  double mean_batch_cols;    /* batching on: members per batched step, averaged over the steps */
} hps_server_stats;

/* A server with a device-memory budget (bytes, for factorizations + work buffers + states)
 * and at most max_active jobs in flight. */
int hps_server_create(size_t mem_budget_bytes, int max_active, hps_server **out);
/* Batching (continuous batching at the kernel level): with max_cols >= 1 (<= 64), jobs whose
 * steps are the same operation -- identical operator (tree, p, coefficients, dt) and identical
 * g -- advance as the columns of one state by ark_step_batch (FP32 sweeps + `refine` FP64
 * refinement sweeps per implicit solve; refine = -1: chosen per operation from its stiffness
 * gamma dt max(a11/hx^2, a22/hy^2) 4 * 0.047 (p-1)^4 -- 1 up to 1e5, one more per factor 100)
 * on a stream of their own, at most max_cols jobs per batch;
 * R = the member count rounded up to 4.  An arriving job joins a running batch of its operation
 * with a free column at that batch's next step boundary (the batch lets its queued steps finish,
 * then repacks its columns), else starts a new batch (its memory -- handle reserved for max_cols
 * columns, two N x max_cols states -- measured against the budget).  A job's result then agrees
 * with its FP64 ark_step result to the mixed-precision tolerance (1e-10) and with its result in
 * another mix to rounding (the split of the FP32 merge sums follows R).  max_cols = 0 (default):
 * every job steps on its own with the FP64 ark_step, results bit-identical alone and in a mix.
 * Jobs with a terms callback share batches only with other jobs that have one: before each
 * batched step every member's callback fills a staging pair, copied into its column of the
 * batch's 6 x N_int x R and 6 x N_bd x R arrays.  For nodal coefficients the stiffness takes the
 * largest |a11|, |a22| over the points. */
int hps_server_set_batching(hps_server *s, int max_cols, int refine);
/* Queue a job; *job_id (may be NULL) receives its index. */
int hps_server_submit(hps_server *s, const hps_job_desc *job, int *job_id);
/* Eviction with checkpoint / resume: once job `job_id` has run `steps` steps (none in flight) its
 * state u and step count -- hence its time t0 + steps dt -- are copied to host memory, its device
 * memory and slot (or batch column) are released and it queues again behind the jobs waiting at
 * that moment; re-admitted, it continues from the checkpoint.  Set before hps_server_run; at most
 * one eviction per job.  Without batching the resumed job's result is bit-identical to an
 * uninterrupted run (the same kernels on the same data); with batching it agrees to the
 * mixed-precision tolerance. */
int hps_server_evict_after(hps_server *s, int job_id, int steps);
/* Run until every queued job is done or rejected (blocks; honours arrival times from now). */
int hps_server_run(hps_server *s);
int hps_server_job_stats(hps_server *s, int job_id, hps_job_stats *out);
int hps_server_summary(hps_server *s, hps_server_stats *out);
void hps_server_free(hps_server *s);

/* Release the handle and all its device memory (synchronizes the device first). */
void hps_free(hps_handle *h);

/* Static description of an error code. */
const char *hps_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HPS_H */
