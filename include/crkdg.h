/*
 * crkdg.h -- C ABI of the GB300 (sm_103a) bound-preserving compact-stencil
 * Runge--Kutta discontinuous Galerkin library (cRKDG; Liu, Sun and Zhang,
 * "A bound-preserving Runge--Kutta discontinuous Galerkin method with compact
 * stencils for hyperbolic conservation laws", arXiv 2412.16002).
 *
 * What one step computes (Scheme 1L, Appendix B.2, eq. rkdg-lim):
 *     u^(1) = u~^n
 *     u^(i) = u~^n + dt sum_{j<i} a_ij G(u~^(j)),  u~^(i) = L(u^(i)),  i = 2..s
 *     u^{n+1} = u~^n + dt sum_i b_i F(u~^(i)),    u~^{n+1} = L(u^{n+1})
 * with G = -div^loc f (interior traces on every edge, Sec. 2.1), F = -div^DG f
 * with the Lax--Friedrichs flux (eq. dxDG), and L the Zhang--Shu scaling limiter
 * (Prop. 2.4 for scalar laws, eq. Euler-limiter1/2 for the Euler equations).
 * If any stage's cell averages leave B (B^eps for Euler) the step is redone
 * from u~^n with dt halved (Sec. 4.1, Algorithm).
 *
 * Discretisation: uniform Cartesian mesh (1D or 2D), tensor-product Q^k basis
 * (k = 1..3), nodal at the (k+1)^d tensor Gauss points; (k+1)-point Gauss on
 * every edge (Prop. 2.1); the limiter point set S_K is the union of the
 * Gauss x Gauss-Lobatto and Gauss-Lobatto x Gauss points (Prop. 2.2, Fig. 1)
 * with L = ceil((k+3)/2) Gauss-Lobatto points.
 *
 * Conventions for every entry point:
 *   - State layout: FP64 nodal values, component-major:
 *       1D  [m][nx][n]            2D  [m][ny][nx][n_y][n_x],  n = k+1,
 *     count = m * nx * ny * n^dim doubles.  m = 1 (advection, Burgers),
 *     3 (1D Euler: rho, m, E), 4 (2D Euler: rho, m_x, m_y, E).
 *   - Pointers are host pointers unless an argument says "device"; an
 *     on_device flag selects which for state transfers.  The caller keeps
 *     ownership of everything it passes; the library copies and owns its own
 *     device buffers, which live until crkdg_destroy.
 *   - Work is issued on options.cuda_stream (NULL = legacy default stream);
 *     calls that return host data synchronise that stream.
 *   - Every call returns a crkdg_status; no C++ exception crosses the ABI.
 *     crkdg_last_error(h) describes the last failure on that handle.  A handle
 *     is not thread-safe: calls on one handle must not overlap.
 */
#ifndef CRKDG_H
#define CRKDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crkdg_ctx *crkdg_t;

typedef enum {
    CRKDG_OK = 0,
    CRKDG_E_ARG = 1,         /* invalid argument (sizes, kinds, tableau, NULL) */
    CRKDG_E_CUDA = 2,        /* a CUDA runtime call failed; see crkdg_last_error */
    CRKDG_E_OOM = 3,         /* device allocation failed */
    CRKDG_E_BOUNDS = 4,      /* averages left B after max_halvings; state unchanged */
    CRKDG_E_TIMEOUT = 5,     /* a bounded device-side wait expired */
    CRKDG_E_UNSUPPORTED = 6  /* valid but not built (e.g. k > 3) */
} crkdg_status;

enum { CRKDG_BC_PERIODIC = 0, CRKDG_BC_OUTFLOW = 1, CRKDG_BC_REFLECT = 2, CRKDG_BC_DIRICHLET = 3 };
enum { CRKDG_FLUX_ADVECTION = 0, CRKDG_FLUX_BURGERS = 1, CRKDG_FLUX_EULER = 2 };
enum { CRKDG_PREC_FP64 = 0, CRKDG_PREC_MIXED = 1 };
enum { CRKDG_IND_OFF = 0, CRKDG_IND_TVB = 1, CRKDG_IND_MLP = 2 };
enum { CRKDG_SCHEME_COMPACT = 0, CRKDG_SCHEME_STANDARD = 1 };
enum { CRKDG_THETA2_RATIO = 0, CRKDG_THETA2_EXACT = 1 };
enum { CRKDG_SOURCE_NONE = 0, CRKDG_SOURCE_SCENARIO1 = 1 };
enum { CRKDG_BASIS_Q = 0, CRKDG_BASIS_P = 1 };

/* Mesh: the domain [x0,x1] (x [y0,y1] in 2D) cut into nx (x ny) equal cells.
 * bc[s] for the sides s = 0 left, 1 right, 2 bottom, 3 top; a periodic side
 * must be paired with a periodic opposite side.  bc_state[s] holds the
 * conservative exterior state of a Dirichlet side.  Boundary data enter only
 * the final stage (compactness, Sec. 1 and the Compactness remark of Sec. 3.2):
 * the exterior trace at a face point is the Dirichlet state, the interior trace
 * with the normal momentum negated (reflect), or the cell average of the same
 * stage value (outflow; a constant state is kept exactly and the Lax--Friedrichs
 * flux keeps its dissipation on outflow faces). */
typedef struct {
    int dim;
    int nx, ny;
    double x0, x1, y0, y1;
    int bc[4];
    double bc_state[4][4];
} crkdg_mesh;

/* Flux f of eq. (claws): kind ADVECTION f = a u (velocity a), BURGERS
 * f = u^2/2 in every direction, EULER eq. (Euler), (Euler-2) with gamma. */
typedef struct {
    int kind;
    double gamma;
    double velocity[2];
} crkdg_flux;

/* Invariant region: scalar B = [lo, hi] (eq. scalar-bound); Euler B^eps with
 * rho >= eps and rho e >= eps (Sec. 2.2.2, eq. Euler-limiter2). */
typedef struct {
    double lo, hi;
    double eps;
} crkdg_bounds;

/* Butcher tableau (eq. butcher): A is s*s row-major, strictly lower triangular,
 * b has s entries, all >= 0 (Sec. 3.3).  s <= 4.  Host pointers. */
typedef struct {
    int s;
    const double *A;
    const double *b;
} crkdg_tableau;

/* Precision.  CRKDG_PREC_FP64: every operation in FP64.  CRKDG_PREC_MIXED: the
 * state is kept as FP64 cell averages plus FP32 nodal deviations; every operator
 * (flux, volume term, traces, Lax--Friedrichs flux, lift) is evaluated in FP32,
 * while the cell-average updates (FP64 sums of the face fluxes, so conservation
 * holds to FP64 round-off), the admissibility test of the averages, the limiter's
 * theta (FP32-screened with a rigorous rounding margin, FP64 where the screen
 * cannot clear a cell) and the time step stay FP64.  Bounds are exact under the
 * FP64 evaluation ubar + (double)(FP32 interpolation of the deviations). */
/* Troubled-cell indicator (optional; the paper applies no anti-oscillation
 * limiter, Sec. 4).  CRKDG_IND_TVB: once per step, after the final stage and
 * before the scaling limiter (so inner stages stay compact), every cell whose
 * face-averaged trace deviations a TVB-modified minmod (threshold tvb_M h^2, per
 * conservative component and direction, against the differences of the
 * neighbouring averages) would change is replaced by its average plus minmod-
 * limited first Legendre moments; averages are kept, and the scaling limiter
 * follows unchanged.  Euler, FP64 path. */
typedef struct {
    int precision;      /* CRKDG_PREC_FP64 (default) or CRKDG_PREC_MIXED */
    int max_halvings;   /* restart cap of the Sec. 4.1 loop (default 20) */
    int indicator;      /* CRKDG_IND_* troubled-cell indicator (default off) */
    double tvb_M;       /* TVB constant of the plain indicator (default 10) */
    void *cuda_stream;  /* cudaStream_t to issue work on (NULL: default stream) */
    int scheme;         /* CRKDG_SCHEME_COMPACT (default): the compact scheme above.
                           CRKDG_SCHEME_STANDARD: the standard RKDG in Butcher form (eq. rkdg,
                           Sec. 2.1), u^(i) = u~^n + dt sum_{j<i} a_ij F(u~^(j)), i.e. F (with
                           its neighbour exchange) in every stage, the same scaling limiter
                           and restart rule; for comparison with the compact scheme.  FP64
                           precision, no indicator (CRKDG_E_UNSUPPORTED otherwise). */
    int theta2;         /* theta_2 of the Euler scaling limiter.  CRKDG_THETA2_RATIO (default):
                           the concavity ratio of eq. (Euler-limiter2), (rho e(ubar) - eps) /
                           (rho e(ubar) - min_q rho e(u_q)).  CRKDG_THETA2_EXACT: for every S_K
                           point q with rho e(u_q) < eps the t in (0, 1) where
                           rho e(ubar + t (u_q - ubar)) = eps, a root of a quadratic in t (rho,
                           m, E are linear in t), and theta_2 = min_q t_q: the least scaling
                           that restores the bound (the per-point solve of the positivity-limiter
                           works the text after eq. Euler-limiter2 refers to).  The
                           same safety margin and verification follow.  FP64 precision
                           (CRKDG_E_UNSUPPORTED otherwise). */
    int source;         /* CRKDG_SOURCE_NONE (default), or CRKDG_SOURCE_SCENARIO1: the source of
                           the manufactured solution of Example 4.2's scenario I (Sec. 4.2),
                           S = d_t U + d_x F(U) + d_y G(U) for rho = e^-t sin 2pi(x+y) + 2,
                           w = (e^-t cos 2pi x sin 2pi y + 2, e^-t sin 2pi x cos 2pi y + 2),
                           e = e^-t cos 2pi(x+y)/2 + 1 (e the specific internal energy), added
                           to the DG operator at every stage at the stage time t + c_i dt
                           (c_i = sum_j a_ij; t: crkdg_set_time, advanced by each accepted
                           step).  For accuracy tests (Table 2): 2D Euler, FP64, the compact
                           scheme, no indicator (CRKDG_E_UNSUPPORTED otherwise). */
    int basis;          /* the DG space: CRKDG_BASIS_Q (default), the tensor-product Q^k, or
                           CRKDG_BASIS_P, the total-degree P^k (Sec. 4.2 reports both).  The
                           state keeps the nodal layout at the (k+1)^2 Gauss points and lies in
                           P^k: every stage value, u* and u^{n+1} (and the state crkdg_set_state
                           receives) is L2-projected onto P^k before the limiter; the Legendre
                           modes L_i(x) L_j(y) being orthogonal, that is the P^k Galerkin
                           scheme with the same quadrature.  In 1D the spaces coincide.  2D:
                           FP64, the compact scheme, no indicator (CRKDG_E_UNSUPPORTED
                           otherwise). */
} crkdg_options;

typedef struct {
    double dt_taken;          /* dt of the accepted attempt */
    int restarts;             /* halvings before acceptance */
    long long cells_limited;  /* cells with theta < 1 over all stages of the accepted attempt */
    double theta_min;         /* smallest theta of the accepted attempt */
    long long troubled;       /* cells flagged by the indicator (0 if off) */
    double mass_drift;        /* (M^{n+1} - M^n) / |M^n| for the first component's total
                                 M = sum_K |K| ubar_K (mass, or the scalar), summed on the
                                 device in a fixed order: the conservation error of the step
                                 (round-off) when no side lets mass in or out (periodic,
                                 reflect); with open sides it also holds the net boundary
                                 inflow of the step.  Ensembles report 0. */
} crkdg_step_info;

/* Fill *opt with the defaults. */
void crkdg_options_default(crkdg_options *opt);

/* Create a solver.  k: polynomial degree 1..3; m must match the flux kind and
 * dim (see the state layout above).  opt may be NULL (defaults).  On success
 * *out receives a handle.  Errors: CRKDG_E_ARG (also for meshes of more than
 * 2e9 cells, or whose cells times face points per cell, 2 d (k+1)^(d-1), reach
 * 2^32 - 1), CRKDG_E_UNSUPPORTED, CRKDG_E_OOM, CRKDG_E_CUDA (no handle is
 * returned). */
crkdg_status crkdg_create(const crkdg_mesh *mesh, int k, int m, const crkdg_flux *flux,
                          const crkdg_bounds *bounds, const crkdg_options *opt, crkdg_t *out);

/* Release every device buffer of h.  h may be NULL. */
crkdg_status crkdg_destroy(crkdg_t h);

/* Copy count doubles of nodal state in (host or device pointer) and apply the
 * scaling limiter once, so that u^n lies in B on every S_K (the hypothesis of
 * Theorem 3.5).  count must equal the state size.  The split-precision path
 * reads a device buffer, or page-locked host memory (cudaHostAlloc,
 * cudaHostRegister), in place with the kernel that splits it; pageable host
 * memory is staged by a copy.  The buffer is not read after the call returns. */
crkdg_status crkdg_set_state(crkdg_t h, const double *nodal, size_t count, int on_device);

/* Copy the current nodal state out (host or device pointer).  The
 * split-precision path writes a device buffer or page-locked host memory in
 * place with the kernel that merges the state; the call returns when the
 * state is there. */
crkdg_status crkdg_get_state(crkdg_t h, double *nodal, size_t count, int on_device);

/* The time of the current state: 0 for a new handle, set by crkdg_set_time (or by the t of
 * crkdg_advance / crkdg_advance_fixed), increased by the dt of every accepted step.  Only a
 * time-dependent source (crkdg_options.source) and the moving shock boundary of a
 * non-rectangular domain (crkdg_set_geometry) read it. */
crkdg_status crkdg_set_time(crkdg_t h, double t);
crkdg_status crkdg_get_time(crkdg_t h, double *t);

/* Trial step of eq. (numerical_experiment:CFL), *dt = cfl * dx / a0, written for
 * Cartesian meshes as *dt = cfl / max_{S_K} sum_d lambda_d / h_d, where
 * lambda_d = |w_d| + c (|u| for Burgers, |a_d| for advection) is the spectral
 * radius in direction d at an S_K point of the current state and h_d the cell
 * size (in 1D exactly cfl*dx/a0; in 2D the form under which the stability CFL
 * numbers of the Remark in Sec. 3.2 keep the scheme linearly stable). */
crkdg_status crkdg_max_dt(crkdg_t h, double cfl, double *dt);

/* One limited cRKDG step of size dt (restarting with dt/2 while any stage's
 * averages leave B, at most max_halvings times).  info may be NULL.
 * CRKDG_E_BOUNDS leaves the state at u^n. */
crkdg_status crkdg_step(crkdg_t h, double dt, const crkdg_tableau *tab, crkdg_step_info *info);

/* Run up to nsteps steps, each of size min(trial step of crkdg_max_dt, t_end - *t),
 * advancing *t; stops early when *t reaches t_end.  *steps_done (nullable)
 * receives the number of accepted steps and *restarts (nullable) the total
 * halvings.  On 1D meshes the whole loop (steps, restarts, trial steps) runs in
 * one persistent cooperative kernel launch with one grid-wide barrier per
 * attempt; CRKDG_E_TIMEOUT reports an expired barrier wait (2 s bound) and
 * CRKDG_E_BOUNDS leaves the state at the last accepted step. */
crkdg_status crkdg_advance(crkdg_t h, int nsteps, double cfl, double t_end,
                           const crkdg_tableau *tab, double *t, int *steps_done, int *restarts);

/* As crkdg_advance with the fixed trial step dt for every step (the step is
 * still halved and redone while a stage's averages leave B; the next step
 * starts again from dt), as in the convergence tests of Sec. 4.2. */
crkdg_status crkdg_advance_fixed(crkdg_t h, int nsteps, double dt, double t_end, const crkdg_tableau *tab,
                                 double *t, int *steps_done, int *restarts);

/* Operator evaluation on device arrays in the state layout, for verification:
 * op 0: out = G(in) (Sec. 2.1), op 1: out = F(in) (eq. dxDG; boundary data at
 * the mesh's BCs), op 2: out = L(in) (the scaling limiter, no admissibility
 * test).  in and out are device pointers of state size; they may not alias. */
enum { CRKDG_OP_G = 0, CRKDG_OP_F = 1, CRKDG_OP_LIMIT = 2 };
crkdg_status crkdg_apply_operator(crkdg_t h, int op, const double *in_dev, double *out_dev);

/* Troubled-cell flags of the last accepted step (one int per cell, row-major
 * [ny][nx]; host or device pointer).  CRKDG_E_ARG if the indicator is off. */
crkdg_status crkdg_troubled_flags(crkdg_t h, int *flags, int on_device);

/* ------------------------------------------------------------------------
 * Learned troubled-cell indicator (CRKDG_IND_MLP; not part of the paper).  A
 * 44 -> 64 -> 64 -> 1 ReLU network with a sigmoid output classifies a cell from
 * its features (2D Euler; layout [cell][44]): per conservative component the
 * 3x3 neighbourhood of cell averages minus their mean, over den = max(range,
 * tvb_M hx hy) + 1e-6 max|v| (36 values, [comp][row-major 3x3]), then the cell's
 * first Legendre moments c_10, c_01 over the same den (8 values, [comp][x,y]).
 * Stencil positions outside the domain take the nearest interior cell's average
 * with the crossed sides' boundary states applied.  A cell is troubled when the
 * probability exceeds 0.6, smooth below 0.4, and takes the plain TVB decision in
 * between; the shock limiter and the scaling limiter then act as for the plain
 * indicator.  Parameters are FP32, layout W1[64][44], b1[64], W2[64][64], b2[64],
 * w3[64], b3 (CRKDG_MLP_NPARAM floats).  All pointers below are device pointers. */
#define CRKDG_MLP_NIN 44
#define CRKDG_MLP_NH 64
#define CRKDG_MLP_NPARAM 7105

/* prob[r] = network(X[r]) for the n rows of X ([n][44]); enqueued on stream.  X must be
 * 16-byte aligned (tiles of 128 rows are moved by bulk asynchronous copies, which need
 * 16-byte aligned addresses; CRKDG_E_ARG otherwise).  The two hidden layers run on the
 * tensor cores with the three-product TF32 split (FP32 accuracy).  If a wait for the
 * tensor cores or for a tile's copy runs out (1 s), the affected probabilities are NaN
 * or unwritten (the learned rule leaves NaN cells to the plain decision) and
 * crkdg_mlp_fault reports it. */
crkdg_status crkdg_mlp_forward(const float *params, const float *X, int n, float *prob, void *stream);
/* *fault = 1 if a crkdg_mlp_forward launch since the last call ran out of time waiting
 * for the tensor cores, else 0; clears the record (synchronises the device). */
crkdg_status crkdg_mlp_fault(int *fault);
/* grad += d loss / d params and *loss += loss, for the mean binary cross-entropy
 * of the n labelled rows (y in {0,1}); the caller zeroes grad and loss. */
crkdg_status crkdg_mlp_grad(const float *params, const float *X, const float *y, int n, float *grad, float *loss,
                            void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8); step is the 1-based count. */
crkdg_status crkdg_mlp_adam(float *params, float *m, float *v, const float *grad, int step, float lr, void *stream);

/* Copy the network the CRKDG_IND_MLP indicator of h uses (params: device). */
crkdg_status crkdg_set_mlp(crkdg_t h, const float *params);
/* While on (indicator on), every step also keeps the features of the unlimited
 * final-stage state on which its indicator decided; crkdg_last_features copies
 * them ([ny][nx][44] floats), matching crkdg_troubled_flags of the same step. */
crkdg_status crkdg_set_harvest(crkdg_t h, int on);
crkdg_status crkdg_last_features(crkdg_t h, float *feat, int on_device);

/* Cell averages of the current state, [ny][nx][m] doubles (host or device). */
crkdg_status crkdg_cell_averages(crkdg_t h, double *avg, int on_device);

/* Smallest bound margins over every S_K point of the current state, evaluated
 * by the limiter's own interpolation: scalar {min(u-lo), min(hi-u)}, Euler
 * {min(rho-eps), min(rho e - eps)}.  Both are >= 0 after every step. */
crkdg_status crkdg_bound_margins(crkdg_t h, double margins[2]);

/* sum_K |K| ubar_K of component comp, summed in a fixed order (deterministic). */
crkdg_status crkdg_total_mass(crkdg_t h, int comp, double *mass);

/* Kernel timing for measurement.  While on, crkdg_step brackets its
 * inner-stage and final-stage launches, and crkdg_advance on 1D meshes its
 * persistent step-loop launch, with CUDA events on the library's stream and
 * accumulates their durations; crkdg_kernel_times returns the milliseconds
 * {inner, final, step loop} and the launch counts since profiling was last
 * switched on.  Off by default; switching on resets the totals. */
crkdg_status crkdg_set_profiling(crkdg_t h, int on);
crkdg_status crkdg_kernel_times(crkdg_t h, double ms[3], long long launches[3]);

/* Testing aid for the failure path of the device-resident loop: with extra > 0
 * the grid barrier of crkdg_advance (1D) waits for `extra` blocks that never
 * arrive, so every block's bounded wait expires after 2 s and the call returns
 * CRKDG_E_TIMEOUT with the state at the last accepted step (nothing faults or
 * hangs).  0 (the default) restores normal operation. */
crkdg_status crkdg_set_barrier_test(crkdg_t h, int extra);

/* Tuning of the 1D device-resident loop: the own cells of one block's chunk (1..30;
 * each chunk also recomputes one halo cell per side).  0 (the default) takes 30, the
 * fastest measured size.  Results do not depend on it (every cell's arithmetic is the
 * same); only the time does. */
crkdg_status crkdg_set_run1d_chunk(crkdg_t h, int cells);

/* Split precision (CRKDG_PREC_MIXED), 2D Euler, k = 3: the inner stages run on the
 * tensor cores (tcgen05.mma kind::tf32 with the three-product split, FP32-level
 * accuracy) for tableaux whose A has only a sub-diagonal (eq. cRKDG2-4); on = 0
 * runs them on the CUDA cores instead (both keep FP64 where the split path does;
 * they differ by FP32 rounding).  On by default; other cases always use the CUDA
 * cores.  A wait for the tensor cores that runs out (1 s) makes crkdg_step return
 * CRKDG_E_TIMEOUT with the state at u^n. */
crkdg_status crkdg_set_tensor_cores(crkdg_t h, int on);

/* Number of doubles of the state. */
size_t crkdg_state_size(crkdg_t h);

/* ------------------------------------------------------------------------
 * One step in two calls, for callers that decide acceptance across several
 * handles (the subdomains of a decomposed mesh, below).  crkdg_step_attempt runs
 * one attempt of size dt from u^n (no restart) and sets *violated to 1 if a
 * stage's cell averages left B (Sec. 4.1 test), else 0; u^n is kept.
 * crkdg_step_accept makes that attempt's result the new state (CRKDG_E_ARG if
 * there is no attempt or it violated); info as for crkdg_step (restarts 0).
 * To restart, call crkdg_step_attempt again with dt/2: crkdg_step is exactly
 * this loop on one handle. */
crkdg_status crkdg_step_attempt(crkdg_t h, double dt, const crkdg_tableau *tab, int *violated);
crkdg_status crkdg_step_accept(crkdg_t h, crkdg_step_info *info);

/* ------------------------------------------------------------------------
 * Non-rectangular domains (Sec. 4.4, Examples 4.8 and 4.9: the shock diffraction
 * on [0,1]x[6,12] U [1,13]x[0,12] and the double Mach reflection on
 * [1,4]x[-1,0] U [0,4]x[0,1]).  The domain is a union of the mesh's cells: the
 * cells of the bounding rectangle outside it are solid.  geo holds one word per
 * cell (host memory, cell order cy * nx + cx, copied into device memory owned
 * by h): bits 4s..4s+3 the boundary kind of side s (0 left, 1 right, 2 bottom,
 * 3 top), bit 16 (CRKDG_GEO_SOLID) a solid cell.  Kinds:
 *   CRKDG_GEO_MESH     the mesh rule: the neighbouring cell, or on the
 *                      rectangle's sides their crkdg_mesh condition;
 *   CRKDG_GEO_WALL     reflective (the interior trace with the normal momentum
 *                      negated);
 *   CRKDG_GEO_OUTFLOW  outflow (the cell average of the same stage value);
 *   CRKDG_GEO_STATE_A, CRKDG_GEO_STATE_B  the fixed state state_a / state_b
 *                      (m doubles each, conservative; nullable: zeros);
 *   CRKDG_GEO_SHOCK    a planar shock's exact trace: state_a at face points with
 *                      x < shock_x0 + shock_speed t, state_b elsewhere, t the
 *                      stage time t^n + c_i dt (crkdg_set_time; advanced by
 *                      every accepted step), as on Example 4.9's top side.
 * Solid cells keep their state (their operators are zero) and count in no
 * admissibility test, limiter statistic, trial-step rate, bound margin or
 * crkdg_total_mass; crkdg_step_info.mass_drift still divides by the totals
 * over every cell.  Every side of a fluid cell that faces a solid cell through
 * the mesh rule must carry another kind.  geo NULL removes the geometry.
 * 2D, FP64, the compact scheme, no indicator, no subdomain
 * (CRKDG_E_UNSUPPORTED otherwise); CRKDG_E_ARG for unknown bits or kinds, an
 * open side facing a solid cell, or a non-finite shock line (the geometry is
 * then unchanged). */
enum { CRKDG_GEO_MESH = 0, CRKDG_GEO_WALL = 1, CRKDG_GEO_OUTFLOW = 2, CRKDG_GEO_STATE_A = 3,
       CRKDG_GEO_STATE_B = 4, CRKDG_GEO_SHOCK = 5 };
#define CRKDG_GEO_SOLID 0x10000u
crkdg_status crkdg_set_geometry(crkdg_t h, const unsigned *geo, const double *state_a, const double *state_b,
                                double shock_x0, double shock_speed);

/* ------------------------------------------------------------------------
 * Subdomains of a block-decomposed mesh (multi-GPU; Sec. 1 and the Compactness
 * remark of Sec. 3.2: the inner stages need no neighbour data, so one exchange of
 * u^n's boundary-cell layer per step suffices when the inner stages are
 * recomputed on a one-cell halo).  A rank builds a handle on its own block of
 * cells plus a one-cell halo ring on every side that borders another block (or
 * wraps periodically), and marks its own cells with crkdg_set_subdomain: only
 * those count in the admissibility flag, the limiter statistics, the trial-step
 * rate (crkdg_max_dt), the bound margins and the totals; the halo cells are
 * stepped as well (their inner stages are exactly those of the cells they
 * copy, which the owned cells' final stage reads) and their results are
 * discarded.  Each step the halo ring is refreshed from the neighbours' owned
 * cells (crkdg_pack_cells on the sender, crkdg_unpack_cells on the receiver),
 * the ranks agree on dt = min of their crkdg_max_dt, and on restarts through
 * crkdg_step_attempt / crkdg_step_accept (OR of the violation flags).  The
 * troubled-cell indicators are not available on a subdomain
 * (CRKDG_E_UNSUPPORTED): they read a 3x3 stencil after the final stage, which
 * needs a second exchange.
 *
 * crkdg_set_subdomain: the owned cells are [i0, i1) x [j0, j1) of this handle's
 * mesh (1D: j ignored; the whole mesh restores the default).  global (nullable)
 * is the undecomposed mesh this one is a window of: the cell sizes are then
 * formed from it exactly as its own handle forms them, so the owned cells'
 * arithmetic is bit-identical to the undecomposed run (a window's own
 * (x1 - x0) / nx can differ in the last bit); CRKDG_E_ARG if the window's cells
 * are not that mesh's cells. */
crkdg_status crkdg_set_subdomain(crkdg_t h, const crkdg_mesh *global, int i0, int i1, int j0, int j1);
/* Bytes of the packed form of `cells` cells: FP64 nodal values
 * [m][rows][cols][n^d] doubles; split precision: the FP64 cell averages
 * [m][rows][cols] doubles followed by the FP32 deviations [m][rows][cols][n^d]
 * floats (the state's own representation, so a copy is exact).  0 on bad
 * arguments. */
size_t crkdg_cells_bytes(crkdg_t h, long long cells);
/* Copy the cells of the box [i0, i1) x [j0, j1) of u^n into buf (pack) or from
 * buf into u^n (unpack; no limiter is applied: the values come from another
 * handle's state).  bytes must equal crkdg_cells_bytes of the box.  Host buffers
 * (on_device 0) are complete / reusable when the call returns; device buffers
 * are stream-ordered on the handle's stream. */
crkdg_status crkdg_pack_cells(crkdg_t h, int i0, int i1, int j0, int j1, void *buf, size_t bytes, int on_device);
crkdg_status crkdg_unpack_cells(crkdg_t h, int i0, int i1, int j0, int j1, const void *buf, size_t bytes,
                                int on_device);

/* Human-readable description of the last error on h (static string if h is NULL). */
const char *crkdg_last_error(crkdg_t h);

/* ------------------------------------------------------------------------
 * Ensembles of 2D Euler problems of uneven size (not part of the paper).  One
 * handle advances many independent problems (each its own mesh, degree k = 2 or
 * 3, tableau, CFL and end time) with the method of crkdg_step: every problem takes
 * its own trial step (crkdg_max_dt rule, clipped to its end time) and its own
 * halve-and-restart loop (Sec. 4.1).  The states live in one concatenated device
 * arena with a per-problem descriptor table; each kernel of a step is one
 * persistent launch per degree whose blocks pull (problem, tile) work items from
 * a device counter, and a step is one CUDA graph launch (attempts after a restart
 * replay a graph that only the restarting problems take part in).  The tile size
 * of the work items is chosen per (degree, size class) by crkdg_ensemble_autotune.
 * Results are bit-identical to stepping each problem alone with crkdg_step at the
 * same trial steps.  FP64 path; indicators as in crkdg_options (the learned
 * indicator runs one network evaluation over all problems' cells per attempt). */
typedef struct crkdg_ensemble_ctx *crkdg_ens_t;

typedef struct {
    crkdg_mesh mesh;              /* dim must be 2 */
    int k;                        /* 2 or 3 */
    const crkdg_tableau *tableau; /* copied at creation */
    double cfl;                   /* trial-step CFL number (> 0) */
    double t_end;                 /* the problem stops when it reaches t_end */
} crkdg_ens_problem;

/* Per-problem progress (crkdg_ensemble_info). */
typedef struct {
    double t;                 /* current time */
    long long steps;          /* accepted steps */
    long long restarts;       /* halvings over all steps */
    int done;                 /* reached t_end */
    int status;               /* CRKDG_OK, or CRKDG_E_BOUNDS if it stopped after max_halvings */
    crkdg_step_info last;     /* the last accepted step */
} crkdg_ens_info;

/* Create an ensemble of count problems (m = 4, flux kind EULER, shared gamma,
 * bounds and options; options.precision must be FP64).  Allocates every buffer
 * at once.  Errors: CRKDG_E_ARG, CRKDG_E_UNSUPPORTED, CRKDG_E_OOM, CRKDG_E_CUDA. */
crkdg_status crkdg_ensemble_create(int count, const crkdg_ens_problem *problems, int m, const crkdg_flux *flux,
                                   const crkdg_bounds *bounds, const crkdg_options *opt, crkdg_ens_t *out);
crkdg_status crkdg_ensemble_destroy(crkdg_ens_t e);
/* Nodal state of problem i (layout and count as for a single handle of its mesh
 * and k); set_state applies the scaling limiter and resets the problem's time to 0. */
crkdg_status crkdg_ensemble_set_state(crkdg_ens_t e, int i, const double *nodal, size_t count, int on_device);
crkdg_status crkdg_ensemble_get_state(crkdg_ens_t e, int i, double *nodal, size_t count, int on_device);
size_t crkdg_ensemble_state_size(crkdg_ens_t e, int i);
/* One step of every problem that has not reached its end time; *active
 * (nullable) receives how many problems are still running afterwards.  A problem
 * whose averages stay outside B^eps after max_halvings restarts stops with status
 * CRKDG_E_BOUNDS (its state stays at its last accepted step); the call itself
 * then returns CRKDG_E_BOUNDS after the other problems have stepped. */
crkdg_status crkdg_ensemble_step(crkdg_ens_t e, int *active);
crkdg_status crkdg_ensemble_info(crkdg_ens_t e, int i, crkdg_ens_info *info);
/* Network of the learned indicator (device pointer, CRKDG_MLP_NPARAM floats). */
crkdg_status crkdg_ensemble_set_mlp(crkdg_ens_t e, const float *params);
/* Training data for the learned indicator from ensemble runs (as crkdg_set_harvest for
 * one handle): while on (indicator on), every step also keeps, per problem, the features
 * of the unlimited final-stage state on which its plain TVB indicator decided
 * (crkdg_ensemble_last_features, [ny][nx][44] floats) and, with the TVB indicator,
 * those decisions (crkdg_ensemble_troubled_flags, one int per cell, the labels).  With
 * the learned indicator the flags are its combined decisions. */
crkdg_status crkdg_ensemble_set_harvest(crkdg_ens_t e, int on);
crkdg_status crkdg_ensemble_last_features(crkdg_ens_t e, int i, float *feat, int on_device);
crkdg_status crkdg_ensemble_troubled_flags(crkdg_ens_t e, int i, int *flags, int on_device);
/* Time one attempt (inner and final kernels) per candidate tile size for every
 * (degree, size class) present, reps times each, keep the fastest and rebuild the
 * step graphs.  Problems' states are not changed.  chosen (nullable, 6 ints)
 * receives the tiles (blocks of cells per work item) for classes
 * {k=2, k=3} x {<= 512^2, <= 1024^2, larger cells}; 0 where a class is empty. */
crkdg_status crkdg_ensemble_autotune(crkdg_ens_t e, int reps, int chosen[6]);
/* Host-only planning (no GPU needed): the work items of one degree group for
 * problems of ncells[i] cells split into blocks of cells_per_block cells, tile[i]
 * blocks per item, largest problems first.  Writes up to cap items as
 * (problem, first block, blocks) triples into items; returns the item count
 * (or -1 on bad arguments). */
int crkdg_ensemble_plan(int count, const long long *ncells, const int *tile, int cells_per_block, int *items,
                        int cap);
/* Device timing: while on, each crkdg_ensemble_step brackets its graph launches
 * (the step and any retry attempts) with CUDA events on the ensemble's stream;
 * crkdg_ensemble_times returns the milliseconds and the number of steps timed
 * since profiling was last switched on (switching on resets them). */
crkdg_status crkdg_ensemble_set_profiling(crkdg_ens_t e, int on);
crkdg_status crkdg_ensemble_times(crkdg_ens_t e, double *ms, long long *steps);
const char *crkdg_ensemble_last_error(crkdg_ens_t e);

/* ------------------------------------------------------------------------
 * Allocation-free DG operator.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code that runs while a
 * CUDA graph is being captured or inside another framework's memory pool,
 * plug-ins whose host forbids allocation after start-up, and real-time loops
 * where an allocation could stall or fail.  It needs no handle.
 *
 * out_dev = F(in_dev) (the DG operator with the Lax--Friedrichs flux and the
 * mesh's boundary conditions), exactly what crkdg_apply_operator(h,
 * CRKDG_OP_F, ...) returns for the same mesh, k and flux.  in_dev and out_dev
 * are caller-owned device arrays in the state layout; they may not alias.
 *
 * Scratch: the interior-trace accumulation, the face traces and the cell
 * averages live in one library-owned static device array of
 * CRKDG_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB), which every GPU that loads
 * the library keeps until the process exits.  A mesh needing more than
 * m * cells * (n^dim + 2*dim*n^(dim-1) + 1) doubles beyond that limit is
 * rejected with CRKDG_E_ARG (e.g. 2D Euler Q^3 fits up to 31775 cells, 1D
 * Euler P^2 up to 233016 cells).  Every word of the
 * scratch that a call reads is written earlier in the same call, so nothing
 * needs clearing; the array keeps the last call's contents.  All calls share
 * the one array: calls whose kernels overlap on the GPU (on different streams
 * or from different threads without ordering) race and give wrong results.
 *
 * The first call on each device does a one-time set-up with that device
 * current: it looks up the array's device address (cudaGetSymbolAddress) and
 * uploads the library's constant nodal tables (cudaMemcpyToSymbol), built by the
 * same routine as a handle's, so handles that already exist on the device see
 * the same bytes they uploaded themselves.  Make that first call before any
 * stream capture.  Afterwards the call only enqueues two kernels on
 * cuda_stream (NULL: the legacy default stream) and returns without
 * synchronising.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: CRKDG_E_ARG (bad mesh, kinds, pointers, or beyond the scratch size),
 * CRKDG_E_UNSUPPORTED (k > 3), CRKDG_E_CUDA (set-up or launch failed). */
#define CRKDG_NOALLOC_SCRATCH_DOUBLES (1 << 22)
crkdg_status crkdg_apply_F_noalloc(const crkdg_mesh *mesh, int k, int m, const crkdg_flux *flux,
                                   const double *in_dev, double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CRKDG_H */
