/*
 * crkdg_oracle.h -- plain FP64 CPU reference of the bound-preserving compact
 * Runge--Kutta discontinuous Galerkin (cRKDG) method of Liu, Sun and Zhang
 * (arXiv 2412.16002).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (paper_2412_16002_gb300/) never links, imports or calls it, and it shares no
 * code, tables or headers with the CUDA path.
 *
 * Representation: modal tensor Legendre basis P_i(xi) P_j(eta) on each cell
 * (the CUDA path is nodal at Gauss points; both define the same discrete
 * scheme because every integral uses the same (k+1)-point Gauss quadrature and
 * both mass matrices are integrated exactly).
 */
#ifndef CRKDG_ORACLE_H
#define CRKDG_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXN 6 /* nodes per direction: k <= 5 */
#define ORC_MAXM 4 /* components: Euler 2D */
#define ORC_MAXS 6 /* RK stages */

enum { ORC_FLUX_ADVECTION = 0, ORC_FLUX_BURGERS = 1, ORC_FLUX_EULER = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_REFLECT = 2, ORC_BC_DIRICHLET = 3,
       ORC_BC_EXACT = 4 };
enum { ORC_OP_G = 0, ORC_OP_F = 1 };

/* exact-solution exterior state (test-only boundary condition, e.g. Sec. 4.2) */
typedef void (*orc_exact_fn)(double x, double y, double t, double *u, void *ctx);

typedef struct orc_problem {
    int dim, nx, ny, k, n, L, m, nmodes, ncell;
    double x0, x1, y0, y1, hx, hy;
    int flux;
    double gamma, vel[2];
    double lo, hi, eps;      /* scalar bounds [lo,hi]; Euler epsilon of B^eps */
    int bc[4];               /* sides: 0 left, 1 right, 2 bottom, 3 top */
    double bc_state[4][ORC_MAXM];
    int limiter_on;          /* 1: scaling limiter after every stage */
    int indicator;           /* 1: TVB troubled-cell indicator + minmod shock limiter after the final stage */
    int standard;            /* 1: standard RKDG (eq. rkdg): F in the inner stages as well */
    int theta2_exact;        /* 1: theta_2 from the exact per-point solve (see orc_set_theta2) */
    int source;              /* 1: the manufactured source of scenario I (see orc_set_source) */
    int pk;                  /* 1: the total-degree space P^k in 2D (see orc_set_basis) */
    unsigned *geo;           /* non-rectangular domain (see orc_set_geometry) or NULL */
    double geo_state[2][ORC_MAXM];
    double shock_x0, shock_speed;
    double tvb_M;            /* TVB constant of the indicator */
    int max_halvings;
    orc_exact_fn exact;
    void *exact_ctx;
    double xg[ORC_MAXN], wg[ORC_MAXN]; /* Gauss-Legendre on [-1,1] */
    double xl[ORC_MAXN], wl[ORC_MAXN]; /* Gauss-Lobatto on [-1,1] */
} orc_problem;

typedef struct orc_info {
    double dt_taken;
    int restarts;
    long long cells_limited;
    double theta_min;
} orc_info;

/* quadrature (Sec. 2.2.1) */
void orc_gauss_legendre(int n, double *x, double *w);
void orc_gauss_lobatto(int L, double *x, double *w);
double orc_legendre(int i, double x);
double orc_dlegendre(int i, double x);

orc_problem *orc_create(int dim, int nx, int ny, int k, double x0, double x1, double y0,
                        double y1, int flux, double gamma, double vx, double vy, double lo,
                        double hi, double eps, const int *bc, const double *bc_state);
void orc_destroy(orc_problem *P);
void orc_set_exact(orc_problem *P, orc_exact_fn fn, void *ctx);
void orc_set_options(orc_problem *P, int limiter_on, int max_halvings);
/* scheme: 0 the compact RKDG (Scheme 1L: G in the inner stages, F in the final one), 1 the
 * standard RKDG in Butcher form (eq. rkdg: F in every stage), with the same limiter */
void orc_set_scheme(orc_problem *P, int standard);
/* theta_2 of the Euler limiter: 0 the concavity ratio of eq. (Euler-limiter2), 1 the exact
 * per-point solve of the positivity-limiter works the text after that equation refers to
 * (the paper prints only the ratio): for every S_K point q where
 * rho e(u_q) < eps, the t in (0, 1) with rho e(ubar + t (u_q - ubar)) = eps, a root of a
 * quadratic (rho, m and E are linear in t); theta_2 = min_q t_q (the same safety margin
 * and verification as the ratio) */
void orc_set_theta2(orc_problem *P, int exact);
/* source: 0 none; 1 the source of Example 4.2's scenario I (2D Euler), S = d_t U + d_x F(U) +
 * d_y G(U) of the manufactured solution rho = exp(-t) sin 2pi(x+y) + 2,
 * w = (exp(-t) cos 2pi x sin 2pi y + 2, exp(-t) sin 2pi x cos 2pi y + 2),
 * e = exp(-t) cos 2pi(x+y) / 2 + 1 (e the specific internal energy), added to G and F as its L2
 * projection (the (k+1)-point Gauss rule) at the stage time */
void orc_set_source(orc_problem *P, int source);
/* basis: 0 the tensor space Q^k; 1 the total-degree space P^k (2D; in 1D the two coincide):
 * the modal tensor Legendre basis restricted to the modes L_i(x) L_j(y) with i + j <= k, which
 * are L2-orthogonal, so the Galerkin equations of P^k are those of Q^k tested against the
 * retained modes only: every operator output, state projection and stage value keeps the
 * modes i + j <= k and has the others zero (Sec. 4.2 tests both spaces) */
void orc_set_basis(orc_problem *P, int pk);
/* the source of scenario I at (x, y, t), m = 4 components */
/* Non-rectangular domains (Examples 4.8 and 4.9): the domain is a union of mesh cells of the
 * bounding rectangle.  geo[cell] holds, in bits 4s..4s+3, the boundary kind of side s
 * (0 left, 1 right, 2 bottom, 3 top) and, in bit 16, whether the cell is solid.  Kinds:
 * ORC_GEO_MESH the mesh rule (the neighbouring cell, or the rectangle side's condition),
 * ORC_GEO_WALL reflective, ORC_GEO_OUTFLOW outflow, ORC_GEO_STATE_A / _B the fixed state
 * state_a / state_b, ORC_GEO_SHOCK state_a at face points with x < shock_x0 + shock_speed t
 * and state_b elsewhere (a planar shock's exact trace on a boundary).  Solid cells take no
 * part: their operators are zero and they count in no test, rate or total.  Every side of a
 * fluid cell that faces a solid cell must carry a kind other than ORC_GEO_MESH.  Returns 0,
 * or -1 (geometry unchanged) on a bad word.  geo is copied; NULL removes the geometry. */
enum { ORC_GEO_MESH = 0, ORC_GEO_WALL = 1, ORC_GEO_OUTFLOW = 2, ORC_GEO_STATE_A = 3,
       ORC_GEO_STATE_B = 4, ORC_GEO_SHOCK = 5 };
#define ORC_GEO_SOLID 0x10000u
int orc_set_geometry(orc_problem *P, const unsigned *geo, const double *state_a,
                     const double *state_b, double shock_x0, double shock_speed);
int orc_is_solid(const orc_problem *P, int cell);
void orc_scenario1_source(double gamma, double x, double y, double t, double *S);
size_t orc_state_size(const orc_problem *P); /* doubles: ncell*m*n^dim */

/* nodal (Gauss points, layout [m][ny][nx][n_y][n_x]) <-> modal */
void orc_nodal_to_modal(const orc_problem *P, const double *nodal, double *modal);
void orc_modal_to_nodal(const orc_problem *P, const double *modal, double *nodal);

/* state evaluation */
void orc_point_state(const orc_problem *P, const double *c, int cell, double xi, double eta,
                     double *u);
void orc_cell_averages(const orc_problem *P, const double *c, double *avg); /* [cell][m] */

/* physics */
void orc_flux(const orc_problem *P, const double *u, int dir, double *f);
double orc_speed(const orc_problem *P, const double *u, int dir);
double orc_pressure(const orc_problem *P, const double *u);

/* spatial operators G = -div^loc f (Sec. 2.1) and F = -div^DG f (eq. dxDG),
 * modal in -> modal out; t is the time at which an exact boundary is sampled */
void orc_apply(const orc_problem *P, int op, const double *in, double *out, double t);

/* scaling limiter (Prop. 2.4 scalar; eq. Euler-limiter), in place.
 * theta_out (optional, [ncell]) receives the combined scaling per cell. */
long long orc_limit(const orc_problem *P, double *c, double *theta_out);
int orc_averages_admissible(const orc_problem *P, const double *c); /* 1 if all in B^eps */
/* minimum over S_K of each bound margin: scalar [u-lo, hi-u]; Euler [rho-eps, rhoe-eps] */
void orc_min_margins(const orc_problem *P, const double *c, double *margins2);

/* plain troubled-cell indicator (TVB-modified minmod on face-averaged traces, per component
 * and direction) and minmod shock limiter; flags[cell] = 1 for a troubled cell */
void orc_set_indicator(orc_problem *P, int on, double tvb_M);
long long orc_troubled_cells(const orc_problem *P, const double *c, int *flags);
void orc_shock_limit(const orc_problem *P, double *c, const int *flags);

/* a0 = max over S_K points and directions of the spectral radius (Sec. 2.1 notation) */
double orc_a0(const orc_problem *P, const double *c);
double orc_max_dt(const orc_problem *P, const double *c, double cfl);

/* one limited cRKDG step (Scheme 1L, eq. rkdg-lim) with the Sec. 4.1 restart loop.
 * A: s*s row-major strictly lower; b: s.  Returns 0 ok, 4 if max_halvings exceeded
 * (state unchanged). */
int orc_step(const orc_problem *P, double *c, double dt, int s, const double *A, const double *b,
             double t, orc_info *info);
/* one attempt without restarts, recording every stage: u_stage and ut_stage are
 * [s+1][state] (index s = final stage).  Returns 0 if every stage average was
 * admissible, else the 1-based stage index that failed (states up to it are filled). */
int orc_step_stages(const orc_problem *P, const double *c, double dt, int s, const double *A,
                    const double *b, double t, double *u_stage, double *ut_stage);

/* diagnostics */
double orc_total_mass(const orc_problem *P, const double *c, int comp);
double orc_l2_error_exact(const orc_problem *P, const double *c, double t, int nq);
double orc_l1_error_exact(const orc_problem *P, const double *c, double t, int nq);

#ifdef __cplusplus
}
#endif
#endif
