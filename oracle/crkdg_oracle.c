/*
 * crkdg_oracle.c -- plain, slow, FP64 reference of the bound-preserving cRKDG
 * method (Liu, Sun, Zhang, arXiv 2412.16002).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py.  The CUDA product path never uses it.
 *
 * Every routine follows the paper's definitions directly, with plain loops over
 * cells, modes and quadrature points and no blocking or fusion:
 *   - V_h with Q^k on Cartesian cells, Sec. 2 (modal tensor Legendre basis here);
 *   - DG operator with the Lax--Friedrichs flux, eq. (dxDG) and the LF formula
 *     below it; local derivative operator div^loc, Sec. 2.1 (interior traces);
 *   - edge quadrature (Prop. 2.1): (k+1)-point Gauss on every edge;
 *   - convex decomposition point set S_K (Prop. 2.2, Fig. 1): Gauss x Gauss-Lobatto
 *     and Gauss-Lobatto x Gauss points;
 *   - scalar scaling limiter, Prop. 2.4; Euler limiter, eq. (Euler-limiter1/2);
 *   - limited Butcher-form cRKDG (Scheme 1L, eq. rkdg-lim, Appendix B.2);
 *   - adaptive time marching with halve-and-restart, Sec. 4.1 (Algorithm).
 *
 * Readings where the paper is silent (all shared with the CUDA path by
 * specification only, never by code):
 *   - the number of Gauss-Lobatto points is L = ceil((k+3)/2), the smallest rule
 *     exact for degree k;
 *   - the LF viscosity alpha on an edge is the maximum over that edge's
 *     quadrature points of the spectral radius of both traces;
 *   - a0 (Sec. 2.1 notation) is the maximum over all S_K points; the trial step
 *     sums the directional radii over the dimensions (orc_max_dt);
 *   - theta is only computed from a bound that is violated (0/0 avoided); every
 *     theta below 1 is multiplied by (1-2^-40), a relative safety margin so that
 *     the rescaled polynomial stays inside the bound after rounding; the limited
 *     polynomial is then re-evaluated on S_K and, if rounding still left a point
 *     outside, the final scaling towards the average (theta, or theta_2 applied
 *     to every component for Euler) is multiplied by (1-2^-30), (1-2^-20),
 *     (1-2^-10) in turn and finally set to 0;
 *   - the Euler energy limiter enforces rho*e >= eps, exactly as eq.
 *     (Euler-limiter2) is written, and the admissibility test of the cell
 *     averages uses the same predicate.
 *
 * Optional, not part of the paper's method (which applies no anti-oscillation
 * limiter, Sec. 4): a plain troubled-cell indicator and shock limiter, applied
 * once per step after the final stage and before the scaling limiter so that the
 * inner stages stay compact:
 *   - per conservative component and direction, with face-averaged traces
 *     ut_R = avg_face(u_R) - ubar and ut_L = ubar - avg_face(u_L) and the neighbour
 *     differences D+ = ubar_{K+1} - ubar_K, D- = ubar_K - ubar_{K-1}, the cell is
 *     troubled if the TVB-modified minmod m~(a, D+, D-) (= a when |a| <= M h^2,
 *     else minmod) changes ut_R or ut_L;
 *   - a troubled cell is replaced by ubar + minmod(c_x, D+x, D-x) P_1(xi)
 *     + minmod(c_y, D+y, D-y) P_1(eta) (its first Legendre moments limited, every
 *     higher mode dropped), which keeps the average;
 *   - neighbour averages across the boundary follow the boundary condition.
 *
 * Non-rectangular domains (Sec. 4.4, Examples 4.8 and 4.9): the domain is a union of
 * cells of the bounding rectangle; the other cells are solid and take no part.  A
 * per-cell word gives each side a boundary kind (reflective wall, outflow, a fixed
 * state, or the exact trace of a planar shock moving at constant speed, evaluated at
 * the stage time); see orc_set_geometry.
 */
#include "crkdg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and quadrature                                       */
/* ------------------------------------------------------------------------ */

double orc_legendre(int i, double x) {
    if (i == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int j = 1; j < i; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

double orc_dlegendre(int i, double x) {
    /* P'_{j+1} = P'_{j-1} + (2j+1) P_j */
    if (i == 0) return 0.0;
    double dm1 = 0.0, d = 1.0; /* P'_0, P'_1 */
    for (int j = 1; j < i; ++j) {
        double dn = dm1 + (2.0 * j + 1.0) * orc_legendre(j, x);
        dm1 = d;
        d = dn;
    }
    return d;
}

static void sort_pairs(int n, double *x, double *w) {
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
            if (x[b] < x[a]) {
                double t = x[a]; x[a] = x[b]; x[b] = t;
                t = w[a]; w[a] = w[b]; w[b] = t;
            }
}

void orc_gauss_legendre(int n, double *x, double *w) {
    /* Newton on P_n from the Chebyshev-like initial guess; w = 2/((1-x^2) P_n'(x)^2) */
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double dz = orc_legendre(n, z) / orc_dlegendre(n, z);
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double dp = orc_dlegendre(n, z);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    sort_pairs(n, x, w);
}

void orc_gauss_lobatto(int L, double *x, double *w) {
    /* end points +-1 and the roots of P'_{L-1}; w = 2/(L(L-1) P_{L-1}(x)^2) */
    const double pi = 3.14159265358979323846;
    int N = L - 1;
    x[0] = -1.0;
    x[L - 1] = 1.0;
    for (int i = 1; i < L - 1; ++i) {
        double z = -cos(pi * i / N);
        for (int it = 0; it < 100; ++it) {
            double p = orc_legendre(N, z), dp = orc_dlegendre(N, z);
            /* (1-z^2) P'' = 2 z P' - N(N+1) P */
            double d2p = (2.0 * z * dp - N * (N + 1.0) * p) / (1.0 - z * z);
            double dz = dp / d2p;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
    for (int i = 0; i < L; ++i) {
        double p = orc_legendre(N, x[i]);
        w[i] = 2.0 / (L * (L - 1.0) * p * p);
    }
    sort_pairs(L, x, w);
}

/* ------------------------------------------------------------------------ */
/* problem set-up                                                            */
/* ------------------------------------------------------------------------ */

orc_problem *orc_create(int dim, int nx, int ny, int k, double x0, double x1, double y0,
                        double y1, int flux, double gamma, double vx, double vy, double lo,
                        double hi, double eps, const int *bc, const double *bc_state) {
    if (dim < 1 || dim > 2 || k < 1 || k + 1 > ORC_MAXN || nx < 1) return NULL;
    orc_problem *P = (orc_problem *)calloc(1, sizeof(orc_problem));
    P->dim = dim;
    P->nx = nx;
    P->ny = dim == 2 ? ny : 1;
    P->k = k;
    P->n = k + 1;
    P->L = (k + 4) / 2; /* ceil((k+3)/2) */
    if (P->L < 2) P->L = 2;
    P->flux = flux;
    P->m = flux == ORC_FLUX_EULER ? dim + 2 : 1;
    P->nmodes = dim == 2 ? P->n * P->n : P->n;
    P->ncell = P->nx * P->ny;
    P->x0 = x0;
    P->x1 = x1;
    P->y0 = dim == 2 ? y0 : 0.0;
    P->y1 = dim == 2 ? y1 : 1.0;
    P->hx = (x1 - x0) / nx;
    P->hy = dim == 2 ? (y1 - y0) / ny : 1.0;
    P->gamma = gamma;
    P->vel[0] = vx;
    P->vel[1] = vy;
    P->lo = lo;
    P->hi = hi;
    P->eps = eps;
    for (int s = 0; s < 4; ++s) {
        P->bc[s] = bc ? bc[s] : ORC_BC_PERIODIC;
        for (int c = 0; c < ORC_MAXM; ++c)
            P->bc_state[s][c] = bc_state ? bc_state[s * ORC_MAXM + c] : 0.0;
    }
    P->limiter_on = 1;
    P->max_halvings = 20;
    P->indicator = 0;
    P->tvb_M = 10.0;
    orc_gauss_legendre(P->n, P->xg, P->wg);
    orc_gauss_lobatto(P->L, P->xl, P->wl);
    return P;
}

void orc_destroy(orc_problem *P) {
    if (P) free(P->geo);
    free(P);
}

void orc_set_exact(orc_problem *P, orc_exact_fn fn, void *ctx) {
    P->exact = fn;
    P->exact_ctx = ctx;
}

void orc_set_options(orc_problem *P, int limiter_on, int max_halvings) {
    P->limiter_on = limiter_on;
    P->max_halvings = max_halvings;
}

void orc_set_scheme(orc_problem *P, int standard) { P->standard = standard ? 1 : 0; }
void orc_set_theta2(orc_problem *P, int exact) { P->theta2_exact = exact ? 1 : 0; }
void orc_set_source(orc_problem *P, int source) { P->source = source; }
void orc_set_basis(orc_problem *P, int pk) { P->pk = pk ? 1 : 0; }

/* boundary kind of side s of a cell (ORC_GEO_MESH without a geometry) */
static int geo_kind(const orc_problem *P, int cell, int s) {
    return P->geo ? (int)((P->geo[cell] >> (4 * s)) & 15u) : ORC_GEO_MESH;
}

int orc_is_solid(const orc_problem *P, int cell) {
    return P->geo && (P->geo[cell] & ORC_GEO_SOLID) ? 1 : 0;
}

int orc_set_geometry(orc_problem *P, const unsigned *geo, const double *state_a,
                     const double *state_b, double shock_x0, double shock_speed) {
    if (!geo) {
        free(P->geo);
        P->geo = NULL;
        return 0;
    }
    if (P->dim != 2) return -1;
    for (int cell = 0; cell < P->ncell; ++cell) {
        unsigned g = geo[cell];
        if (g & ~(ORC_GEO_SOLID | 0xFFFFu)) return -1;
        if (g & ORC_GEO_SOLID) continue;
        int cx = cell % P->nx, cy = cell / P->nx;
        for (int s = 0; s < 4; ++s) {
            int kind = (int)((g >> (4 * s)) & 15u);
            if (kind > ORC_GEO_SHOCK) return -1;
            if (kind != ORC_GEO_MESH) continue;
            /* the mesh neighbour (periodic wrap included) must be a fluid cell */
            int nb;
            if (s == 0) nb = cx > 0 ? cell - 1 : (P->bc[0] == ORC_BC_PERIODIC ? cell + P->nx - 1 : -1);
            else if (s == 1) nb = cx < P->nx - 1 ? cell + 1 : (P->bc[1] == ORC_BC_PERIODIC ? cell - P->nx + 1 : -1);
            else if (s == 2) nb = cy > 0 ? cell - P->nx : (P->bc[2] == ORC_BC_PERIODIC ? cell + (P->ny - 1) * P->nx : -1);
            else nb = cy < P->ny - 1 ? cell + P->nx : (P->bc[3] == ORC_BC_PERIODIC ? cell - (P->ny - 1) * P->nx : -1);
            if (nb >= 0 && (geo[nb] & ORC_GEO_SOLID)) return -1;
        }
    }
    unsigned *copy = (unsigned *)malloc(sizeof(unsigned) * P->ncell);
    if (!copy) return -1;
    memcpy(copy, geo, sizeof(unsigned) * P->ncell);
    free(P->geo);
    P->geo = copy;
    for (int comp = 0; comp < ORC_MAXM; ++comp) {
        P->geo_state[0][comp] = comp < P->m && state_a ? state_a[comp] : 0.0;
        P->geo_state[1][comp] = comp < P->m && state_b ? state_b[comp] : 0.0;
    }
    P->shock_x0 = shock_x0;
    P->shock_speed = shock_speed;
    return 0;
}

/* Scenario I (Example 4.2): S = d_t U + d_x F + d_y G by the chain rule from the primitive
 * fields q in {rho, wx, wy, e} and their partial derivatives in t, x and y. */
void orc_scenario1_source(double gamma, double x, double y, double t, double *S) {
    const double tp = 2.0 * 3.14159265358979323846, a = exp(-t);
    const double s1 = sin(tp * (x + y)), c1 = cos(tp * (x + y));
    const double sx = sin(tp * x), cx = cos(tp * x), sy = sin(tp * y), cy = cos(tp * y);
    /* primitive fields and their derivatives (index 0: value, 1: d_t, 2: d_x, 3: d_y) */
    double r[4], u[4], v[4], e[4];
    r[0] = a * s1 + 2.0;        r[1] = -a * s1;                r[2] = a * tp * c1;        r[3] = a * tp * c1;
    u[0] = a * cx * sy + 2.0;   u[1] = -a * cx * sy;           u[2] = -a * tp * sx * sy;  u[3] = a * tp * cx * cy;
    v[0] = a * sx * cy + 2.0;   v[1] = -a * sx * cy;           v[2] = a * tp * cx * cy;   v[3] = -a * tp * sx * sy;
    e[0] = 0.5 * a * c1 + 1.0;  e[1] = -0.5 * a * c1;          e[2] = -0.5 * a * tp * s1; e[3] = -0.5 * a * tp * s1;
    /* derived quantities and their derivatives, d = 1, 2, 3 */
    double p[4], E[4], K[4];
    for (int d = 0; d < 4; ++d) {
        if (d == 0) {
            K[0] = 0.5 * (u[0] * u[0] + v[0] * v[0]);
            p[0] = (gamma - 1.0) * r[0] * e[0];
            E[0] = r[0] * e[0] + r[0] * K[0];
        } else {
            K[d] = u[0] * u[d] + v[0] * v[d];
            p[d] = (gamma - 1.0) * (r[d] * e[0] + r[0] * e[d]);
            E[d] = r[d] * e[0] + r[0] * e[d] + r[d] * K[0] + r[0] * K[d];
        }
    }
    /* S_rho = rho_t + (rho u)_x + (rho v)_y */
    S[0] = r[1] + (r[2] * u[0] + r[0] * u[2]) + (r[3] * v[0] + r[0] * v[3]);
    /* S_mx = (rho u)_t + (rho u^2 + p)_x + (rho u v)_y */
    S[1] = (r[1] * u[0] + r[0] * u[1]) + (r[2] * u[0] * u[0] + 2.0 * r[0] * u[0] * u[2] + p[2]) +
           (r[3] * u[0] * v[0] + r[0] * u[3] * v[0] + r[0] * u[0] * v[3]);
    /* S_my = (rho v)_t + (rho u v)_x + (rho v^2 + p)_y */
    S[2] = (r[1] * v[0] + r[0] * v[1]) + (r[2] * u[0] * v[0] + r[0] * u[2] * v[0] + r[0] * u[0] * v[2]) +
           (r[3] * v[0] * v[0] + 2.0 * r[0] * v[0] * v[3] + p[3]);
    /* S_E = E_t + ((E + p) u)_x + ((E + p) v)_y */
    S[3] = E[1] + ((E[2] + p[2]) * u[0] + (E[0] + p[0]) * u[2]) + ((E[3] + p[3]) * v[0] + (E[0] + p[0]) * v[3]);
}

void orc_set_indicator(orc_problem *P, int on, double tvb_M) {
    P->indicator = on;
    P->tvb_M = tvb_M;
}

size_t orc_state_size(const orc_problem *P) { return (size_t)P->ncell * P->m * P->nmodes; }

static const double *cell_coef(const orc_problem *P, const double *c, int cell, int comp) {
    return c + ((size_t)cell * P->m + comp) * P->nmodes;
}
static double *cell_coef_w(const orc_problem *P, double *c, int cell, int comp) {
    return c + ((size_t)cell * P->m + comp) * P->nmodes;
}

/* ------------------------------------------------------------------------ */
/* nodal <-> modal                                                           */
/* ------------------------------------------------------------------------ */

/* P^k: zero the modes L_i(x) L_j(y) with i + j > k of every cell and component */
static void drop_high_modes(const orc_problem *P, double *modal) {
    if (!P->pk || P->dim != 2) return;
    int n = P->n;
    for (int comp = 0; comp < P->m; ++comp)
        for (int cell = 0; cell < P->ncell; ++cell) {
            double *c = cell_coef_w(P, modal, cell, comp);
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i)
                    if (i + j > P->k) c[j * n + i] = 0.0;
        }
}

void orc_nodal_to_modal(const orc_problem *P, const double *nodal, double *modal) {
    /* L2 projection by the (k+1)-point Gauss rule, exact for Q^k */
    int n = P->n, nyn = P->dim == 2 ? n : 1;
    for (int comp = 0; comp < P->m; ++comp)
        for (int cell = 0; cell < P->ncell; ++cell) {
            const double *u = nodal + ((size_t)comp * P->ncell + cell) * P->nmodes;
            double *c = cell_coef_w(P, modal, cell, comp);
            for (int j = 0; j < nyn; ++j)
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int b = 0; b < nyn; ++b)
                        for (int a = 0; a < n; ++a) {
                            double wy = P->dim == 2 ? P->wg[b] * orc_legendre(j, P->xg[b]) : 1.0;
                            s += P->wg[a] * orc_legendre(i, P->xg[a]) * wy * u[b * n + a];
                        }
                    double norm = 2.0 / (2.0 * i + 1.0);
                    if (P->dim == 2) norm *= 2.0 / (2.0 * j + 1.0);
                    c[j * n + i] = s / norm;
                }
        }
    drop_high_modes(P, modal);  /* P^k: the L2 projection keeps the retained modes */
}

static double eval_modal(const orc_problem *P, const double *c, double xi, double eta) {
    int n = P->n;
    if (P->dim == 1) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += c[i] * orc_legendre(i, xi);
        return s;
    }
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        double pj = orc_legendre(j, eta);
        for (int i = 0; i < n; ++i) s += c[j * n + i] * orc_legendre(i, xi) * pj;
    }
    return s;
}

void orc_modal_to_nodal(const orc_problem *P, const double *modal, double *nodal) {
    int n = P->n, nyn = P->dim == 2 ? n : 1;
    for (int comp = 0; comp < P->m; ++comp)
        for (int cell = 0; cell < P->ncell; ++cell) {
            double *u = nodal + ((size_t)comp * P->ncell + cell) * P->nmodes;
            const double *c = cell_coef(P, modal, cell, comp);
            for (int b = 0; b < nyn; ++b)
                for (int a = 0; a < n; ++a)
                    u[b * n + a] = eval_modal(P, c, P->xg[a], P->dim == 2 ? P->xg[b] : 0.0);
        }
}

void orc_point_state(const orc_problem *P, const double *c, int cell, double xi, double eta,
                     double *u) {
    for (int comp = 0; comp < P->m; ++comp) u[comp] = eval_modal(P, cell_coef(P, c, cell, comp), xi, eta);
}

void orc_cell_averages(const orc_problem *P, const double *c, double *avg) {
    /* P_0 = 1 and the other modes have zero mean: the average is mode (0,0) */
    for (int cell = 0; cell < P->ncell; ++cell)
        for (int comp = 0; comp < P->m; ++comp) avg[cell * P->m + comp] = cell_coef(P, c, cell, comp)[0];
}

/* ------------------------------------------------------------------------ */
/* physics: eq. (claws), Burgers, Euler eq. (Euler), (Euler-2)               */
/* ------------------------------------------------------------------------ */

double orc_pressure(const orc_problem *P, const double *u) {
    if (P->dim == 1) return (P->gamma - 1.0) * (u[2] - 0.5 * u[1] * u[1] / u[0]);
    return (P->gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

static double rho_e(const orc_problem *P, const double *u) {
    if (P->dim == 1) return u[2] - 0.5 * u[1] * u[1] / u[0];
    return u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0];
}

void orc_flux(const orc_problem *P, const double *u, int dir, double *f) {
    switch (P->flux) {
    case ORC_FLUX_ADVECTION:
        f[0] = P->vel[dir] * u[0];
        break;
    case ORC_FLUX_BURGERS:
        f[0] = 0.5 * u[0] * u[0];
        break;
    default: {
        double p = orc_pressure(P, u);
        if (P->dim == 1) {
            double w = u[1] / u[0];
            f[0] = u[1];
            f[1] = u[1] * w + p;
            f[2] = (u[2] + p) * w;
        } else {
            double wd = u[1 + dir] / u[0];
            f[0] = u[1 + dir];
            f[1] = u[1] * wd + (dir == 0 ? p : 0.0);
            f[2] = u[2] * wd + (dir == 1 ? p : 0.0);
            f[3] = (u[3] + p) * wd;
        }
    }
    }
}

double orc_speed(const orc_problem *P, const double *u, int dir) {
    switch (P->flux) {
    case ORC_FLUX_ADVECTION:
        return fabs(P->vel[dir]);
    case ORC_FLUX_BURGERS:
        return fabs(u[0]);
    default: {
        double p = orc_pressure(P, u);
        double c2 = P->gamma * p / u[0];
        double c = c2 > 0.0 ? sqrt(c2) : 0.0;
        return fabs(u[1 + dir] / u[0]) + c;
    }
    }
}

/* ------------------------------------------------------------------------ */
/* boundary exterior states                                                  */
/* ------------------------------------------------------------------------ */

/* neighbour across side s (0 L, 1 R, 2 B, 3 T) or -1 if the side is a boundary */
static int neighbour(const orc_problem *P, int cell, int s) {
    if (geo_kind(P, cell, s) != ORC_GEO_MESH) return -1; /* a boundary of the domain's geometry */
    int cx = cell % P->nx, cy = cell / P->nx;
    int nx = P->nx, ny = P->ny;
    switch (s) {
    case 0:
        if (cx > 0) return cell - 1;
        return P->bc[0] == ORC_BC_PERIODIC ? cy * nx + nx - 1 : -1;
    case 1:
        if (cx < nx - 1) return cell + 1;
        return P->bc[1] == ORC_BC_PERIODIC ? cy * nx : -1;
    case 2:
        if (cy > 0) return cell - nx;
        return P->bc[2] == ORC_BC_PERIODIC ? (ny - 1) * nx + cx : -1;
    default:
        if (cy < ny - 1) return cell + nx;
        return P->bc[3] == ORC_BC_PERIODIC ? cx : -1;
    }
}

/* Exterior state on boundary side s of a cell whose side has the geometry kind `kind`
 * (ORC_GEO_MESH: the rectangle side's condition bc[s]): uin is the interior trace, avg the
 * cell average of the same polynomial, (x, y) the face point, t the stage time.  Outflow
 * takes the cell average (the Lax--Friedrichs flux keeps its dissipation on outflow faces;
 * a constant state is kept exactly). */
static void exterior_state(const orc_problem *P, int kind, int s, const double *uin, const double *avg,
                           double x, double y, double t, double *uex) {
    int m = P->m;
    int bc = P->bc[s];
    switch (kind) {
    case ORC_GEO_WALL: bc = ORC_BC_REFLECT; break;
    case ORC_GEO_OUTFLOW: bc = ORC_BC_OUTFLOW; break;
    case ORC_GEO_STATE_A:
    case ORC_GEO_STATE_B:
    case ORC_GEO_SHOCK: {
        /* behind the shock (x < its position at time t) state_a, ahead of it state_b */
        int which = kind == ORC_GEO_STATE_A ? 0 : kind == ORC_GEO_STATE_B ? 1
                    : (x < P->shock_x0 + P->shock_speed * t ? 0 : 1);
        for (int c = 0; c < m; ++c) uex[c] = P->geo_state[which][c];
        return;
    }
    default: break;
    }
    switch (bc) {
    case ORC_BC_DIRICHLET:
        for (int c = 0; c < m; ++c) uex[c] = P->bc_state[s][c];
        break;
    case ORC_BC_EXACT:
        P->exact(x, y, t, uex, P->exact_ctx);
        break;
    case ORC_BC_REFLECT:
        for (int c = 0; c < m; ++c) uex[c] = uin[c];
        if (P->flux == ORC_FLUX_EULER) uex[1 + s / 2] = -uin[1 + s / 2];
        break;
    default: /* outflow */
        for (int c = 0; c < m; ++c) uex[c] = avg[c];
    }
}

/* ------------------------------------------------------------------------ */
/* spatial operators                                                         */
/* ------------------------------------------------------------------------ */

/* reference coordinates of the q-th quadrature point of side s */
static void face_point(const orc_problem *P, int s, int q, double *xi, double *eta) {
    double e = P->dim == 2 ? P->xg[q] : 0.0;
    switch (s) {
    case 0: *xi = -1.0; *eta = e; break;
    case 1: *xi = 1.0; *eta = e; break;
    case 2: *xi = e; *eta = -1.0; break;
    default: *xi = e; *eta = 1.0;
    }
}

void orc_apply(const orc_problem *P, int op, const double *in, double *out, double t) {
    int n = P->n, m = P->m, dim = P->dim;
    int nyq = dim == 2 ? n : 1;     /* y quadrature points of the volume rule */
    int nfp = dim == 2 ? n : 1;     /* quadrature points per edge */
    int nside = 2 * dim;
    double hx = P->hx, hy = P->hy;
    double *rhs = (double *)malloc(sizeof(double) * m * P->nmodes);
    for (int cell = 0; cell < P->ncell; ++cell) {
        int cx = cell % P->nx, cy = cell / P->nx;
        memset(rhs, 0, sizeof(double) * m * P->nmodes);
        if (orc_is_solid(P, cell)) { /* outside the domain: no operator */
            for (int c = 0; c < m; ++c) memset(cell_coef_w(P, out, cell, c), 0, sizeof(double) * P->nmodes);
            continue;
        }
        /* volume term: int_K f(u) : grad v */
        for (int r = 0; r < nyq; ++r)
            for (int q = 0; q < n; ++q) {
                double xi = P->xg[q], eta = dim == 2 ? P->xg[r] : 0.0;
                double u[ORC_MAXM], fx[ORC_MAXM], fy[ORC_MAXM];
                orc_point_state(P, in, cell, xi, eta, u);
                orc_flux(P, u, 0, fx);
                if (dim == 2) orc_flux(P, u, 1, fy);
                for (int j = 0; j < nyq; ++j)
                    for (int i = 0; i < n; ++i) {
                        double vx, vy = 0.0, jac;
                        if (dim == 1) {
                            jac = hx / 2.0 * P->wg[q];
                            vx = orc_dlegendre(i, xi) * 2.0 / hx;
                        } else {
                            jac = hx * hy / 4.0 * P->wg[q] * P->wg[r];
                            vx = orc_dlegendre(i, xi) * 2.0 / hx * orc_legendre(j, eta);
                            vy = orc_legendre(i, xi) * orc_dlegendre(j, eta) * 2.0 / hy;
                        }
                        for (int c = 0; c < m; ++c)
                            rhs[c * P->nmodes + j * n + i] += jac * (fx[c] * vx + (dim == 2 ? fy[c] * vy : 0.0));
                    }
            }
        /* edge terms: - sum_l int_e (f.nu) v */
        for (int s = 0; s < nside; ++s) {
            int dir = s / 2;
            double sgn = (s % 2) ? 1.0 : -1.0;
            int nb = neighbour(P, cell, s);
            double fnu[ORC_MAXN][ORC_MAXM];
            if (op == ORC_OP_G) {
                for (int q = 0; q < nfp; ++q) {
                    double xi, eta, u[ORC_MAXM], f[ORC_MAXM];
                    face_point(P, s, q, &xi, &eta);
                    orc_point_state(P, in, cell, xi, eta, u);
                    orc_flux(P, u, dir, f);
                    for (int c = 0; c < m; ++c) fnu[q][c] = sgn * f[c];
                }
            } else {
                /* canonical orientation: uL on the lower side, uR on the upper side */
                double uL[ORC_MAXN][ORC_MAXM], uR[ORC_MAXN][ORC_MAXM];
                double alpha = 0.0;
                for (int q = 0; q < nfp; ++q) {
                    double xi, eta, ui[ORC_MAXM], ue[ORC_MAXM];
                    face_point(P, s, q, &xi, &eta);
                    orc_point_state(P, in, cell, xi, eta, ui);
                    if (nb >= 0) {
                        double xo = xi, eo = eta;
                        if (dir == 0) xo = -xi; else eo = -eta;
                        orc_point_state(P, in, nb, xo, eo, ue);
                    } else {
                        double x = P->x0 + (cx + 0.5 * (xi + 1.0)) * hx;
                        double y = P->y0 + (cy + 0.5 * (eta + 1.0)) * hy;
                        double av[ORC_MAXM];
                        for (int c = 0; c < m; ++c) av[c] = cell_coef(P, in, cell, c)[0];
                        exterior_state(P, geo_kind(P, cell, s), s, ui, av, x, y, t, ue);
                    }
                    for (int c = 0; c < m; ++c) {
                        uL[q][c] = (s % 2) ? ui[c] : ue[c];
                        uR[q][c] = (s % 2) ? ue[c] : ui[c];
                    }
                    double a1 = orc_speed(P, uL[q], dir), a2 = orc_speed(P, uR[q], dir);
                    if (a1 > alpha) alpha = a1;
                    if (a2 > alpha) alpha = a2;
                }
                for (int q = 0; q < nfp; ++q) {
                    double fL[ORC_MAXM], fR[ORC_MAXM];
                    orc_flux(P, uL[q], dir, fL);
                    orc_flux(P, uR[q], dir, fR);
                    for (int c = 0; c < m; ++c) {
                        double fhat = 0.5 * (fL[c] + fR[c]) - 0.5 * alpha * (uR[q][c] - uL[q][c]);
                        fnu[q][c] = sgn * fhat;
                    }
                }
            }
            for (int q = 0; q < nfp; ++q) {
                double xi, eta;
                face_point(P, s, q, &xi, &eta);
                double len = dim == 1 ? 1.0 : (dir == 0 ? hy : hx) / 2.0 * P->wg[q];
                for (int j = 0; j < nyq; ++j)
                    for (int i = 0; i < n; ++i) {
                        double v = orc_legendre(i, xi) * (dim == 2 ? orc_legendre(j, eta) : 1.0);
                        for (int c = 0; c < m; ++c) rhs[c * P->nmodes + j * n + i] -= len * fnu[q][c] * v;
                    }
            }
        }
        /* the source (scenario I): + int_K S v, (k+1)-point Gauss rule, at the stage time t */
        if (P->source == 1 && dim == 2) {
            for (int r = 0; r < n; ++r)
                for (int q = 0; q < n; ++q) {
                    double xi = P->xg[q], eta = P->xg[r];
                    double x = P->x0 + (cx + 0.5 * (xi + 1.0)) * hx, y = P->y0 + (cy + 0.5 * (eta + 1.0)) * hy;
                    double src[ORC_MAXM];
                    orc_scenario1_source(P->gamma, x, y, t, src);
                    double jac = hx * hy / 4.0 * P->wg[q] * P->wg[r];
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i) {
                            double v = orc_legendre(i, xi) * orc_legendre(j, eta);
                            for (int c = 0; c < m; ++c) rhs[c * P->nmodes + j * n + i] += jac * src[c] * v;
                        }
                }
        }
        /* divide by the (diagonal, exact) mass matrix */
        for (int j = 0; j < nyq; ++j)
            for (int i = 0; i < n; ++i) {
                double mass = hx / 2.0 * 2.0 / (2.0 * i + 1.0);
                if (dim == 2) mass *= hy / 2.0 * 2.0 / (2.0 * j + 1.0);
                for (int c = 0; c < m; ++c)
                    cell_coef_w(P, out, cell, c)[j * n + i] = rhs[c * P->nmodes + j * n + i] / mass;
            }
    }
    free(rhs);
    drop_high_modes(P, out);  /* P^k: only the retained modes are test functions */
}

/* ------------------------------------------------------------------------ */
/* S_K and the scaling limiter                                               */
/* ------------------------------------------------------------------------ */

/* S_K points (Prop. 2.2 / Fig. 1): 1D the Gauss-Lobatto points; 2D the union of
 * (GL_alpha, G_beta) and (G_beta, GL_alpha).  Returns the count. */
static int sk_points(const orc_problem *P, double *xs, double *ys) {
    int np = 0;
    if (P->dim == 1) {
        for (int a = 0; a < P->L; ++a) { xs[np] = P->xl[a]; ys[np] = 0.0; ++np; }
        return np;
    }
    for (int b = 0; b < P->n; ++b)
        for (int a = 0; a < P->L; ++a) { xs[np] = P->xl[a]; ys[np] = P->xg[b]; ++np; }
    for (int b = 0; b < P->n; ++b)
        for (int a = 0; a < P->L; ++a) { xs[np] = P->xg[b]; ys[np] = P->xl[a]; ++np; }
    return np;
}

#define ORC_MAXP (2 * ORC_MAXN * ORC_MAXN)

static void scale_cell(const orc_problem *P, const double *src, double *dst, int cell, int comp, double theta) {
    const double *a = cell_coef(P, src, cell, comp);
    double *b = cell_coef_w(P, dst, cell, comp);
    b[0] = a[0];
    for (int i = 1; i < P->nmodes; ++i) b[i] = theta * a[i];
}

/* safety margin applied to every theta < 1, then the retry factors */
static const double margin_factor = 1.0 - 9.094947017729282e-13; /* 1 - 2^-40 */
static const double retry_factors[4] = {
    1.0 - 9.313225746154785e-10, /* 1 - 2^-30 */
    1.0 - 9.5367431640625e-07,   /* 1 - 2^-20 */
    1.0 - 0.0009765625,          /* 1 - 2^-10 */
    0.0,
};

static double safe_ratio(double num, double den) {
    if (!(den > 0.0)) return 0.0;
    double t = num / den;
    if (!(t >= 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* The exact theta_2 of one S_K point: along u(t) = ubar + t (u - ubar), rho, m and E are
 * linear in t, so with rho(t) > 0
 *   rho e(u(t)) >= eps  <=>  h(t) = (E(t) - eps) rho(t) - |m(t)|^2 / 2 >= 0,
 * h(t) = a t^2 + b t + c.  h(0) = rho_bar (rho e(ubar) - eps) > 0 for an admissible average
 * and h(1) < 0 at a violating point, so h has exactly one root in (0, 1): the answer.  The
 * roots are taken in the cancellation-free form q = -(b + sign(b) sqrt(b^2 - 4ac)) / 2,
 * roots q / a and c / q.  Returns 1 when the point does not violate (h(1) >= 0). */
static double theta2_point(const orc_problem *P, const double *ubar, const double *u) {
    int dim = P->dim;
    double eps = P->eps;
    double dr = u[0] - ubar[0], dE = u[dim + 1] - ubar[dim + 1];
    double mm = 0.0, md = 0.0, dd = 0.0;
    for (int d = 1; d <= dim; ++d) {
        double dm = u[d] - ubar[d];
        mm += ubar[d] * ubar[d];
        md += ubar[d] * dm;
        dd += dm * dm;
    }
    double c = (ubar[dim + 1] - eps) * ubar[0] - 0.5 * mm;
    double b = (ubar[dim + 1] - eps) * dr + dE * ubar[0] - md;
    double a = dE * dr - 0.5 * dd;
    if (!(c > 0.0)) return 0.0;     /* the average itself is not strictly inside */
    if (a + b + c >= 0.0) return 1.0; /* h(1) >= 0: no violation at this point */
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) disc = 0.0;
    double q = -0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
    double best = 0.0;
    int found = 0;
    double r[2];
    int nr = 0;
    if (a != 0.0) r[nr++] = q / a;
    if (q != 0.0) r[nr++] = c / q;
    for (int i = 0; i < nr; ++i)
        if (r[i] > 0.0 && r[i] < 1.0 && (!found || r[i] < best)) {
            best = r[i];
            found = 1;
        }
    return found ? best : 0.0;
}

long long orc_limit(const orc_problem *P, double *c, double *theta_out) {
    double xs[ORC_MAXP], ys[ORC_MAXP];
    int np = sk_points(P, xs, ys);
    int m = P->m;
    long long nlim = 0;
    double *trial = (double *)malloc(sizeof(double) * orc_state_size(P));
    memcpy(trial, c, sizeof(double) * orc_state_size(P));
    for (int cell = 0; cell < P->ncell; ++cell) {
        if (orc_is_solid(P, cell)) { /* outside the domain */
            if (theta_out) theta_out[cell] = 1.0;
            continue;
        }
        double theta_rep = 1.0;
        if (P->flux != ORC_FLUX_EULER) {
            double ub = cell_coef(P, c, cell, 0)[0];
            double Mk = -INFINITY, mk = INFINITY;
            for (int p = 0; p < np; ++p) {
                double v = eval_modal(P, cell_coef(P, c, cell, 0), xs[p], ys[p]);
                if (v > Mk) Mk = v;
                if (v < mk) mk = v;
            }
            double th = 1.0;
            if (Mk > P->hi) { double t1 = safe_ratio(P->hi - ub, Mk - ub); if (t1 < th) th = t1; }
            if (mk < P->lo) { double t2 = safe_ratio(ub - P->lo, ub - mk); if (t2 < th) th = t2; }
            if (th < 1.0) {
                th *= margin_factor;
                double tha = th;
                for (int attempt = 0; attempt <= 4; ++attempt) {
                    tha = attempt == 0 ? th : th * retry_factors[attempt - 1];
                    scale_cell(P, c, trial, cell, 0, tha);
                    int ok = 1;
                    for (int p = 0; p < np && ok; ++p) {
                        double v = eval_modal(P, cell_coef(P, trial, cell, 0), xs[p], ys[p]);
                        if (!(v >= P->lo && v <= P->hi)) ok = 0;
                    }
                    if (ok) break;
                }
                scale_cell(P, c, c, cell, 0, tha);
                theta_rep = tha;
                ++nlim;
            }
        } else {
            double eps = P->eps;
            /* eq. (Euler-limiter1): density */
            double rb = cell_coef(P, c, cell, 0)[0];
            double rmin = INFINITY;
            for (int p = 0; p < np; ++p) {
                double v = eval_modal(P, cell_coef(P, c, cell, 0), xs[p], ys[p]);
                if (v < rmin) rmin = v;
            }
            double th1 = 1.0;
            if (rmin < eps) {
                th1 = safe_ratio(rb - eps, rb - rmin) * margin_factor;
                scale_cell(P, c, c, cell, 0, th1);
            }
            /* eq. (Euler-limiter2): internal energy rho*e with the limited density */
            double ubar[ORC_MAXM];
            for (int comp = 0; comp < m; ++comp) ubar[comp] = cell_coef(P, c, cell, comp)[0];
            double reb = rho_e(P, ubar);
            double remin = INFINITY;
            for (int p = 0; p < np; ++p) {
                double u[ORC_MAXM];
                orc_point_state(P, c, cell, xs[p], ys[p], u);
                double re = rho_e(P, u);
                if (!(re >= remin)) remin = re; /* NaN propagates as a violation */
            }
            double th2 = 1.0;
            if (!(remin >= eps)) {
                if (P->theta2_exact) {
                    /* the smallest per-point solution over the violating points */
                    double tmin = 1.0;
                    for (int p = 0; p < np; ++p) {
                        double u[ORC_MAXM];
                        orc_point_state(P, c, cell, xs[p], ys[p], u);
                        double re = rho_e(P, u);
                        if (re >= eps) continue;
                        double tq = re == re ? theta2_point(P, ubar, u) : 0.0;
                        if (tq < tmin) tmin = tq;
                    }
                    th2 = tmin * margin_factor;
                } else {
                    th2 = safe_ratio(reb - eps, reb - remin) * margin_factor;
                }
            }
            if (th1 < 1.0 || th2 < 1.0) {
                /* verify rho >= eps and rho e >= eps on S_K; shrink the final scaling */
                double tha = th2;
                for (int attempt = 0; attempt <= 4; ++attempt) {
                    tha = attempt == 0 ? th2 : th2 * retry_factors[attempt - 1];
                    for (int comp = 0; comp < m; ++comp) scale_cell(P, c, trial, cell, comp, tha);
                    int ok = 1;
                    for (int p = 0; p < np && ok; ++p) {
                        double u[ORC_MAXM];
                        orc_point_state(P, trial, cell, xs[p], ys[p], u);
                        if (!(u[0] >= eps && rho_e(P, u) >= eps)) ok = 0;
                    }
                    if (ok) break;
                }
                for (int comp = 0; comp < m; ++comp) scale_cell(P, c, c, cell, comp, tha);
                th2 = tha;
            }
            theta_rep = th1 < th2 ? th1 : th2;
            if (theta_rep < 1.0) ++nlim;
        }
        if (theta_out) theta_out[cell] = theta_rep;
    }
    free(trial);
    return nlim;
}

int orc_averages_admissible(const orc_problem *P, const double *c) {
    int m = P->m;
    for (int cell = 0; cell < P->ncell; ++cell) {
        if (orc_is_solid(P, cell)) continue;
        double ub[ORC_MAXM];
        for (int comp = 0; comp < m; ++comp) ub[comp] = cell_coef(P, c, cell, comp)[0];
        if (P->flux == ORC_FLUX_EULER) {
            if (!(ub[0] >= P->eps)) return 0;
            if (!(rho_e(P, ub) >= P->eps)) return 0;
        } else {
            if (!(ub[0] >= P->lo && ub[0] <= P->hi)) return 0;
        }
    }
    return 1;
}

void orc_min_margins(const orc_problem *P, const double *c, double *margins2) {
    double xs[ORC_MAXP], ys[ORC_MAXP];
    int np = sk_points(P, xs, ys);
    double m0 = INFINITY, m1 = INFINITY;
    for (int cell = 0; cell < P->ncell; ++cell)
        for (int p = 0; p < np && !orc_is_solid(P, cell); ++p) {
            double u[ORC_MAXM];
            orc_point_state(P, c, cell, xs[p], ys[p], u);
            double a, b;
            if (P->flux == ORC_FLUX_EULER) {
                a = u[0] - P->eps;
                b = rho_e(P, u) - P->eps;
            } else {
                a = u[0] - P->lo;
                b = P->hi - u[0];
            }
            if (!(a >= m0)) m0 = a;
            if (!(b >= m1)) m1 = b;
        }
    margins2[0] = m0;
    margins2[1] = m1;
}

double orc_a0(const orc_problem *P, const double *c) {
    double xs[ORC_MAXP], ys[ORC_MAXP];
    int np = sk_points(P, xs, ys);
    double a0 = 0.0;
    for (int cell = 0; cell < P->ncell; ++cell)
        for (int p = 0; p < np && !orc_is_solid(P, cell); ++p) {
            double u[ORC_MAXM];
            orc_point_state(P, c, cell, xs[p], ys[p], u);
            for (int d = 0; d < P->dim; ++d) {
                double s = orc_speed(P, u, d);
                if (s > a0) a0 = s;
            }
        }
    return a0;
}

double orc_max_dt(const orc_problem *P, const double *c, double cfl) {
    /* eq. (numerical_experiment:CFL), dt = CFL dx / a0, with the directional spectral
     * radii summed over the dimensions: dt = CFL / max_{S_K} sum_d lambda_d / h_d.  In 1D this
     * is the printed formula; in 2D it is the Cartesian form for which the (1D, Fourier)
     * stability CFL numbers of the Remark in Sec. 3.2 keep the scheme linearly stable. */
    double xs[ORC_MAXP], ys[ORC_MAXP];
    int np = sk_points(P, xs, ys);
    double rate = 0.0;
    for (int cell = 0; cell < P->ncell; ++cell)
        for (int p = 0; p < np && !orc_is_solid(P, cell); ++p) {
            double u[ORC_MAXM];
            orc_point_state(P, c, cell, xs[p], ys[p], u);
            double r = orc_speed(P, u, 0) / P->hx;
            if (P->dim == 2) r += orc_speed(P, u, 1) / P->hy;
            if (r > rate) rate = r;
        }
    return cfl / rate;
}

/* ------------------------------------------------------------------------ */
/* troubled-cell indicator and shock limiter (optional; not in the paper)    */
/* ------------------------------------------------------------------------ */

static double minmod3(double a, double b, double c) {
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* average of the neighbour across side s, following the boundary condition */
static void neighbour_average(const orc_problem *P, const double *c, int cell, int s, double *ub) {
    int nb = neighbour(P, cell, s);
    int m = P->m;
    if (nb >= 0) {
        for (int comp = 0; comp < m; ++comp) ub[comp] = cell_coef(P, c, nb, comp)[0];
        return;
    }
    double own[ORC_MAXM];
    for (int comp = 0; comp < m; ++comp) own[comp] = cell_coef(P, c, cell, comp)[0];
    exterior_state(P, geo_kind(P, cell, s), s, own, own, 0.0, 0.0, 0.0, ub);
}

long long orc_troubled_cells(const orc_problem *P, const double *c, int *flags) {
    int n = P->n, m = P->m;
    long long count = 0;
    for (int cell = 0; cell < P->ncell; ++cell) {
        int troubled = 0;
        for (int dir = 0; dir < P->dim && !troubled && !orc_is_solid(P, cell); ++dir) {
            double h = dir == 0 ? P->hx : P->hy;
            double ulo[ORC_MAXM], uhi[ORC_MAXM];
            neighbour_average(P, c, cell, 2 * dir, ulo);
            neighbour_average(P, c, cell, 2 * dir + 1, uhi);
            for (int comp = 0; comp < m && !troubled; ++comp) {
                const double *a = cell_coef(P, c, cell, comp);
                /* face averages of the traces: only the modes constant along the face survive */
                double fp = 0.0, fm = 0.0;
                for (int i = 1; i < n; ++i) {
                    double ci = dir == 0 ? a[i] : a[i * n];
                    fp += ci;                       /* P_i(+1) = 1 */
                    fm += (i % 2 ? -1.0 : 1.0) * ci; /* P_i(-1) = (-1)^i */
                }
                double utR = fp, utL = -fm;
                double dp = uhi[comp] - a[0], dm = a[0] - ulo[comp];
                double thr = P->tvb_M * h * h;
                double mR = fabs(utR) <= thr ? utR : minmod3(utR, dp, dm);
                double mL = fabs(utL) <= thr ? utL : minmod3(utL, dp, dm);
                if (mR != utR || mL != utL) troubled = 1;
            }
        }
        flags[cell] = troubled;
        count += troubled;
    }
    return count;
}

void orc_shock_limit(const orc_problem *P, double *c, const int *flags) {
    int n = P->n, m = P->m;
    double *out = (double *)malloc(sizeof(double) * orc_state_size(P));
    memcpy(out, c, sizeof(double) * orc_state_size(P));
    for (int cell = 0; cell < P->ncell; ++cell) {
        if (!flags[cell]) continue;
        double nbr[4][ORC_MAXM];
        for (int s = 0; s < 2 * P->dim; ++s) neighbour_average(P, c, cell, s, nbr[s]);
        for (int comp = 0; comp < m; ++comp) {
            const double *a = cell_coef(P, c, cell, comp);
            double *b = cell_coef_w(P, out, cell, comp);
            double ub = a[0];
            double cx = n > 1 ? a[1] : 0.0;
            double newx = minmod3(cx, nbr[1][comp] - ub, ub - nbr[0][comp]);
            double newy = 0.0;
            if (P->dim == 2) newy = minmod3(a[n], nbr[3][comp] - ub, ub - nbr[2][comp]);
            for (int q = 0; q < P->nmodes; ++q) b[q] = 0.0;
            b[0] = ub;
            b[1] = newx;
            if (P->dim == 2) b[n] = newy;
        }
    }
    memcpy(c, out, sizeof(double) * orc_state_size(P));
    free(out);
}

/* ------------------------------------------------------------------------ */
/* time stepping: Scheme 1L                                                  */
/* ------------------------------------------------------------------------ */

/* one attempt; ws holds (2s+2) states of scratch.  Returns 0 or the failing stage. */
static int attempt_step(const orc_problem *P, const double *cn, double dt, int s, const double *A,
                        const double *b, double t, double *out, double *u_stage, double *ut_stage,
                        long long *nlim, double *thmin) {
    size_t N = orc_state_size(P);
    double *ut = (double *)malloc(sizeof(double) * N * s);    /* limited stages */
    double *Gs = (double *)malloc(sizeof(double) * N * s);    /* G(ut_j) */
    double *Fs = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * N);
    double *theta = (double *)malloc(sizeof(double) * P->ncell);
    int *have_g = (int *)calloc(s, sizeof(int));
    double cst[ORC_MAXS];
    int fail = 0;
    for (int i = 0; i < s; ++i) {
        cst[i] = 0.0;
        for (int j = 0; j < s; ++j) cst[i] += A[i * s + j];
    }
    memcpy(ut, cn, sizeof(double) * N); /* stage 1: u^(1) = u^n, already limited */
    if (u_stage) { memcpy(u_stage, cn, sizeof(double) * N); memcpy(ut_stage, cn, sizeof(double) * N); }
    for (int i = 1; i < s && !fail; ++i) {
        /* u^(i) = u^n + dt sum_{j<i} a_ij G(ut^(j)); the standard RKDG (eq. rkdg) takes F */
        memcpy(u, cn, sizeof(double) * N);
        for (int j = 0; j < i; ++j) {
            double a = A[i * s + j];
            if (a == 0.0) continue;
            if (!have_g[j]) {
                orc_apply(P, P->standard ? ORC_OP_F : ORC_OP_G, ut + N * j, Gs + N * j, t + cst[j] * dt);
                have_g[j] = 1;
            }
            for (size_t q = 0; q < N; ++q) u[q] += dt * a * Gs[N * j + q];
        }
        if (u_stage) memcpy(u_stage + N * i, u, sizeof(double) * N);
        if (!orc_averages_admissible(P, u)) { fail = i + 1; break; }
        if (P->limiter_on) {
            *nlim += orc_limit(P, u, theta);
            for (int q = 0; q < P->ncell; ++q) if (theta[q] < *thmin) *thmin = theta[q];
        }
        memcpy(ut + N * i, u, sizeof(double) * N);
        if (ut_stage) memcpy(ut_stage + N * i, u, sizeof(double) * N);
    }
    if (!fail) {
        /* u^{n+1} = u^n + dt sum_i b_i F(ut^(i)) */
        memcpy(u, cn, sizeof(double) * N);
        for (int i = 0; i < s; ++i) {
            if (b[i] == 0.0) continue;
            orc_apply(P, ORC_OP_F, ut + N * i, Fs, t + cst[i] * dt);
            for (size_t q = 0; q < N; ++q) u[q] += dt * b[i] * Fs[q];
        }
        if (u_stage) memcpy(u_stage + N * s, u, sizeof(double) * N);
        if (!orc_averages_admissible(P, u)) {
            fail = s + 1;
        } else {
            if (P->indicator) {
                int *flags = (int *)malloc(sizeof(int) * P->ncell);
                orc_troubled_cells(P, u, flags);
                orc_shock_limit(P, u, flags);
                free(flags);
            }
            if (P->limiter_on) {
                *nlim += orc_limit(P, u, theta);
                for (int q = 0; q < P->ncell; ++q) if (theta[q] < *thmin) *thmin = theta[q];
            }
            if (ut_stage) memcpy(ut_stage + N * s, u, sizeof(double) * N);
            if (out) memcpy(out, u, sizeof(double) * N);
        }
    }
    free(ut); free(Gs); free(Fs); free(u); free(theta); free(have_g);
    return fail;
}

int orc_step(const orc_problem *P, double *c, double dt, int s, const double *A, const double *b,
             double t, orc_info *info) {
    size_t N = orc_state_size(P);
    double *out = (double *)malloc(sizeof(double) * N);
    int rc = 4;
    for (int r = 0; r <= P->max_halvings; ++r) {
        long long nlim = 0;
        double thmin = 1.0;
        int fail = attempt_step(P, c, dt, s, A, b, t, out, NULL, NULL, &nlim, &thmin);
        if (!fail) {
            memcpy(c, out, sizeof(double) * N);
            if (info) {
                info->dt_taken = dt;
                info->restarts = r;
                info->cells_limited = nlim;
                info->theta_min = thmin;
            }
            rc = 0;
            break;
        }
        dt *= 0.5;
    }
    free(out);
    return rc;
}

int orc_step_stages(const orc_problem *P, const double *c, double dt, int s, const double *A,
                    const double *b, double t, double *u_stage, double *ut_stage) {
    long long nlim = 0;
    double thmin = 1.0;
    return attempt_step(P, c, dt, s, A, b, t, NULL, u_stage, ut_stage, &nlim, &thmin);
}

/* ------------------------------------------------------------------------ */
/* diagnostics                                                               */
/* ------------------------------------------------------------------------ */

double orc_total_mass(const orc_problem *P, const double *c, int comp) {
    /* sum_K |K| ubar_K over the domain's cells, summed in cell order */
    double s = 0.0;
    for (int cell = 0; cell < P->ncell; ++cell)
        if (!orc_is_solid(P, cell)) s += cell_coef(P, c, cell, comp)[0];
    return s * P->hx * P->hy;
}

static double error_norm(const orc_problem *P, const double *c, double t, int nq, int p) {
    double xq[16], wq[16];
    if (nq > 16) nq = 16;
    orc_gauss_legendre(nq, xq, wq);
    int nyq = P->dim == 2 ? nq : 1;
    double s = 0.0;
    for (int cell = 0; cell < P->ncell; ++cell) {
        int cx = cell % P->nx, cy = cell / P->nx;
        for (int r = 0; r < nyq; ++r)
            for (int q = 0; q < nq; ++q) {
                double xi = xq[q], eta = P->dim == 2 ? xq[r] : 0.0;
                double u[ORC_MAXM], ue[ORC_MAXM];
                orc_point_state(P, c, cell, xi, eta, u);
                double x = P->x0 + (cx + 0.5 * (xi + 1.0)) * P->hx;
                double y = P->y0 + (cy + 0.5 * (eta + 1.0)) * P->hy;
                P->exact(x, y, t, ue, P->exact_ctx);
                double wgt = (P->dim == 2 ? wq[q] * wq[r] * P->hx * P->hy / 4.0 : wq[q] * P->hx / 2.0);
                for (int comp = 0; comp < P->m; ++comp) {
                    double d = fabs(u[comp] - ue[comp]);
                    s += wgt * (p == 2 ? d * d : d);
                }
            }
    }
    return p == 2 ? sqrt(s) : s;
}

double orc_l2_error_exact(const orc_problem *P, const double *c, double t, int nq) {
    return error_norm(P, c, t, nq, 2);
}

double orc_l1_error_exact(const orc_problem *P, const double *c, double t, int nq) {
    return error_norm(P, c, t, nq, 1);
}
