// dg_types.h -- plain data shared by the host API and the kernels of the cRKDG
// library (no device code here).  Nodal Q^k tables, step parameters and the
// device buffer set one launch works on.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace crkdg {

constexpr int MAXN = 4;  // nodes per direction (k <= 3)
constexpr int MAXM = 4;  // conservative components (2D Euler)
constexpr int MAXS = 4;  // Runge--Kutta stages

enum Phys { PH_ADV = 0, PH_BURG = 1, PH_EULER = 2 };
enum Bc { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2, BC_DIRICHLET = 3 };

// Operator modes of the inner / final kernels.
enum Mode {
    MODE_STEP = 0,   // one limited cRKDG step (Scheme 1L)
    MODE_OP_G = 1,   // inner kernel writes G(u) instead of the stage accumulation
    MODE_OP_F = 2,   // final kernel adds the face correction only (no limiter, no checks)
    MODE_RATE = 3,   // scan kernels: the trial-step rate only (no bound margins)
    MODE_LIMIT_CHECK = 4,  // limiter kernel: also test the averages and count limited cells
    MODE_LIMIT_FINAL = 5,  // as MODE_LIMIT_CHECK, and post the trial-step rate of the result
};

__host__ __device__ constexpr int ncomp(int phys, int dim) { return phys == PH_EULER ? dim + 2 : 1; }
// Gauss--Lobatto points of S_K: L = ceil((k+3)/2), the smallest rule exact for degree k.
__host__ __device__ constexpr int nlob(int n) { return (n + 3) / 2; }
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
// Cells per block of the thread-per-node kernels: whole warps of whole cells,
// at least 128 threads.
__host__ __device__ constexpr int warp_cells(int nn) { return nn * 32 / gcd_c(nn, 32); }  // lcm(nn, 32)
__host__ __device__ constexpr int cells_per_block(int dim, int n) {
    return (warp_cells(dim == 2 ? n * n : n) / (dim == 2 ? n * n : n)) *
           (warp_cells(dim == 2 ? n * n : n) >= 128 ? 1 : 128 / warp_cells(dim == 2 ? n * n : n));
}

// One-dimensional nodal tables for n = k+1 Gauss points on [-1, 1].
struct NodalTables {
    double xg[MAXN], wg[MAXN];  // Gauss--Legendre nodes / weights (sum 2)
    double xl[MAXN], wl[MAXN];  // Gauss--Lobatto nodes / weights
    double Dhat[MAXN][MAXN];    // Dhat[a][q] = w_q l_a'(x_q) / w_a  (volume term)
    double lm[MAXN], lp[MAXN];  // l_a(-1), l_a(+1)                 (traces)
    double liftm[MAXN], liftp[MAXN];  // l_a(-1)/w_a, l_a(+1)/w_a    (lift)
    double Igl[MAXN][MAXN];     // Igl[alpha][a] = l_a(xl_alpha)   (S_K interpolation)
    double w1[MAXN];            // w_a / 2                          (1D average weights)
    double w2[MAXN * MAXN];     // (w_a/2)(w_b/2) at node b*n+a      (2D average weights)
    // products of the tables the troubled-cell and feature kernels weigh node values by,
    // host-computed with the kernels' association of the factors (the sums are unchanged)
    double mom2[MAXN * MAXN];        // (3 w1_a) w1_b at node b*n+a: 2D first moments
    double trw2[2][2][MAXN * MAXN];  // [dir][R, L] w1_across l_along(+1 / -1): 2D face averages
    double pm2[2][MAXN * MAXN];      // [dir] ((3 w1_a) w1_b) x_along: 2D first moments along dir
    double pm1[MAXN];                // (3 w1_a) x_a: 1D first moment
    float momxf[MAXN * MAXN], momyf[MAXN * MAXN];  // FP32 ((3 w1_a) w1_b) x_a, ... x_b: 2D first moments
    // FP32 copies for the split-precision path
    float Dhatf[MAXN][MAXN], lmf[MAXN], lpf[MAXN], liftmf[MAXN], liftpf[MAXN], Iglf[MAXN][MAXN];
    float w1f[MAXN], w2f[MAXN * MAXN];
    // the L2 projection of Q^k nodal values onto the total-degree space P^k (2D): node b*n+a
    // from node q, sum over the Legendre modes i + j <= k of L_i(x_a) L_j(x_b) times the
    // Gauss-rule coefficient of that mode at node q
    double pk[MAXN * MAXN][MAXN * MAXN];
};

// FP32 copies of the parameters for the split-precision kernels, rounded once by
// the host at launch (the kernels then never convert a double parameter).
struct ParamsF {
    float rhx, rhy, gamma, gm1, velx, vely, lo, hi, eps;
    float thr[2];  // (float) of Params::thr
    float bcs[4][MAXM];
    float dtA[MAXS][MAXS];  // (float)(dt a_ij)
    float dtb[MAXS];        // (float)(dt b_i)
    float b[MAXS];
    float dt;
};

struct Params {
    int nx, ny, ncell;
    double rhx, rhy;  // 2/hx, 2/hy
    double gamma, velx, vely;
    double lo, hi, eps;
    int bc[4];
    double bcs[4][MAXM];
    int s;
    double A[MAXS][MAXS];
    double b[MAXS];
    int slot[MAXS];  // trace slot of stage i, -1 when b_i = 0
    int nslot;
    double dt;
    int mode;
    int defer_limit;  // final kernel leaves the limiter to the troubled-cell kernel
    double tvb_M;     // TVB constant of the plain indicator
    double thr[2];    // its thresholds M h_x^2, M h_y^2 (h_d = 2 / rh_d), set by tvb_thresholds
    double thr_feat;  // M h_x h_y: the learned indicator's feature scale floor
    // FP32 bounds of the FP64 limiter's screen, set by screen_bounds: eps and lo rounded up,
    // hi rounded down (scr_on = 0: the screen clears nothing)
    int scr_on;
    float scr_eps, scr_lo, scr_hi;
    int ind_stage;    // troubled-cell kernel: 0 decide and limit, 2 limit the given flags (the feature
                      // kernel decided), 3 combine the given plain flags with the learned
                      // probabilities, then limit; 4 (split path) decide, combine with the
                      // learned probabilities, then limit
    ParamsF f;        // split-precision kernels only
    // Owned box of a subdomain (domain decomposition): cells [own[0], own[1]) x [own[2], own[3])
    // of this mesh.  With own_on, only those cells count in the admissibility flag, the limiter
    // statistics, the trial-step rate and the bound margins; the other cells (the halo ring)
    // are still computed, so that the owned cells' final stage reads their traces.
    int own_on;
    int own[4];
    // theta_2 of the Euler limiter: 0 the concavity ratio of eq. (Euler-limiter2), 1 the exact
    // per-point solve (theta2_point)
    int theta2_exact;
    // the manufactured source of Example 4.2's scenario I (2D Euler) added to G at the nodes:
    // 0 off, 1 on; t0 the time of u^n (stage i at t0 + c_i dt), x0, y0 the mesh's lower corner
    int source;
    double t0, x0, y0;
    // 1: the total-degree space P^k (2D): stage values, u* and u^{n+1} projected (NodalTables::pk)
    int pk;
    // Non-rectangular domain (Examples 4.8 and 4.9) or null: one word per cell (device memory),
    // bits 4s..4s+3 the boundary kind of side s (GEO_*), GEO_SOLID a cell outside the domain.
    // Solid cells keep u^n (their operators are zero) and count in no test, statistic or rate.
    const unsigned *geo;
    double gstate[2][MAXM];          // the fixed states A and B of the GEO_STATE_* / GEO_SHOCK kinds
    double shock_x0, shock_speed;    // GEO_SHOCK: state A where x < shock_x0 + shock_speed t
};

// Boundary kinds of a side in a geometry word: the mesh rule (the neighbouring cell, or the
// rectangle side's condition), reflective wall, outflow, fixed state A, fixed state B, and a
// planar shock's exact trace (state A behind x_s(t) = shock_x0 + shock_speed t, B ahead).
enum GeoKind { GEO_MESH = 0, GEO_WALL = 1, GEO_OUTFLOW = 2, GEO_STATE_A = 3, GEO_STATE_B = 4, GEO_SHOCK = 5 };
constexpr unsigned GEO_SOLID = 0x10000u;

// A cell outside a non-rectangular domain (device side; never without a geometry).
__device__ __forceinline__ bool solid_cell(const Params &P, int cell) {
    return P.geo != nullptr && (P.geo[cell] & GEO_SOLID) != 0u;
}

// Cells outside the owned box are halo cells (never when own_on is 0).
__host__ __device__ __forceinline__ bool owned(const Params &P, int cell) {
    if (!P.own_on) return true;
    const int cy = cell / P.nx, cx = cell - cy * P.nx;
    return cx >= P.own[0] && cx < P.own[1] && cy >= P.own[2] && cy < P.own[3];
}

// The TVB thresholds from rhx, rhy and tvb_M (host side, once per parameter set).
inline void tvb_thresholds(Params &P) {
    const double hx = 2.0 / P.rhx, hy = 2.0 / P.rhy;
    P.thr[0] = P.tvb_M * hx * hx;
    P.thr[1] = P.tvb_M * hy * hy;
    P.thr_feat = P.tvb_M * (2.0 / P.rhx) * (2.0 / P.rhy);
}

// The FP32 bounds of the FP64 limiter's screen (host side): floats on the safe side of
// eps, lo and hi, moved a further 2^-20 inwards.
inline float float_at_least(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}
inline float float_at_most(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}
inline void screen_bounds(Params &P) {
    const float in = 9.5367431640625e-07f;  // 2^-20
    P.scr_eps = float_at_least(P.eps) * (1.0f + in);
    P.scr_lo = float_at_least(P.lo);
    P.scr_lo = P.scr_lo + in * fabsf(P.scr_lo);
    P.scr_hi = float_at_most(P.hi);
    P.scr_hi = P.scr_hi - in * fabsf(P.scr_hi);
    P.scr_on = 1;
}

struct Bufs {
    const double *un;   // u^n (nodal, state layout)
    double *ustar;      // u^n + dt sum_i b_i G(u~^(i))   (or G(u) in MODE_OP_G)
    double *unew;       // u^{n+1}
    double *tr;         // face traces of u~^(i): [slot][m][cell][face point]
    double *tavg;       // cell averages of the same u~^(i): [slot][m][cell] (outflow exterior state)
    double *tfs = nullptr;  // optional: normal fluxes and spectral radii of the traces,
                            // [slot][m + 1][cell][face point] (the final kernel recomputes them when null)
    int *flag;          // set when a stage average leaves B
    unsigned long long *nlim;   // limited cells
    unsigned long long *thmin;  // bits of the smallest theta (non-negative double)
    unsigned long long *a0;     // bits of the largest spectral radius (non-negative double)
    double *aux;        // per-cell output of the utility kernels
    unsigned long long *ord;    // two order-preserving mins (margins)
    int *tflags;        // troubled-cell flags (one per cell) or nullptr
    unsigned long long *ntrb;   // number of troubled cells
    float *feat;        // MLP features [cell][44]
    const float *prob;  // MLP probabilities [cell]
};

enum KernelId { K_INNER = 0, K_FINAL = 1, K_LIMIT = 2, K_A0 = 3, K_MARGINS = 4, K_AVG = 5, K_TROUBLE = 6,
                K_FEATURES = 7 };

// Buffers of the split-precision path: FP64 cell averages plus FP32 nodal
// deviations (the polynomial is ubar + (dev - mean_w dev)).
struct MixBufs {
    const double *ub;   // averages of u^n            [m][cell]
    const float *dv;    // deviations of u^n          [m][cell][n^d]
    float *dv_s;        // deviations of u* = u^n + dt sum_i b_i G(u~^(i))
    double *ub_n;       // averages of u^{n+1}
    float *dv_n;        // deviations of u^{n+1}
    float *tr;          // FP32 face traces           [slot][m][cell][face point]
    float *tavg;        // FP32 cell averages of the traced stages [slot][m][cell]
    const double *nod_in;  // FP64 nodal input (split, operators)
    double *nod_out;       // FP64 nodal output (merge, operators)
    int *flag;
    unsigned long long *nlim, *thmin, *a0, *ord;
    double *aux;
    int *tflags;              // troubled-cell flags (indicator on)
    const float *prob;        // learned probabilities (ind_stage 3, 4)
    float *feat;              // learned indicator's features [cell][44] (k_features_x)
    unsigned long long *ntrb; // troubled cells
};

enum MixKernelId { KX_SPLIT = 0, KX_MERGE = 1, KX_LIMIT = 2, KX_INNER = 3, KX_FINAL = 4, KX_SCAN = 5, KX_AVG = 6,
                   KX_TROUBLE = 7, KX_FEATURES = 8 };

// ---------------------------------------------------------------- ensembles (2D Euler)

// Scalars of one problem's current attempt.
struct EnsScal {
    int flag;                 // a stage average left B^eps
    int pad;
    unsigned long long nlim;  // limited cells
    unsigned long long thmin; // bits of the smallest theta
    unsigned long long a0;    // bits of the rate of the new state
    unsigned long long ord[2];
    unsigned long long ntrb;  // troubled cells
};

// Descriptor of one problem of an ensemble (device table, one per problem).
struct EnsProblem {
    Params P;                // its parameters; P.dt is the step of the current attempt
    double *u[2];            // u[cur] holds u^n, u[cur ^ 1] receives u^{n+1}
    double *ustar, *tr, *tavg, *aux;
    int *tflags;
    float *feat;
    const float *prob;
    EnsScal *sc;
    int n;                   // k + 1
    int cur;
    int pending;             // takes part in the current attempt
    int done;                // reached t_end
    int status;              // 0, or CRKDG_E_BOUNDS after max_halvings
    int restarts;            // halvings of the current step
    int klass;               // (n - 3) * 3 + size class, for tuning
    int pad;
    double t, t_end, cfl, a0;
    long long steps, restarts_total;
    // the last accepted step
    double last_dt, last_thmin;
    long long last_nlim, last_ntrb;
    int last_restarts, pad2;
};

// Work item: blocks [blk, blk + nblk) of problem prob.
struct EnsItem {
    int prob, blk, nblk, pad;
};

enum { ENS_COUNTERS = 16 };
enum EnsKernelKind { ENS_INNER = 0, ENS_FINAL = 1, ENS_TROUBLE = 2, ENS_FEATURES = 3 };
struct EnsCtl {
    unsigned int counter[ENS_COUNTERS];  // one work counter per persistent launch of an attempt
    int any_pending;
    int pad[3];
};

// Scalars of one attempt of the device-resident step loop (three rotate).
struct RunSlot {
    int flag;
    int pad;
    unsigned long long nlim;
    unsigned long long thmin;
    unsigned long long rate;  // bits of max over S_K of sum_d lambda_d / h_d
};

// Control block of the persistent 1D run kernel (device memory).
struct RunCtl {
    // inputs
    double t, t_end, dt0, cfl;
    int nsteps, max_halvings, cur;
    int extra_arrivals;  // testing aid: > 0 makes the barrier wait for blocks that never come
    // outputs
    double t_out, rate_out;
    int steps, restarts, cur_out, status;
    unsigned long long nlim_total;
    // grid barrier: arrivals so far (zero at launch)
    unsigned bar_count, pad_;
    RunSlot slot[3];
};

// Status values written by the run kernel (match crkdg_status).
enum RunStatus { RUN_OK = 0, RUN_BOUNDS = 4, RUN_TIMEOUT = 5 };

}  // namespace crkdg

// Per-dimension launchers (defined in dg_1d.cu / dg_2d.cu).
extern "C++" {
cudaError_t crkdg_upload_tables_1d(const crkdg::NodalTables *t);
cudaError_t crkdg_upload_tables_2d(const crkdg::NodalTables *t);
cudaError_t crkdg_launch_1d(int kernel, int n, int phys, int nblocks, cudaStream_t st,
                            const crkdg::Params &P, const crkdg::Bufs &B);
cudaError_t crkdg_launch_2d(int kernel, int n, int phys, int nblocks, cudaStream_t st,
                            const crkdg::Params &P, const crkdg::Bufs &B);
cudaError_t crkdg_launch_mx_1d(int kernel, int n, int phys, int nblocks, cudaStream_t st,
                               const crkdg::Params &P, const crkdg::MixBufs &B);
cudaError_t crkdg_launch_mx_2d(int kernel, int n, int phys, int nblocks, cudaStream_t st,
                               const crkdg::Params &P, const crkdg::MixBufs &B);
// Ensembles of 2D Euler problems (defined in dg_ens.cu).
cudaError_t crkdg_upload_tables_ens(const crkdg::NodalTables *t);
cudaError_t crkdg_ens_launch(int kind, int n, int grid, cudaStream_t st, crkdg::EnsProblem *E,
                             const crkdg::EnsItem *items, int nitems, crkdg::EnsCtl *ctl, int counter, int stage);
int crkdg_ens_occupancy(int kind, int n);
int crkdg_ens_cells_per_block(int kind, int n);
// which: 0 open a step (arg: size class or -1), 1 clear the counters, 2 close an attempt (arg: max_halvings)
cudaError_t crkdg_ens_control(int which, cudaStream_t st, crkdg::EnsProblem *E, int np, crkdg::EnsCtl *ctl, int arg);
// Inner stages of the split-precision path on the tensor cores (2D Euler, n = 4, MODE_STEP,
// tableaux whose A has only a sub-diagonal; defined in dg_2d.cu).
cudaError_t crkdg_launch_inner_tc(cudaStream_t st, const crkdg::Params &P, const crkdg::MixBufs &X);
// Closed-form nodal tables for n = 2, 3, 4 (defined in crkdg_api.cu).
void crkdg_build_tables(crkdg::NodalTables *tab);
// Persistent 1D step loop (cooperative launch); chunk: own cells per block chunk (0: fill
// every block slot of the GPU); *nblocks receives the grid used.
cudaError_t crkdg_run_1d(int n, int phys, cudaStream_t st, const crkdg::Params &P, double *u0, double *u1,
                         crkdg::RunCtl *ctl, int chunk, int *nblocks);
}
