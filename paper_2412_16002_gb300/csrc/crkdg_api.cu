// crkdg_api.cu -- the C ABI of include/crkdg.h: argument checks, device
// buffers, the nodal tables, and the Sec. 4.1 restart loop around the
// inner-stage and final-stage kernels.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/crkdg.h"
#include "dg_types.h"

using namespace crkdg;

namespace {

// Device-side scalars written by the kernels of one step.
struct DevScal {
    int flag;
    int pad;
    unsigned long long nlim;
    unsigned long long thmin;
    unsigned long long a0;
    unsigned long long ord[2];
    unsigned long long ntrb;
    double mass[MAXM];  // sum over cells of the cell averages, per component (fixed order)
};

uint64_t bits_of(double x) {
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
}
double from_bits(uint64_t u) {
    double x;
    memcpy(&x, &u, 8);
    return x;
}
double from_ordbits(uint64_t u) {
    return from_bits((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u);
}

// ---------------------------------------------------------------- component totals
// Deterministic sums over the cells of per-cell values x[cell * cs + comp * ms] (the cell
// averages, in either buffer layout): block b sums cells [b * kSumCells, (b + 1) * kSumCells)
// by a fixed pairwise tree, then one block adds the block sums in block order.  The result
// does not depend on scheduling, so repeated runs give the same bits.
constexpr int kSumThreads = 256, kSumCells = 4 * kSumThreads;

// The cells summed are those of the box [i0, i0 + w) x [j0, j0 + count / w) of a mesh nx wide
// (the whole mesh: i0 = j0 = 0, w = nx).
__global__ void k_colsum_part(const double *x, long long cs, long long ms, int count, int nx, int i0, int j0, int w,
                              int m, double *part) {
    __shared__ double sh[kSumThreads];
    const int b = blockIdx.x, t = threadIdx.x;
    for (int c = 0; c < m; ++c) {
        double v = 0.0;
        for (int j = 0; j < kSumCells / kSumThreads; ++j) {
            long long r = (long long)b * kSumCells + (long long)j * kSumThreads + t;
            if (r < count) {
                const long long cell = (j0 + r / w) * (long long)nx + i0 + r % w;
                v += x[cell * cs + c * ms];
            }
        }
        sh[t] = v;
        __syncthreads();
        for (int w = kSumThreads / 2; w > 0; w >>= 1) {
            if (t < w) sh[t] += sh[t + w];
            __syncthreads();
        }
        if (t == 0) part[(size_t)b * m + c] = sh[0];
        __syncthreads();
    }
}

// One warp per component: lane l adds the block sums l, l + 32, ... in order, then a fixed
// butterfly combines the lanes (the same order every run).
__global__ void k_colsum_final(const double *part, int nblk, int m, double *out) {
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (c >= m) return;
    double v = 0.0;
    for (int b = l; b < nblk; b += 32) v += part[(size_t)b * m + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) out[c] = v;
}

// ---------------------------------------------------------------- nodal tables
// Closed-form Gauss--Legendre and Gauss--Lobatto rules (n <= 4, L <= 3) and
// the Lagrange basis on the Gauss nodes.
void gauss_rule(int n, double *x, double *w) {
    if (n == 2) {
        double a = 1.0 / sqrt(3.0);
        x[0] = -a; x[1] = a;
        w[0] = w[1] = 1.0;
    } else if (n == 3) {
        double a = sqrt(0.6);
        x[0] = -a; x[1] = 0.0; x[2] = a;
        w[0] = w[2] = 5.0 / 9.0;
        w[1] = 8.0 / 9.0;
    } else {
        double r = 2.0 / 7.0 * sqrt(6.0 / 5.0);
        double a = sqrt(3.0 / 7.0 - r), b = sqrt(3.0 / 7.0 + r);
        double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
        x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
        w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
    }
}

void lobatto_rule(int L, double *x, double *w) {
    if (L == 2) {
        x[0] = -1.0; x[1] = 1.0;
        w[0] = w[1] = 1.0;
    } else {
        x[0] = -1.0; x[1] = 0.0; x[2] = 1.0;
        w[0] = w[2] = 1.0 / 3.0;
        w[1] = 4.0 / 3.0;
    }
}

double lagrange(int n, const double *x, int a, double t) {
    double v = 1.0;
    for (int b = 0; b < n; ++b)
        if (b != a) v *= (t - x[b]) / (x[a] - x[b]);
    return v;
}

double dlagrange(int n, const double *x, int a, double t) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) {
        if (c == a) continue;
        double v = 1.0 / (x[a] - x[c]);
        for (int b = 0; b < n; ++b)
            if (b != a && b != c) v *= (t - x[b]) / (x[a] - x[b]);
        s += v;
    }
    return s;
}

void build_tables(NodalTables *tab) {
    for (int n = 2; n <= 4; ++n) {
        NodalTables &T = tab[n - 2];
        memset(&T, 0, sizeof(T));
        int L = nlob(n);
        gauss_rule(n, T.xg, T.wg);
        lobatto_rule(L, T.xl, T.wl);
        for (int a = 0; a < n; ++a) {
            for (int q = 0; q < n; ++q) T.Dhat[a][q] = T.wg[q] * dlagrange(n, T.xg, a, T.xg[q]) / T.wg[a];
            T.lm[a] = lagrange(n, T.xg, a, -1.0);
            T.lp[a] = lagrange(n, T.xg, a, 1.0);
            T.liftm[a] = T.lm[a] / T.wg[a];
            T.liftp[a] = T.lp[a] / T.wg[a];
            for (int al = 0; al < L; ++al) T.Igl[al][a] = lagrange(n, T.xg, a, T.xl[al]);
            T.w1[a] = 0.5 * T.wg[a];
        }
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) T.w2[b * n + a] = 0.25 * T.wg[a] * T.wg[b];
        for (int a = 0; a < MAXN; ++a) {
            for (int q = 0; q < MAXN; ++q) {
                T.Dhatf[a][q] = (float)T.Dhat[a][q];
                T.Iglf[a][q] = (float)T.Igl[a][q];
            }
            T.lmf[a] = (float)T.lm[a];
            T.lpf[a] = (float)T.lp[a];
            T.liftmf[a] = (float)T.liftm[a];
            T.liftpf[a] = (float)T.liftp[a];
            T.w1f[a] = (float)T.w1[a];
        }
        for (int q = 0; q < MAXN * MAXN; ++q) T.w2f[q] = (float)T.w2[q];
        {  // P^k projection: modes L_i(x) L_j(y), i + j <= n - 1, Legendre by the recurrence
            auto leg = [](int i, double x) {
                double p0 = 1.0, p1 = x;
                if (i == 0) return p0;
                for (int l = 1; l < i; ++l) {
                    const double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
                    p0 = p1;
                    p1 = p2;
                }
                return p1;
            };
            const int k = n - 1;
            for (int node = 0; node < n * n; ++node) {
                const int a = node % n, b = node / n;
                for (int q = 0; q < n * n; ++q) {
                    const int qa = q % n, qb = q / n;
                    double v = 0.0;
                    for (int j = 0; j <= k; ++j)
                        for (int i = 0; i + j <= k; ++i)
                            v += leg(i, T.xg[a]) * leg(j, T.xg[b]) * (0.5 * (2 * i + 1)) * (0.5 * (2 * j + 1)) *
                                 T.wg[qa] * T.wg[qb] * leg(i, T.xg[qa]) * leg(j, T.xg[qb]);
                    T.pk[node][q] = v;
                }
            }
        }
        for (int q = 0; q < n * n; ++q) {
            const int qa = q % n, qb = q / n;
            T.mom2[q] = (3.0 * T.w1[qa]) * T.w1[qb];
            for (int d = 0; d < 2; ++d) {
                const int along = d == 0 ? qa : qb, across = d == 0 ? qb : qa;
                T.trw2[d][0][q] = T.w1[across] * T.lp[along];
                T.trw2[d][1][q] = T.w1[across] * T.lm[along];
                T.pm2[d][q] = ((3.0 * T.w1[qa]) * T.w1[qb]) * T.xg[along];
            }
            T.momxf[q] = (float)(T.mom2[q] * T.xg[qa]);
            T.momyf[q] = (float)(T.mom2[q] * T.xg[qb]);
        }
        for (int a = 0; a < n; ++a) T.pm1[a] = (3.0 * T.w1[a]) * T.xg[a];
    }
}

}  // namespace

void crkdg_build_tables(NodalTables *tab) { build_tables(tab); }

struct crkdg_ctx {
    crkdg_mesh mesh;
    crkdg_flux flux;
    crkdg_bounds bounds;
    crkdg_options opt;
    int k = 0, n = 0, m = 0, dim = 0, phys = 0;
    int ncell = 0, nn = 0, ntr = 0;
    size_t nstate = 0;
    cudaStream_t st = nullptr;
    double *u = nullptr, *unew = nullptr, *ustar = nullptr, *tr = nullptr, *aux = nullptr;
    int tr_slots = 0;
    DevScal *scal = nullptr;
    DevScal *hs = nullptr;      // pinned readback
    DevScal *hinit = nullptr;   // pinned initial values
    bool a0_valid = false;
    double t = 0.0;  // time of the current state (stage times of a time-dependent source)
    double a0 = 0.0;
    bool prof = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    double prof_ms[3] = {0.0, 0.0, 0.0};
    long long prof_n[3] = {0, 0, 0};
    // split-precision state (CRKDG_PREC_MIXED): FP64 averages + FP32 deviations
    bool mixed = false;
    double *xub[2] = {nullptr, nullptr};
    float *xdv[2] = {nullptr, nullptr};
    float *xdvs = nullptr;
    float *xtr = nullptr;
    int xtr_slots = 0;
    int xcur = 0;
    int *tflags = nullptr;   // troubled-cell flags of the last step (indicator on)
    float *feat = nullptr;   // MLP features [cell][44]
    float *prob = nullptr;   // MLP probabilities [cell]
    float *mlp = nullptr;    // MLP parameters of the learned indicator
    bool harvest = false;
    int barrier_extra = 0;   // testing aid (crkdg_set_barrier_test)
    int run1d_chunk = 0;     // own cells per block chunk of the 1D step loop (0: automatic)
    RunCtl *ctl = nullptr;   // device control block of the 1D step loop
    RunCtl *hctl = nullptr;  // pinned host copy
    bool pending = false;         // an attempt (crkdg_step_attempt) waits for crkdg_step_accept
    double pending_dt = 0.0;
    bool own_on = false;          // owned box of a subdomain (crkdg_set_subdomain)
    int own[4] = {0, 0, 0, 0};
    bool metric_on = false;       // cell sizes taken from the global mesh of a subdomain
    double rhx_g = 0.0, rhy_g = 0.0;
    bool tc_on = true;            // split path: inner stages on the tensor cores where built
    double *fst = nullptr;        // standard RKDG: F of each stage, then two stage buffers
    int fst_slots = 0;
    double *mass_part = nullptr;  // block sums of the component totals
    double mass_n[MAXM] = {};     // component totals of u^n (valid when mass_valid)
    bool mass_valid = false;
    unsigned *geo = nullptr;          // geometry words of a non-rectangular domain (device)
    std::vector<unsigned> geo_host;   // their host copy (solid cells of the totals)
    double gstate[2][MAXM] = {};
    double shock_x0 = 0.0, shock_speed = 0.0;
    std::string err;
};

namespace {

crkdg_status fail(crkdg_t h, crkdg_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(h, e_ == cudaErrorMemoryAllocation ? CRKDG_E_OOM : CRKDG_E_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

Params base_params(const crkdg_ctx *h) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.nx = h->mesh.nx;
    P.ny = h->dim == 2 ? h->mesh.ny : 1;
    P.ncell = h->ncell;
    P.rhx = h->metric_on ? h->rhx_g : 2.0 * h->mesh.nx / (h->mesh.x1 - h->mesh.x0);
    P.rhy = h->dim == 2 ? (h->metric_on ? h->rhy_g : 2.0 * h->mesh.ny / (h->mesh.y1 - h->mesh.y0)) : 0.0;
    P.gamma = h->flux.gamma;
    P.velx = h->flux.velocity[0];
    P.vely = h->flux.velocity[1];
    P.lo = h->bounds.lo;
    P.hi = h->bounds.hi;
    P.eps = h->bounds.eps;
    P.tvb_M = h->opt.tvb_M;
    tvb_thresholds(P);
    screen_bounds(P);
    for (int s = 0; s < 4; ++s) {
        P.bc[s] = (h->dim == 1 && s >= 2) ? BC_OUTFLOW : h->mesh.bc[s];
        for (int c = 0; c < MAXM; ++c) P.bcs[s][c] = h->mesh.bc_state[s][c];
    }
    P.own_on = h->own_on ? 1 : 0;
    for (int i = 0; i < 4; ++i) P.own[i] = h->own[i];
    P.theta2_exact = h->opt.theta2 == CRKDG_THETA2_EXACT ? 1 : 0;
    P.source = h->opt.source == CRKDG_SOURCE_SCENARIO1 ? 1 : 0;
    P.t0 = h->t;
    P.x0 = h->mesh.x0;
    P.y0 = h->mesh.y0;
    P.pk = (h->opt.basis == CRKDG_BASIS_P && h->dim == 2) ? 1 : 0;
    P.geo = h->geo;
    for (int w = 0; w < 2; ++w)
        for (int c = 0; c < MAXM; ++c) P.gstate[w][c] = h->gstate[w][c];
    P.shock_x0 = h->shock_x0;
    P.shock_speed = h->shock_speed;
    for (int i = 0; i < MAXS; ++i) P.slot[i] = -1;
    return P;
}

Bufs base_bufs(const crkdg_ctx *h) {
    Bufs B;
    B.un = h->u;
    B.ustar = h->ustar;
    B.unew = h->unew;
    B.tr = h->tr;
    B.tavg = h->tr ? h->tr + (size_t)h->tr_slots * h->m * h->ncell * h->ntr : nullptr;
    B.tfs = h->tr ? h->tr + (size_t)h->tr_slots * h->m * h->ncell * (h->ntr + 1) : nullptr;
    B.flag = &h->scal->flag;
    B.nlim = &h->scal->nlim;
    B.thmin = &h->scal->thmin;
    B.a0 = &h->scal->a0;
    B.aux = h->aux;
    B.ord = h->scal->ord;
    B.tflags = h->tflags;
    B.ntrb = &h->scal->ntrb;
    B.feat = h->feat;
    B.prob = h->prob;
    return B;
}

// Stages with a trace slot write their traces and cell averages (inner kernel) and the
// final kernel reads them: refuse a launch whose buffers are missing.
bool slots_ok(const Params &P, const void *tr, const void *tavg) {
    for (int i = 0; i < P.s && i < MAXS; ++i)
        if (P.slot[i] >= 0 && (!tr || !tavg)) return false;
    return true;
}

cudaError_t launch(crkdg_ctx *h, int kernel, const Params &P, const Bufs &B) {
    if ((kernel == K_INNER || kernel == K_FINAL) && !slots_ok(P, B.tr, B.tavg)) return cudaErrorInvalidValue;
    int ncb = cells_per_block(h->dim, h->n);
    int nblocks = (h->ncell + ncb - 1) / ncb;
    if (h->dim == 1) return crkdg_launch_1d(kernel, h->n, h->phys, nblocks, h->st, P, B);
    return crkdg_launch_2d(kernel, h->n, h->phys, nblocks, h->st, P, B);
}

MixBufs base_xbufs(const crkdg_ctx *h) {
    MixBufs X;
    memset(&X, 0, sizeof(X));
    X.ub = h->xub[h->xcur];
    X.dv = h->xdv[h->xcur];
    X.dv_s = h->xdvs;
    X.ub_n = h->xub[1 - h->xcur];
    X.dv_n = h->xdv[1 - h->xcur];
    X.tr = h->xtr;
    X.tavg = h->xtr ? h->xtr + (size_t)h->xtr_slots * h->m * h->ncell * h->ntr : nullptr;
    X.flag = &h->scal->flag;
    X.nlim = &h->scal->nlim;
    X.thmin = &h->scal->thmin;
    X.a0 = &h->scal->a0;
    X.ord = h->scal->ord;
    X.aux = h->aux;
    X.tflags = h->tflags;
    X.prob = h->prob;
    X.feat = h->feat;
    X.ntrb = &h->scal->ntrb;
    return X;
}

void fill_f32(Params &P) {
    ParamsF &F = P.f;
    F.rhx = (float)P.rhx;
    F.rhy = (float)P.rhy;
    F.gamma = (float)P.gamma;
    F.gm1 = (float)(P.gamma - 1.0);
    F.velx = (float)P.velx;
    F.vely = (float)P.vely;
    F.lo = (float)P.lo;
    F.hi = (float)P.hi;
    F.eps = (float)P.eps;
    F.thr[0] = (float)P.thr[0];
    F.thr[1] = (float)P.thr[1];
    for (int s = 0; s < 4; ++s)
        for (int c = 0; c < MAXM; ++c) F.bcs[s][c] = (float)P.bcs[s][c];
    for (int i = 0; i < MAXS; ++i) {
        for (int j = 0; j < MAXS; ++j) F.dtA[i][j] = (float)(P.dt * P.A[i][j]);
        F.dtb[i] = (float)(P.dt * P.b[i]);
        F.b[i] = (float)P.b[i];
    }
    F.dt = (float)P.dt;
}

// The tensor-core inner stages serve 2D Euler Q^3 steps whose tableau has only a
// sub-diagonal (every tableau of the paper); other cases run k_inner_x.
bool use_tc(const crkdg_ctx *h, const Params &P) {
    if (!h->tc_on || h->dim != 2 || h->phys != PH_EULER || h->n != 4 || P.mode != MODE_STEP) return false;
    for (int i = 0; i < P.s; ++i)
        for (int j = 0; j + 1 < i; ++j)
            if (P.A[i][j] != 0.0) return false;
    return true;
}

cudaError_t launch_x(crkdg_ctx *h, int kernel, const Params &P0, const MixBufs &X) {
    if ((kernel == KX_INNER || kernel == KX_FINAL) && !slots_ok(P0, X.tr, X.tavg)) return cudaErrorInvalidValue;
    Params P = P0;
    fill_f32(P);
    if (kernel == KX_INNER && use_tc(h, P)) return crkdg_launch_inner_tc(h->st, P, X);
    int ncb = cells_per_block(h->dim, h->n);
    int nblocks = (h->ncell + ncb - 1) / ncb;
    if (h->dim == 1) return crkdg_launch_mx_1d(kernel, h->n, h->phys, nblocks, h->st, P, X);
    return crkdg_launch_mx_2d(kernel, h->n, h->phys, nblocks, h->st, P, X);
}

crkdg_status reset_scalars(crkdg_ctx *h) {
    CK(h, cudaMemcpyAsync(h->scal, h->hinit, sizeof(DevScal), cudaMemcpyHostToDevice, h->st));
    return CRKDG_OK;
}

crkdg_status read_scalars(crkdg_ctx *h) {
    CK(h, cudaMemcpyAsync(h->hs, h->scal, sizeof(DevScal), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

// Stage combination of the standard RKDG (eq. rkdg): out = un + sum_j c_j F_j over the state,
// the terms added in stage order.
struct Combo {
    const double *f[MAXS];
    double c[MAXS];
    int nf;
};
__global__ void k_combine(const double *__restrict__ un, Combo cb, size_t count, double *__restrict__ out) {
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x) {
        double v = un[q];
        for (int j = 0; j < cb.nf; ++j) v = fma(cb.c[j], cb.f[j][q], v);
        out[q] = v;
    }
}

crkdg_status ensure_fstages(crkdg_ctx *h, int s) {
    const int need = s + 2;
    if (need <= h->fst_slots) return CRKDG_OK;
    if (h->fst) cudaFree(h->fst);
    h->fst = nullptr;
    h->fst_slots = 0;
    CK(h, cudaMalloc(&h->fst, (size_t)need * h->nstate * sizeof(double)));
    h->fst_slots = need;
    return CRKDG_OK;
}

// Queue the component totals of a state into scal->mass (read by the next read_scalars).
// FP64 path: the averages of the nodal state `nodal` (aux is overwritten); split path: the
// stored FP64 averages `ub` ([m][cell]).
crkdg_status queue_mass(crkdg_ctx *h, const double *nodal, const double *ub) {
    const double *x;
    long long cs, ms;
    if (h->mixed) {
        x = ub;
        cs = 1;
        ms = h->ncell;
    } else {
        Bufs B = base_bufs(h);
        B.un = nodal;
        CK(h, launch(h, K_AVG, base_params(h), B));
        x = h->aux;
        cs = h->m;
        ms = 1;
    }
    int i0 = 0, j0 = 0, w = h->mesh.nx, count = h->ncell;
    if (h->own_on) {
        i0 = h->own[0];
        j0 = h->own[2];
        w = h->own[1] - h->own[0];
        count = w * (h->own[3] - h->own[2]);
    }
    const int nblk = (count + kSumCells - 1) / kSumCells;
    k_colsum_part<<<nblk, kSumThreads, 0, h->st>>>(x, cs, ms, count, h->mesh.nx, i0, j0, w, h->m, h->mass_part);
    CK(h, cudaGetLastError());
    k_colsum_final<<<1, 32 * MAXM, 0, h->st>>>(h->mass_part, nblk, h->m, h->scal->mass);
    CK(h, cudaGetLastError());
    return CRKDG_OK;
}

void take_mass(crkdg_ctx *h) {
    for (int c = 0; c < h->m; ++c) h->mass_n[c] = h->hs->mass[c];
    h->mass_valid = true;
}

crkdg_status ensure_traces(crkdg_ctx *h, int slots) {
    if (slots <= h->tr_slots) return CRKDG_OK;
    if (h->tr) cudaFree(h->tr);
    h->tr = nullptr;
    h->tr_slots = 0;
    // traces [slot][m][cell][face point], the traced stages' cell averages [slot][m][cell],
    // then the traces' normal fluxes and spectral radii [slot][m + 1][cell][face point]
    size_t bytes = ((size_t)slots * h->m * h->ncell * (h->ntr + 1) + (size_t)slots * (h->m + 1) * h->ncell * h->ntr) *
                   sizeof(double);
    CK(h, cudaMalloc(&h->tr, bytes));
    h->tr_slots = slots;
    return CRKDG_OK;
}

crkdg_status ensure_traces_x(crkdg_ctx *h, int slots) {
    if (slots <= h->xtr_slots) return CRKDG_OK;
    if (h->xtr) cudaFree(h->xtr);
    h->xtr = nullptr;
    h->xtr_slots = 0;
    CK(h, cudaMalloc(&h->xtr, (size_t)slots * h->m * h->ncell * (h->ntr + 1) * sizeof(float)));
    h->xtr_slots = slots;
    return CRKDG_OK;
}

crkdg_status check_tableau(crkdg_t h, const crkdg_tableau *tab) {
    if (!tab || !tab->A || !tab->b) return fail(h, CRKDG_E_ARG, "tableau: NULL");
    if (tab->s < 1 || tab->s > MAXS) return fail(h, CRKDG_E_ARG, "tableau: need 1 <= s <= 4");
    for (int i = 0; i < tab->s; ++i) {
        if (!isfinite(tab->b[i]) || tab->b[i] < 0.0) return fail(h, CRKDG_E_ARG, "tableau: b must be finite and >= 0");
        for (int j = 0; j < tab->s; ++j) {
            double a = tab->A[i * tab->s + j];
            if (!isfinite(a)) return fail(h, CRKDG_E_ARG, "tableau: A not finite");
            if (j >= i && a != 0.0) return fail(h, CRKDG_E_ARG, "tableau: A must be strictly lower triangular");
        }
    }
    return CRKDG_OK;
}

void fill_tableau(Params &P, const crkdg_tableau *tab) {
    P.s = tab->s;
    int ns = 0;
    for (int i = 0; i < tab->s; ++i) {
        P.b[i] = tab->b[i];
        for (int j = 0; j < tab->s; ++j) P.A[i][j] = tab->A[i * tab->s + j];
        P.slot[i] = tab->b[i] != 0.0 ? ns++ : -1;
    }
    P.nslot = ns;
}

crkdg_status compute_a0(crkdg_ctx *h) {
    crkdg_status s = reset_scalars(h);
    if (s) return s;
    Params P = base_params(h);
    P.mode = MODE_RATE;
    if (h->mixed) {
        CK(h, launch_x(h, KX_SCAN, P, base_xbufs(h)));
    } else {
        Bufs B = base_bufs(h);
        CK(h, launch(h, K_A0, P, B));
    }
    s = read_scalars(h);
    if (s) return s;
    h->a0 = from_bits(h->hs->a0);
    h->a0_valid = true;
    return CRKDG_OK;
}

}  // namespace

extern "C" {

void crkdg_options_default(crkdg_options *opt) {
    if (!opt) return;
    opt->precision = CRKDG_PREC_FP64;
    opt->max_halvings = 20;
    opt->indicator = CRKDG_IND_OFF;
    opt->tvb_M = 10.0;
    opt->cuda_stream = nullptr;
    opt->scheme = CRKDG_SCHEME_COMPACT;
    opt->theta2 = CRKDG_THETA2_RATIO;
    opt->source = CRKDG_SOURCE_NONE;
    opt->basis = CRKDG_BASIS_Q;
}

crkdg_status crkdg_create(const crkdg_mesh *mesh, int k, int m, const crkdg_flux *flux,
                          const crkdg_bounds *bounds, const crkdg_options *opt, crkdg_t *out) {
    if (!out) return CRKDG_E_ARG;
    *out = nullptr;
    if (!mesh || !flux || !bounds) return CRKDG_E_ARG;
    if (mesh->dim != 1 && mesh->dim != 2) return CRKDG_E_ARG;
    if (k < 1) return CRKDG_E_ARG;
    if (k > 3) return CRKDG_E_UNSUPPORTED;
    if (flux->kind < CRKDG_FLUX_ADVECTION || flux->kind > CRKDG_FLUX_EULER) return CRKDG_E_ARG;
    if (m != ncomp(flux->kind, mesh->dim)) return CRKDG_E_ARG;
    int ny = mesh->dim == 2 ? mesh->ny : 1;
    if (mesh->nx < 1 || ny < 1) return CRKDG_E_ARG;
    if ((double)mesh->nx * ny * m * 64.0 > 9.0e15) return CRKDG_E_ARG;
    if ((double)mesh->nx * ny > 2.0e9) return CRKDG_E_ARG;
    // the split kernels address a component's face points with 32-bit offsets
    if ((double)mesh->nx * ny * 2 * mesh->dim * (mesh->dim == 2 ? k + 1 : 1) >= 4294967295.0) return CRKDG_E_ARG;
    if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0))) return CRKDG_E_ARG;
    int nsides = 2 * mesh->dim;
    for (int s = 0; s < nsides; ++s)
        if (mesh->bc[s] < CRKDG_BC_PERIODIC || mesh->bc[s] > CRKDG_BC_DIRICHLET) return CRKDG_E_ARG;
    for (int d = 0; d < mesh->dim; ++d)
        if ((mesh->bc[2 * d] == CRKDG_BC_PERIODIC) != (mesh->bc[2 * d + 1] == CRKDG_BC_PERIODIC)) return CRKDG_E_ARG;
    if (flux->kind == CRKDG_FLUX_EULER && !(flux->gamma > 1.0 && bounds->eps > 0.0)) return CRKDG_E_ARG;
    if (flux->kind != CRKDG_FLUX_EULER && !(bounds->lo <= bounds->hi)) return CRKDG_E_ARG;
    crkdg_options o;
    crkdg_options_default(&o);
    if (opt) o = *opt;
    if (o.max_halvings < 0 || o.max_halvings > 60) return CRKDG_E_ARG;
    if (o.precision != CRKDG_PREC_FP64 && o.precision != CRKDG_PREC_MIXED) return CRKDG_E_ARG;
    if (o.indicator < CRKDG_IND_OFF || o.indicator > CRKDG_IND_MLP || !(o.tvb_M >= 0.0)) return CRKDG_E_ARG;
    if (o.indicator != CRKDG_IND_OFF && flux->kind != CRKDG_FLUX_EULER) return CRKDG_E_UNSUPPORTED;
    if (o.indicator == CRKDG_IND_MLP && mesh->dim != 2) return CRKDG_E_UNSUPPORTED;
    if (o.scheme != CRKDG_SCHEME_COMPACT && o.scheme != CRKDG_SCHEME_STANDARD) return CRKDG_E_ARG;
    if (o.theta2 != CRKDG_THETA2_RATIO && o.theta2 != CRKDG_THETA2_EXACT) return CRKDG_E_ARG;
    if (o.theta2 == CRKDG_THETA2_EXACT && o.precision != CRKDG_PREC_FP64) return CRKDG_E_UNSUPPORTED;
    if (o.source != CRKDG_SOURCE_NONE && o.source != CRKDG_SOURCE_SCENARIO1) return CRKDG_E_ARG;
    if (o.basis != CRKDG_BASIS_Q && o.basis != CRKDG_BASIS_P) return CRKDG_E_ARG;
    if (o.basis == CRKDG_BASIS_P && mesh->dim == 2 &&
        (o.precision != CRKDG_PREC_FP64 || o.scheme != CRKDG_SCHEME_COMPACT || o.indicator != CRKDG_IND_OFF))
        return CRKDG_E_UNSUPPORTED;
    if (o.source == CRKDG_SOURCE_SCENARIO1 &&
        (mesh->dim != 2 || flux->kind != CRKDG_FLUX_EULER || o.precision != CRKDG_PREC_FP64 ||
         o.scheme != CRKDG_SCHEME_COMPACT || o.indicator != CRKDG_IND_OFF))
        return CRKDG_E_UNSUPPORTED;
    if (o.scheme == CRKDG_SCHEME_STANDARD && (o.precision != CRKDG_PREC_FP64 || o.indicator != CRKDG_IND_OFF))
        return CRKDG_E_UNSUPPORTED;

    crkdg_ctx *h = new (std::nothrow) crkdg_ctx();
    if (!h) return CRKDG_E_OOM;
    try {
        h->mesh = *mesh;
        h->mesh.ny = ny;
        h->flux = *flux;
        h->bounds = *bounds;
        h->opt = o;
        h->k = k;
        h->n = k + 1;
        h->m = m;
        h->dim = mesh->dim;
        h->phys = flux->kind;
        h->ncell = mesh->nx * ny;
        h->nn = h->dim == 2 ? h->n * h->n : h->n;
        h->ntr = h->dim == 2 ? 4 * h->n : 2;
        h->nstate = (size_t)h->ncell * h->nn * h->m;
        h->st = (cudaStream_t)o.cuda_stream;
        NodalTables tab[3];
        build_tables(tab);
        crkdg_status s = CRKDG_OK;
        auto chk = [&](cudaError_t e, const char *what) {
            if (e != cudaSuccess && s == CRKDG_OK) {
                s = e == cudaErrorMemoryAllocation ? CRKDG_E_OOM : CRKDG_E_CUDA;
                h->err = std::string(what) + ": " + cudaGetErrorString(e);
            }
        };
        chk(h->dim == 1 ? crkdg_upload_tables_1d(tab) : crkdg_upload_tables_2d(tab), "upload tables");
        size_t bytes = h->nstate * sizeof(double);
        if (s == CRKDG_OK) chk(cudaMalloc(&h->u, bytes), "cudaMalloc state");
        if (s == CRKDG_OK) chk(cudaMalloc(&h->unew, bytes), "cudaMalloc state");
        if (s == CRKDG_OK) chk(cudaMalloc(&h->ustar, bytes), "cudaMalloc state");
        if (s == CRKDG_OK) chk(cudaMalloc(&h->aux, (size_t)h->ncell * h->m * sizeof(double)), "cudaMalloc aux");
        if (s == CRKDG_OK) chk(cudaMalloc(&h->scal, sizeof(DevScal)), "cudaMalloc scalars");
        if (s == CRKDG_OK)
            chk(cudaMalloc(&h->mass_part, (size_t)((h->ncell + kSumCells - 1) / kSumCells) * h->m * sizeof(double)),
                "cudaMalloc totals");
        if (s == CRKDG_OK) chk(cudaMallocHost(&h->hs, sizeof(DevScal)), "cudaMallocHost");
        if (s == CRKDG_OK) chk(cudaMallocHost(&h->hinit, sizeof(DevScal)), "cudaMallocHost");
        h->mixed = o.precision == CRKDG_PREC_MIXED;
        if (s == CRKDG_OK && h->mixed) {
            size_t nb = (size_t)h->ncell * h->m;
            for (int i = 0; i < 2 && s == CRKDG_OK; ++i) {
                chk(cudaMalloc(&h->xub[i], nb * sizeof(double)), "cudaMalloc averages");
                if (s == CRKDG_OK) chk(cudaMalloc(&h->xdv[i], h->nstate * sizeof(float)), "cudaMalloc deviations");
            }
            if (s == CRKDG_OK) chk(cudaMalloc(&h->xdvs, h->nstate * sizeof(float)), "cudaMalloc deviations");
            if (s == CRKDG_OK) chk(cudaMemsetAsync(h->xub[0], 0, nb * sizeof(double), h->st), "cudaMemset");
            if (s == CRKDG_OK) chk(cudaMemsetAsync(h->xdv[0], 0, h->nstate * sizeof(float), h->st), "cudaMemset");
        }
        if (s == CRKDG_OK && o.indicator != CRKDG_IND_OFF)
            chk(cudaMalloc(&h->tflags, (size_t)h->ncell * sizeof(int)), "cudaMalloc flags");
        if (s == CRKDG_OK && o.indicator != CRKDG_IND_OFF && h->dim == 2) {
            chk(cudaMalloc(&h->feat, (size_t)h->ncell * CRKDG_MLP_NIN * sizeof(float)), "cudaMalloc features");
            if (s == CRKDG_OK) chk(cudaMalloc(&h->prob, (size_t)h->ncell * sizeof(float)), "cudaMalloc prob");
            if (s == CRKDG_OK) chk(cudaMalloc(&h->mlp, CRKDG_MLP_NPARAM * sizeof(float)), "cudaMalloc mlp");
            if (s == CRKDG_OK) chk(cudaMemsetAsync(h->mlp, 0, CRKDG_MLP_NPARAM * sizeof(float), h->st), "cudaMemset");
        }
        if (s == CRKDG_OK) chk(cudaMemsetAsync(h->u, 0, bytes, h->st), "cudaMemset");
        if (s == CRKDG_OK) chk(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
        if (s != CRKDG_OK) {
            crkdg_destroy(h);
            return s;
        }
        memset(h->hinit, 0, sizeof(DevScal));
        h->hinit->thmin = bits_of(1.0);
        h->hinit->ord[0] = h->hinit->ord[1] = ~0ull;
        *out = h;
        return CRKDG_OK;
    } catch (...) {
        crkdg_destroy(h);
        return CRKDG_E_OOM;
    }
}

crkdg_status crkdg_destroy(crkdg_t h) {
    if (!h) return CRKDG_OK;
    if (h->st || h->u) cudaStreamSynchronize(h->st);
    for (int i = 0; i < 3; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    cudaFree(h->u);
    cudaFree(h->unew);
    cudaFree(h->ustar);
    cudaFree(h->geo);
    cudaFree(h->tr);
    cudaFree(h->aux);
    cudaFree(h->mass_part);
    cudaFree(h->fst);
    cudaFree(h->scal);
    cudaFreeHost(h->hs);
    cudaFreeHost(h->hinit);
    cudaFree(h->ctl);
    cudaFreeHost(h->hctl);
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->xub[i]);
        cudaFree(h->xdv[i]);
    }
    cudaFree(h->xdvs);
    cudaFree(h->xtr);
    cudaFree(h->tflags);
    cudaFree(h->feat);
    cudaFree(h->prob);
    cudaFree(h->mlp);
    delete h;
    return CRKDG_OK;
}

size_t crkdg_state_size(crkdg_t h) { return h ? h->nstate : 0; }

crkdg_status crkdg_set_profiling(crkdg_t h, int on) {
    if (!h) return CRKDG_E_ARG;
    if (on && !h->ev[0])
        for (int i = 0; i < 3; ++i) CK(h, cudaEventCreate(&h->ev[i]));
    h->prof = on != 0;
    for (int i = 0; i < 3; ++i) {
        h->prof_ms[i] = 0.0;
        h->prof_n[i] = 0;
    }
    return CRKDG_OK;
}

crkdg_status crkdg_set_tensor_cores(crkdg_t h, int on) {
    if (!h) return CRKDG_E_ARG;
    h->tc_on = on != 0;
    return CRKDG_OK;
}

crkdg_status crkdg_set_run1d_chunk(crkdg_t h, int cells) {
    if (!h || cells < 0 || cells > 30) return CRKDG_E_ARG;
    h->run1d_chunk = cells;
    return CRKDG_OK;
}

crkdg_status crkdg_set_barrier_test(crkdg_t h, int extra) {
    if (!h || extra < 0) return CRKDG_E_ARG;
    h->barrier_extra = extra;
    return CRKDG_OK;
}

crkdg_status crkdg_kernel_times(crkdg_t h, double ms[3], long long launches[3]) {
    if (!h || !ms || !launches) return CRKDG_E_ARG;
    for (int i = 0; i < 3; ++i) {
        ms[i] = h->prof_ms[i];
        launches[i] = h->prof_n[i];
    }
    return CRKDG_OK;
}

const char *crkdg_last_error(crkdg_t h) { return h ? h->err.c_str() : "invalid handle"; }

// The device address under which a kernel can read or write the caller's buffer in place: a
// device pointer itself, or page-locked host memory mapped into the device's address space
// (a split-precision state is split or merged over the host link by the kernel, with no staging
// copy).  nullptr for pageable host memory, which is staged by cudaMemcpyAsync.
static void *direct_ptr(const void *p, int on_device) {
    if (on_device) return const_cast<void *>(p);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA-known pointer: clear the error, stage it
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

crkdg_status crkdg_set_state(crkdg_t h, const double *nodal, size_t count, int on_device) {
    if (!h) return CRKDG_E_ARG;
    if (!nodal || count != h->nstate) return fail(h, CRKDG_E_ARG, "set_state: count must equal the state size");
    try {
        const double *src = h->mixed ? static_cast<const double *>(direct_ptr(nodal, on_device)) : nullptr;
        if (!src) {
            CK(h, cudaMemcpyAsync(h->unew, nodal, count * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
            src = h->unew;
        }
        Params P = base_params(h);
        CK(h, reset_scalars(h) == CRKDG_OK ? cudaSuccess : cudaErrorUnknown);
        if (h->mixed) {
            MixBufs X = base_xbufs(h);
            X.nod_in = src;
            X.ub_n = h->xub[h->xcur];
            X.dv_n = h->xdv[h->xcur];
            CK(h, launch_x(h, KX_SPLIT, P, X));
            X = base_xbufs(h);
            X.dv_n = h->xdv[h->xcur];
            P.mode = MODE_RATE;  // the limiter also posts the trial-step rate of the limited state
            CK(h, launch_x(h, KX_LIMIT, P, X));
            crkdg_status s = queue_mass(h, nullptr, h->xub[h->xcur]);
            if (s == CRKDG_OK) s = read_scalars(h);
            if (s) return s;
            take_mass(h);
            h->a0 = from_bits(h->hs->a0);
            h->a0_valid = true;
            return CRKDG_OK;
        }
        // FP64: the limiter also posts the trial-step rate of the limited state, so
        // crkdg_max_dt needs no pass of its own
        Bufs B = base_bufs(h);
        B.un = h->unew;
        B.unew = h->u;
        P.mode = MODE_RATE;
        CK(h, launch(h, K_LIMIT, P, B));
        crkdg_status s = queue_mass(h, h->u, nullptr);
        if (s == CRKDG_OK) s = read_scalars(h);
        if (s) return s;
        take_mass(h);
        h->a0 = from_bits(h->hs->a0);
        h->a0_valid = true;
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

crkdg_status crkdg_get_state(crkdg_t h, double *nodal, size_t count, int on_device) {
    if (!h) return CRKDG_E_ARG;
    if (!nodal || count != h->nstate) return fail(h, CRKDG_E_ARG, "get_state: count must equal the state size");
    double *dst = nullptr;
    if (h->mixed) {
        dst = static_cast<double *>(direct_ptr(nodal, on_device));
        MixBufs X = base_xbufs(h);
        X.nod_out = dst ? dst : h->u;
        CK(h, launch_x(h, KX_MERGE, base_params(h), X));
    }
    if (!dst)
        CK(h, cudaMemcpyAsync(nodal, h->u, count * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

crkdg_status crkdg_set_time(crkdg_t h, double t) {
    if (!h || !isfinite(t)) return CRKDG_E_ARG;
    h->t = t;
    return CRKDG_OK;
}

crkdg_status crkdg_get_time(crkdg_t h, double *t) {
    if (!h || !t) return CRKDG_E_ARG;
    *t = h->t;
    return CRKDG_OK;
}

crkdg_status crkdg_max_dt(crkdg_t h, double cfl, double *dt) {
    if (!h || !dt) return CRKDG_E_ARG;
    if (!(cfl > 0.0)) return fail(h, CRKDG_E_ARG, "max_dt: cfl must be > 0");
    try {
        if (!h->a0_valid) {
            crkdg_status s = compute_a0(h);
            if (s) return s;
        }
        // h->a0 holds max over S_K points of sum_d lambda_d / h_d
        *dt = h->a0 > 0.0 ? cfl / h->a0 : INFINITY;
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

}  // extern "C"

namespace {

// Parameters and trace buffers of a step with tableau tab (shared by crkdg_step and the
// attempt / accept pair); with want_mass the totals of u^n are made current.
crkdg_status prepare_step(crkdg_t h, double dt, const crkdg_tableau *tab, bool want_mass, Params &P) {
    crkdg_status s = check_tableau(h, tab);
    if (s) return s;
    if (!(dt > 0.0) || !isfinite(dt)) return fail(h, CRKDG_E_ARG, "step: dt must be finite and > 0");
    P = base_params(h);
    P.s = tab->s;
    P.mode = MODE_STEP;
    P.defer_limit = h->opt.indicator != CRKDG_IND_OFF ? 1 : 0;
    int ns = 0;
    for (int i = 0; i < tab->s; ++i) {
        P.b[i] = tab->b[i];
        for (int j = 0; j < tab->s; ++j) P.A[i][j] = tab->A[i * tab->s + j];
        P.slot[i] = tab->b[i] != 0.0 ? ns++ : -1;
    }
    P.nslot = ns;
    s = h->mixed ? ensure_traces_x(h, ns > 0 ? ns : 1) : ensure_traces(h, ns > 0 ? ns : 1);
    if (s) return s;
    if (h->opt.scheme == CRKDG_SCHEME_STANDARD) {
        s = ensure_fstages(h, tab->s);
        if (s) return s;
    }
    if (want_mass && !h->mass_valid) {
        s = reset_scalars(h);
        if (s == CRKDG_OK) s = queue_mass(h, h->u, h->mixed ? h->xub[h->xcur] : nullptr);
        if (s == CRKDG_OK) s = read_scalars(h);
        if (s) return s;
        take_mass(h);
    }
    return CRKDG_OK;
}

// F(in) -> out with the operator kernels (the inner kernel's G plus the final kernel's face
// correction, as crkdg_apply_operator); traces in slot 0.
crkdg_status apply_F(crkdg_t h, const double *in, double *out) {
    Params P = base_params(h);
    P.s = 1;
    P.dt = 1.0;
    P.b[0] = 1.0;
    P.slot[0] = 0;
    P.nslot = 1;
    P.mode = MODE_OP_G;
    Bufs B = base_bufs(h);
    B.un = in;
    B.ustar = h->ustar;
    CK(h, launch(h, K_INNER, P, B));
    P.mode = MODE_OP_F;
    B.unew = out;
    CK(h, launch(h, K_FINAL, P, B));
    return CRKDG_OK;
}

crkdg_status combine(crkdg_t h, const double *un, const Combo &cb, double *out) {
    const size_t n = h->nstate;
    int grid = (int)((n + 255) / 256);
    if (grid > 65535) grid = 65535;
    k_combine<<<grid, 256, 0, h->st>>>(un, cb, n, out);
    CK(h, cudaGetLastError());
    return CRKDG_OK;
}

// One attempt of the standard RKDG (eq. rkdg): every stage value is u^n plus its combination of
// the previous stages' F (each F with its own neighbour exchange), tested and limited like the
// compact scheme's stages; the result lands in h->unew.
crkdg_status attempt_standard(crkdg_t h, const Params &Ps, double dt, bool want_mass) {
    crkdg_status s = reset_scalars(h);
    if (s) return s;
    const int ns = Ps.s;
    double *F = h->fst, *comb = h->fst + (size_t)ns * h->nstate, *ut = comb + h->nstate;
    bool need[MAXS] = {};
    for (int j = 0; j < ns; ++j) {
        need[j] = Ps.b[j] != 0.0;
        for (int i = j + 1; i < ns; ++i) need[j] = need[j] || Ps.A[i][j] != 0.0;
    }
    if (h->prof) CK(h, cudaEventRecord(h->ev[0], h->st));
    for (int i = 0; i < ns; ++i) {
        const double *stage = h->u;  // u~^(1) = u~^n
        if (i > 0) {
            Combo cb;
            memset(&cb, 0, sizeof(cb));
            for (int j = 0; j < i; ++j)
                if (Ps.A[i][j] != 0.0) {
                    cb.f[cb.nf] = F + (size_t)j * h->nstate;
                    cb.c[cb.nf++] = dt * Ps.A[i][j];
                }
            s = combine(h, h->u, cb, comb);
            if (s) return s;
            Params P = base_params(h);
            P.mode = MODE_LIMIT_CHECK;
            Bufs B = base_bufs(h);
            B.un = comb;
            B.unew = ut;
            CK(h, launch(h, K_LIMIT, P, B));
            stage = ut;
        }
        if (need[i]) {
            s = apply_F(h, stage, F + (size_t)i * h->nstate);
            if (s) return s;
        }
    }
    if (h->prof) CK(h, cudaEventRecord(h->ev[1], h->st));
    Combo cb;
    memset(&cb, 0, sizeof(cb));
    for (int i = 0; i < ns; ++i)
        if (Ps.b[i] != 0.0) {
            cb.f[cb.nf] = F + (size_t)i * h->nstate;
            cb.c[cb.nf++] = dt * Ps.b[i];
        }
    s = combine(h, h->u, cb, comb);
    if (s) return s;
    Params P = base_params(h);
    P.mode = MODE_LIMIT_FINAL;
    Bufs B = base_bufs(h);
    B.un = comb;
    B.unew = h->unew;
    CK(h, launch(h, K_LIMIT, P, B));
    if (h->prof) CK(h, cudaEventRecord(h->ev[2], h->st));
    if (want_mass) {
        s = queue_mass(h, h->unew, nullptr);
        if (s) return s;
    }
    s = read_scalars(h);
    if (s) return s;
    if (h->prof) {
        float t0 = 0.f, t1 = 0.f;
        CK(h, cudaEventElapsedTime(&t0, h->ev[0], h->ev[1]));
        CK(h, cudaEventElapsedTime(&t1, h->ev[1], h->ev[2]));
        h->prof_ms[0] += t0;
        h->prof_ms[1] += t1;
        h->prof_n[0] += 1;
        h->prof_n[1] += 1;
    }
    return CRKDG_OK;
}

// One attempt of size dt from u^n into the second state buffer; h->hs holds its flag and
// statistics afterwards (synchronises the stream).
crkdg_status attempt_once(crkdg_t h, Params &P, double dt, bool want_mass) {
    if (h->opt.scheme == CRKDG_SCHEME_STANDARD) return attempt_standard(h, P, dt, want_mass);
    const bool ind = h->opt.indicator != CRKDG_IND_OFF;
    crkdg_status s;
    P.dt = dt;
    Bufs B = base_bufs(h);
    B.un = h->u;
    B.unew = h->unew;
    s = reset_scalars(h);
    if (s) return s;
    if (h->prof) CK(h, cudaEventRecord(h->ev[0], h->st));
    if (h->mixed) {
        CK(h, launch_x(h, KX_INNER, P, base_xbufs(h)));
    } else {
        CK(h, launch(h, K_INNER, P, B));
    }
    if (h->prof) CK(h, cudaEventRecord(h->ev[1], h->st));
    if (h->mixed) {
        CK(h, launch_x(h, KX_FINAL, P, base_xbufs(h)));
        if (ind) {
            // the final stage left the unlimited u^{n+1} and its averages (aux); the plain
            // decision is taken in the troubled-cell pass, unless features are wanted:
            // then the FP64 feature kernel takes it on the merged nodal values
            const bool learned = h->opt.indicator == CRKDG_IND_MLP;
            if (learned && !h->harvest) {
                // features from the split state; the troubled-cell pass takes the plain
                // decision itself and combines it with the network's
                CK(h, launch_x(h, KX_FEATURES, P, base_xbufs(h)));
                if (crkdg_mlp_forward(h->mlp, h->feat, h->ncell, h->prob, h->st) != CRKDG_OK)
                    return fail(h, CRKDG_E_CUDA, "step: MLP forward failed");
                P.ind_stage = 4;
            } else if (h->harvest) {
                MixBufs Xn = base_xbufs(h);
                Xn.ub = h->xub[1 - h->xcur];
                Xn.dv = h->xdv[1 - h->xcur];
                Xn.nod_out = h->unew;
                CK(h, launch_x(h, KX_MERGE, P, Xn));
                Bufs Bf = base_bufs(h);
                Bf.unew = h->unew;
                CK(h, launch(h, K_FEATURES, P, Bf));
                if (learned && crkdg_mlp_forward(h->mlp, h->feat, h->ncell, h->prob, h->st) != CRKDG_OK)
                    return fail(h, CRKDG_E_CUDA, "step: MLP forward failed");
                P.ind_stage = learned ? 3 : 2;
            } else {
                P.ind_stage = 0;
            }
            CK(h, launch_x(h, KX_TROUBLE, P, base_xbufs(h)));
            P.ind_stage = 0;
        }
    } else {
        CK(h, launch(h, K_FINAL, P, B));
        if (ind) {
            const bool learned = h->opt.indicator == CRKDG_IND_MLP;
            if (learned || h->harvest) {
                // features and the plain decision of the unlimited state in one pass
                CK(h, launch(h, K_FEATURES, P, B));
                if (learned && crkdg_mlp_forward(h->mlp, h->feat, h->ncell, h->prob, h->st) != CRKDG_OK)
                    return fail(h, CRKDG_E_CUDA, "step: MLP forward failed");
                P.ind_stage = learned ? 3 : 2;  // (combine the learned flags and) limit the flagged cells
            } else {
                P.ind_stage = 0;
            }
            CK(h, launch(h, K_TROUBLE, P, B));
        }
    }
    if (h->prof) CK(h, cudaEventRecord(h->ev[2], h->st));
    if (want_mass) {
        // component totals of the new state (after the event: not part of the kernel times)
        s = queue_mass(h, h->unew, h->mixed ? h->xub[1 - h->xcur] : nullptr);
        if (s) return s;
    }
    s = read_scalars(h);
    if (s) return s;
    if (h->hs->flag & 2) return fail(h, CRKDG_E_TIMEOUT, "step: a wait for the tensor cores ran out");
    if (h->prof) {
        float t0 = 0.f, t1 = 0.f;
        CK(h, cudaEventElapsedTime(&t0, h->ev[0], h->ev[1]));
        CK(h, cudaEventElapsedTime(&t1, h->ev[1], h->ev[2]));
        h->prof_ms[0] += t0;
        h->prof_ms[1] += t1;
        h->prof_n[0] += 1;
        h->prof_n[1] += 1;
    }
    return CRKDG_OK;
}

// Accept the attempt in h->hs: the new state becomes u^n.
void accept_attempt(crkdg_t h, double dt, int restarts, crkdg_step_info *info) {
    h->t += dt;
    if (h->mixed) {
        h->xcur = 1 - h->xcur;
    } else {
        double *t = h->u;
        h->u = h->unew;
        h->unew = t;
    }
    h->a0 = from_bits(h->hs->a0);
    h->a0_valid = true;
    if (info) {
        info->dt_taken = dt;
        info->restarts = restarts;
        info->cells_limited = (long long)h->hs->nlim;
        info->theta_min = from_bits(h->hs->thmin);
        info->troubled = (long long)h->hs->ntrb;
        // relative change of the first component's total over the step
        const double m0 = h->mass_n[0], m1 = h->hs->mass[0];
        info->mass_drift = (m1 - m0) / (m0 != 0.0 ? fabs(m0) : 1.0);
        take_mass(h);
    } else {
        h->mass_valid = false;
    }
}

}  // namespace

extern "C" {

crkdg_status crkdg_step(crkdg_t h, double dt, const crkdg_tableau *tab, crkdg_step_info *info) {
    if (!h) return CRKDG_E_ARG;
    try {
        Params P;
        crkdg_status s = prepare_step(h, dt, tab, info != nullptr, P);
        if (s) return s;
        h->pending = false;
        for (int r = 0; r <= h->opt.max_halvings; ++r) {
            s = attempt_once(h, P, dt, info != nullptr);
            if (s) return s;
            if (h->hs->flag == 0) {
                accept_attempt(h, dt, r, info);
                return CRKDG_OK;
            }
            dt *= 0.5;
        }
        return fail(h, CRKDG_E_BOUNDS, "step: cell averages left the admissible set after max_halvings restarts");
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

crkdg_status crkdg_step_attempt(crkdg_t h, double dt, const crkdg_tableau *tab, int *violated) {
    if (!h || !violated) return CRKDG_E_ARG;
    try {
        Params P;
        h->pending = false;
        crkdg_status s = prepare_step(h, dt, tab, true, P);
        if (s) return s;
        s = attempt_once(h, P, dt, true);
        if (s) return s;
        *violated = h->hs->flag != 0;
        h->pending = true;
        h->pending_dt = dt;
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

crkdg_status crkdg_step_accept(crkdg_t h, crkdg_step_info *info) {
    if (!h) return CRKDG_E_ARG;
    if (!h->pending) return fail(h, CRKDG_E_ARG, "step_accept: no attempt to accept");
    if (h->hs->flag != 0) return fail(h, CRKDG_E_ARG, "step_accept: the attempt left the admissible set");
    h->pending = false;
    crkdg_step_info tmp;
    accept_attempt(h, h->pending_dt, 0, info ? info : &tmp);
    return CRKDG_OK;
}

// 1D meshes: one persistent cooperative launch runs the whole step loop.
// cfl > 0: adaptive trial steps; cfl <= 0: the fixed trial step dt_fixed every step.
static crkdg_status advance_1d(crkdg_t h, int nsteps, double cfl, double dt_fixed, double t_end,
                               const crkdg_tableau *tab, double *t, int *steps_done, int *restarts) {
    crkdg_status s = check_tableau(h, tab);
    if (s) return s;
    if (steps_done) *steps_done = 0;
    if (restarts) *restarts = 0;
    if (nsteps <= 0 || !(*t < t_end)) return CRKDG_OK;
    if (!h->ctl) {
        CK(h, cudaMalloc(&h->ctl, sizeof(RunCtl)));
        CK(h, cudaMallocHost(&h->hctl, sizeof(RunCtl)));
    }
    if (cfl > 0.0 && !h->a0_valid) {
        s = compute_a0(h);
        if (s) return s;
    }
    Params P = base_params(h);
    fill_tableau(P, tab);
    P.mode = MODE_STEP;
    RunCtl *c = h->hctl;
    memset(c, 0, sizeof(RunCtl));
    c->t = *t;
    c->t_end = t_end;
    c->dt0 = cfl > 0.0 ? (h->a0 > 0.0 ? cfl / h->a0 : INFINITY) : dt_fixed;
    c->cfl = cfl > 0.0 ? cfl : 0.0;
    c->nsteps = nsteps;
    c->max_halvings = h->opt.max_halvings;
    c->cur = 0;
    c->extra_arrivals = h->barrier_extra;
    for (int i = 0; i < 3; ++i) c->slot[i].thmin = bits_of(1.0);
    CK(h, cudaMemcpyAsync(h->ctl, c, sizeof(RunCtl), cudaMemcpyHostToDevice, h->st));
    int nb = 0;
    if (h->prof) CK(h, cudaEventRecord(h->ev[0], h->st));
    CK(h, crkdg_run_1d(h->n, h->phys, h->st, P, h->u, h->unew, h->ctl, h->run1d_chunk, &nb));
    if (h->prof) CK(h, cudaEventRecord(h->ev[1], h->st));
    CK(h, cudaMemcpyAsync(c, h->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (h->prof) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        h->prof_ms[2] += ms;
        h->prof_n[2] += 1;
    }
    if (c->cur_out) {
        double *tmp = h->u;
        h->u = h->unew;
        h->unew = tmp;
    }
    if (c->steps > 0) h->mass_valid = false;  // the loop keeps no component totals
    *t = c->t_out;
    h->t = *t;
    if (steps_done) *steps_done = c->steps;
    if (restarts) *restarts = c->restarts;
    if (c->steps > 0 && c->rate_out >= 0.0) {
        h->a0 = c->rate_out;
        h->a0_valid = true;
    }
    if (c->status == RUN_BOUNDS)
        return fail(h, CRKDG_E_BOUNDS, "advance: cell averages left the admissible set after max_halvings restarts");
    if (c->status == RUN_TIMEOUT) return fail(h, CRKDG_E_TIMEOUT, "advance: grid barrier wait expired");
    return CRKDG_OK;
}

crkdg_status crkdg_advance(crkdg_t h, int nsteps, double cfl, double t_end, const crkdg_tableau *tab,
                           double *t, int *steps_done, int *restarts) {
    if (!h || !t) return CRKDG_E_ARG;
    if (!(cfl > 0.0)) return fail(h, CRKDG_E_ARG, "advance: cfl must be > 0");
    h->t = *t;  // the caller's time is the state's
    if (h->dim == 1 && !h->mixed && h->opt.indicator == CRKDG_IND_OFF && !h->own_on &&
        h->opt.scheme == CRKDG_SCHEME_COMPACT) {
        try {
            return advance_1d(h, nsteps, cfl, 0.0, t_end, tab, t, steps_done, restarts);
        } catch (...) {
            return CRKDG_E_OOM;
        }
    }
    int done = 0, rs = 0;
    crkdg_status s = CRKDG_OK;
    for (int i = 0; i < nsteps; ++i) {
        if (!(*t < t_end)) break;
        double dt;
        s = crkdg_max_dt(h, cfl, &dt);
        if (s) break;
        if (dt > t_end - *t) dt = t_end - *t;
        crkdg_step_info info;
        s = crkdg_step(h, dt, tab, &info);
        if (s) break;
        *t += info.dt_taken;
        ++done;
        rs += info.restarts;
    }
    if (steps_done) *steps_done = done;
    if (restarts) *restarts = rs;
    return s;
}

crkdg_status crkdg_advance_fixed(crkdg_t h, int nsteps, double dt, double t_end, const crkdg_tableau *tab,
                                 double *t, int *steps_done, int *restarts) {
    if (!h || !t) return CRKDG_E_ARG;
    if (!(dt > 0.0) || !isfinite(dt)) return fail(h, CRKDG_E_ARG, "advance_fixed: dt must be finite and > 0");
    h->t = *t;  // the caller's time is the state's
    if (h->dim == 1 && !h->mixed && h->opt.indicator == CRKDG_IND_OFF && !h->own_on &&
        h->opt.scheme == CRKDG_SCHEME_COMPACT) {
        try {
            return advance_1d(h, nsteps, 0.0, dt, t_end, tab, t, steps_done, restarts);
        } catch (...) {
            return CRKDG_E_OOM;
        }
    }
    int done = 0, rs = 0;
    crkdg_status s = CRKDG_OK;
    for (int i = 0; i < nsteps; ++i) {
        if (!(*t < t_end)) break;
        double d = dt < t_end - *t ? dt : t_end - *t;
        crkdg_step_info info;
        s = crkdg_step(h, d, tab, &info);
        if (s) break;
        *t += info.dt_taken;
        if (t_end - *t <= 1e-14 * fabs(t_end)) *t = t_end;
        ++done;
        rs += info.restarts;
    }
    if (steps_done) *steps_done = done;
    if (restarts) *restarts = rs;
    return s;
}

crkdg_status crkdg_apply_operator(crkdg_t h, int op, const double *in_dev, double *out_dev) {
    if (!h) return CRKDG_E_ARG;
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(h, CRKDG_E_ARG, "apply_operator: bad pointers");
    try {
        Params P = base_params(h);
        Bufs B = base_bufs(h);
        P.s = 1;
        P.dt = 1.0;
        P.b[0] = 1.0;
        if (h->mixed) {
            if (op != CRKDG_OP_G && op != CRKDG_OP_F && op != CRKDG_OP_LIMIT)
                return fail(h, CRKDG_E_ARG, "apply_operator: unknown op");
            crkdg_status s = ensure_traces_x(h, 1);
            if (s) return s;
            // split the input into the spare (averages, deviations) pair
            MixBufs X = base_xbufs(h);
            X.nod_in = in_dev;
            CK(h, launch_x(h, KX_SPLIT, P, X));
            MixBufs Y = base_xbufs(h);
            Y.ub = h->xub[1 - h->xcur];
            Y.dv = h->xdv[1 - h->xcur];
            Y.dv_n = h->xdv[1 - h->xcur];
            if (op == CRKDG_OP_LIMIT) {
                CK(h, launch_x(h, KX_LIMIT, P, Y));
                Y.nod_out = out_dev;
                CK(h, launch_x(h, KX_MERGE, P, Y));
            } else {
                P.mode = MODE_OP_G;
                P.slot[0] = op == CRKDG_OP_F ? 0 : -1;
                P.nslot = op == CRKDG_OP_F ? 1 : 0;
                Y.nod_out = op == CRKDG_OP_F ? h->ustar : out_dev;
                CK(h, launch_x(h, KX_INNER, P, Y));
                if (op == CRKDG_OP_F) {
                    P.mode = MODE_OP_F;
                    Y.nod_in = h->ustar;
                    Y.nod_out = out_dev;
                    CK(h, launch_x(h, KX_FINAL, P, Y));
                }
            }
            CK(h, cudaStreamSynchronize(h->st));
            return CRKDG_OK;
        }
        if (op == CRKDG_OP_G) {
            P.mode = MODE_OP_G;
            B.un = in_dev;
            B.ustar = out_dev;
            CK(h, launch(h, K_INNER, P, B));
        } else if (op == CRKDG_OP_F) {
            crkdg_status s = ensure_traces(h, 1);
            if (s) return s;
            B = base_bufs(h);  // the trace buffer (and its stage averages) may be new
            P.slot[0] = 0;
            P.nslot = 1;
            P.mode = MODE_OP_G;
            B.un = in_dev;
            B.ustar = h->ustar;
            CK(h, launch(h, K_INNER, P, B));
            P.mode = MODE_OP_F;
            B.unew = out_dev;
            CK(h, launch(h, K_FINAL, P, B));
        } else if (op == CRKDG_OP_LIMIT) {
            B.un = in_dev;
            B.unew = out_dev;
            CK(h, launch(h, K_LIMIT, P, B));
        } else {
            return fail(h, CRKDG_E_ARG, "apply_operator: unknown op");
        }
        CK(h, cudaStreamSynchronize(h->st));
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

crkdg_status crkdg_troubled_flags(crkdg_t h, int *flags, int on_device) {
    if (!h || !flags) return CRKDG_E_ARG;
    if (!h->tflags) return fail(h, CRKDG_E_ARG, "troubled_flags: the indicator is off");
    CK(h, cudaMemcpyAsync(flags, h->tflags, (size_t)h->ncell * sizeof(int),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

crkdg_status crkdg_set_mlp(crkdg_t h, const float *params) {
    if (!h || !params) return CRKDG_E_ARG;
    if (!h->mlp) return fail(h, CRKDG_E_ARG, "set_mlp: needs a 2D handle with an indicator");
    CK(h, cudaMemcpyAsync(h->mlp, params, CRKDG_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

crkdg_status crkdg_set_harvest(crkdg_t h, int on) {
    if (!h) return CRKDG_E_ARG;
    if (on && !h->feat) return fail(h, CRKDG_E_ARG, "set_harvest: needs a 2D handle with an indicator");
    h->harvest = on != 0;
    return CRKDG_OK;
}

crkdg_status crkdg_last_features(crkdg_t h, float *feat, int on_device) {
    if (!h || !feat) return CRKDG_E_ARG;
    if (!h->feat) return fail(h, CRKDG_E_ARG, "last_features: needs a 2D handle with an indicator");
    CK(h, cudaMemcpyAsync(feat, h->feat, (size_t)h->ncell * CRKDG_MLP_NIN * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

crkdg_status crkdg_cell_averages(crkdg_t h, double *avg, int on_device) {
    if (!h || !avg) return CRKDG_E_ARG;
    Params P = base_params(h);
    if (h->mixed) {
        CK(h, launch_x(h, KX_AVG, P, base_xbufs(h)));
    } else {
        Bufs B = base_bufs(h);
        CK(h, launch(h, K_AVG, P, B));
    }
    CK(h, cudaMemcpyAsync(avg, h->aux, (size_t)h->ncell * h->m * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRKDG_OK;
}

crkdg_status crkdg_bound_margins(crkdg_t h, double margins[2]) {
    if (!h || !margins) return CRKDG_E_ARG;
    crkdg_status s = reset_scalars(h);
    if (s) return s;
    Params P = base_params(h);
    if (h->mixed) {
        CK(h, launch_x(h, KX_SCAN, P, base_xbufs(h)));
    } else {
        Bufs B = base_bufs(h);
        CK(h, launch(h, K_MARGINS, P, B));
    }
    s = read_scalars(h);
    if (s) return s;
    margins[0] = from_ordbits(h->hs->ord[0]);
    margins[1] = from_ordbits(h->hs->ord[1]);
    return CRKDG_OK;
}

crkdg_status crkdg_total_mass(crkdg_t h, int comp, double *mass) {
    if (!h || !mass || comp < 0 || comp >= h->m) return CRKDG_E_ARG;
    try {
        std::string tmp;
        double *host = new (std::nothrow) double[(size_t)h->ncell * h->m];
        if (!host) return CRKDG_E_OOM;
        crkdg_status s = crkdg_cell_averages(h, host, 0);
        if (s) {
            delete[] host;
            return s;
        }
        double acc = 0.0;  // fixed cell order: deterministic; cells of the domain only
        const bool geo = !h->geo_host.empty();
        for (int c = 0; c < h->ncell; ++c)
            if (!geo || !(h->geo_host[c] & GEO_SOLID)) acc += host[(size_t)c * h->m + comp];
        delete[] host;
        double hx = (h->mesh.x1 - h->mesh.x0) / h->mesh.nx;
        double hy = h->dim == 2 ? (h->mesh.y1 - h->mesh.y0) / h->mesh.ny : 1.0;
        *mass = acc * hx * hy;
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

// ---------------------------------------------------------------- non-rectangular domains

crkdg_status crkdg_set_geometry(crkdg_t h, const unsigned *geo, const double *state_a, const double *state_b,
                                double shock_x0, double shock_speed) {
    if (!h) return CRKDG_E_ARG;
    try {
        if (!geo) {
            if (h->geo) CK(h, cudaFree(h->geo));
            h->geo = nullptr;
            h->geo_host.clear();
            h->a0_valid = false;
            return CRKDG_OK;
        }
        if (h->dim != 2) return fail(h, CRKDG_E_UNSUPPORTED, "set_geometry: 2D meshes only");
        if (h->mixed || h->opt.scheme != CRKDG_SCHEME_COMPACT || h->opt.indicator != CRKDG_IND_OFF || h->own_on)
            return fail(h, CRKDG_E_UNSUPPORTED,
                        "set_geometry: FP64, the compact scheme, no indicator, no subdomain");
        if (!(isfinite(shock_x0) && isfinite(shock_speed)))
            return fail(h, CRKDG_E_ARG, "set_geometry: the shock line must be finite");
        const int nx = h->mesh.nx, ny = h->mesh.ny;
        auto solid = [&](int cell) { return (geo[cell] & GEO_SOLID) != 0u; };
        for (int cell = 0; cell < h->ncell; ++cell) {
            const unsigned g = geo[cell];
            if (g & ~(GEO_SOLID | 0xFFFFu)) return fail(h, CRKDG_E_ARG, "set_geometry: unknown bits in a word");
            if (solid(cell)) continue;
            const int cx = cell % nx, cy = cell / nx;
            for (int s = 0; s < 4; ++s) {
                const unsigned kind = (g >> (4 * s)) & 15u;
                if (kind > GEO_SHOCK) return fail(h, CRKDG_E_ARG, "set_geometry: unknown boundary kind");
                if (kind != GEO_MESH) continue;
                int nb;
                const int *bc = h->mesh.bc;
                if (s == 0) nb = cx > 0 ? cell - 1 : (bc[0] == CRKDG_BC_PERIODIC ? cell + nx - 1 : -1);
                else if (s == 1) nb = cx < nx - 1 ? cell + 1 : (bc[1] == CRKDG_BC_PERIODIC ? cell - nx + 1 : -1);
                else if (s == 2) nb = cy > 0 ? cell - nx : (bc[2] == CRKDG_BC_PERIODIC ? cell + (ny - 1) * nx : -1);
                else nb = cy < ny - 1 ? cell + nx : (bc[3] == CRKDG_BC_PERIODIC ? cell - (ny - 1) * nx : -1);
                if (nb >= 0 && solid(nb))
                    return fail(h, CRKDG_E_ARG, "set_geometry: a fluid side faces a solid cell without a boundary kind");
            }
        }
        if (!h->geo) CK(h, cudaMalloc(&h->geo, sizeof(unsigned) * h->ncell));
        CK(h, cudaMemcpyAsync(h->geo, geo, sizeof(unsigned) * h->ncell, cudaMemcpyHostToDevice, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        h->geo_host.assign(geo, geo + h->ncell);
        for (int c = 0; c < MAXM; ++c) {
            h->gstate[0][c] = state_a && c < h->m ? state_a[c] : 0.0;
            h->gstate[1][c] = state_b && c < h->m ? state_b[c] : 0.0;
        }
        h->shock_x0 = shock_x0;
        h->shock_speed = shock_speed;
        h->a0_valid = false;
        return CRKDG_OK;
    } catch (...) {
        return CRKDG_E_OOM;
    }
}

// ---------------------------------------------------------------- subdomains

crkdg_status crkdg_set_subdomain(crkdg_t h, const crkdg_mesh *global, int i0, int i1, int j0, int j1) {
    if (!h) return CRKDG_E_ARG;
    if (h->dim == 1) {
        j0 = 0;
        j1 = 1;
    }
    if (!(0 <= i0 && i0 < i1 && i1 <= h->mesh.nx && 0 <= j0 && j0 < j1 && j1 <= h->mesh.ny))
        return fail(h, CRKDG_E_ARG, "set_subdomain: need 0 <= i0 < i1 <= nx and 0 <= j0 < j1 <= ny");
    if (h->opt.indicator != CRKDG_IND_OFF)
        return fail(h, CRKDG_E_UNSUPPORTED, "set_subdomain: the troubled-cell indicators need a second exchange");
    if (h->geo) return fail(h, CRKDG_E_UNSUPPORTED, "set_subdomain: not with a non-rectangular domain");
    double rhx = 0.0, rhy = 0.0;
    if (global) {
        if (global->dim != h->dim || global->nx < 1 || (h->dim == 2 && global->ny < 1) ||
            !(global->x1 > global->x0) || (h->dim == 2 && !(global->y1 > global->y0)))
            return fail(h, CRKDG_E_ARG, "set_subdomain: bad global mesh");
        // the global handle's own formula, so that the window's arithmetic is the same bits
        rhx = 2.0 * global->nx / (global->x1 - global->x0);
        rhy = h->dim == 2 ? 2.0 * global->ny / (global->y1 - global->y0) : 0.0;
        const double lx = 2.0 * h->mesh.nx / (h->mesh.x1 - h->mesh.x0);
        const double ly = h->dim == 2 ? 2.0 * h->mesh.ny / (h->mesh.y1 - h->mesh.y0) : 0.0;
        if (fabs(lx - rhx) > 1e-9 * rhx || (h->dim == 2 && fabs(ly - rhy) > 1e-9 * rhy))
            return fail(h, CRKDG_E_ARG, "set_subdomain: the local cells are not the global mesh's cells");
    }
    const bool whole = i0 == 0 && i1 == h->mesh.nx && j0 == 0 && j1 == h->mesh.ny;
    h->own_on = !whole;
    h->own[0] = i0;
    h->own[1] = i1;
    h->own[2] = j0;
    h->own[3] = j1;
    h->metric_on = global != nullptr;
    h->rhx_g = rhx;
    h->rhy_g = rhy;
    h->a0_valid = false;
    h->mass_valid = false;
    h->pending = false;
    return CRKDG_OK;
}

size_t crkdg_cells_bytes(crkdg_t h, long long cells) {
    if (!h || cells < 0) return 0;
    if (h->mixed) return (size_t)cells * h->m * (sizeof(double) + h->nn * sizeof(float));
    return (size_t)cells * h->m * h->nn * sizeof(double);
}

namespace {

// Copy the cells of the box [i0, i1) x [j0, j1) between the current state u^n and a packed
// buffer (out: state -> buffer).  One strided copy per component and array.
crkdg_status copy_cells(crkdg_t h, int i0, int i1, int j0, int j1, void *buf, size_t bytes, int on_device,
                        bool out) {
    if (!buf) return fail(h, CRKDG_E_ARG, "pack/unpack: NULL buffer");
    if (h->dim == 1) {
        j0 = 0;
        j1 = 1;
    }
    if (!(0 <= i0 && i0 < i1 && i1 <= h->mesh.nx && 0 <= j0 && j0 < j1 && j1 <= h->mesh.ny))
        return fail(h, CRKDG_E_ARG, "pack/unpack: box outside the mesh");
    const long long w = i1 - i0, rows = j1 - j0, cells = w * rows;
    if (bytes != crkdg_cells_bytes(h, cells)) return fail(h, CRKDG_E_ARG, "pack/unpack: wrong byte count");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    const size_t nx = (size_t)h->mesh.nx, nc = (size_t)h->ncell, nn = (size_t)h->nn;
    char *pb = (char *)buf;
    auto copy2d = [&](char *dev, size_t elem, size_t per_cell, char *packed) -> cudaError_t {
        // device rows: component plane base + (j0 + r) nx + i0, pitch nx cells
        char *d0 = dev + ((size_t)j0 * nx + i0) * per_cell * elem;
        const size_t dpitch = nx * per_cell * elem, width = (size_t)w * per_cell * elem;
        return out ? cudaMemcpy2DAsync(packed, width, d0, dpitch, width, rows, kind, h->st)
                   : cudaMemcpy2DAsync(d0, dpitch, packed, width, width, rows, kind, h->st);
    };
    if (h->mixed) {
        double *ub = h->xub[h->xcur];
        float *dv = h->xdv[h->xcur];
        for (int c = 0; c < h->m; ++c)
            CK(h, copy2d((char *)(ub + (size_t)c * nc), sizeof(double), 1, pb + (size_t)c * cells * sizeof(double)));
        char *pd = pb + (size_t)h->m * cells * sizeof(double);
        for (int c = 0; c < h->m; ++c)
            CK(h, copy2d((char *)(dv + (size_t)c * nc * nn), sizeof(float), nn, pd + (size_t)c * cells * nn * sizeof(float)));
    } else {
        for (int c = 0; c < h->m; ++c)
            CK(h, copy2d((char *)(h->u + (size_t)c * nc * nn), sizeof(double), nn,
                         pb + (size_t)c * cells * nn * sizeof(double)));
    }
    if (!on_device) CK(h, cudaStreamSynchronize(h->st));
    if (!out) {
        h->pending = false;
        // cells inside the owned box change what the rate and the totals were taken over
        const bool hits_own = !h->own_on || !(i1 <= h->own[0] || i0 >= h->own[1] || j1 <= h->own[2] || j0 >= h->own[3]);
        if (hits_own) {
            h->a0_valid = false;
            h->mass_valid = false;
        }
    }
    return CRKDG_OK;
}

}  // namespace

crkdg_status crkdg_pack_cells(crkdg_t h, int i0, int i1, int j0, int j1, void *buf, size_t bytes, int on_device) {
    if (!h) return CRKDG_E_ARG;
    return copy_cells(h, i0, i1, j0, j1, buf, bytes, on_device, true);
}

crkdg_status crkdg_unpack_cells(crkdg_t h, int i0, int i1, int j0, int j1, const void *buf, size_t bytes,
                                int on_device) {
    if (!h) return CRKDG_E_ARG;
    return copy_cells(h, i0, i1, j0, j1, const_cast<void *>(buf), bytes, on_device, false);
}

}  // extern "C"
