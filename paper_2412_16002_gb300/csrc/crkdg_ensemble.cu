// crkdg_ensemble.cu -- host side of the ensemble entry points (include/crkdg.h).
//
// One descriptor per problem lives in a device table; all problems' buffers are
// slices of shared arenas.  A step is one CUDA graph: open the step (trial steps),
// the persistent inner and final launches of each degree, the indicator launches,
// close the attempt, and copy the "someone must retry" flag to pinned memory.  While
// that flag is set, a second graph (the same launches without the opening kernel)
// runs again for the problems that halved their step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/crkdg.h"
#include "dg_types.h"

using namespace crkdg;

namespace {

constexpr int NCLASS = 6;  // {k=2, k=3} x {<= 512^2, <= 1024^2, larger}
constexpr int TILES[] = {1, 2, 4, 8, 16};

int size_class(long long ncell) { return ncell <= 512LL * 512 ? 0 : (ncell <= 1024LL * 1024 ? 1 : 2); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct crkdg_ensemble_ctx {
    int np = 0;
    crkdg_flux flux{};
    crkdg_bounds bounds{};
    crkdg_options opt{};
    std::vector<crkdg_ens_problem> spec;
    std::vector<std::vector<double>> tabA, tabB;
    cudaStream_t st = nullptr;
    int nsm = 0;
    // descriptor table and scalars
    EnsProblem *dprob = nullptr;
    std::vector<EnsProblem> hprob;
    EnsScal *dsc = nullptr;
    EnsCtl *dctl = nullptr;
    int *hpend = nullptr;  // pinned
    // arenas
    double *arena_u[2] = {nullptr, nullptr};
    double *arena_ustar = nullptr, *arena_tr = nullptr, *arena_tavg = nullptr, *arena_aux = nullptr;
    int *arena_flags = nullptr;
    float *arena_feat = nullptr, *arena_prob = nullptr, *mlp = nullptr;
    long long total_cells = 0;
    bool harvest = false;
    // work items: [group n=3,4][0 cell blocks, 1 feature blocks]
    EnsItem *ditems[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int nitems[2][2] = {{0, 0}, {0, 0}};
    int cap_items[2][2] = {{0, 0}, {0, 0}};
    int tile[NCLASS] = {4, 4, 4, 4, 4, 4};
    int occ[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // resident blocks per SM, [group][kind]
    cudaGraphExec_t g_step = nullptr, g_attempt = nullptr;
    bool graphs_valid = false;
    bool prof = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double prof_ms = 0.0;
    long long prof_n = 0;
    std::string err;
};

namespace {

crkdg_status efail(crkdg_ens_t e, crkdg_status s, const std::string &msg) {
    if (e) e->err = msg;
    return s;
}

#define ECK(e, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return efail(e, e_ == cudaErrorMemoryAllocation ? CRKDG_E_OOM : CRKDG_E_CUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

int group_of(int n) { return n - 3; }  // n = k + 1 in {3, 4}

// Work items of one degree group: problems of that degree, largest first.
crkdg_status build_items(crkdg_ens_t e, int g) {
    const int n = g + 3;
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<int> idx;
        std::vector<long long> nc;
        std::vector<int> tl;
        for (int i = 0; i < e->np; ++i)
            if (e->hprob[i].n == n) {
                idx.push_back(i);
                nc.push_back(e->hprob[i].P.ncell);
                tl.push_back(kind == 0 ? e->tile[e->hprob[i].klass] : 4);
            }
        const int cpb = crkdg_ens_cells_per_block(kind == 0 ? ENS_INNER : ENS_FEATURES, n);
        int cnt = crkdg_ensemble_plan((int)idx.size(), nc.data(), tl.data(), cpb, nullptr, 0);
        std::vector<int> raw((size_t)std::max(cnt, 0) * 3);
        if (cnt > 0) crkdg_ensemble_plan((int)idx.size(), nc.data(), tl.data(), cpb, raw.data(), cnt);
        std::vector<EnsItem> items((size_t)std::max(cnt, 0));
        for (int j = 0; j < cnt; ++j) items[j] = EnsItem{idx[raw[3 * j]], raw[3 * j + 1], raw[3 * j + 2], 0};
        if (cnt > e->cap_items[g][kind]) {
            if (e->ditems[g][kind]) cudaFree(e->ditems[g][kind]);
            e->ditems[g][kind] = nullptr;
            e->cap_items[g][kind] = 0;
            ECK(e, cudaMalloc(&e->ditems[g][kind], sizeof(EnsItem) * (size_t)cnt));
            e->cap_items[g][kind] = cnt;
        }
        if (cnt > 0)
            ECK(e, cudaMemcpyAsync(e->ditems[g][kind], items.data(), sizeof(EnsItem) * (size_t)cnt,
                                   cudaMemcpyHostToDevice, e->st));
        e->nitems[g][kind] = std::max(cnt, 0);
    }
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

// Persistent grid: every resident block slot of the GPU, at most one block per item.
int grid_of(crkdg_ens_t e, int kind, int n, int nitems) {
    int g = std::max(1, e->occ[n - 3][kind]) * e->nsm;
    return std::max(1, std::min(g, nitems));
}

// The persistent launches of one attempt (counters 0..9), then the closing kernel
// and the copy of the retry flag.
crkdg_status enqueue_attempt(crkdg_ens_t e) {
    int counter = 0;
    auto run = [&](int kind, int stage) -> cudaError_t {
        for (int g = 0; g < 2; ++g) {
            const int which = kind == ENS_FEATURES ? 1 : 0;
            const int cnt = e->nitems[g][which];
            const int c = counter++;
            if (cnt == 0) continue;
            cudaError_t r = crkdg_ens_launch(kind, g + 3, grid_of(e, kind, g + 3, cnt), e->st, e->dprob,
                                             e->ditems[g][which], cnt, e->dctl, c, stage);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    ECK(e, run(ENS_INNER, 0));
    ECK(e, run(ENS_FINAL, 0));
    const int ind = e->opt.indicator;
    if (ind != CRKDG_IND_OFF) {
        const bool learned = ind == CRKDG_IND_MLP;
        if (learned || e->harvest) {
            ECK(e, run(ENS_FEATURES, 0));  // features and the plain decision in one pass
            if (learned && crkdg_mlp_forward(e->mlp, e->arena_feat, (int)e->total_cells, e->arena_prob, e->st) !=
                               CRKDG_OK)
                return efail(e, CRKDG_E_CUDA, "ensemble: MLP forward failed");
            ECK(e, run(ENS_TROUBLE, learned ? 3 : 2));
        } else {
            ECK(e, run(ENS_TROUBLE, 0));
        }
    }
    ECK(e, crkdg_ens_control(2, e->st, e->dprob, e->np, e->dctl, e->opt.max_halvings));
    ECK(e, cudaMemcpyAsync(e->hpend, &e->dctl->any_pending, sizeof(int), cudaMemcpyDeviceToHost, e->st));
    return CRKDG_OK;
}

crkdg_status capture(crkdg_ens_t e, bool open_step, cudaGraphExec_t *out) {
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t graph = nullptr;
    ECK(e, cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t r = open_step ? crkdg_ens_control(0, e->st, e->dprob, e->np, e->dctl, -1)
                              : crkdg_ens_control(1, e->st, e->dprob, e->np, e->dctl, 0);
    crkdg_status s = r == cudaSuccess ? enqueue_attempt(e) : CRKDG_E_CUDA;
    cudaError_t r2 = cudaStreamEndCapture(e->st, &graph);
    if (s != CRKDG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (r != cudaSuccess) return efail(e, CRKDG_E_CUDA, std::string("ensemble capture: ") + cudaGetErrorString(r));
    ECK(e, r2);
    cudaError_t r3 = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    ECK(e, r3);
    return CRKDG_OK;
}

crkdg_status ensure_graphs(crkdg_ens_t e) {
    if (e->graphs_valid) return CRKDG_OK;
    crkdg_status s = capture(e, true, &e->g_step);
    if (s) return s;
    s = capture(e, false, &e->g_attempt);
    if (s) return s;
    e->graphs_valid = true;
    return CRKDG_OK;
}

crkdg_status pull_table(crkdg_ens_t e) {
    ECK(e, cudaMemcpyAsync(e->hprob.data(), e->dprob, sizeof(EnsProblem) * e->np, cudaMemcpyDeviceToHost, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

crkdg_status push_problem(crkdg_ens_t e, int i) {
    ECK(e, cudaMemcpyAsync(e->dprob + i, &e->hprob[i], sizeof(EnsProblem), cudaMemcpyHostToDevice, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

Bufs single_bufs(const EnsProblem &p) {
    Bufs B;
    memset(&B, 0, sizeof(B));
    B.un = p.u[p.cur];
    B.unew = p.u[p.cur ^ 1];
    B.ustar = p.ustar;
    B.tr = p.tr;
    B.tavg = p.tavg;
    B.flag = &p.sc->flag;
    B.nlim = &p.sc->nlim;
    B.thmin = &p.sc->thmin;
    B.a0 = &p.sc->a0;
    B.aux = p.aux;
    B.ord = p.sc->ord;
    B.tflags = p.tflags;
    B.ntrb = &p.sc->ntrb;
    B.feat = p.feat;
    B.prob = p.prob;
    return B;
}

double from_bits(unsigned long long u) {
    double x;
    memcpy(&x, &u, 8);
    return x;
}
unsigned long long to_bits(double x) {
    unsigned long long u;
    memcpy(&u, &x, 8);
    return u;
}

crkdg_status check_problem(crkdg_ens_t e, const crkdg_ens_problem &q) {
    const crkdg_mesh &M = q.mesh;
    if (M.dim != 2 || M.nx < 1 || M.ny < 1) return efail(e, CRKDG_E_ARG, "ensemble: meshes must be 2D with nx, ny >= 1");
    if (!(M.x1 > M.x0) || !(M.y1 > M.y0)) return efail(e, CRKDG_E_ARG, "ensemble: empty domain");
    if ((long long)M.nx * M.ny > (1LL << 30)) return efail(e, CRKDG_E_ARG, "ensemble: mesh too large");
    for (int s = 0; s < 4; ++s)
        if (M.bc[s] < CRKDG_BC_PERIODIC || M.bc[s] > CRKDG_BC_DIRICHLET) return efail(e, CRKDG_E_ARG, "ensemble: bad bc");
    for (int d = 0; d < 2; ++d)
        if ((M.bc[2 * d] == CRKDG_BC_PERIODIC) != (M.bc[2 * d + 1] == CRKDG_BC_PERIODIC))
            return efail(e, CRKDG_E_ARG, "ensemble: periodic sides must come in pairs");
    if (q.k < 2 || q.k > 3) return efail(e, CRKDG_E_UNSUPPORTED, "ensemble: k must be 2 or 3");
    const crkdg_tableau *t = q.tableau;
    if (!t || !t->A || !t->b || t->s < 1 || t->s > MAXS) return efail(e, CRKDG_E_ARG, "ensemble: bad tableau");
    for (int i = 0; i < t->s; ++i) {
        if (!std::isfinite(t->b[i]) || t->b[i] < 0.0) return efail(e, CRKDG_E_ARG, "ensemble: b must be >= 0");
        for (int j = 0; j < t->s; ++j) {
            double a = t->A[i * t->s + j];
            if (!std::isfinite(a) || (j >= i && a != 0.0))
                return efail(e, CRKDG_E_ARG, "ensemble: A must be finite and strictly lower triangular");
        }
    }
    if (!(q.cfl > 0.0) || !std::isfinite(q.cfl)) return efail(e, CRKDG_E_ARG, "ensemble: cfl must be > 0");
    if (!(q.t_end > 0.0)) return efail(e, CRKDG_E_ARG, "ensemble: t_end must be > 0");
    return CRKDG_OK;
}

void release(crkdg_ens_t e) {
    for (cudaEvent_t v : e->ev)
        if (v) cudaEventDestroy(v);
    if (e->g_step) cudaGraphExecDestroy(e->g_step);
    if (e->g_attempt) cudaGraphExecDestroy(e->g_attempt);
    for (int g = 0; g < 2; ++g)
        for (int k = 0; k < 2; ++k)
            if (e->ditems[g][k]) cudaFree(e->ditems[g][k]);
    for (double *p : {e->arena_u[0], e->arena_u[1], e->arena_ustar, e->arena_tr, e->arena_tavg, e->arena_aux})
        if (p) cudaFree(p);
    if (e->arena_flags) cudaFree(e->arena_flags);
    if (e->arena_feat) cudaFree(e->arena_feat);
    if (e->arena_prob) cudaFree(e->arena_prob);
    if (e->mlp) cudaFree(e->mlp);
    if (e->dprob) cudaFree(e->dprob);
    if (e->dsc) cudaFree(e->dsc);
    if (e->dctl) cudaFree(e->dctl);
    if (e->hpend) cudaFreeHost(e->hpend);
    if (e->st) cudaStreamDestroy(e->st);
}

}  // namespace

extern "C" {

int crkdg_ensemble_plan(int count, const long long *ncells, const int *tile, int cells_per_block, int *items,
                        int cap) {
    if (count < 0 || (count > 0 && (!ncells || !tile)) || cells_per_block < 1) return -1;
    std::vector<int> order((size_t)count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ncells[a] > ncells[b]; });
    long long total = 0;
    for (int i : order) {
        if (ncells[i] < 0 || tile[i] < 1) return -1;
        const long long nb = (ncells[i] + cells_per_block - 1) / cells_per_block;
        for (long long b = 0; b < nb; b += tile[i]) {
            if (items && total < cap) {
                items[3 * total] = i;
                items[3 * total + 1] = (int)b;
                items[3 * total + 2] = (int)std::min<long long>(tile[i], nb - b);
            }
            ++total;
            if (total > (1LL << 30)) return -1;
        }
    }
    return (int)total;
}

crkdg_status crkdg_ensemble_create(int count, const crkdg_ens_problem *problems, int m, const crkdg_flux *flux,
                                   const crkdg_bounds *bounds, const crkdg_options *opt, crkdg_ens_t *out) {
    if (!out || !problems || !flux || !bounds || count < 1) return CRKDG_E_ARG;
    *out = nullptr;
    crkdg_ens_t e = nullptr;
    try {
        e = new crkdg_ensemble_ctx();
    } catch (...) {
        return CRKDG_E_OOM;
    }
    auto bail = [&](crkdg_status s) {
        release(e);
        delete e;
        return s;
    };
    e->np = count;
    e->flux = *flux;
    e->bounds = *bounds;
    if (opt) {
        e->opt = *opt;
    } else {
        crkdg_options_default(&e->opt);
    }
    if (m != 4 || flux->kind != CRKDG_FLUX_EULER || !(flux->gamma > 1.0)) return bail(CRKDG_E_ARG);
    if (e->opt.precision != CRKDG_PREC_FP64 || e->opt.scheme != CRKDG_SCHEME_COMPACT) return bail(CRKDG_E_UNSUPPORTED);
    if (e->opt.indicator < CRKDG_IND_OFF || e->opt.indicator > CRKDG_IND_MLP || e->opt.max_halvings < 0)
        return bail(CRKDG_E_ARG);
    if (!(bounds->eps > 0.0)) return bail(CRKDG_E_ARG);
    e->spec.assign(problems, problems + count);
    for (int i = 0; i < count; ++i) {
        crkdg_status s = check_problem(e, problems[i]);
        if (s) return bail(s);
        const crkdg_tableau *t = problems[i].tableau;
        e->tabA.emplace_back(t->A, t->A + t->s * t->s);
        e->tabB.emplace_back(t->b, t->b + t->s);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return bail(CRKDG_E_CUDA);
    if (cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking) != cudaSuccess) return bail(CRKDG_E_CUDA);
    for (int g = 0; g < 2; ++g)
        for (int kind = 0; kind < 4; ++kind) e->occ[g][kind] = crkdg_ens_occupancy(kind, g + 3);
    NodalTables tab[3];
    crkdg_build_tables(tab);
    if (crkdg_upload_tables_2d(tab) != cudaSuccess || crkdg_upload_tables_ens(tab) != cudaSuccess)
        return bail(CRKDG_E_CUDA);

    // sizes and arena offsets (slices aligned to 32 doubles)
    const bool ind = e->opt.indicator != CRKDG_IND_OFF;
    std::vector<size_t> off_u(count), off_tr(count), off_tavg(count), off_aux(count);
    std::vector<long long> off_cell(count);
    size_t tot_u = 0, tot_tr = 0, tot_tavg = 0, tot_aux = 0;
    long long tot_cells = 0;
    for (int i = 0; i < count; ++i) {
        const int n = problems[i].k + 1;
        const long long nc = (long long)problems[i].mesh.nx * problems[i].mesh.ny;
        int ns = 0;
        for (int j = 0; j < problems[i].tableau->s; ++j) ns += problems[i].tableau->b[j] != 0.0;
        off_u[i] = tot_u;
        tot_u += align_up((size_t)4 * nc * n * n, 32);
        off_tr[i] = tot_tr;
        tot_tr += align_up((size_t)std::max(ns, 1) * 4 * nc * 4 * n, 32);
        off_tavg[i] = tot_tavg;
        tot_tavg += align_up((size_t)std::max(ns, 1) * 4 * nc, 32);
        off_aux[i] = tot_aux;
        tot_aux += align_up((size_t)4 * nc, 32);
        off_cell[i] = tot_cells;
        tot_cells += nc;
    }
    e->total_cells = tot_cells;
    auto alloc = [&](void **p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 256)) == cudaSuccess; };
    bool ok = alloc((void **)&e->arena_u[0], tot_u * 8) && alloc((void **)&e->arena_u[1], tot_u * 8) &&
              alloc((void **)&e->arena_ustar, tot_u * 8) && alloc((void **)&e->arena_tr, tot_tr * 8) &&
              alloc((void **)&e->arena_tavg, tot_tavg * 8) &&
              alloc((void **)&e->arena_aux, tot_aux * 8) && alloc((void **)&e->dsc, sizeof(EnsScal) * count) &&
              alloc((void **)&e->dctl, sizeof(EnsCtl)) && alloc((void **)&e->dprob, sizeof(EnsProblem) * count);
    if (ok && ind) ok = alloc((void **)&e->arena_flags, sizeof(int) * (size_t)tot_cells);
    if (ok && ind) {
        ok = alloc((void **)&e->arena_feat, sizeof(float) * CRKDG_MLP_NIN * (size_t)tot_cells) &&
             alloc((void **)&e->arena_prob, sizeof(float) * (size_t)tot_cells) &&
             alloc((void **)&e->mlp, sizeof(float) * CRKDG_MLP_NPARAM);
    }
    if (!ok) return bail(CRKDG_E_OOM);
    if (cudaMallocHost(&e->hpend, sizeof(int)) != cudaSuccess) return bail(CRKDG_E_OOM);
    if (cudaMemsetAsync(e->dctl, 0, sizeof(EnsCtl), e->st) != cudaSuccess ||
        cudaMemsetAsync(e->dsc, 0, sizeof(EnsScal) * count, e->st) != cudaSuccess)
        return bail(CRKDG_E_CUDA);
    if (ind && (cudaMemsetAsync(e->arena_flags, 0, sizeof(int) * (size_t)tot_cells, e->st) != cudaSuccess ||
                cudaMemsetAsync(e->arena_prob, 0, sizeof(float) * (size_t)tot_cells, e->st) != cudaSuccess ||
                cudaMemsetAsync(e->mlp, 0, sizeof(float) * CRKDG_MLP_NPARAM, e->st) != cudaSuccess))
        return bail(CRKDG_E_CUDA);

    // descriptors (parameters formed exactly as for a single handle)
    e->hprob.resize(count);
    for (int i = 0; i < count; ++i) {
        const crkdg_ens_problem &q = problems[i];
        EnsProblem &p = e->hprob[i];
        memset(&p, 0, sizeof(p));
        Params &P = p.P;
        P.nx = q.mesh.nx;
        P.ny = q.mesh.ny;
        P.ncell = q.mesh.nx * q.mesh.ny;
        P.rhx = 2.0 * q.mesh.nx / (q.mesh.x1 - q.mesh.x0);
        P.rhy = 2.0 * q.mesh.ny / (q.mesh.y1 - q.mesh.y0);
        P.gamma = flux->gamma;
        P.velx = flux->velocity[0];
        P.vely = flux->velocity[1];
        P.lo = bounds->lo;
        P.hi = bounds->hi;
        P.eps = bounds->eps;
        P.tvb_M = e->opt.tvb_M;
        tvb_thresholds(P);
        screen_bounds(P);
        for (int s = 0; s < 4; ++s) {
            P.bc[s] = q.mesh.bc[s];
            for (int c = 0; c < MAXM; ++c) P.bcs[s][c] = q.mesh.bc_state[s][c];
        }
        for (int j = 0; j < MAXS; ++j) P.slot[j] = -1;
        const crkdg_tableau *t = q.tableau;
        P.s = t->s;
        int ns = 0;
        for (int a = 0; a < t->s; ++a) {
            P.b[a] = t->b[a];
            for (int b = 0; b < t->s; ++b) P.A[a][b] = t->A[a * t->s + b];
            P.slot[a] = t->b[a] != 0.0 ? ns++ : -1;
        }
        P.nslot = ns;
        P.mode = MODE_STEP;
        P.defer_limit = ind ? 1 : 0;
        p.u[0] = e->arena_u[0] + off_u[i];
        p.u[1] = e->arena_u[1] + off_u[i];
        p.ustar = e->arena_ustar + off_u[i];
        p.tr = e->arena_tr + off_tr[i];
        p.tavg = e->arena_tavg + off_tavg[i];
        p.aux = e->arena_aux + off_aux[i];
        p.tflags = ind ? e->arena_flags + off_cell[i] : nullptr;
        p.feat = ind ? e->arena_feat + (size_t)off_cell[i] * CRKDG_MLP_NIN : nullptr;
        p.prob = ind ? e->arena_prob + off_cell[i] : nullptr;
        p.sc = e->dsc + i;
        p.n = q.k + 1;
        p.klass = (p.n - 3) * 3 + size_class(P.ncell);
        p.t = 0.0;
        p.t_end = q.t_end;
        p.cfl = q.cfl;
        p.a0 = 0.0;
        p.done = 1;  // until its state is set
    }
    if (cudaMemcpyAsync(e->dprob, e->hprob.data(), sizeof(EnsProblem) * count, cudaMemcpyHostToDevice, e->st) !=
        cudaSuccess)
        return bail(CRKDG_E_CUDA);
    for (int g = 0; g < 2; ++g)
        if (build_items(e, g) != CRKDG_OK) return bail(CRKDG_E_CUDA);
    if (cudaStreamSynchronize(e->st) != cudaSuccess) return bail(CRKDG_E_CUDA);
    *out = e;
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_destroy(crkdg_ens_t e) {
    if (!e) return CRKDG_OK;
    if (e->st) cudaStreamSynchronize(e->st);
    release(e);
    delete e;
    return CRKDG_OK;
}

size_t crkdg_ensemble_state_size(crkdg_ens_t e, int i) {
    if (!e || i < 0 || i >= e->np) return 0;
    const EnsProblem &p = e->hprob[i];
    return (size_t)4 * p.P.ncell * p.n * p.n;
}

crkdg_status crkdg_ensemble_set_state(crkdg_ens_t e, int i, const double *nodal, size_t count, int on_device) {
    if (!e || !nodal || i < 0 || i >= e->np) return CRKDG_E_ARG;
    if (count != crkdg_ensemble_state_size(e, i)) return efail(e, CRKDG_E_ARG, "ensemble set_state: count");
    crkdg_status s = pull_table(e);
    if (s) return s;
    EnsProblem &p = e->hprob[i];
    double *scratch = p.u[p.cur ^ 1];
    ECK(e, cudaMemcpyAsync(scratch, nodal, count * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, e->st));
    // limiter (as crkdg_set_state), then the rate of the limited state (as crkdg_max_dt)
    const int nblocks = (p.P.ncell + crkdg_ens_cells_per_block(ENS_INNER, p.n) - 1) /
                        crkdg_ens_cells_per_block(ENS_INNER, p.n);
    Bufs B = single_bufs(p);
    B.un = scratch;
    B.unew = p.u[p.cur];
    Params P = p.P;
    ECK(e, crkdg_launch_2d(K_LIMIT, p.n, PH_EULER, nblocks, e->st, P, B));
    EnsScal init;
    memset(&init, 0, sizeof(init));
    init.thmin = to_bits(1.0);
    init.ord[0] = init.ord[1] = ~0ull;
    ECK(e, cudaMemcpyAsync(p.sc, &init, sizeof(init), cudaMemcpyHostToDevice, e->st));
    B = single_bufs(p);
    ECK(e, crkdg_launch_2d(K_A0, p.n, PH_EULER, nblocks, e->st, P, B));
    EnsScal back;
    ECK(e, cudaMemcpyAsync(&back, p.sc, sizeof(back), cudaMemcpyDeviceToHost, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    p.a0 = from_bits(back.a0);
    p.t = 0.0;
    p.done = 0;
    p.status = 0;
    p.pending = 0;
    p.steps = p.restarts_total = 0;
    p.last_dt = p.last_thmin = 0.0;
    p.last_nlim = p.last_ntrb = 0;
    p.last_restarts = 0;
    return push_problem(e, i);
}

crkdg_status crkdg_ensemble_get_state(crkdg_ens_t e, int i, double *nodal, size_t count, int on_device) {
    if (!e || !nodal || i < 0 || i >= e->np) return CRKDG_E_ARG;
    if (count != crkdg_ensemble_state_size(e, i)) return efail(e, CRKDG_E_ARG, "ensemble get_state: count");
    crkdg_status s = pull_table(e);
    if (s) return s;
    const EnsProblem &p = e->hprob[i];
    ECK(e, cudaMemcpyAsync(nodal, p.u[p.cur], count * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_step(crkdg_ens_t e, int *active) {
    if (!e) return CRKDG_E_ARG;
    crkdg_status s = pull_table(e);
    if (s) return s;
    int failed_before = 0;
    for (const EnsProblem &p : e->hprob) failed_before += p.status != 0;
    s = ensure_graphs(e);
    if (s) return s;
    if (e->prof) ECK(e, cudaEventRecord(e->ev[0], e->st));
    ECK(e, cudaGraphLaunch(e->g_step, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    // every retry halves some problem's dt; max_halvings bounds the rounds
    for (int round = 0; *e->hpend && round <= e->opt.max_halvings + 1; ++round) {
        ECK(e, cudaGraphLaunch(e->g_attempt, e->st));
        ECK(e, cudaStreamSynchronize(e->st));
    }
    if (e->prof) {
        ECK(e, cudaEventRecord(e->ev[1], e->st));
        ECK(e, cudaEventSynchronize(e->ev[1]));
        float ms = 0.0f;
        ECK(e, cudaEventElapsedTime(&ms, e->ev[0], e->ev[1]));
        e->prof_ms += ms;
        e->prof_n += 1;
    }
    if (*e->hpend) return efail(e, CRKDG_E_CUDA, "ensemble step: attempts did not settle");
    s = pull_table(e);
    if (s) return s;
    int running = 0, failed = 0;
    for (const EnsProblem &p : e->hprob) {
        running += !p.done && p.status == 0;
        failed += p.status != 0;
    }
    if (active) *active = running;
    if (failed > failed_before)
        return efail(e, CRKDG_E_BOUNDS, "ensemble step: a problem's averages left B^eps after max_halvings restarts");
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_info(crkdg_ens_t e, int i, crkdg_ens_info *info) {
    if (!e || !info || i < 0 || i >= e->np) return CRKDG_E_ARG;
    crkdg_status s = pull_table(e);
    if (s) return s;
    const EnsProblem &p = e->hprob[i];
    info->t = p.t;
    info->steps = p.steps;
    info->restarts = p.restarts_total;
    info->done = p.done;
    info->status = p.status;
    info->last.dt_taken = p.last_dt;
    info->last.restarts = p.last_restarts;
    info->last.cells_limited = p.last_nlim;
    info->last.theta_min = p.last_thmin;
    info->last.troubled = p.last_ntrb;
    info->last.mass_drift = 0.0;
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_set_mlp(crkdg_ens_t e, const float *params) {
    if (!e || !params) return CRKDG_E_ARG;
    if (!e->mlp) return efail(e, CRKDG_E_ARG, "ensemble set_mlp: the indicator is off");
    ECK(e, cudaMemcpyAsync(e->mlp, params, sizeof(float) * CRKDG_MLP_NPARAM, cudaMemcpyDeviceToDevice, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_set_harvest(crkdg_ens_t e, int on) {
    if (!e) return CRKDG_E_ARG;
    if (on && (e->opt.indicator == CRKDG_IND_OFF || !e->arena_feat))
        return efail(e, CRKDG_E_ARG, "ensemble set_harvest: needs an indicator");
    if (e->harvest != (on != 0)) {
        e->harvest = on != 0;
        e->graphs_valid = false;  // the step graph gains (or drops) the feature pass
    }
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_last_features(crkdg_ens_t e, int i, float *feat, int on_device) {
    if (!e || !feat || i < 0 || i >= e->np) return CRKDG_E_ARG;
    if (!e->arena_feat) return efail(e, CRKDG_E_ARG, "ensemble last_features: the indicator is off");
    const EnsProblem &p = e->hprob[i];
    const size_t n = (size_t)p.P.ncell * CRKDG_MLP_NIN;
    ECK(e, cudaMemcpyAsync(feat, p.feat, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_troubled_flags(crkdg_ens_t e, int i, int *flags, int on_device) {
    if (!e || !flags || i < 0 || i >= e->np) return CRKDG_E_ARG;
    if (!e->arena_flags) return efail(e, CRKDG_E_ARG, "ensemble troubled_flags: the indicator is off");
    const EnsProblem &p = e->hprob[i];
    ECK(e, cudaMemcpyAsync(flags, p.tflags, (size_t)p.P.ncell * sizeof(int),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->st));
    ECK(e, cudaStreamSynchronize(e->st));
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_autotune(crkdg_ens_t e, int reps, int chosen[6]) {
    if (!e || reps < 1) return CRKDG_E_ARG;
    crkdg_status s = pull_table(e);
    if (s) return s;
    bool present[NCLASS] = {false, false, false, false, false, false};
    for (const EnsProblem &p : e->hprob)
        if (!p.done && p.status == 0) present[p.klass] = true;
    cudaEvent_t ev0, ev1;
    ECK(e, cudaEventCreate(&ev0));
    ECK(e, cudaEventCreate(&ev1));
    crkdg_status res = CRKDG_OK;
    for (int c = 0; c < NCLASS && res == CRKDG_OK; ++c) {
        if (!present[c]) continue;
        const int g = c / 3;
        float best = INFINITY;
        int best_tile = e->tile[c];
        for (int tl : TILES) {
            e->tile[c] = tl;
            if ((res = build_items(e, g)) != CRKDG_OK) break;
            float tot = 0.0f;
            for (int r = 0; r < reps + 1 && res == CRKDG_OK; ++r) {
                // open a step for this class only; inner and final kernels of its degree
                cudaError_t err = crkdg_ens_control(0, e->st, e->dprob, e->np, e->dctl, c);
                if (err == cudaSuccess) err = cudaEventRecord(ev0, e->st);
                const int cnt = e->nitems[g][0];
                if (err == cudaSuccess)
                    err = crkdg_ens_launch(ENS_INNER, g + 3, grid_of(e, ENS_INNER, g + 3, cnt), e->st, e->dprob,
                                           e->ditems[g][0], cnt, e->dctl, 0, 0);
                if (err == cudaSuccess)
                    err = crkdg_ens_launch(ENS_FINAL, g + 3, grid_of(e, ENS_FINAL, g + 3, cnt), e->st, e->dprob,
                                           e->ditems[g][0], cnt, e->dctl, 1, 0);
                if (err == cudaSuccess) err = cudaEventRecord(ev1, e->st);
                if (err == cudaSuccess) err = cudaEventSynchronize(ev1);
                float ms = 0.0f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ev0, ev1);
                if (err != cudaSuccess) res = efail(e, CRKDG_E_CUDA, std::string("autotune: ") + cudaGetErrorString(err));
                if (r > 0) tot += ms;  // the first repetition warms up
            }
            if (res == CRKDG_OK && tot < best) {
                best = tot;
                best_tile = tl;
            }
        }
        e->tile[c] = best_tile;
    }
    // nobody pending; the problems' states and times are untouched
    if (res == CRKDG_OK) {
        cudaError_t err = crkdg_ens_control(0, e->st, e->dprob, e->np, e->dctl, NCLASS);
        if (err == cudaSuccess) err = cudaStreamSynchronize(e->st);
        if (err != cudaSuccess) res = efail(e, CRKDG_E_CUDA, std::string("autotune: ") + cudaGetErrorString(err));
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    for (int g = 0; g < 2 && res == CRKDG_OK; ++g) res = build_items(e, g);
    e->graphs_valid = false;
    if (chosen)
        for (int c = 0; c < NCLASS; ++c) chosen[c] = present[c] ? e->tile[c] : 0;
    return res;
}

crkdg_status crkdg_ensemble_set_profiling(crkdg_ens_t e, int on) {
    if (!e) return CRKDG_E_ARG;
    for (cudaEvent_t &v : e->ev)
        if (!v) ECK(e, cudaEventCreate(&v));
    e->prof = on != 0;
    e->prof_ms = 0.0;
    e->prof_n = 0;
    return CRKDG_OK;
}

crkdg_status crkdg_ensemble_times(crkdg_ens_t e, double *ms, long long *steps) {
    if (!e || !ms || !steps) return CRKDG_E_ARG;
    *ms = e->prof_ms;
    *steps = e->prof_n;
    return CRKDG_OK;
}

const char *crkdg_ensemble_last_error(crkdg_ens_t e) {
    if (!e) return "invalid ensemble handle";
    return e->err.c_str();
}

}  // extern "C"
