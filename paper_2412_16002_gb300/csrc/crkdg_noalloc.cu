// crkdg_noalloc.cu -- the DG operator F without any device allocation.
//
// For callers that cannot call cudaMalloc: code running inside a CUDA graph
// capture or another framework's memory pool, plug-ins whose host forbids
// allocation after start-up, or hard real-time loops where an allocation could
// stall or fail.  They pass their own input and output buffers; the scratch the
// operator needs (the interior-trace stage accumulation and the face traces
// shared between neighbouring cells) lives in one file-scope device array.
//
// The array is a static __device__ symbol: every GPU that loads this library
// holds its CRKDG_NOALLOC_SCRATCH_DOUBLES doubles until the process exits.  In
// host code its name is only a host-side stand-in, so the device address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) and passed to the kernels.
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/crkdg.h"
#include "dg_types.h"

using namespace crkdg;

static __device__ __align__(256) double g_noalloc_scratch[CRKDG_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_ptr[kMaxDevices] = {};  // device address of the scratch array, per device
bool g_tables[kMaxDevices] = {};

// Closed-form Gauss / Gauss--Lobatto rules and the Lagrange tables on the Gauss
// nodes (same definitions as the handle-based path, built here independently
// so that no existing code path changes).
void rules(int n, double *x, double *w, double *xl) {
    if (n == 2) {
        x[0] = -1.0 / sqrt(3.0); x[1] = -x[0];
        w[0] = w[1] = 1.0;
        xl[0] = -1.0; xl[1] = 1.0;
    } else if (n == 3) {
        x[0] = -sqrt(0.6); x[1] = 0.0; x[2] = sqrt(0.6);
        w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
        xl[0] = -1.0; xl[1] = 0.0; xl[2] = 1.0;
    } else {
        double r = 2.0 / 7.0 * sqrt(6.0 / 5.0);
        double a = sqrt(3.0 / 7.0 - r), b = sqrt(3.0 / 7.0 + r);
        x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
        w[1] = w[2] = (18.0 + sqrt(30.0)) / 36.0;
        w[0] = w[3] = (18.0 - sqrt(30.0)) / 36.0;
        xl[0] = -1.0; xl[1] = 0.0; xl[2] = 1.0;
    }
}

double lag(int n, const double *x, int a, double t) {
    double v = 1.0;
    for (int b = 0; b < n; ++b)
        if (b != a) v *= (t - x[b]) / (x[a] - x[b]);
    return v;
}

double dlag(int n, const double *x, int a, double t) {
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

void tables(NodalTables *tab) {
    for (int n = 2; n <= 4; ++n) {
        NodalTables &T = tab[n - 2];
        memset(&T, 0, sizeof(T));
        int L = nlob(n);
        rules(n, T.xg, T.wg, T.xl);
        for (int a = 0; a < n; ++a) {
            for (int q = 0; q < n; ++q) T.Dhat[a][q] = T.wg[q] * dlag(n, T.xg, a, T.xg[q]) / T.wg[a];
            T.lm[a] = lag(n, T.xg, a, -1.0);
            T.lp[a] = lag(n, T.xg, a, 1.0);
            T.liftm[a] = T.lm[a] / T.wg[a];
            T.liftp[a] = T.lp[a] / T.wg[a];
            for (int al = 0; al < L; ++al) T.Igl[al][a] = lag(n, T.xg, a, T.xl[al]);
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
    }
}

// Once per device, with that device current: the scratch address and the tables.
crkdg_status setup(int dev, int dim, double **ptr) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return CRKDG_E_UNSUPPORTED;
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CRKDG_E_CUDA;
        g_ptr[dev] = (double *)p;
    }
    if (!g_tables[dev]) {
        NodalTables tab[3];
        tables(tab);
        if (crkdg_upload_tables_1d(tab) != cudaSuccess) return CRKDG_E_CUDA;
        if (crkdg_upload_tables_2d(tab) != cudaSuccess) return CRKDG_E_CUDA;
        g_tables[dev] = true;
    }
    (void)dim;
    *ptr = g_ptr[dev];
    return CRKDG_OK;
}

}  // namespace

extern "C" crkdg_status crkdg_apply_F_noalloc(const crkdg_mesh *mesh, int k, int m, const crkdg_flux *flux,
                                              const double *in_dev, double *out_dev, void *cuda_stream) {
    if (!mesh || !flux || !in_dev || !out_dev || in_dev == out_dev) return CRKDG_E_ARG;
    if (mesh->dim != 1 && mesh->dim != 2) return CRKDG_E_ARG;
    if (k < 1) return CRKDG_E_ARG;
    if (k > 3) return CRKDG_E_UNSUPPORTED;
    if (flux->kind < CRKDG_FLUX_ADVECTION || flux->kind > CRKDG_FLUX_EULER) return CRKDG_E_ARG;
    if (m != ncomp(flux->kind, mesh->dim)) return CRKDG_E_ARG;
    if (flux->kind == CRKDG_FLUX_EULER && !(flux->gamma > 1.0)) return CRKDG_E_ARG;
    int ny = mesh->dim == 2 ? mesh->ny : 1;
    if (mesh->nx < 1 || ny < 1) return CRKDG_E_ARG;
    if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0))) return CRKDG_E_ARG;
    for (int s = 0; s < 2 * mesh->dim; ++s)
        if (mesh->bc[s] < CRKDG_BC_PERIODIC || mesh->bc[s] > CRKDG_BC_DIRICHLET) return CRKDG_E_ARG;
    for (int d = 0; d < mesh->dim; ++d)
        if ((mesh->bc[2 * d] == CRKDG_BC_PERIODIC) != (mesh->bc[2 * d + 1] == CRKDG_BC_PERIODIC)) return CRKDG_E_ARG;
    int n = k + 1;
    int nn = mesh->dim == 2 ? n * n : n;
    int ntr = mesh->dim == 2 ? 4 * n : 2;
    double cells = (double)mesh->nx * ny;
    // scratch: the accumulated G (state size), one slot of face traces, the cell averages
    double need = cells * nn * m + cells * ntr * m + cells * m;
    if (need > (double)CRKDG_NOALLOC_SCRATCH_DOUBLES) return CRKDG_E_ARG;  // beyond the fixed scratch size
    int ncell = mesh->nx * ny;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CRKDG_E_CUDA;
    double *scratch = nullptr;
    crkdg_status s = setup(dev, mesh->dim, &scratch);
    if (s) return s;

    Params P;
    memset(&P, 0, sizeof(P));
    P.nx = mesh->nx;
    P.ny = ny;
    P.ncell = ncell;
    P.rhx = 2.0 * mesh->nx / (mesh->x1 - mesh->x0);
    P.rhy = mesh->dim == 2 ? 2.0 * ny / (mesh->y1 - mesh->y0) : 0.0;
    P.gamma = flux->gamma;
    P.velx = flux->velocity[0];
    P.vely = flux->velocity[1];
    for (int side = 0; side < 4; ++side) {
        P.bc[side] = (mesh->dim == 1 && side >= 2) ? BC_OUTFLOW : mesh->bc[side];
        for (int c = 0; c < MAXM; ++c) P.bcs[side][c] = mesh->bc_state[side][c];
    }
    for (int i = 0; i < MAXS; ++i) P.slot[i] = -1;
    P.s = 1;
    P.dt = 1.0;
    P.b[0] = 1.0;
    P.slot[0] = 0;
    P.nslot = 1;

    Bufs B;
    memset(&B, 0, sizeof(B));
    B.un = in_dev;
    B.ustar = scratch;                              // G(in), fully written by the inner kernel
    B.tr = scratch + (size_t)ncell * nn * m;        // traces of in, fully written before they are read
    B.tavg = B.tr + (size_t)ncell * ntr * m;        // cell averages of in, likewise
    B.unew = out_dev;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    int ncb = cells_per_block(mesh->dim, n);
    int nblocks = (ncell + ncb - 1) / ncb;
    auto go = [&](int kernel) {
        return mesh->dim == 1 ? crkdg_launch_1d(kernel, n, flux->kind, nblocks, st, P, B)
                              : crkdg_launch_2d(kernel, n, flux->kind, nblocks, st, P, B);
    };
    P.mode = MODE_OP_G;
    if (go(K_INNER) != cudaSuccess) return CRKDG_E_CUDA;
    P.mode = MODE_OP_F;
    if (go(K_FINAL) != cudaSuccess) return CRKDG_E_CUDA;
    return CRKDG_OK;
}
