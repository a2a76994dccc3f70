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
        // The handle path's own table builder: the upload rewrites the constant tables
        // that every handle on this device reads with the same bytes, so a handle
        // created earlier keeps computing with complete, identical tables.
        NodalTables tab[3];
        crkdg_build_tables(tab);
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
