// dg_ens.cu -- persistent ensemble kernels for 2D Euler (Q^2 and Q^3), see dg_ensemble.cuh.
#include "dg_ensemble.cuh"

using namespace crkdg;

cudaError_t crkdg_upload_tables_ens(const NodalTables *t) {
    return cudaMemcpyToSymbol(c_tab, t, sizeof(NodalTables) * 3);
}

cudaError_t crkdg_ens_launch(int kind, int n, int grid, cudaStream_t st, EnsProblem *E, const EnsItem *items,
                             int nitems, EnsCtl *ctl, int counter, int stage) {
#define CRKDG_ENS_CASE(NV, KV) \
    if (n == NV && kind == KV) return ens_launch_one<NV, KV>(grid, st, E, items, nitems, ctl, counter, stage);
    CRKDG_ENS_CASE(3, ENS_INNER) CRKDG_ENS_CASE(3, ENS_FINAL) CRKDG_ENS_CASE(3, ENS_TROUBLE)
    CRKDG_ENS_CASE(3, ENS_FEATURES) CRKDG_ENS_CASE(4, ENS_INNER) CRKDG_ENS_CASE(4, ENS_FINAL)
    CRKDG_ENS_CASE(4, ENS_TROUBLE) CRKDG_ENS_CASE(4, ENS_FEATURES)
#undef CRKDG_ENS_CASE
    return cudaErrorInvalidValue;
}

int crkdg_ens_occupancy(int kind, int n) {
#define CRKDG_ENS_OCC(NV, KV) \
    if (n == NV && kind == KV) return ens_occupancy<NV, KV>();
    CRKDG_ENS_OCC(3, ENS_INNER) CRKDG_ENS_OCC(3, ENS_FINAL) CRKDG_ENS_OCC(3, ENS_TROUBLE)
    CRKDG_ENS_OCC(3, ENS_FEATURES) CRKDG_ENS_OCC(4, ENS_INNER) CRKDG_ENS_OCC(4, ENS_FINAL)
    CRKDG_ENS_OCC(4, ENS_TROUBLE) CRKDG_ENS_OCC(4, ENS_FEATURES)
#undef CRKDG_ENS_OCC
    return 0;
}

int crkdg_ens_cells_per_block(int kind, int n) {
    if (kind == ENS_FEATURES) return 128;
    return n == 3 ? Cfg<2, 3, PH_EULER>::NCB : Cfg<2, 4, PH_EULER>::NCB;
}

cudaError_t crkdg_ens_control(int which, cudaStream_t st, EnsProblem *E, int np, EnsCtl *ctl, int arg) {
    switch (which) {
    case 0: k_ens_begin<<<1, 256, 0, st>>>(E, np, ctl, arg); break;
    case 1: k_ens_reset<<<1, 32, 0, st>>>(ctl); break;
    case 2: k_ens_end<<<1, 256, 0, st>>>(E, np, ctl, arg); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
