// dg_1d.cu -- 1D instantiations of the FP64 cRKDG kernels (see dg_core.cuh).
#include "dg_core.cuh"
#include "dg_mixed.cuh"
#include "dg_run1d.cuh"

using namespace crkdg;

cudaError_t crkdg_upload_tables_1d(const NodalTables *t) {
    return cudaMemcpyToSymbol(c_tab, t, sizeof(NodalTables) * 3);
}

cudaError_t crkdg_launch_1d(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                            const Bufs &B) {
    return launch_dim<1>(kernel, n, phys, nblocks, st, P, B);
}

cudaError_t crkdg_run_1d(int n, int phys, cudaStream_t st, const Params &P, double *u0, double *u1, RunCtl *ctl,
                         int chunk, int *nblocks) {
#define CRKDG_RUN(NV, PV) \
    if (n == NV && phys == PV) return run1d_launch<NV, PV>(st, P, u0, u1, ctl, chunk, nblocks);
    CRKDG_RUN(2, PH_ADV) CRKDG_RUN(2, PH_BURG) CRKDG_RUN(2, PH_EULER)
    CRKDG_RUN(3, PH_ADV) CRKDG_RUN(3, PH_BURG) CRKDG_RUN(3, PH_EULER)
    CRKDG_RUN(4, PH_ADV) CRKDG_RUN(4, PH_BURG) CRKDG_RUN(4, PH_EULER)
#undef CRKDG_RUN
    return cudaErrorInvalidValue;
}

cudaError_t crkdg_launch_mx_1d(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                               const MixBufs &X) {
    return launch_dim_x<1>(kernel, n, phys, nblocks, st, P, X);
}
