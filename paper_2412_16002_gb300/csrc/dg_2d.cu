// dg_2d.cu -- 2D instantiations of the FP64 cRKDG kernels (see dg_core.cuh).
#include "dg_core.cuh"
#include "dg_mixed.cuh"
#include "dg_tc.cuh"

using namespace crkdg;

cudaError_t crkdg_upload_tables_2d(const NodalTables *t) {
    return cudaMemcpyToSymbol(c_tab, t, sizeof(NodalTables) * 3);
}

cudaError_t crkdg_launch_2d(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                            const Bufs &B) {
    return launch_dim<2>(kernel, n, phys, nblocks, st, P, B);
}

cudaError_t crkdg_launch_mx_2d(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                               const MixBufs &X) {
    return launch_dim_x<2>(kernel, n, phys, nblocks, st, P, X);
}

cudaError_t crkdg_launch_inner_tc(cudaStream_t st, const Params &P, const MixBufs &X) {
    return launch_inner_tc(st, P, X);
}
