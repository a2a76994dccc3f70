// dg_1d.cu -- 1D instantiations of the FP64 cRKDG kernels (see dg_core.cuh).
#include "dg_core.cuh"

using namespace crkdg;

cudaError_t crkdg_upload_tables_1d(const NodalTables *t) {
    return cudaMemcpyToSymbol(c_tab, t, sizeof(NodalTables) * 3);
}

cudaError_t crkdg_launch_1d(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                            const Bufs &B) {
    return launch_dim<1>(kernel, n, phys, nblocks, st, P, B);
}
