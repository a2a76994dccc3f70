"""The kernels' double reciprocal (Newton-Raphson from the hardware's approximate
reciprocal, dg_core.cuh: recip_nr) against CUDA's IEEE quotient 1.0/x: within one ulp
on random arguments over the whole normal range, both signs, and exact at the edges
the fallback covers (zero, subnormal, huge, inf, NaN take the IEEE division)."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include "dg_core.cuh"
#include <cstdio>
#include <cstdlib>
__global__ void k(const double *x, double *a, double *b, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i] = crkdg::recip_nr(x[i]); b[i] = 1.0 / x[i]; }
}
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int n = atoi(argv[3]);
    double *hx = (double *)malloc(n * 8), *ha = (double *)malloc(n * 8), *hb = (double *)malloc(n * 8);
    if (fread(hx, 8, n, f) != (size_t)n) return 2;
    fclose(f);
    double *x, *a, *b;
    cudaMalloc(&x, n * 8); cudaMalloc(&a, n * 8); cudaMalloc(&b, n * 8);
    cudaMemcpy(x, hx, n * 8, cudaMemcpyHostToDevice);
    k<<<(n + 255) / 256, 256>>>(x, a, b, n);
    cudaMemcpy(ha, a, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(hb, b, n * 8, cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) return 3;
    f = fopen(argv[2], "wb");
    fwrite(ha, 8, n, f); fwrite(hb, 8, n, f);
    fclose(f);
    return 0;
}
"""


def test_recip_nr_within_one_ulp_of_the_quotient():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(5)
    n = 1 << 20
    mant = 1.0 + rng.random(n)
    expo = rng.integers(-1020, 1021, n)
    x = np.ldexp(mant, expo) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    edges = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2e-308, 1.0, -1.0, 2.0 ** -1000, 2.0 ** 1000, 2.0 ** -1001,
                      2.0 ** 1001, 1.7e308, np.inf, -np.inf, np.nan, 1e-13, 3.0])
    x = np.concatenate([edges, x])
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cu")
        open(src, "w").write(SRC)
        exe = os.path.join(d, "t")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I",
                        os.path.join(ROOT, "paper_2412_16002_gb300", "csrc"), src, "-o", exe], check=True)
        xin, out = os.path.join(d, "x.bin"), os.path.join(d, "o.bin")
        x.tofile(xin)
        subprocess.run([exe, xin, out, str(x.size)], check=True)
        r = np.fromfile(out, dtype=np.float64)
    a, b = r[: x.size], r[x.size:]
    ne = len(edges)
    # the fallback range: bit-identical to the quotient (NaN stays NaN)
    fa, fb = a[:ne], b[:ne]
    out_of_range = (np.abs(x[:ne]) < 2.0 ** -1000 + 0) | (np.abs(x[:ne]) >= 2.0 ** 1001) | ~np.isfinite(x[:ne])
    assert np.array_equal(fa[out_of_range], fb[out_of_range], equal_nan=True)
    ia, ib = a[ne:].view(np.int64), b[ne:].view(np.int64)
    ulp = np.abs(ia - ib)
    print(f"recip_nr against 1.0/x: {np.count_nonzero(ulp)} of {ulp.size} differ, max {ulp.max()} ulp")
    assert ulp.max() <= 1
    assert np.array_equal(a[ne:] > 0, x[ne:] > 0)
