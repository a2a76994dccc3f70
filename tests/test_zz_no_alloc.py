"""The allocation-free DG operator entry point against the handle-based one.

crkdg_apply_F_noalloc serves callers that cannot allocate device memory (for
example code that runs inside a CUDA graph capture or inside another
framework's memory pool): it takes their input and output buffers and keeps its
scratch in a fixed device array.  It must give the same F(u) as
crkdg_apply_operator(CRKDG_OP_F) on two calls in a row, whether it runs first
in a fresh process or after every other test.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import rel_linf
from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300 import build

    build()
    lib = L.load()
    return lib


def _mesh(L, dim, nx, ny, bc, st):
    mesh = L.Mesh()
    mesh.dim, mesh.nx, mesh.ny = dim, nx, ny
    mesh.x0, mesh.x1, mesh.y0, mesh.y1 = 0.0, 1.0, 0.0, 2.0
    for s in range(4):
        mesh.bc[s] = L.BC[bc[s]]
        for c in range(4):
            mesh.bc_state[s][c] = st[c]
    return mesh


@pytest.mark.parametrize("dim,nx,ny,k,bc", [
    (1, 37, 1, 2, ("dirichlet", "outflow", "outflow", "outflow")),
    (2, 19, 13, 3, ("reflect", "outflow", "periodic", "periodic")),
    (2, 24, 24, 2, ("outflow",) * 4),
])
def test_noalloc_F_matches_handle_path_twice(lib, dim, nx, ny, k, bc):
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    st = [1.1, 0.2, -0.1, 2.3] if dim == 2 else [1.1, 0.2, 2.3, 0.0]
    g = Solver(dim, nx, ny, k, (0.0, 1.0, 0.0, 2.0), "euler", bc=bc,
               bc_state={s: st[: dim + 2] for s in range(4)})
    U = inputs.random_euler(dim, nx, ny, k, seed=17, osc=0.4)
    x = torch.from_numpy(U).cuda()
    ref = torch.empty_like(x)
    g.apply("F", x, ref)
    mesh = _mesh(L, dim, nx, ny, bc, st)
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(x, float("nan"))
        rc = lib.crkdg_apply_F_noalloc(C.byref(mesh), k, dim + 2, C.byref(fl), C.c_void_p(x.data_ptr()),
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == L.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_linf(got, ref.cpu().numpy(), dim + 2) < 1e-12, call


def test_noalloc_rejects_meshes_beyond_the_scratch(lib):
    from paper_2412_16002_gb300 import _lib as L

    mesh = _mesh(L, 2, 4096, 4096, ("outflow",) * 4, [1.0, 0.0, 0.0, 2.5])
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.crkdg_apply_F_noalloc(C.byref(mesh), 3, 4, C.byref(fl), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(y.data_ptr()), None)
    assert rc == L.E_ARG
