"""The allocation-free DG operator entry point against the handle-based one.

crkdg_apply_F_noalloc serves callers that cannot allocate device memory (for
example code that runs inside a CUDA graph capture or inside another
framework's memory pool): it takes their input and output buffers and keeps its
scratch in a fixed device array.  It must give the same F(u) as
crkdg_apply_operator(CRKDG_OP_F) on two calls in a row, whether it runs first
in a fresh process or after every other test, and its one-time set-up must
leave the constant tables of handles that already exist on the device as they
were (their troubled-cell decisions read tables the operator itself does not
use).  The file sorts last so that a run stopping at its first failure has run
every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import ORACLE_TABS, rel_linf
from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCRATCH = 1 << 22  # CRKDG_NOALLOC_SCRATCH_DOUBLES


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300 import build

    build()
    lib = L.load()
    return lib


def _mesh(L, dim, nx, ny, bc, st, dom=(0.0, 1.0, 0.0, 2.0)):
    mesh = L.Mesh()
    mesh.dim, mesh.nx, mesh.ny = dim, nx, ny
    mesh.x0, mesh.x1, mesh.y0, mesh.y1 = dom
    for s in range(4):
        mesh.bc[s] = L.BC[bc[s]]
        for c in range(4):
            mesh.bc_state[s][c] = st[c]
    return mesh


def _noalloc(lib, L, mesh, k, m, fl, x):
    out = torch.full_like(x, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.crkdg_apply_F_noalloc(C.byref(mesh), k, m, C.byref(fl), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    return rc, out


def _euler_state(dim):
    return [1.1, 0.2, -0.1, 2.3] if dim == 2 else [1.1, 0.2, 2.3, 0.0]


@pytest.mark.parametrize("dim,nx,ny,k,bc", [
    (1, 37, 1, 2, ("dirichlet", "outflow", "outflow", "outflow")),
    (1, 29, 1, 1, ("reflect", "dirichlet", "outflow", "outflow")),
    (2, 19, 13, 3, ("reflect", "outflow", "periodic", "periodic")),
    (2, 24, 24, 2, ("outflow",) * 4),
    (2, 17, 11, 1, ("dirichlet", "reflect", "outflow", "dirichlet")),
])
def test_noalloc_F_matches_handle_path_twice(lib, dim, nx, ny, k, bc):
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    st = _euler_state(dim)
    g = Solver(dim, nx, ny, k, (0.0, 1.0, 0.0, 2.0), "euler", bc=bc,
               bc_state={s: st[: dim + 2] for s in range(4)})
    U = inputs.random_euler(dim, nx, ny, k, seed=17, osc=0.4)
    x = torch.from_numpy(U).cuda()
    ref = torch.empty_like(x)
    g.apply("F", x, ref)
    mesh = _mesh(L, dim, nx, ny, bc, st)
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    for call in range(2):
        rc, out = _noalloc(lib, L, mesh, k, dim + 2, fl, x)
        assert rc == L.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_linf(got, ref.cpu().numpy(), dim + 2) < 1e-12, call


@pytest.mark.parametrize("flux,dim,nx,ny,k,vel,bc", [
    ("advection", 1, 41, 1, 1, (-0.7, 0.0), ("periodic",) * 4),
    ("advection", 2, 15, 21, 3, (0.6, -1.3), ("periodic", "periodic", "outflow", "dirichlet")),
    ("advection", 2, 12, 9, 1, (-0.4, 0.9), ("dirichlet", "outflow", "periodic", "periodic")),
    ("burgers", 1, 33, 1, 2, (1.0, 0.0), ("periodic",) * 4),
    ("burgers", 2, 14, 18, 2, (1.0, 0.0), ("outflow", "dirichlet", "periodic", "periodic")),
    ("burgers", 2, 10, 10, 1, (1.0, 0.0), ("periodic",) * 4),
])
def test_noalloc_F_scalar_laws_match_handle_path(lib, flux, dim, nx, ny, k, vel, bc):
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    st = [0.3, 0.0, 0.0, 0.0]
    g = Solver(dim, nx, ny, k, (0.0, 1.0, 0.0, 2.0), flux, velocity=vel, bounds=(-2.0, 2.0), bc=bc,
               bc_state={s: st[:1] for s in range(4)})
    U = inputs.random_scalar(dim, nx, ny, k, seed=23, lo=-1.0, hi=1.0)
    x = torch.from_numpy(U).cuda()
    ref = torch.empty_like(x)
    g.apply("F", x, ref)
    mesh = _mesh(L, dim, nx, ny, bc, st)
    fl = L.Flux(L.FLUX[flux], 1.4, (C.c_double * 2)(*vel))
    for call in range(2):
        rc, out = _noalloc(lib, L, mesh, k, 1, fl, x)
        assert rc == L.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_linf(got, ref.cpu().numpy(), 1) < 1e-12, call


def test_noalloc_leaves_live_handles_tables_intact(lib):
    """A TVB-indicator handle created before the entry point's first call keeps taking the
    oracle's troubled-cell decisions after it (the face-average and moment weights those
    decisions use live in the same constant tables the set-up writes)."""
    from oracle import Oracle
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.riemann_quadrants(4, 32, 2)
    g = Solver.from_workload(wl, indicator="tvb", tvb_M=1.0)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, eps=wl.eps, bc=wl.bc,
               bc_state=wl.bc_state, indicator=True, tvb_M=1.0)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t = 0.0
    total = 0
    for step in range(3):
        if step == 1:
            # a different mesh and degree, so that every n's tables are uploaded again
            st = _euler_state(2)
            mesh = _mesh(L, 2, 9, 7, ("outflow",) * 4, st)
            fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
            x = torch.from_numpy(inputs.random_euler(2, 9, 7, 3, seed=5, osc=0.3)).cuda()
            rc, _ = _noalloc(lib, L, mesh, 3, 4, fl, x)
            assert rc == L.OK
            torch.cuda.synchronize()
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        before = o.c.copy()
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"] == 0
        rc2, us, uts = o.step_stages(dt, ORACLE_TABS[wl.tableau], t, modal=before)
        flags_o = o.troubled(us[-1])
        flags_g = g.troubled_flags()
        assert np.array_equal(flags_g, flags_o), (step, np.nonzero(flags_g != flags_o))
        total += int(flags_g.sum())
        assert rel_linf(g.get_state(), o.get_state(), o.m) < 1e-10, step
        t += dt
    assert total > 0


def test_noalloc_rejects_meshes_beyond_the_scratch(lib):
    from paper_2412_16002_gb300 import _lib as L

    mesh = _mesh(L, 2, 4096, 4096, ("outflow",) * 4, [1.0, 0.0, 0.0, 2.5])
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.crkdg_apply_F_noalloc(C.byref(mesh), 3, 4, C.byref(fl), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(y.data_ptr()), None)
    assert rc == L.E_ARG


def test_noalloc_scratch_limit_is_exact(lib):
    """2D Euler Q^3 needs 4 * (16 + 16 + 1) doubles per cell: 31775 cells fit, 31776 do not."""
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    per_cell = 4 * (16 + 16 + 1)
    assert 31775 * per_cell <= SCRATCH < 31776 * per_cell
    st = _euler_state(2)
    bc = ("outflow",) * 4
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    # 775 x 41 = 31775 cells: accepted, and equal to the handle path
    U = inputs.random_euler(2, 775, 41, 3, seed=3, osc=0.2)
    x = torch.from_numpy(U).cuda()
    mesh = _mesh(L, 2, 775, 41, bc, st)
    rc, out = _noalloc(lib, L, mesh, 3, 4, fl, x)
    assert rc == L.OK
    g = Solver(2, 775, 41, 3, (0.0, 1.0, 0.0, 2.0), "euler", bc=bc, bc_state={s: st for s in range(4)})
    ref = torch.empty_like(x)
    g.apply("F", x, ref)
    torch.cuda.synchronize()
    assert rel_linf(out.cpu().numpy(), ref.cpu().numpy(), 4) < 1e-12
    # 96 x 331 = 31776 cells: one cell beyond the scratch
    mesh = _mesh(L, 2, 96, 331, bc, st)
    y = torch.zeros(96 * 331 * 64, dtype=torch.float64, device="cuda")
    rc = lib.crkdg_apply_F_noalloc(C.byref(mesh), 3, 4, C.byref(fl), C.c_void_p(y.data_ptr()),
                                   C.c_void_p(x.data_ptr()), None)
    assert rc == L.E_ARG
