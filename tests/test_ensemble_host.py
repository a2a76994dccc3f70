"""Host-side logic of the ensemble path (no GPU): the work-item plan covers every block of
every problem exactly once, largest problems first, within each problem's tile; argument
checks run before any device call; the device-side initial state equals the host one."""
import ctypes as C

import numpy as np
import pytest

from paper_2412_16002_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300 import build

    build()
    L._lib = None
    return L.load()


def test_plan_covers_every_block_once(lib):
    from paper_2412_16002_gb300.ensemble import plan

    rng = np.random.default_rng(5)
    ncells = [int(x) for x in rng.integers(1, 5000, size=9)] + [0, 128]
    tiles = [int(x) for x in rng.choice([1, 2, 4, 8, 16], size=len(ncells))]
    cpb = 32
    items = plan(ncells, tiles, cpb)
    seen = {i: np.zeros((nc + cpb - 1) // cpb, dtype=int) for i, nc in enumerate(ncells)}
    order = []
    for p, b0, nb in items:
        assert 1 <= nb <= tiles[p]
        seen[p][b0:b0 + nb] += 1
        if not order or order[-1] != p:
            order.append(p)
    for i, cnt in seen.items():
        assert np.all(cnt == 1), i
    # problem-major, largest first (ties keep the input order)
    assert len(order) == len(set(order))
    sizes = [ncells[p] for p in order]
    assert sizes == sorted(sizes, reverse=True)
    assert len(items) == sum(-(-((nc + cpb - 1) // cpb) // t) for nc, t in zip(ncells, tiles))


def test_plan_rejects_bad_arguments(lib):
    nc = (C.c_longlong * 2)(10, 20)
    tl = (C.c_int * 2)(1, 0)
    assert lib.crkdg_ensemble_plan(2, nc, tl, 32, None, 0) == -1
    tl = (C.c_int * 2)(1, 1)
    assert lib.crkdg_ensemble_plan(2, nc, tl, 0, None, 0) == -1
    assert lib.crkdg_ensemble_plan(-1, nc, tl, 32, None, 0) == -1
    assert lib.crkdg_ensemble_plan(0, None, None, 32, None, 0) == 0


def test_ensemble_create_argument_checks(lib):
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import _Tab

    tab = _Tab("heun3")
    arr = (L.EnsProblem * 2)()
    for q in arr:
        q.mesh.dim, q.mesh.nx, q.mesh.ny = 2, 8, 8
        q.mesh.x0, q.mesh.x1, q.mesh.y0, q.mesh.y1 = 0.0, 1.0, 0.0, 1.0
        for s in range(4):
            q.mesh.bc[s] = L.BC["outflow"]
        q.k, q.tableau, q.cfl, q.t_end = 2, C.pointer(tab.c), 0.1, 1.0
    fl = L.Flux(L.FLUX["euler"], 1.4, (C.c_double * 2)(0.0, 0.0))
    bd = L.Bounds(0.0, 1.0, 1e-13)
    e = C.c_void_p()

    def create(m=4, flux=fl, opt=None):
        return lib.crkdg_ensemble_create(2, arr, m, C.byref(flux), C.byref(bd), opt, C.byref(e))

    assert create(m=3) == L.E_ARG
    assert create(flux=L.Flux(L.FLUX["burgers"], 1.4, (C.c_double * 2)(0.0, 0.0))) == L.E_ARG
    opt = L.Options()
    lib.crkdg_options_default(C.byref(opt))
    opt.precision = L.PREC["mixed"]
    assert create(opt=C.byref(opt)) == L.E_UNSUPPORTED
    arr[1].k = 1
    assert create() == L.E_UNSUPPORTED
    arr[1].k = 2
    arr[1].mesh.dim = 1
    assert create() == L.E_ARG
    arr[1].mesh.dim = 2
    arr[1].mesh.bc[0] = L.BC["periodic"]
    assert create() == L.E_ARG
    arr[1].mesh.bc[0] = L.BC["outflow"]
    arr[0].cfl = 0.0
    assert create() == L.E_ARG
    assert not e.value
    assert lib.crkdg_ensemble_destroy(None) == L.OK
    assert lib.crkdg_ensemble_state_size(None, 0) == 0


@pytest.mark.parametrize("seed,n,k", [(3, 16, 2), (7, 24, 3)])
def test_device_initial_state_equals_host(seed, n, k):
    a = inputs.riemann_quadrants(seed, n, k).state
    b = inputs.riemann_quadrants_device(seed, n, k, device="cpu").numpy()
    assert np.array_equal(a, b)


def test_ensemble_specs_are_seeded():
    from paper_2412_16002_gb300.ensemble import riemann_ensemble_specs

    a = riemann_ensemble_specs(64, seed=0)
    assert a == riemann_ensemble_specs(64, seed=0)
    assert {k for _, _, k in a} == {2, 3}
    assert all(256 <= n <= 1536 and n % 128 == 0 for _, n, _ in a)
