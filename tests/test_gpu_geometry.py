"""Non-rectangular domains on the GPU (Examples 4.8 and 4.9) against the CPU oracle.

The shock diffraction and the double Mach reflection run on the bounding rectangle with the
solid cells masked, walls on the sides facing them, an inflow side, a fixed state on part of
a wall and the exact moving shock on a side.  Through the C ABI: the operator F at a stage
time (rel L-inf 1e-12, or the oracle's own rounding envelope where larger), steps of both benchmarks (rel L-inf
1e-10, identical restarts, bounds exact at every step), solid cells untouched, and the
argument checks of crkdg_set_geometry.
"""
import numpy as np
import pytest

from gpu_helpers import ORACLE_TABS, pair, rel_linf
from paper_2412_16002_gb300 import inputs
from paper_2412_16002_gb300.inputs import GEO_SOLID, GEO_WALL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _workload(example, k):
    if example == "diffraction":
        return inputs.shock_diffraction(cells_per_unit=2, k=k)
    return inputs.double_mach(cells_per_unit=6, k=k)


def _pair(wl):
    g, o = pair(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, eps=wl.eps, bc=wl.bc,
                bc_state=wl.bc_state)
    g.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
    o.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
    return g, o


@pytest.mark.parametrize("example", ["diffraction", "double_mach"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_geometry_operator_F(example, k):
    """F on a seeded oscillating state: walls, fixed states, inflow, outflow and (double Mach)
    the shock line at t = 0.05, where it has left its initial cell on the top side.

    Held to 1e-12 relative, or to 10 times the oracle's own response to a one-ulp relative
    perturbation of its input where that is larger: on the 26 x 24 diffraction mesh the
    seeded state has near-vacuum points whose Lax-Friedrichs viscosity amplifies rounding
    (the oracle against itself: 2.5e-12 for Q^2, 1.4e-12 for Q^3)."""
    wl = _workload(example, k)
    g, o = _pair(wl)
    U = inputs.random_euler(2, wl.nx, wl.ny, k, seed=90 + k, osc=0.3)
    t = 0.05
    g.set_time(t)
    x = torch.from_numpy(U).cuda()
    out = torch.empty_like(x)
    g.apply("F", x, out)
    ref = o.to_nodal(o.apply("F", o.to_modal(U), t=t))
    rng = np.random.default_rng(5)
    envelope = max(rel_linf(o.to_nodal(o.apply("F", o.to_modal(U * (1.0 + 2.2e-16 * rng.standard_normal(U.shape))),
                                               t=t)), ref, 4) for _ in range(3))
    got = out.cpu().numpy()
    assert rel_linf(got, ref, 4) < max(1e-12, 10.0 * envelope)
    solid = ((wl.geo & GEO_SOLID) != 0).reshape(wl.ny, wl.nx)
    assert not got.reshape(4, wl.ny, wl.nx, -1)[:, solid].any()  # no operator outside the domain


@pytest.mark.parametrize("example,k,tab", [("diffraction", 2, "heun3"), ("diffraction", 3, "rk4"),
                                           ("double_mach", 1, "midpoint2"), ("double_mach", 2, "heun3")])
def test_geometry_steps(example, k, tab):
    """Steps of each benchmark from its initial data: the shock runs into the corner region,
    the scaling limiter works at every stage, and both sides restart alike."""
    wl = _workload(example, k)
    g, o = _pair(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    s0 = g.get_state().copy()
    assert rel_linf(s0, o.get_state(), 4) < 1e-12
    t = 0.0
    for _ in range(25):
        dt = o.max_dt(wl.cfl)
        assert abs(g.max_dt(wl.cfl) - dt) <= 1e-10 * dt
        ig = g.step(dt, tab)
        rc, io = o.step(dt, ORACLE_TABS[tab], t)
        assert rc == 0 and ig["restarts"] == io["restarts"]
        m = g.margins()
        assert m[0] >= 0.0 and m[1] >= 0.0, m
        t += io["dt_taken"]
    assert rel_linf(g.get_state(), o.get_state(), 4) < 1e-10
    solid = ((wl.geo & GEO_SOLID) != 0).reshape(wl.ny, wl.nx)
    s1 = g.get_state()
    assert np.array_equal(s1.reshape(4, wl.ny, wl.nx, -1)[:, solid], s0.reshape(4, wl.ny, wl.nx, -1)[:, solid])
    assert g.mass(0) == pytest.approx(o.total_mass(0), rel=1e-12)
    assert g.time() == pytest.approx(t, rel=1e-15)


def test_geometry_arguments():
    """crkdg_set_geometry: an open side facing a solid cell and unknown kinds are refused with
    CRKDG_E_ARG (geometry unchanged); the split-precision path is refused as unsupported."""
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    g = Solver(2, 4, 4, 1, (0.0, 1.0, 0.0, 1.0), "euler", bc=("outflow",) * 4)
    geo = np.zeros((4, 4), dtype=np.uint32)
    geo[0, 0] = GEO_SOLID
    with pytest.raises(L.CrkdgError) as e:
        g.set_geometry(geo)
    assert e.value.status == L.E_ARG
    geo[0, 1] = GEO_WALL
    geo[1, 0] = GEO_WALL << 8
    g.set_geometry(geo)
    bad = geo.copy()
    bad[2, 2] = 9
    with pytest.raises(L.CrkdgError):
        g.set_geometry(bad)
    g.set_geometry(None)
    x = Solver(2, 4, 4, 2, (0.0, 1.0, 0.0, 1.0), "euler", bc=("outflow",) * 4, precision="mixed")
    with pytest.raises(L.CrkdgError) as e:
        x.set_geometry(geo)
    assert e.value.status == L.E_UNSUPPORTED
