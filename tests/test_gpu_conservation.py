"""Conservation drift reported by crkdg_step (crkdg_step_info.mass_drift) on the GPU.

The scheme is conservative (the cell-average update is the sum of the face fluxes, each
face flux formed identically by both of its cells; the limiters keep the averages), so on a
mesh whose sides let no mass through (periodic, reflective) the total sum_K |K| rho_K of a
step changes by round-off only.  With open sides the reported change is the net boundary
inflow of the step and must equal the change of crkdg_total_mass (a host sum in another
order) to round-off.
"""
import numpy as np
import pytest

from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _solver(dim, nx, k, bc, precision, flux="euler"):
    from paper_2412_16002_gb300.solver import Solver

    dom = (0.0, 1.0, 0.0, 1.0)
    return Solver(dim, nx, nx if dim == 2 else 1, k, dom, flux, bc=bc, precision=precision,
                  bounds=(-1.0, 2.0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dim,k,bc", [
    (2, 3, ("periodic",) * 4),
    (2, 2, ("reflect", "reflect", "periodic", "periodic")),
    (2, 2, ("reflect",) * 4),
    (1, 2, ("reflect", "reflect", "outflow", "outflow")),
])
def test_closed_domains_report_round_off_drift(precision, dim, k, bc):
    nx = 24 if dim == 2 else 96
    g = _solver(dim, nx, k, bc, precision)
    g.set_state(inputs.random_euler(dim, nx, nx if dim == 2 else 1, k, seed=11, osc=0.5))
    m0 = g.mass(0)
    tab = "rk4" if k == 3 else "heun3"
    for _ in range(20):
        info = g.step(g.max_dt(0.1), tab)
        assert abs(info["mass_drift"]) < 1e-13, info
    assert abs(g.mass(0) - m0) < 1e-13 * abs(m0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_open_domain_drift_equals_total_mass_change(precision):
    wl = inputs.riemann_quadrants(3, 32, 2)
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, precision=precision)
    g.set_state(wl.state)
    seen = 0.0
    for _ in range(15):
        before = g.mass(0)
        info = g.step(g.max_dt(wl.cfl), wl.tableau)
        after = g.mass(0)
        expect = (after - before) / abs(before)
        assert abs(info["mass_drift"] - expect) < 1e-13, (info["mass_drift"], expect)
        seen = max(seen, abs(info["mass_drift"]))
    assert seen > 1e-8  # outflow sides do let mass through


def test_steps_without_info_then_with_info_stay_consistent():
    """A step taken through crkdg_advance (which keeps no totals on 1D meshes) is followed by
    a crkdg_step whose drift is measured against the state it actually started from."""
    wl = inputs.euler_blast_tube(256, 2)
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl)
    g.set_state(wl.state)
    t, done, _ = g.advance(10, wl.cfl, 1e30, wl.tableau)
    assert done == 10
    before = g.mass(0)
    info = g.step(g.max_dt(wl.cfl), wl.tableau)
    after = g.mass(0)
    assert abs(info["mass_drift"] - (after - before) / abs(before)) < 1e-13
