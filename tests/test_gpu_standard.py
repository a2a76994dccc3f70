"""The standard RKDG (eq. rkdg: F, with its neighbour exchange, in every stage; the same scaling
limiter and restart rule) on the GPU against the oracle's standard scheme, and against the
compact scheme it is compared with."""
import numpy as np
import pytest

from gpu_helpers import ORACLE_TABS, rel_linf
from oracle import Oracle
from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _pair(wl, **kw):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, scheme="standard", **kw)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
               bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state, scheme="standard")
    return g, o


def _random(dim, k, bc, seed):
    nx, ny = (13, 1) if dim == 1 else (11, 9)
    return inputs.Workload("rnd", dim, nx, ny, k, (0.0, 1.0, 0.0, 1.0), "euler", bc,
                           inputs.random_euler(dim, nx, ny, k, seed=seed, osc=0.8), cfl=0.1,
                           bc_state={s: ([1.1, 0.2, -0.1, 2.3] if dim == 2 else [1.1, 0.2, 2.3]) for s in range(4)})


@pytest.mark.parametrize("tab", ["midpoint2", "heun3", "rk4"])
@pytest.mark.parametrize("dim,k,bc", [(1, 2, ("dirichlet", "outflow", "outflow", "outflow")),
                                      (2, 3, ("reflect", "outflow", "periodic", "periodic")),
                                      (2, 1, ("outflow",) * 4)])
def test_standard_steps_match_oracle(tab, dim, k, bc):
    wl = _random(dim, k, bc, seed=21)
    g, o = _pair(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t = 0.0
    for _ in range(5):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, tab)
        rc, io = o.step(dt, ORACLE_TABS[tab], t)
        assert rc == 0 and ig["restarts"] == io["restarts"]
        t += io["dt_taken"]
        assert g.margins().min() >= 0.0
    assert rel_linf(g.get_state(), o.get_state(), o.m) < 1e-11


def test_standard_smooth_100_steps_and_conservation():
    wl = inputs.scenario2(12, 2)
    g, o = _pair(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    m0 = g.mass(0)
    t = 0.0
    for _ in range(100):
        dt = o.max_dt(wl.cfl)
        info = g.step(dt, wl.tableau)
        rc, _ = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0
        assert abs(info["mass_drift"]) < 1e-13
        t += dt
    assert rel_linf(g.get_state(), o.get_state(), 4) < 1e-10
    assert abs(g.mass(0) - m0) <= 1e-13 * abs(m0)


def test_standard_blast_restarts_match_oracle():
    """Sedov-type blast at CFL 0.9: the standard scheme's stage averages leave the set and the
    step is halved exactly when the oracle halves it; bounds hold after every step."""
    wl = inputs.sedov(16, 3)
    wl.cfl = 0.9
    g, o = _pair(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t, total = 0.0, 0
    for _ in range(10):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"]
        total += io["restarts"]
        t += io["dt_taken"]
        assert g.margins().min() >= 0.0
    assert total > 0
    assert rel_linf(g.get_state(), o.get_state(), 4) < 1e-9


def test_standard_differs_from_compact_and_rejects_unsupported():
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.riemann_quadrants(4, 20, 2)
    a = Solver.from_workload(wl, scheme="standard")
    b = Solver.from_workload(wl)
    a.set_state(wl.state)
    b.set_state(wl.state)
    dt = b.max_dt(wl.cfl)
    a.step(dt, wl.tableau)
    b.step(dt, wl.tableau)
    d = np.abs(a.get_state() - b.get_state()).max()
    assert d > 1e-8  # the schemes differ (G against F in the inner stages)
    for kw in (dict(precision="mixed"), dict(indicator="tvb")):
        with pytest.raises(L.CrkdgError) as e:
            Solver.from_workload(wl, scheme="standard", **kw)
        assert e.value.status == L.E_UNSUPPORTED
