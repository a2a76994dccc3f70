"""Plain troubled-cell indicator + shock limiter on the GPU against the oracle: the flags are
integer decisions taken in FP64 on both sides and must agree exactly; the limited states to
1e-10; averages are kept and the scaling limiter still leaves every S_K point in bounds."""
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


def _pair(wl, M):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, indicator="tvb", tvb_M=M)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, eps=wl.eps, bc=wl.bc,
               bc_state=wl.bc_state, indicator=True, tvb_M=M)
    return g, o


@pytest.mark.parametrize("name,M", [("riemann32_q2", 1.0), ("riemann24_q3", 10.0), ("blast1d_256_p2", 1.0)])
def test_indicator_steps_match_oracle(name, M):
    if name == "riemann32_q2":
        wl = inputs.riemann_quadrants(4, 32, 2)
    elif name == "riemann24_q3":
        wl = inputs.riemann_quadrants(5, 24, 3)
    else:
        wl = inputs.euler_blast_tube(256, 2)
    g, o = _pair(wl, M)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t = 0.0
    total = 0
    for step in range(5):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        before = o.c.copy()
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"] == 0
        # the oracle's flags of this step: recompute them from its unlimited final stage
        rc2, us, uts = o.step_stages(dt, ORACLE_TABS[wl.tableau], t, modal=before)
        flags_o = o.troubled(us[-1])
        flags_g = g.troubled_flags()
        assert np.array_equal(flags_g, flags_o), (step, np.nonzero(flags_g != flags_o))
        total += int(flags_g.sum())
        assert ig["troubled"] == int(flags_g.sum())
        assert rel_linf(g.get_state(), o.get_state(), o.m) < 1e-10
        assert g.margins().min() >= 0.0
        t += dt
    assert total > 0, "the case must flag cells"
