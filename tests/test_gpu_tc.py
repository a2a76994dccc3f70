"""Split precision's inner stages on the tensor cores (tcgen05.mma kind::tf32 with the
three-product split; 2D Euler, Q^3) against the same stages on the CUDA cores and against
the FP64 oracle.

The two kernels evaluate the same maps in FP32-level arithmetic with different rounding
(tensor-core products of TF32 halves against fused multiply-adds), so states agree to a few
units of FP32 rounding of the largest values: 2e-5 relative L-inf after one step, the bound
the split path's operators are held to.  What FP64 keeps must agree exactly in kind: bounds
at every S_K point, conservation to FP64 round-off, and the restart decisions."""
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


def _solver(wl, tc=True):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, precision="mixed")
    g.set_tensor_cores(tc)
    return g


def _oracle(wl):
    return Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
                  bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state)


def _rel_l1(a, b, m):
    a, b = np.asarray(a).reshape(m, -1), np.asarray(b).reshape(m, -1)
    return max(np.abs(a[c] - b[c]).sum() / max(np.abs(b[c]).sum(), 1e-300) for c in range(m))


def _random(nx, ny, seed, osc):
    return inputs.Workload("rnd", 2, nx, ny, 3, (0.0, 1.0, 0.0, 1.0), "euler", ("periodic",) * 4,
                           inputs.random_euler(2, nx, ny, 3, seed=seed, osc=osc), cfl=0.103, tableau="rk4")


@pytest.mark.parametrize("case", ["ragged", "sedov", "oscillating"])
def test_tensor_core_step_matches_cuda_core_step(case):
    """One RK4 step from the same state: 37 x 29 cells (9 tiles, the last one ragged), the
    Sedov-type blast, and a state whose inner stages need the limiter."""
    if case == "ragged":
        wl = _random(37, 29, seed=3, osc=0.3)
    elif case == "sedov":
        wl = inputs.sedov(48, 3)
    else:
        wl = _random(24, 20, seed=8, osc=1.2)
    a, b = _solver(wl, True), _solver(wl, False)
    a.set_state(wl.state)
    b.set_state(wl.state)
    dt = b.max_dt(wl.cfl)
    ia, ib = a.step(dt, wl.tableau), b.step(dt, wl.tableau)
    assert ia["restarts"] == ib["restarts"]
    sa, sb = a.get_state(), b.get_state()
    assert not np.array_equal(sa, sb), "the tensor-core path did not run"
    assert rel_linf(sa, sb, 4) < 2e-5
    assert a.margins().min() >= 0.0
    if case == "oscillating":
        assert ib["cells_limited"] > 0 and ia["cells_limited"] > 0
    # conservation: the averages change only through the FP64 face sums of the final stage,
    # which read the traces of the inner stages
    assert abs(a.mass(0) - b.mass(0)) <= 1e-6 * abs(b.mass(0))


def test_tensor_core_smooth_run_against_oracle():
    """Smooth 2D Euler (scenario II on the periodic square), Q^3, 100 steps on the tensor cores:
    relative L1 gap to the FP64 oracle <= 1e-4 and every component conserved to round-off."""
    wl = inputs.scenario2(12, 3)
    g, o = _solver(wl), _oracle(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    m0 = [g.mass(c) for c in range(4)]
    t = 0.0
    for _ in range(100):
        dt = o.max_dt(wl.cfl)
        g.step(dt, wl.tableau)
        rc, _ = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0
        t += dt
        assert g.margins().min() >= 0.0
    assert _rel_l1(g.get_state(), o.get_state(), 4) < 1e-4
    for c in range(4):
        assert abs(g.mass(c) - m0[c]) <= 1e-13 * max(1.0, abs(m0[c]))


def test_tensor_core_blast_against_oracle():
    """Sedov-type blast 48^2, Q^3, RK4 at the oracle's trial steps: bounds every step, equal
    restart decisions, conservation, and the L1 gap <= 1e-4 at step 10 (the blast's own
    conditioning amplifies FP32-level differences beyond that, as for the CUDA-core path)."""
    wl = inputs.sedov(48, 3)
    g, o = _solver(wl), _oracle(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    m0 = g.mass(0)
    t = 0.0
    for step in range(1, 31):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0
        t += dt
        if step <= 10:
            assert ig["restarts"] == io["restarts"]
        assert g.margins().min() >= 0.0
        assert abs(ig["mass_drift"]) < 1e-13
        if step == 10:
            assert _rel_l1(g.get_state(), o.get_state(), 4) < 1e-4
    assert abs(g.mass(0) - m0) <= 1e-13 * abs(m0)


def test_tensor_core_restarts_match_oracle():
    """At CFL 0.9 the blast's stage averages leave the admissible set: the tensor-core path
    halves the step exactly when the oracle does (the test of the averages is FP64)."""
    wl = inputs.sedov(16, 3)
    wl.cfl = 0.9
    g, o = _solver(wl), _oracle(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t, total = 0.0, 0
    for _ in range(8):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"]
        t += io["dt_taken"]
        total += io["restarts"]
        assert g.margins().min() >= 0.0
    assert total > 0


def test_tensor_core_switch_and_fallbacks():
    """Q^2 and general tableaux keep the CUDA-core kernel (the results do not depend on the
    switch); the switch restores the CUDA-core path for Q^3."""
    wl = inputs.riemann_quadrants(1, 24, 2)
    a, b = _solver(wl, True), _solver(wl, False)
    a.set_state(wl.state)
    b.set_state(wl.state)
    for _ in range(3):
        dt = b.max_dt(wl.cfl)
        a.step(dt, wl.tableau)
        b.step(dt, wl.tableau)
    assert np.array_equal(a.get_state(), b.get_state())
    # a tableau with a_31 != 0 (not sub-diagonal) runs on the CUDA cores
    wl3 = _random(12, 10, seed=2, osc=0.3)
    tab = ([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.25, 0.25, 0.0]], [1 / 6, 1 / 6, 2 / 3])
    a, b = _solver(wl3, True), _solver(wl3, False)
    a.set_state(wl3.state)
    b.set_state(wl3.state)
    dt = b.max_dt(0.1)
    a.step(dt, tab)
    b.step(dt, tab)
    assert np.array_equal(a.get_state(), b.get_state())
