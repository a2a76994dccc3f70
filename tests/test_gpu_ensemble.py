"""Ensembles of uneven 2D Euler problems in persistent launches under CUDA graphs: every
member is bit-identical to the same problem stepped alone by crkdg_step at the same trial
steps (the kernels run the same block bodies), through restarts, both indicators, clipping
at the end time and after autotuning."""
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


SPECS = [(11, 16, 2), (12, 24, 3), (13, 20, 2), (14, 12, 3), (15, 40, 2), (16, 9, 3)]


def _riemann(specs):
    return [inputs.riemann_quadrants(seed, n, k) for seed, n, k in specs]


def _run_and_compare(wls, steps, indicator="off", cfl_scale=1.0, t_end=None, mlp=None, autotune=False):
    from paper_2412_16002_gb300.ensemble import Ensemble
    from paper_2412_16002_gb300.solver import Solver

    probs = [dict(nx=w.nx, ny=w.ny, k=w.k, domain=w.domain, bc=w.bc, tableau=w.tableau, cfl=w.cfl * cfl_scale,
                  t_end=1e30 if t_end is None else t_end[i]) for i, w in enumerate(wls)]
    ens = Ensemble(probs, gamma=wls[0].gamma, eps=wls[0].eps, indicator=indicator)
    for i, w in enumerate(wls):
        ens.set_state(i, w.state)
    if mlp is not None:
        ens.set_mlp(mlp)
    if autotune:
        before = [ens.get_state(i).copy() for i in range(len(wls))]
        tiles = ens.autotune(reps=1)
        assert all(t in (0, 1, 2, 4, 8, 16) for t in tiles) and any(tiles)
        for i in range(len(wls)):
            assert np.array_equal(ens.get_state(i), before[i])
    singles = []
    for w in wls:
        g = Solver.from_workload(w, indicator=indicator)
        if mlp is not None:
            g.set_mlp(mlp)
        g.set_state(w.state)
        singles.append(g)
    times = [0.0] * len(wls)
    restarts = 0
    for _ in range(steps):
        ens.step()
        for i, g in enumerate(singles):
            te = probs[i]["t_end"]
            if not times[i] < te:
                continue
            dt = min(g.max_dt(probs[i]["cfl"]), te - times[i])
            info = g.step(dt, probs[i]["tableau"])
            times[i] += info["dt_taken"]
            e = ens.info(i)
            assert e["t"] == times[i], (i, e["t"], times[i])
            assert e["last_restarts"] == info["restarts"]
            assert e["troubled"] == info["troubled"]
            restarts += info["restarts"]
    for i, g in enumerate(singles):
        assert np.array_equal(ens.get_state(i), g.get_state()), i
    return ens, restarts


def test_ensemble_matches_single_problems_bitwise():
    _run_and_compare(_riemann(SPECS), 8)


def test_ensemble_restarts_match():
    """Sedov-type blasts (reflecting and outflow sides) at 5x their CFL number restart; each
    problem halves its own step, the others are not redone."""
    wls = [inputs.sedov(16, 3), inputs.sedov(12, 2), inputs.riemann_quadrants(11, 16, 2)]
    ens, restarts = _run_and_compare(wls, 6, cfl_scale=5.0)
    assert restarts > 0


def test_ensemble_end_times_and_tvb_indicator():
    t_end = [0.004, 1e30, 0.002, 1e30, 1e30, 0.003]
    ens, _ = _run_and_compare(_riemann(SPECS), 10, indicator="tvb", t_end=t_end)
    for i, te in enumerate(t_end):
        inf = ens.info(i)
        if te < 1:
            assert inf["done"] and inf["t"] == pytest.approx(te, rel=0, abs=1e-15)


def test_ensemble_learned_indicator_and_autotune():
    from paper_2412_16002_gb300.indicator import init_params

    theta = init_params(3)
    _run_and_compare(_riemann(SPECS), 5, indicator="mlp", mlp=theta, autotune=True)


def test_ensemble_harvest_equals_single_problem_harvest():
    """The indicator's training set from one ensemble run (features of the unlimited final
    stage and the plain TVB labels, every problem, every few steps) equals the single-handle
    harvest of the same seeds bit for bit."""
    from paper_2412_16002_gb300 import indicator as ind

    seeds, n, steps, every = [11, 12, 13], 24, 12, 4
    Xe, Ye = ind.harvest_ensemble(seeds, n=n, k=2, steps=steps, every=every)
    Xs, Ys = ind.harvest(seeds, n=n, k=2, steps=steps, every=every)
    assert Xe.shape == Xs.shape == (len(seeds) * (steps // every) * n * n, 44)
    assert torch.equal(Xe, Xs) and torch.equal(Ye, Ys)
    assert float(Ye.sum()) > 0
