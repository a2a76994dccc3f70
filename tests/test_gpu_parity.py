"""CUDA path vs the CPU oracle, element by element, on seeded inputs (through the C ABI).

Tolerance: relative L-infinity 1e-10 per component (the stated bound for the
all-FP64 build); single operators are held to 1e-12.  Bounds are checked with
the library's own S_K evaluation, which must show margins >= 0 exactly.
"""
import math

import numpy as np
import pytest

from gpu_helpers import ORACLE_TABS, pair, pair_from_workload, rel_linf
from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _state(dim, nx, ny, k, flux, seed, osc):
    if flux == "euler":
        return inputs.random_euler(dim, nx, ny, k, seed=seed, osc=osc)
    return inputs.random_scalar(dim, nx, ny, k, seed=seed, osc=osc)


OP_CASES = [(1, 11, 1, k, f) for k in (1, 2, 3) for f in ("advection", "burgers", "euler")] + \
           [(2, 7, 5, k, f) for k in (1, 2, 3) for f in ("advection", "burgers", "euler")]


@pytest.mark.parametrize("dim,nx,ny,k,flux", OP_CASES)
@pytest.mark.parametrize("op", ["G", "F", "limit"])
def test_operator_parity(dim, nx, ny, k, flux, op):
    """G (Sec. 2.1), F (eq. dxDG, periodic) and the limiter (Prop. 2.4 / eq. Euler-limiter)."""
    g, o = pair(dim, nx, ny, k, (0.0, 1.0, 0.0, 2.0), flux, velocity=(0.9, -0.6), bounds=(-0.5, 1.5))
    U = _state(dim, nx, ny, k, flux, seed=7 + k, osc=1.4 if op == "limit" else 0.3)
    x = torch.from_numpy(U).cuda()
    out = torch.empty_like(x)
    g.apply(op, x, out)
    c = o.to_modal(U)
    if op == "limit":
        o.limit(c)
        ref = o.to_nodal(c)
    else:
        ref = o.to_nodal(o.apply(op, c))
    err = rel_linf(out.cpu().numpy(), ref, o.m)
    assert err < 1e-12, err


@pytest.mark.parametrize("bc", [("outflow",) * 4, ("reflect", "outflow", "reflect", "outflow"),
                                ("dirichlet",) * 4])
@pytest.mark.parametrize("dim", [1, 2])
def test_F_boundary_conditions(dim, bc):
    """Exterior traces of the final stage: outflow, reflective walls, Dirichlet states."""
    st = {s: [1.1, 0.2, -0.1, 2.3][: dim + 2] if dim == 2 else [1.1, 0.2, 2.3] for s in range(4)}
    g, o = pair(dim, 6, 5, 2, (0.0, 1.0, 0.0, 1.0), "euler", bc=bc, bc_state=st)
    U = inputs.random_euler(dim, 6, 5, 2, seed=3, osc=0.3)
    x = torch.from_numpy(U).cuda()
    out = torch.empty_like(x)
    g.apply("F", x, out)
    ref = o.to_nodal(o.apply("F", o.to_modal(U)))
    assert rel_linf(out.cpu().numpy(), ref, o.m) < 1e-12


STEP_CASES = [(1, 16, 1, 1, "euler", "midpoint2"), (1, 16, 1, 2, "euler", "heun3"), (1, 16, 1, 3, "burgers", "rk4"),
              (2, 6, 5, 2, "euler", "heun3"), (2, 6, 5, 3, "euler", "rk4"), (2, 6, 5, 1, "advection", "midpoint2"),
              (2, 6, 5, 3, "burgers", "heun3")]


@pytest.mark.parametrize("dim,nx,ny,k,flux,tab", STEP_CASES)
def test_one_step_parity(dim, nx, ny, k, flux, tab):
    """One limited step (Scheme 1L): every stage, limiter and the final LF stage."""
    g, o = pair(dim, nx, ny, k, (0.0, 1.0, 0.0, 1.0), flux, velocity=(0.9, -0.6), bounds=(-0.5, 1.5))
    U = _state(dim, nx, ny, k, flux, seed=21, osc=1.2)
    g.set_state(U)
    o.set_state(U)
    assert rel_linf(g.get_state(), o.get_state(), o.m) < 1e-12
    dt = o.max_dt(0.1)
    assert abs(g.max_dt(0.1) - dt) < 1e-12 * dt
    ig = g.step(dt, tab)
    rc, io = o.step(dt, ORACLE_TABS[tab])
    assert rc == 0 and ig["restarts"] == io["restarts"]
    assert rel_linf(g.get_state(), o.get_state(), o.m) < 1e-11
    assert g.margins().min() >= 0.0


def _run_pair(g, o, steps, cfl, tab, t_end=math.inf):
    t = 0.0
    for _ in range(steps):
        dt = min(o.max_dt(cfl), t_end - t)
        if dt <= 0:
            break
        dg = g.max_dt(cfl)
        assert abs(dg - o.max_dt(cfl)) <= 1e-10 * dt
        ig = g.step(dt, tab)
        rc, io = o.step(dt, ORACLE_TABS[tab], t)
        assert rc == 0
        assert ig["restarts"] == io["restarts"]
        assert abs(ig["dt_taken"] - io["dt_taken"]) <= 1e-15 * dt
        m = g.margins()
        assert m[0] >= 0.0 and m[1] >= 0.0, m
        t += io["dt_taken"]
    return t


@pytest.mark.parametrize("name", ["burgers200", "euler1d_4096", "sedov32_q3", "riemann32_q2"])
def test_hundred_steps(name):
    """100 steps of the workloads (full size in 1D, 32x32 in 2D): rel L-inf <= 1e-10, bounds
    exact at every step, identical restart counts."""
    if name == "burgers200":
        wl = inputs.burgers_sine(200, 2)
    elif name == "euler1d_4096":
        wl = inputs.euler_blast_tube(4096, 2)
    elif name == "sedov32_q3":
        wl = inputs.sedov(32, 3)
    else:
        wl = inputs.riemann_quadrants(0, 32, 2)
    g, o = pair_from_workload(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    m0 = g.mass(0)
    _run_pair(g, o, 100, wl.cfl, wl.tableau)
    err = rel_linf(g.get_state(), o.get_state(), o.m)
    assert err < 1e-10, err
    if name == "burgers200":  # periodic: conservation to round-off
        assert abs(g.mass(0) - m0) < 1e-13 * abs(m0)


def test_conservation_periodic_euler_2d():
    """Sec. 3.2: global conservation of every component on a periodic mesh."""
    from paper_2412_16002_gb300.solver import Solver

    U = inputs.random_euler(2, 16, 12, 2, seed=5, osc=0.8)
    g = Solver(2, 16, 12, 2, (0.0, 1.0, 0.0, 1.0), "euler")
    g.set_state(U)
    m0 = [g.mass(c) for c in range(4)]
    for _ in range(20):
        g.step(g.max_dt(0.1), "heun3")
    for c in range(4):
        assert abs(g.mass(c) - m0[c]) <= 1e-13 * max(1.0, abs(m0[c]))
