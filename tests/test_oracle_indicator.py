"""Pins of the oracle's plain troubled-cell indicator and minmod shock limiter (an optional
anti-oscillation stage that the paper itself leaves out, Sec. 4): hand-computed TVB
decisions on small stencils, invariants of the limiter."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2412_16002_gb300 import inputs


def _modal_1d(o, coeffs):
    """modal state from per-cell Legendre coefficient lists"""
    c = np.zeros(o.N)
    n = o.n
    for cell, cc in enumerate(coeffs):
        c[cell * n: cell * n + len(cc)] = cc
    return c


def test_linear_data_is_never_troubled():
    """u = a + b x is exactly P1: face deviations b h/2 against neighbour differences b h."""
    for k in (1, 2, 3):
        X = inputs.node_coords(1, 10, 1, k, (0.0, 1.0))
        o = Oracle(1, 10, 1, k, (0.0, 1.0), "advection", bounds=(-100, 100), bc=("outflow",) * 4, tvb_M=0.0)
        f = o.troubled(o.to_modal((3.0 * X - 1.0)[None]))
        assert f[1:-1].sum() == 0  # boundary cells see a zero outflow difference


def test_hand_computed_stencil():
    """Three cells (outflow), P1, averages (0, 1, 1) and centre slope c = 0.4:
    ut_R = ut_L = 0.4, D+ = 0, D- = 1 -> minmod(0.4, 0, 1) = 0 != 0.4 -> troubled (M = 0).
    With M h^2 >= 0.4 the TVB modification keeps 0.4 -> not troubled."""
    o = Oracle(1, 3, 1, 1, (0.0, 3.0), "advection", bounds=(-10, 10), bc=("outflow",) * 4, tvb_M=0.0)
    c = _modal_1d(o, [[0.0, 0.0], [1.0, 0.4], [1.0, 0.0]])
    assert list(o.troubled(c)) == [0, 1, 0]
    o2 = Oracle(1, 3, 1, 1, (0.0, 3.0), "advection", bounds=(-10, 10), bc=("outflow",) * 4, tvb_M=0.4)
    assert list(o2.troubled(c)) == [0, 0, 0]
    # centre slope 0.3 between averages 0, 0.5, 1: minmod(0.3, 0.5, 0.5) = 0.3 -> smooth
    c3 = _modal_1d(o, [[0.0, 0.0], [0.5, 0.3], [1.0, 0.0]])
    assert o.troubled(c3)[1] == 0
    # centre slope 0.7 > 0.5: limited -> troubled; the limited slope is minmod = 0.5
    c4 = _modal_1d(o, [[0.0, 0.0], [0.5, 0.7], [1.0, 0.0]])
    f = o.troubled(c4)
    assert f[1] == 1
    o.shock_limit(f, c4)
    assert abs(c4[2] - 0.5) < 1e-15 and abs(c4[3] - 0.5) < 1e-15


def test_discontinuity_inside_a_cell_is_troubled():
    o = Oracle(1, 16, 1, 2, (0.0, 1.0), "advection", bounds=(-10, 10), bc=("outflow",) * 4, tvb_M=1.0)
    X = inputs.node_coords(1, 16, 1, 2, (0.0, 1.0))
    U = np.where(X < 0.53, 1.0, 0.0)[None]  # the jump falls inside cell 8
    f = o.troubled(o.to_modal(U))
    assert f[8] == 1 and f.sum() <= 3


@pytest.mark.parametrize("dim,k", [(1, 2), (2, 2), (2, 3)])
def test_shock_limiter_keeps_averages_and_is_linear(dim, k):
    o = Oracle(dim, 8, 6, k, (0.0, 1.0, 0.0, 1.0), "euler", tvb_M=0.0)
    U = inputs.random_euler(dim, 8, 6, k, seed=2, osc=0.8)
    c = o.to_modal(U)
    avg0 = o.averages(c).copy()
    f = o.troubled(c)
    assert f.sum() > 0
    o.shock_limit(f, c)
    assert np.array_equal(o.averages(c), avg0)
    n = k + 1
    per = o.N // (o.nx * o.ny)
    for cell in np.nonzero(f)[0]:
        for comp in range(o.m):
            modes = c[cell * per + comp * (per // o.m): cell * per + (comp + 1) * (per // o.m)]
            keep = {0, 1} | ({n} if dim == 2 else set())
            assert all(modes[q] == 0.0 for q in range(len(modes)) if q not in keep)


def test_indicator_step_keeps_bounds_and_conservation():
    """With the indicator on, a limited step still conserves (periodic) and keeps the bounds."""
    o = Oracle(2, 12, 12, 2, (0.0, 1.0, 0.0, 1.0), "euler", indicator=True, tvb_M=1.0)
    o.set_state(inputs.random_euler(2, 12, 12, 2, seed=3, osc=0.6))
    m0 = [o.total_mass(c) for c in range(4)]
    for _ in range(5):
        rc, info = o.step(o.max_dt(0.1), (np.array([[0, 0, 0], [1 / 3, 0, 0], [0, 2 / 3, 0]]), np.array([0.25, 0, 0.75])))
        assert rc == 0
    assert o.min_margins().min() >= 0
    for c in range(4):
        assert abs(o.total_mass(c) - m0[c]) < 1e-13 * max(1, abs(m0[c]))
