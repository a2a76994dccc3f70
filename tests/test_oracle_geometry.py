"""Pins of the oracle's non-rectangular domains (Examples 4.8 and 4.9, Sec. 4.4).

The two benchmarks run on unions of rectangles: the bounding rectangle's cells, with the
cells outside the domain (the solid) masked, reflective walls on the sides that face the
solid, an inflow side, and for the double Mach reflection a fixed state on part of the wall
and the exact shock motion on the top side.  Each pin ties the geometry to something fixed
independently: the rectangular problem with the same wall (itself pinned by mirror
symmetry), the Rankine-Hugoniot relations and the paper's printed post-shock state,
conservation in a closed box, and the shock's kinematics.
"""
import math

import numpy as np
import pytest

from oracle.oracle import HEUN3, MIDPOINT2, Oracle
from paper_2412_16002_gb300 import inputs
from paper_2412_16002_gb300.inputs import (GEO_SHOCK, GEO_SOLID, GEO_STATE_A, GEO_STATE_B,
                                           GEO_WALL)


def _euler(nx, ny, k, dom, bc, **kw):
    return Oracle(2, nx, ny, k, dom, "euler", bc=bc, **kw)


def _run(o, steps, cfl=0.1, t=0.0):
    for _ in range(steps):
        dt = o.max_dt(cfl)
        rc, _ = o.step(dt, HEUN3, t)
        assert rc == 0
        t += dt
    return t


# ----------------------------------------------------------------------------- shock states


@pytest.mark.parametrize("mach", [5.09, 10.0])
def test_normal_shock_states_satisfy_rankine_hugoniot(mach):
    """The inflow and post-shock states of Examples 4.8 and 4.9 come from the normal-shock
    relations; in the shock's frame the mass, momentum and energy fluxes must be continuous."""
    g = 1.4
    rho1, p1 = 1.4, 1.0
    rho2, u2, p2, s = inputs.normal_shock(mach, rho1, p1, g)
    assert s == pytest.approx(mach * math.sqrt(g * p1 / rho1), rel=1e-15)

    def fluxes(rho, u, p):
        v = u - s  # velocity relative to the shock
        E = p / (g - 1.0) + 0.5 * rho * v * v
        return np.array([rho * v, rho * v * v + p, v * (E + p)])

    f1, f2 = fluxes(rho1, 0.0, p1), fluxes(rho2, u2, p2)
    assert np.abs(f1 - f2).max() <= 1e-12 * np.abs(f1).max()
    assert rho2 > rho1 and p2 > p1 and u2 > 0.0  # a compressive shock, not its expansion twin


def test_double_mach_post_shock_state_is_the_papers():
    """Example 4.9 prints the post-shock state of its Mach 10 shock: rho = 8,
    w = (4.125 sqrt 3, -4.125), p = 116.5, and a shock through (1/6, 0) at 60 degrees whose
    trace on y = 1 moves as x = 1/6 + (1 + 20 t)/sqrt 3."""
    wl = inputs.double_mach(cells_per_unit=6, k=1)
    post = np.array(wl.geo_states[0])
    rho, mx, my, E = post
    assert rho == pytest.approx(8.0, rel=1e-14)
    assert mx / rho == pytest.approx(4.125 * math.sqrt(3.0), rel=1e-14)
    assert my / rho == pytest.approx(-4.125, rel=1e-14)
    p = 0.4 * (E - 0.5 * (mx * mx + my * my) / rho)
    assert p == pytest.approx(116.5, rel=1e-13)
    x0, speed = wl.shock
    assert x0 == pytest.approx(1.0 / 6.0 + 1.0 / math.sqrt(3.0), rel=1e-15)
    assert speed == pytest.approx(20.0 / math.sqrt(3.0), rel=1e-15)


def test_benchmark_geometries_follow_the_paper():
    """The masks and walls of both examples at a coarse resolution: the solid blocks, and a
    wall on exactly the fluid sides that touch them."""
    sd = inputs.shock_diffraction(cells_per_unit=2, k=1)
    g = sd.geo.reshape(sd.ny, sd.nx)
    solid = (g & GEO_SOLID) != 0
    assert solid.sum() == 2 * 12  # [0,1]x[0,6] at h = 1/2
    assert solid[:12, :2].all() and not solid[12:, :].any() and not solid[:, 2:].any()
    assert (((g[12, :2] >> 8) & 15) == GEO_WALL).all()   # y = 6, x <= 1: bottom walls
    assert (((g[:12, 2] >> 0) & 15) == GEO_WALL).all()   # x = 1, y <= 6: left walls
    assert ((g[~solid] & 0xFFFF) != 0).sum() == 2 + 12   # nothing else carries a kind
    dm = inputs.double_mach(cells_per_unit=12, k=1)
    g = dm.geo.reshape(dm.ny, dm.nx)
    solid = (g & GEO_SOLID) != 0
    assert solid[:12, :12].all() and solid.sum() == 144
    bottom = (g[12, :12] >> 8) & 15
    assert (bottom[:2] == GEO_STATE_A).all() and (bottom[2:] == GEO_WALL).all()  # x < 1/6
    assert (((g[:12, 12] >> 0) & 15) == GEO_WALL).all()
    assert (((g[-1, :] >> 12) & 15) == GEO_SHOCK).all()


# ----------------------------------------------------------------------------- the oracle


@pytest.mark.parametrize("axis", ["x", "y"])
def test_masked_cells_with_walls_equal_the_rectangular_wall(axis):
    """A mesh whose first two columns (rows) are solid, with walls on the sides facing them,
    is the rectangular problem with a reflective side: every fluid cell's state, the trial
    step and the limiter's decisions must agree to the last bit of rounding.  The
    rectangular reflective wall is pinned by mirror symmetry in test_oracle_pins."""
    k, nx, ny, m = 2, 8, 6, 4
    U = inputs.random_euler(2, nx, ny, k, seed=71, osc=0.4).reshape(m, ny, nx, k + 1, k + 1)
    amb = np.array([1.4, 0.0, 0.0, 2.5])
    if axis == "x":
        bc_r = ("reflect", "outflow", "outflow", "outflow")
        dom_r, dom_g = (0.0, 1.0, 0.0, 0.75), (-0.25, 1.0, 0.0, 0.75)
        nxg, nyg = nx + 2, ny
        big = np.empty((m, ny, nx + 2, k + 1, k + 1))
        big[:, :, 2:] = U
        big[:, :, :2] = amb.reshape(m, 1, 1, 1, 1)
        sl = (slice(None), slice(None), slice(2, None))
    else:
        bc_r = ("outflow", "outflow", "reflect", "outflow")
        dom_r, dom_g = (0.0, 1.0, 0.0, 0.75), (0.0, 1.0, -0.25, 0.75)
        nxg, nyg = nx, ny + 2
        big = np.empty((m, ny + 2, nx, k + 1, k + 1))
        big[:, 2:] = U
        big[:, :2] = amb.reshape(m, 1, 1, 1, 1)
        sl = (slice(None), slice(2, None), slice(None))
    geo = np.zeros((nyg, nxg), dtype=np.uint32)
    if axis == "x":
        geo[:, :2] = GEO_SOLID
        geo[:, 2] = GEO_WALL  # left side
    else:
        geo[:2, :] = GEO_SOLID
        geo[2, :] = GEO_WALL << 8  # bottom side
    o_r = _euler(nx, ny, k, dom_r, bc_r)
    o_g = _euler(nxg, nyg, k, dom_g, ("outflow",) * 4)
    o_g.set_geometry(geo)
    o_r.set_state(U)
    o_g.set_state(big)
    g0 = o_g.get_state().copy()
    t = 0.0
    for _ in range(8):
        dt = o_r.max_dt(0.1)
        assert o_g.max_dt(0.1) == dt
        r1, i1 = o_r.step(dt, HEUN3, t)
        r2, i2 = o_g.step(dt, HEUN3, t)
        assert r1 == 0 and r2 == 0 and i1["cells_limited"] == i2["cells_limited"]
        t += dt
    a, b = o_r.get_state(), o_g.get_state()
    assert np.array_equal(a, b[sl])
    # the solid cells kept their state exactly
    rest = b[:, :, :2] if axis == "x" else b[:, :2]
    assert np.array_equal(rest, g0[:, :, :2] if axis == "x" else g0[:, :2])
    assert o_g.total_mass(0) == pytest.approx(o_r.total_mass(0), rel=1e-14)


def test_state_and_shock_kinds_equal_dirichlet_sides():
    """A fixed-state kind on the left column is the rectangle's Dirichlet side; the moving
    shock kind is state A behind the line and state B ahead of it."""
    k, nx, ny, m = 2, 6, 5, 4
    U = inputs.random_euler(2, nx, ny, k, seed=73, osc=0.3)
    sa = [2.0, 0.5, -0.2, 6.0]
    sb = [0.7, -0.1, 0.3, 1.9]
    dom = (0.0, 1.0, 0.0, 1.0)
    ref_a = _euler(nx, ny, k, dom, ("dirichlet", "outflow", "outflow", "outflow"), bc_state={0: sa})
    ref_b = _euler(nx, ny, k, dom, ("dirichlet", "outflow", "outflow", "outflow"), bc_state={0: sb})
    for o in (ref_a, ref_b):
        o.set_state(U)
    fa, fb = ref_a.apply("F", t=0.3), ref_b.apply("F", t=0.3)
    cases = [
        (GEO_STATE_A, (0.0, 0.0), fa),
        (GEO_STATE_B, (0.0, 0.0), fb),
        (GEO_SHOCK, (1e9, 0.0), fa),      # the line far ahead: every point behind it
        (GEO_SHOCK, (-1.0, 0.0), fb),     # the line behind the domain: every point ahead
        (GEO_SHOCK, (-0.5, 2.0), fa),     # it passes x = 0 at t = 0.25: at t = 0.3 behind
        (GEO_SHOCK, (-0.7, 2.0), fb),     # it passes x = 0 at t = 0.35: at t = 0.3 ahead
    ]
    for kind, shock, want in cases:
        geo = np.zeros((ny, nx), dtype=np.uint32)
        geo[:, 0] = kind
        o = _euler(nx, ny, k, dom, ("outflow",) * 4)
        o.set_geometry(geo, sa, sb, *shock)
        o.set_state(U)
        assert np.array_equal(o.apply("F", t=0.3), want), (kind, shock)
    assert not np.array_equal(fa, fb)


def test_shock_kind_switches_point_by_point_along_a_face():
    """On the top side the moving shock kind gives state A at face points with
    x < x0 + s t and state B beyond: against the rectangle's exact-solution side evaluated
    from the same step function of (x, t)."""
    k, nx, ny = 3, 5, 4
    U = inputs.random_euler(2, nx, ny, k, seed=75, osc=0.3)
    sa = np.array([2.0, 0.5, -0.2, 6.0])
    sb = np.array([0.7, -0.1, 0.3, 1.9])
    x0, s = 0.13, 1.7
    dom = (0.0, 1.0, 0.0, 1.0)
    ref = _euler(nx, ny, k, dom, ("outflow", "outflow", "outflow", "exact"),
                 exact=lambda x, y, t: sa if x < x0 + s * t else sb)
    geo = np.zeros((ny, nx), dtype=np.uint32)
    geo[-1, :] = GEO_SHOCK << 12
    o = _euler(nx, ny, k, dom, ("outflow",) * 4)
    o.set_geometry(geo, sa, sb, x0, s)
    ref.set_state(U)
    o.set_state(U)
    for t in (0.0, 0.11, 0.26, 0.4):
        assert np.array_equal(o.apply("F", t=t), ref.apply("F", t=t)), t
    # and the line really crosses the face points in that time window
    assert not np.array_equal(o.apply("F", t=0.0), o.apply("F", t=0.4))


def test_closed_l_shaped_box_conserves_mass_and_energy():
    """An L-shaped box (a solid block in one corner) closed by walls on every side: the walls
    carry no mass or energy flux, so both totals over the fluid cells stay fixed to rounding,
    the solid cells keep their state, and the averages stay in B^eps."""
    k, nx, ny, m = 2, 8, 8, 4
    U = inputs.random_euler(2, nx, ny, k, seed=77, osc=0.4).reshape(m, ny, nx, k + 1, k + 1)
    geo = np.zeros((ny, nx), dtype=np.uint32)
    geo[:3, :3] = GEO_SOLID
    geo[3, :3] |= GEO_WALL << 8
    geo[:3, 3] |= GEO_WALL
    geo[:, 0] |= np.where(geo[:, 0] & GEO_SOLID, 0, GEO_WALL).astype(np.uint32)
    geo[0, :] |= np.where(geo[0, :] & GEO_SOLID, 0, GEO_WALL << 8).astype(np.uint32)
    geo[:, -1] |= GEO_WALL << 4
    geo[-1, :] |= GEO_WALL << 12
    o = _euler(nx, ny, k, (0.0, 1.0, 0.0, 1.0), ("outflow",) * 4)
    o.set_geometry(geo)
    o.set_state(U)
    s0 = o.get_state().copy()
    mass0, en0 = o.total_mass(0), o.total_mass(3)
    _run(o, 12)
    assert abs(o.total_mass(0) - mass0) <= 1e-14 * abs(mass0)
    assert abs(o.total_mass(3) - en0) <= 1e-14 * abs(en0)
    s1 = o.get_state()
    solid = (geo & GEO_SOLID) != 0
    assert np.array_equal(s1[:, solid], s0[:, solid])
    assert not np.array_equal(s1[:, ~solid], s0[:, ~solid])
    # the totals exclude the solid cells
    o2 = _euler(nx, ny, k, (0.0, 1.0, 0.0, 1.0), ("outflow",) * 4)
    o2.set_state(s1)
    avg = o2.averages().reshape(ny, nx, m)
    assert o.total_mass(0) == pytest.approx(avg[~solid, 0].sum() / (nx * ny), rel=1e-13)
    assert o.admissible()


def test_geometry_rejects_an_open_side_facing_a_solid_cell():
    o = _euler(4, 4, 1, (0.0, 1.0, 0.0, 1.0), ("outflow",) * 4)
    geo = np.zeros((4, 4), dtype=np.uint32)
    geo[0, 0] = GEO_SOLID
    with pytest.raises(ValueError):
        o.set_geometry(geo)  # cells (1, 0) and (0, 1) face it through the mesh rule
    geo[0, 1] = GEO_WALL
    geo[1, 0] = GEO_WALL << 8
    o.set_geometry(geo)
    geo[2, 2] = 9  # no such kind
    with pytest.raises(ValueError):
        o.set_geometry(geo)


@pytest.mark.parametrize("example", ["diffraction", "double_mach"])
def test_benchmarks_keep_positivity_and_the_shock_moves(example):
    """A few steps of each benchmark at a coarse mesh: the averages stay in B^eps, every S_K
    point satisfies the bounds (Theorem 3.5), the solid cells keep their state, and the
    shock has moved by its speed times the elapsed time (within two cells)."""
    if example == "diffraction":
        wl = inputs.shock_diffraction(cells_per_unit=2, k=2)
    else:
        wl = inputs.double_mach(cells_per_unit=6, k=2)
    o = Oracle(2, wl.nx, wl.ny, wl.k, wl.domain, "euler", bc=wl.bc, bc_state=wl.bc_state, eps=wl.eps)
    o.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
    o.set_state(wl.state)
    s0 = o.get_state().copy()
    t = _run(o, 10, cfl=wl.cfl)
    assert o.admissible()
    mg = o.min_margins()
    assert mg[0] >= 0.0 and mg[1] >= 0.0
    s1 = o.get_state()
    solid = ((wl.geo & GEO_SOLID) != 0).reshape(wl.ny, wl.nx)
    assert np.array_equal(s1[:, solid], s0[:, solid])
    # the shock front: the first column (along the top fluid row) whose density is still ambient
    rho = o.averages().reshape(wl.ny, wl.nx, 4)[..., 0]
    row = rho[-1]
    h = (wl.domain[1] - wl.domain[0]) / wl.nx
    front = h * np.argmax(row < 1.4 + 0.05)
    if example == "diffraction":
        x_exp = 0.5 + 5.09 * t
    else:
        x_exp = wl.shock[0] + wl.shock[1] * t
    assert abs(front - x_exp) <= 2.0 * h, (front, x_exp)


@pytest.mark.parametrize("example", ["diffraction", "double_mach"])
def test_benchmarks_run_to_their_end_times(example):
    """Examples 4.8 and 4.9 to their end times (2.3 and 0.2) at coarse meshes, Q^1 with the
    explicit midpoint scheme: no step fails (the restart loop of Sec. 4.1 always finds an
    admissible step), every S_K point of every step's result keeps rho >= eps and
    rho e >= eps (Theorem 3.5: the paper reports positivity at the corner, where density and
    pressure fall), the solid cells are untouched, and the undisturbed incident shock on the
    top side is where it must be at the end time (within 2.5 cells)."""
    if example == "diffraction":
        wl = inputs.shock_diffraction(cells_per_unit=4, k=1)
        T = 2.3
    else:
        wl = inputs.double_mach(cells_per_unit=16, k=1)
        T = 0.2
    o = Oracle(2, wl.nx, wl.ny, 1, wl.domain, "euler", bc=wl.bc, bc_state=wl.bc_state, eps=wl.eps)
    o.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
    o.set_state(wl.state)
    s0 = o.get_state().copy()
    t = 0.0
    while t < T - 1e-14:
        dt = min(o.max_dt(wl.cfl), T - t)
        rc, info = o.step(dt, MIDPOINT2, t)
        assert rc == 0, t
        t += info["dt_taken"]
        mg = o.min_margins()
        assert mg[0] >= 0.0 and mg[1] >= 0.0, (t, mg)
    assert o.admissible()
    solid = ((wl.geo & GEO_SOLID) != 0).reshape(wl.ny, wl.nx)
    assert np.array_equal(o.get_state()[:, solid], s0[:, solid])
    rho = o.averages().reshape(wl.ny, wl.nx, 4)[..., 0]
    h = (wl.domain[1] - wl.domain[0]) / wl.nx
    front = h * (np.where(rho[-1] > 1.4 + 0.05)[0].max() + 1)
    x_exact = 0.5 + 5.09 * T if example == "diffraction" else wl.shock[0] + wl.shock[1] * T
    assert abs(front - x_exact) <= 2.5 * h, (front, x_exact)
    # the corner expansion drops the density well below the ambient 1.4 (the diffraction's
    # low-density region) while staying positive
    assert rho[~solid].min() < 1.0


def test_transposed_diffraction_is_the_transpose():
    """The shock diffraction with x and y exchanged (the step [0,6]x[0,1] at the left of the
    bottom side, the shock entering through the bottom and running up) must be the
    transpose of the original at every step, the two momenta exchanged: walls on left and
    bottom sides, the inflow side and the re-entrant corner treated alike in both
    directions.  The summation orders of the two runs differ, so the pin is 1e-12 relative."""
    wl = inputs.shock_diffraction(cells_per_unit=2, k=2)
    nx, ny, n = wl.nx, wl.ny, wl.k + 1
    o = Oracle(2, nx, ny, wl.k, wl.domain, "euler", bc=wl.bc, bc_state=wl.bc_state, eps=wl.eps)
    o.set_geometry(wl.geo)
    o.set_state(wl.state)

    def transpose_state(U):  # [4][ny][nx][n_y][n_x] -> the transposed problem's layout
        V = U.transpose(0, 2, 1, 4, 3)[[0, 2, 1, 3]]
        return np.ascontiguousarray(V)

    g = wl.geo.reshape(ny, nx)
    sides = [(g >> (4 * s)) & 15 for s in range(4)]
    gt = (sides[2].T | sides[3].T << 4 | sides[0].T << 8 | sides[1].T << 12) | (g.T & GEO_SOLID)
    post = list(wl.bc_state[0])
    post_t = [post[0], post[2], post[1], post[3]]
    ot = Oracle(2, ny, nx, wl.k, (0.0, 12.0, 0.0, 13.0), "euler", bc=("outflow", "outflow", "dirichlet", "outflow"),
                bc_state={2: post_t}, eps=wl.eps)
    ot.set_geometry(np.ascontiguousarray(gt, dtype=np.uint32))
    ot.set_state(transpose_state(wl.state))
    t = 0.0
    for _ in range(30):  # the shock passes the corner (x = 1) at t ~ 0.1
        dt = o.max_dt(wl.cfl)
        assert ot.max_dt(wl.cfl) == pytest.approx(dt, rel=1e-14)
        rc1, _ = o.step(dt, HEUN3, t)
        rc2, _ = ot.step(dt, HEUN3, t)
        assert rc1 == 0 and rc2 == 0
        t += dt
    a = transpose_state(o.get_state().reshape(4, ny, nx, n, n))
    b = ot.get_state()
    for c in range(4):
        assert np.abs(a[c] - b[c]).max() <= 1e-12 * np.abs(b[c]).max(), c
