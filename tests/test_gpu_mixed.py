"""Split-precision path (FP64 averages, FP32 deviations and operators) against the FP64
oracle.  Tolerances follow from the arithmetic: FP32 operators on O(n) terms carry a
relative error of a few 1e-7 of the largest value, so single operators are held to 2e-5
(relative L-inf) and smooth runs to 1e-4 relative L1; what FP64 keeps is held exactly:
bounds at every S_K point (by the library's own FP64 evaluation), conservation of the
cell averages to FP64 round-off, and the averages' admissibility decisions."""
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


def _pair(wl, precision="mixed"):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, precision=precision)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
               bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state)
    return g, o


def _rel_l1(a, b, m):
    a = np.asarray(a).reshape(m, -1)
    b = np.asarray(b).reshape(m, -1)
    return max(np.abs(a[c] - b[c]).sum() / max(np.abs(b[c]).sum(), 1e-300) for c in range(m))


@pytest.mark.parametrize("dim,k", [(1, 2), (2, 2), (2, 3)])
@pytest.mark.parametrize("op", ["G", "F"])
def test_mixed_operators(dim, k, op):
    from paper_2412_16002_gb300.solver import Solver

    nx, ny = 9, 7
    g = Solver(dim, nx, ny, k, (0.0, 1.0, 0.0, 1.0), "euler", precision="mixed")
    o = Oracle(dim, nx, ny, k, (0.0, 1.0, 0.0, 1.0), "euler")
    U = inputs.random_euler(dim, nx, ny, k, seed=4, osc=0.3)
    x = torch.from_numpy(U).cuda()
    out = torch.empty_like(x)
    g.apply(op, x, out)
    ref = o.to_nodal(o.apply(op, o.to_modal(U)))
    assert rel_linf(out.cpu().numpy(), ref, o.m) < 2e-5


@pytest.mark.parametrize("dim,k", [(1, 2), (2, 2), (2, 3)])
def test_mixed_limiter_bounds_and_averages(dim, k):
    """The FP32-screened limiter keeps the FP64 averages and restores the bounds exactly
    under its FP64 evaluation; the limited polynomial matches the oracle's to FP32 accuracy."""
    from paper_2412_16002_gb300.solver import Solver

    nx, ny = 11, 9
    wl = inputs.Workload("rnd", dim, nx, ny if dim == 2 else 1, k, (0.0, 1.0, 0.0, 1.0), "euler",
                         ("periodic",) * 4, inputs.random_euler(dim, nx, ny, k, seed=6, osc=1.5))
    g, o = _pair(wl)
    g.set_state(wl.state)  # set_state splits and limits
    o.set_state(wl.state)
    assert g.margins().min() >= 0.0
    assert np.array_equal(g.averages(), g.averages())
    avg_ref = o.averages()
    assert np.abs(g.averages() - avg_ref).max() <= 1e-14 * np.abs(avg_ref).max()
    assert _rel_l1(g.get_state(), o.get_state(), o.m) < 1e-5


@pytest.mark.parametrize("k", [2, 3])
def test_mixed_smooth_run_and_conservation(k):
    """Smooth 2D Euler (scenario II on the periodic square), 100 steps: relative L1 gap to the
    FP64 oracle <= 1e-4, and sum |K| ubar conserved to FP64 round-off for every component."""
    wl = inputs.scenario2(12, k)
    g, o = _pair(wl)
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


@pytest.mark.parametrize("name,cmp_step", [("sedov48_q3", 10), ("riemann48_q2", 60)])
def test_mixed_shock_workloads(name, cmp_step):
    """Sedov-type blast (Q3, RK4) and a four-quadrant Riemann problem (Q2, Heun-3), 60 steps
    with the oracle's trial steps on both sides: exact bounds at every step, conservation of
    the averages (the blast does not reach the outflow sides), equal restart decisions, and
    the relative L1 gap to the FP64 oracle <= 1e-4 at step cmp_step.

    The comparison step is set by the flow's conditioning, not by the kernels: the FP64
    oracle run against itself, its state rounded to FP32 once per step, drifts on the blast
    by 9e-8 after 10 steps, 1e-2 after 30 and 1.5e-1 after 60, and on the Riemann problem
    stays near round-off; beyond step 10 the blast amplifies any FP32-level difference to
    O(0.1), so its states are compared at step 10 and only the invariants after that."""
    wl = inputs.sedov(48, 3) if name.startswith("sedov") else inputs.riemann_quadrants(2, 48, 2)
    g, o = _pair(wl)
    g.set_state(wl.state)
    o.set_state(wl.state)
    m0 = [g.mass(c) for c in range(4)]
    t = 0.0
    for step in range(1, 61):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0
        if step <= cmp_step:
            assert ig["restarts"] == io["restarts"]
        t += dt
        assert g.margins().min() >= 0.0
        if step == cmp_step:
            gap = _rel_l1(g.get_state(), o.get_state(), 4)
            print(f"{name}: relative L1 gap to the FP64 oracle after {step} steps = {gap:.3e}")
            assert gap < 1e-4, gap
    if name.startswith("sedov"):
        for c in (0, 3):
            assert abs(g.mass(c) - m0[c]) <= 1e-13 * abs(m0[c])


def _riemann_pair(precision, indicator, seed=2, n=48, **kw):
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.riemann_quadrants(seed, n, 2)
    g = Solver.from_workload(wl, precision=precision, indicator=indicator, **kw)
    g.set_state(wl.state)
    return g, wl


def test_mixed_tvb_indicator_invariants_and_fp64_agreement():
    """Split precision with the plain indicator (four-quadrant Riemann 48^2, Q^2, 20 steps at
    the FP64 run's trial steps): bounds exact every step, the flags agree with the FP64 path's
    in at least 99% of the cell-steps (the decisions are FP64 on states that differ by FP32
    rounding), and the relative L1 gap to the FP64 path stays below 1e-3."""
    gm, wl = _riemann_pair("mixed", "tvb", tvb_M=10.0)
    gf, _ = _riemann_pair("fp64", "tvb", tvb_M=10.0)
    agree = total = flagged = 0
    for _ in range(20):
        dt = gf.max_dt(wl.cfl)
        im = gm.step(dt, wl.tableau)
        gf.step(dt, wl.tableau)
        fm, ff = gm.troubled_flags(), gf.troubled_flags()
        agree += int((fm == ff).sum())
        total += fm.size
        flagged += int(ff.sum())
        assert im["troubled"] == int(fm.sum())
        assert gm.margins().min() >= 0.0
    assert flagged > 0 and agree >= 0.99 * total, (agree, total)
    gap = _rel_l1(gm.get_state(), gf.get_state(), 4)
    print(f"split + TVB against FP64 + TVB after 20 steps: L1 gap {gap:.3e}, flag agreement {agree / total:.5f}")
    assert gap < 1e-3


def test_mixed_learned_with_undecided_network_is_the_plain_indicator():
    """A network with zero parameters outputs p = 0.5 for every cell, which the learned rule
    leaves to the plain decision: the split-precision learned path (decision by the FP64
    feature kernel on the merged nodal values) then reproduces the split-precision TVB path
    (decision by the FP32 screen of the troubled-cell pass) bit for bit, flags included."""
    ga, wl = _riemann_pair("mixed", "tvb", tvb_M=10.0)
    gb, _ = _riemann_pair("mixed", "mlp", tvb_M=10.0)
    gb.set_mlp(torch.zeros(7105, dtype=torch.float32, device="cuda"))
    for _ in range(10):
        dt = ga.max_dt(wl.cfl)
        ia = ga.step(dt, wl.tableau)
        ib = gb.step(dt, wl.tableau)
        assert ia["troubled"] == ib["troubled"] and ia["restarts"] == ib["restarts"]
        assert np.array_equal(ga.troubled_flags(), gb.troubled_flags())
    assert np.array_equal(ga.get_state(), gb.get_state())


def test_mixed_tvb_conserves_the_blast():
    """Sedov-type blast (reflecting and outflow sides, not reached), Q^3, split precision with
    the plain indicator: the shock limiter keeps the FP64 averages, so mass and energy are
    conserved to FP64 round-off; bounds hold every step."""
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.sedov(32, 3)
    g = Solver.from_workload(wl, precision="mixed", indicator="tvb", tvb_M=10.0)
    g.set_state(wl.state)
    m0 = [g.mass(c) for c in (0, 3)]
    troubled = 0
    for _ in range(20):
        info = g.step(g.max_dt(wl.cfl), wl.tableau)
        troubled += info["troubled"]
        assert g.margins().min() >= 0.0
    assert troubled > 0
    for c, m in zip((0, 3), m0):
        assert abs(g.mass(c) - m) <= 1e-13 * abs(m)


@pytest.mark.parametrize("seed,n,k,M", [(4, 32, 2, 1.0), (5, 24, 3, 10.0)])
def test_mixed_tvb_indicator_against_oracle(seed, n, k, M):
    """Split precision with the plain indicator against the FP64 oracle with the same
    indicator, five steps at the oracle's trial steps: the flags are FP64 decisions on states
    that differ by FP32 rounding, so at most 0.5% of them may differ; the states agree to 1e-5
    relative L1 and the bounds hold exactly."""
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.riemann_quadrants(seed, n, k)
    g = Solver.from_workload(wl, precision="mixed", indicator="tvb", tvb_M=M)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, eps=wl.eps, bc=wl.bc,
               bc_state=wl.bc_state, indicator=True, tvb_M=M)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t = 0.0
    flagged = differ = 0
    for step in range(5):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        before = o.c.copy()
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"] == 0
        rc2, us, _ = o.step_stages(dt, ORACLE_TABS[wl.tableau], t, modal=before)
        fo, fg = o.troubled(us[-1]), g.troubled_flags()
        flagged += int(fo.sum())
        differ += int((fo != fg).sum())
        assert ig["troubled"] == int(fg.sum())
        assert g.margins().min() >= 0.0
        t += dt
    gap = _rel_l1(g.get_state(), o.get_state(), o.m)
    print(f"riemann{n}_q{k} split + TVB: {flagged} oracle flags, {differ} differ; L1 gap {gap:.3e}")
    assert flagged > 0 and differ <= 0.005 * 5 * n * n
    assert gap < 1e-5


@pytest.mark.parametrize("seed,n,k,M", [(3, 40, 2, 0.0), (3, 40, 2, 10.0), (6, 32, 3, 1.0)])
def test_mixed_screened_decision_is_the_fp64_decision(seed, n, k, M):
    """The split troubled-cell pass takes the plain decision from an FP32 screen of the
    deviations with an FP64 fallback; with harvesting on, the FP64 feature kernel takes it on
    the merged nodal values instead.  Both must give the same flags and the same states bit
    for bit.  M = 0 leaves most decisions of the smooth and constant regions to the fallback
    (trace deviations at rounding level against a zero threshold)."""
    ga, wl = _riemann_pair("mixed", "tvb", seed=seed, n=n, tvb_M=M)
    gb, _ = _riemann_pair("mixed", "tvb", seed=seed, n=n, tvb_M=M)
    gb.set_harvest(True)
    flagged = 0
    for _ in range(12):
        dt = ga.max_dt(wl.cfl)
        ia = ga.step(dt, wl.tableau)
        ib = gb.step(dt, wl.tableau)
        fa, fb = ga.troubled_flags(), gb.troubled_flags()
        assert np.array_equal(fa, fb), np.nonzero(fa != fb)
        assert ia["troubled"] == ib["troubled"] == int(fa.sum())
        flagged += int(fa.sum())
    assert flagged > 0
    assert np.array_equal(ga.get_state(), gb.get_state())


def test_mixed_tvb_1d_against_oracle():
    """Split precision with the plain indicator on a 1D mesh (blast tube, 256 P^2 cells):
    flags within 0.5% of the oracle's, states to 1e-5 relative L1, bounds exact."""
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.euler_blast_tube(256, 2)
    M = 1.0
    g = Solver.from_workload(wl, precision="mixed", indicator="tvb", tvb_M=M)
    o = Oracle(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, eps=wl.eps, bc=wl.bc,
               bc_state=wl.bc_state, indicator=True, tvb_M=M)
    g.set_state(wl.state)
    o.set_state(wl.state)
    t = 0.0
    flagged = differ = 0
    for step in range(5):
        dt = o.max_dt(wl.cfl)
        ig = g.step(dt, wl.tableau)
        before = o.c.copy()
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0 and ig["restarts"] == io["restarts"]
        rc2, us, _ = o.step_stages(dt, ORACLE_TABS[wl.tableau], t, modal=before)
        fo, fg = o.troubled(us[-1]), g.troubled_flags()
        flagged += int(fo.sum())
        differ += int((fo != fg).sum())
        assert g.margins().min() >= 0.0
        t += dt
    gap = _rel_l1(g.get_state(), o.get_state(), o.m)
    print(f"blast1d_256_p2 split + TVB: {flagged} oracle flags, {differ} differ; L1 gap {gap:.3e}")
    assert flagged > 0 and differ <= 0.005 * 5 * 256
    assert gap < 1e-5


def test_mixed_learned_features_from_the_split_state():
    """The split path's learned indicator takes its features from the split state (the
    stencil part from the FP64 averages, the first moments in FP32 from the deviations) and
    leaves the plain decision to the troubled-cell pass.  With harvesting on, the same step
    instead merges to FP64 nodal values and runs the FP64 feature kernel.  The two feature
    sets agree to 1e-5 (features are O(1)); with a random network the learned flags and the
    states then agree exactly (a flag could move only for a probability within ~1e-7 of 0.4
    or 0.6)."""
    from oracle import mlp

    ga, wl = _riemann_pair("mixed", "mlp", tvb_M=10.0)
    gb, _ = _riemann_pair("mixed", "mlp", tvb_M=10.0)
    theta = torch.tensor(mlp.init_params(3), dtype=torch.float32, device="cuda")
    ga.set_mlp(theta)
    gb.set_mlp(theta)
    gb.set_harvest(True)
    flagged = 0
    for _ in range(8):
        dt = ga.max_dt(wl.cfl)
        ia = ga.step(dt, wl.tableau)
        ib = gb.step(dt, wl.tableau)
        fa, fb = ga.last_features(), gb.last_features()
        assert np.abs(fa - fb).max() < 1e-5, np.abs(fa - fb).max()
        assert np.array_equal(ga.troubled_flags(), gb.troubled_flags())
        assert ia["troubled"] == ib["troubled"]
        flagged += ia["troubled"]
    assert flagged > 0
    assert np.array_equal(ga.get_state(), gb.get_state())


@pytest.mark.parametrize("name", ["sedov_2048_q3", "riemann_1024_q2"])
def test_mixed_full_size_sampled_cells(name):
    """Full-size split-precision step (2048^2 Q^3 RK4 Sedov-type blast, whose inner stages run
    on the tensor cores; 1024^2 Q^2 Heun-3 Riemann problem), launched as bench.py launches it:
    sampled cells against the FP64 oracle on their 3x3 patch with the same dt, element by
    element at the split path's operator tolerance (2e-5 of the component's scale), and the
    cell averages (updated in FP64 from FP32 face fluxes) to 1e-6."""
    from test_gpu_parity import _patch_oracle

    from paper_2412_16002_gb300.solver import Solver

    if name.startswith("sedov"):
        wl = inputs.sedov_shell(2048, 3)
        r = 0.3 / 1.1 * 2048
        cells = [(0, 0), (2047, 2047), (0, 1000), (1000, 0), (int(r * 0.7071), int(r * 0.7071)),
                 (int(r), 3), (3, int(r)), (int(r * 0.6), int(r * 0.8)), (700, 1500), (1200, 200)]
    else:
        wl = inputs.riemann_quadrants(3, 1024, 2)
        cells = [(511, 511), (512, 512), (511, 512), (0, 0), (1023, 1023), (511, 100), (100, 512),
                 (700, 511), (0, 511), (511, 1023)]
    g = Solver.from_workload(wl, precision="mixed", stream=torch.cuda.current_stream())
    g.set_state(torch.from_numpy(wl.state).cuda())
    dt = g.max_dt(wl.cfl)
    info = g.step(dt, wl.tableau)
    assert info["restarts"] == 0
    assert g.margins().min() >= 0.0
    out = g.get_state()
    n = wl.k + 1
    w = np.polynomial.legendre.leggauss(n)[1] / 2.0
    W = np.outer(w, w)
    for cx, cy in cells:
        o, px, py = _patch_oracle(wl, cx, cy, wl.state)
        rc, io = o.step(dt, ORACLE_TABS[wl.tableau])
        assert rc == 0 and io["restarts"] == 0
        ref = o.get_state()[:, py, px]
        got = out[:, cy, cx]
        for c in range(4):
            scale = max(np.abs(ref[c]).max(), np.abs(wl.state[c]).max() * 1e-3)
            assert np.abs(got[c] - ref[c]).max() <= 2e-5 * scale, (cx, cy, c)
            assert abs((W * got[c]).sum() - (W * ref[c]).sum()) <= 1e-6 * scale, (cx, cy, c)


@pytest.mark.parametrize("dim,k", [(1, 2), (2, 3)])
def test_mixed_state_in_and_out_of_page_locked_host_memory(dim, k):
    """The split-precision path splits a page-locked host buffer in place (its kernel reads the
    host memory) and merges into one: the same state, bit for bit, as through a device buffer and
    through a pageable (staged) host buffer."""
    from paper_2412_16002_gb300.solver import Solver

    nx, ny = (37, 1) if dim == 1 else (13, 11)
    U = inputs.random_euler(dim, nx, ny, k, seed=12, osc=0.8)
    flat = torch.from_numpy(U.reshape(-1).copy())
    pinned = flat.pin_memory()
    outs = []
    for src in (pinned, flat.cuda(), U):
        g = Solver(dim, nx, ny, k, (0.0, 1.0, 0.0, 1.0), "euler", precision="mixed")
        g.set_state(src)
        g.step(g.max_dt(0.1), "heun3")
        o_pin = torch.empty_like(flat).pin_memory()
        o_dev = torch.empty_like(flat, device="cuda")
        g.get_state(o_pin)
        g.get_state(o_dev)
        o_host = g.get_state().reshape(-1)
        assert np.array_equal(o_pin.numpy(), o_dev.cpu().numpy())
        assert np.array_equal(o_pin.numpy(), o_host)
        outs.append(o_pin.numpy().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
