"""Block domain decomposition through the CUDA library: subdomain handles with a halo ring,
the owned box masking the flag, statistics and rate, the packed cell copies of the halo
exchange, and the attempt / accept pair of the global restart decision.  The assembled owned
cells must equal the undecomposed GPU run bit for bit (FP64 and split precision), on meshes
whose cell size is not exactly representable (the subdomain takes the global mesh's).

Ranks run as threads of one process (each with its own handle) or as two processes with the
gloo transport and host-staged halos; in both the host orchestrates every exchange between
kernel launches, so no kernel waits on another."""
import os
import sys
import threading

import numpy as np
import pytest

from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _workload(case):
    if case == "sedov":
        return inputs.sedov(40, 3)  # [0, 1.1]^2: cells not exactly representable
    if case == "riemann":
        return inputs.riemann_quadrants(2, 36, 2)
    if case == "periodic":
        wl = inputs.riemann_quadrants(3, 30, 2)
        wl.bc = ("periodic",) * 4
        wl.state = inputs.random_euler(2, 30, 30, 2, seed=9, osc=0.5)
        return wl
    if case == "tube1d":
        return inputs.euler_blast_tube(300, 2)
    raise KeyError(case)


def _make_rank(wl, grid, rank, transport, precision):
    from paper_2412_16002_gb300.decomp import DomainSolver, Layout
    from paper_2412_16002_gb300.solver import Solver

    per = (wl.bc[0] == "periodic", wl.bc[2] == "periodic")
    lay = Layout(wl.dim, wl.nx, wl.ny, grid[0], grid[1], rank, per)
    dom, bc = lay.local_mesh(wl.domain, wl.bc)
    s = Solver(wl.dim, lay.nxl, lay.nyl, wl.k, dom, wl.flux, gamma=wl.gamma, bounds=wl.bounds, eps=wl.eps,
               bc=bc, bc_state=wl.bc_state, precision=precision)
    return DomainSolver(lay, s, transport, wl.domain)


def _run_rank(wl, grid, rank, transport, precision, steps):
    ds = _make_rank(wl, grid, rank, transport, precision)
    ds.set_global_state(wl.state)
    dts, rs = [], []
    for _ in range(steps):
        dt = ds.max_dt(wl.cfl)
        info = ds.step(dt, wl.tableau)
        dts.append(dt)
        rs.append(info["restarts"])
    out = ds.gather_state(), dts, rs
    ds.s.close()
    return out


def _reference(wl, precision, steps):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver.from_workload(wl, precision=precision)
    g.set_state(wl.state)
    dts, rs = [], []
    for _ in range(steps):
        dt = g.max_dt(wl.cfl)
        info = g.step(dt, wl.tableau)
        dts.append(dt)
        rs.append(info["restarts"])
    return g.get_state(), dts, rs


def _threads(wl, grid, precision, steps):
    from paper_2412_16002_gb300.decomp import LocalWorld

    world = grid[0] * grid[1]
    W = LocalWorld(world)
    res, errs = {}, []

    def go(r):
        try:
            res[r] = _run_rank(wl, grid, r, W.transport(r), precision, steps)
        except BaseException as e:
            errs.append(e)
            W.barrier.abort()

    th = [threading.Thread(target=go, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return res[0]


def _compare(got, ref):
    state, dts, rs = got
    rstate, rdts, rrs = ref
    assert dts == rdts
    assert rs == rrs
    assert np.array_equal(state, rstate), np.abs(state - rstate).max()


@pytest.mark.parametrize("case,grid,precision", [
    ("sedov", (2, 2), "fp64"),
    ("sedov", (2, 2), "mixed"),
    ("riemann", (3, 2), "fp64"),
    ("riemann", (2, 3), "mixed"),
    ("periodic", (2, 2), "fp64"),
    ("periodic", (3, 1), "mixed"),
    ("tube1d", (3, 1), "fp64"),
])
def test_thread_ranks_equal_undecomposed_gpu_run(case, grid, precision):
    wl = _workload(case)
    steps = 20
    _compare(_threads(wl, grid, precision, steps), _reference(wl, precision, steps))


@pytest.mark.parametrize("n,k,precision", [(16, 3, "fp64"), (12, 2, "fp64"), (16, 3, "mixed")])
def test_blast_restarts_together(n, k, precision):
    """Restarts (Sedov-type blasts at CFL 0.9, where the oracle halves the step in 3 of the
    first 8 steps) are decided by all subdomains together."""
    wl = inputs.sedov(n, k)
    wl.cfl = 0.9
    ref = _reference(wl, precision, 8)
    assert sum(ref[2]) > 0
    _compare(_threads(wl, (2, 2), precision, 8), ref)


def test_owned_box_masks_flag_rate_and_totals():
    """A handle whose owned box excludes a poisoned cell keeps its trial step, margins and
    totals to the owned cells, and the poisoned cell does not force a restart.  The poisoned
    cell is a corner two cells away from the owned box, so no owned cell's final stage reads
    its traces (a halo cell next to the box is, in a decomposition, an exact copy)."""
    from paper_2412_16002_gb300.solver import Solver

    wl = _workload("riemann")
    g = Solver.from_workload(wl)
    U = wl.state.copy()
    g.set_state(U)
    dt_all = g.max_dt(wl.cfl)
    # poison a corner cell with a negative density and a huge speed
    U[0, 0, 0] = -1.0
    U[1, 0, 0] = 1e6
    h = Solver.from_workload(wl)
    h.set_subdomain((2, wl.nx, 2, wl.ny), dict(dim=2, nx=wl.nx, ny=wl.ny, domain=wl.domain))
    h.set_state(U)
    assert np.isfinite(h.max_dt(wl.cfl)) and h.max_dt(wl.cfl) >= dt_all
    assert h.margins().min() >= 0.0
    assert h.step_attempt(0.5 * dt_all, wl.tableau) is False
    h.step_accept()


def _gloo_worker(rank, world, port, case, grid, precision, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2412_16002_gb300.decomp import TorchTransport

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = _run_rank(_workload(case), grid, rank, TorchTransport(), precision, steps)
        if rank == 0:
            out["res"] = res
    finally:
        dist.destroy_process_group()


def test_two_processes_gloo_host_staged_halos():
    import torch.multiprocessing as mp

    wl = _workload("riemann")
    grid, steps = (2, 1), 10
    port = 29700 + os.getpid() % 2000
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_gloo_worker, args=(2, port, "riemann", grid, "fp64", steps, out), nprocs=2,
                           join=True, start_method="spawn")
        got = out["res"]
    _compare(got, _reference(wl, "fp64", steps))
