"""Block domain decomposition of one mesh (multi-GPU path) on CPU ranks.

The ranks drive the CPU oracle through the same subdomain logic (partition, one halo
exchange per step with the inner stages recomputed on the halo, global trial step, global
restart decision) that drives the CUDA library on GPUs; the transports are torch.distributed
over gloo (separate processes) and the in-process thread transport.  The assembled state of
the owned cells must equal the undecomposed oracle run bit for bit: the inner stages are
cell-local and the final stage reads only face neighbours (Sec. 1, Compactness remark of
Sec. 3.2), so every owned cell computes exactly what it computes in the whole mesh.
"""
import os
import sys
import threading

import numpy as np
import pytest

from decomp_oracle import OracleStepper, modal_state_layout
from oracle import HEUN3, RK4, Oracle
from paper_2412_16002_gb300 import inputs
from paper_2412_16002_gb300.decomp import DomainSolver, Layout, LocalWorld, partition

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABS = {"heun3": HEUN3, "rk4": RK4}


# --------------------------------------------------------------------------- host logic


def test_partition_balanced_and_contiguous():
    for n in (1, 7, 12, 2048):
        for p in range(1, min(n, 9) + 1):
            parts = partition(n, p)
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition(3, 4)


def test_layout_neighbours_halos_and_wrap():
    # 2 x 2, periodic in x, walls in y
    L = [Layout(2, 10, 9, 2, 2, r, (True, False)) for r in range(4)]
    assert L[0].own == (0, 5, 0, 5) and L[3].own == (5, 10, 5, 9)
    assert L[0].nbr == (1, 1, None, 2)       # x wraps onto the other column, no rank below
    assert L[3].nbr == (2, 2, 1, None)
    assert L[0].halo == (1, 1, 0, 1)
    assert (L[0].nxl, L[0].nyl) == (7, 6)
    assert L[0].own_local == (1, 6, 0, 5)
    assert L[0].gx == [9, 0, 1, 2, 3, 4, 5]  # the west halo column is global column 9
    assert L[0].gy == [0, 1, 2, 3, 4, 5]
    dom, bc = L[0].local_mesh((0.0, 10.0, 0.0, 9.0), ("periodic", "periodic", "reflect", "outflow"))
    assert dom == (-1.0, 6.0, 0.0, 6.0)
    assert bc == ("outflow", "outflow", "reflect", "outflow")
    # a single block keeps the mesh's own periodic sides
    S = Layout(2, 6, 6, 1, 1, 0, (True, True))
    assert S.nbr == (None,) * 4 and S.own_local == (0, 6, 0, 6)
    assert S.local_mesh((0.0, 1.0, 0.0, 1.0), ("periodic",) * 4)[1] == ("periodic",) * 4
    # 1D, three blocks, walls
    L1 = [Layout(1, 10, 1, 3, 1, r, (False, False)) for r in range(3)]
    assert [l.nbr[:2] for l in L1] == [(None, 1), (0, 2), (1, None)]
    assert L1[1].own_local == (1, 4, 0, 1) and L1[1].gx == [3, 4, 5, 6, 7]


# --------------------------------------------------------------------------- runs


def _problem(case):
    """(dim, nx, ny, k, domain, bc, tableau, cfl, state, blast): meshes with power-of-two cells
    (hx = hy = 1/16), so a window's cell size is the global one exactly in the oracle."""
    if case == "periodic":
        dim, nx, ny, k, bc = 2, 12, 8, 2, ("periodic",) * 4
        U = inputs.random_euler(2, nx, ny, k, seed=5, osc=0.5)
        return dim, nx, ny, k, (0.0, nx / 16, 0.0, ny / 16), bc, "heun3", 0.178, U
    if case == "reflect":
        dim, nx, ny, k, bc = 2, 10, 9, 3, ("reflect", "reflect", "periodic", "periodic")
        U = inputs.random_euler(2, nx, ny, k, seed=6, osc=0.5)
        return dim, nx, ny, k, (0.0, nx / 16, 0.0, ny / 16), bc, "rk4", 0.103, U
    if case == "walls":
        dim, nx, ny, k, bc = 2, 11, 10, 2, ("reflect", "outflow", "reflect", "outflow")
        U = inputs.random_euler(2, nx, ny, k, seed=7, osc=0.5)
        return dim, nx, ny, k, (0.0, nx / 16, 0.0, ny / 16), bc, "heun3", 0.178, U
    if case == "blast":  # restarts: a hot corner at 5x the stability CFL number
        dim, nx, ny, k, bc = 2, 12, 12, 2, ("reflect", "outflow", "reflect", "outflow")
        wl = inputs.sedov(nx, k)
        return dim, nx, ny, k, (0.0, nx / 16, 0.0, ny / 16), bc, "heun3", 0.9, wl.state
    if case == "tube1d":
        wl = inputs.euler_blast_tube(48, 2)
        return 1, 48, 1, 2, (0.0, 48 / 16), ("dirichlet", "dirichlet", "outflow", "outflow"), "heun3", 0.178, wl.state
    raise KeyError(case)


def _bc_state(case):
    if case == "tube1d":
        wl = inputs.euler_blast_tube(48, 2)
        return wl.bc_state
    return None


def _run_rank(case, grid, rank, transport, steps):
    dim, nx, ny, k, dom, bc, tab, cfl, U = _problem(case)
    px, py = grid
    lay = Layout(dim, nx, ny, px, py, rank, (bc[0] == "periodic", bc[2] == "periodic"))
    ldom, lbc = lay.local_mesh(dom, bc)
    st = OracleStepper(dim, lay.nxl, lay.nyl, k, ldom, "euler", bc=lbc, bc_state=_bc_state(case))
    ds = DomainSolver(lay, st, transport, dom)
    ds.set_global_state(U)
    dts, restarts = [], []
    for _ in range(steps):
        dt = ds.max_dt(cfl)
        info = ds.step(dt, TABS[tab])
        dts.append(dt)
        restarts.append(info["restarts"])
    return ds.gather_state(), dts, restarts


def _reference(case, steps):
    dim, nx, ny, k, dom, bc, tab, cfl, U = _problem(case)
    o = Oracle(dim, nx, ny, k, dom, "euler", bc=bc, bc_state=_bc_state(case))
    o.set_state(U)
    dts, restarts = [], []
    t = 0.0
    for _ in range(steps):
        dt = o.max_dt(cfl)
        rc, info = o.step(dt, TABS[tab], t)
        assert rc == 0
        t += info["dt_taken"]
        dts.append(dt)
        restarts.append(info["restarts"])
    return modal_state_layout(o), dts, restarts


def _check(case, got, steps):
    state, dts, restarts = got
    ref, rdts, rrestarts = _reference(case, steps)
    assert dts == rdts  # the global trial step is the undecomposed one, bit for bit
    assert restarts == rrestarts
    assert np.array_equal(state, ref), np.abs(state - ref).max()
    return rrestarts


def _gloo_worker(rank, world, port, case, grid, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2412_16002_gb300.decomp import TorchTransport

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = _run_rank(case, grid, rank, TorchTransport(), steps)
        if rank == 0:
            out["res"] = res
    finally:
        dist.destroy_process_group()


def _gloo(case, grid, steps):
    world = grid[0] * grid[1]
    port = 29600 + (os.getpid() * 7 + world) % 2000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_gloo_worker, args=(world, port, case, grid, steps, out), nprocs=world, join=True)
        return out["res"]


@pytest.mark.parametrize("case,grid", [("periodic", (2, 1)), ("periodic", (2, 2)), ("reflect", (2, 2)),
                                       ("tube1d", (2, 1))])
def test_gloo_ranks_equal_undecomposed_oracle(case, grid):
    _check(case, _gloo(case, grid, 20), 20)


def _threads(case, grid, steps):
    world = grid[0] * grid[1]
    W = LocalWorld(world)
    res, errs = {}, []

    def go(r):
        try:
            res[r] = _run_rank(case, grid, r, W.transport(r), steps)
        except BaseException as e:  # surface a rank's failure in the test
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


@pytest.mark.parametrize("case,grid", [("walls", (3, 2)), ("reflect", (1, 3)), ("tube1d", (3, 1))])
def test_thread_ranks_equal_undecomposed_oracle(case, grid):
    _check(case, _threads(case, grid, 20), 20)


def test_restarts_are_decided_for_all_ranks_together():
    """A blast at 5x the stability CFL number restarts; every rank halves together, and the
    halvings and the state equal the undecomposed run's."""
    restarts = _check("blast", _threads("blast", (2, 2), 12), 12)
    assert sum(restarts) > 0
