"""Table 3 of the paper (Example 4.2, scenario II) on the GPU: 2D Euler with the exact solution
rho = 0.99 sin pi(x + y - 2t) + 1, w = (1, 1), p = 1, Q^k with the printed schemes (Q^1 midpoint,
Q^2 Heun, Q^3 RK4) at the printed fixed time steps to T = 0.1024.  The solution is 2-periodic in
x and y, so the runs use the periodic square [0, 2]^2 with twice the printed cell count (the
printed cell size) and measure the L2 error (all four components, (k+3)-point Gauss quadrature
per cell, reading C18) on [0, 1]^2, the paper's domain, where the periodic data are the exact
boundary data the paper imposes.

The errors sit a factor 3-5 below the printed ones (as the oracle's own pin finds on [0, 1]^2:
the paper does not state its nodes, initial projection or norm quadrature), so they are held to
[printed / 8, 1.5 printed]; the rates to 0.35 of the printed ones or 0.15 of k + 1."""
import math
import os

import numpy as np
import pytest

from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import build

    build()


def _rows():
    rows = []
    with open(os.path.join(GOLDEN, "table3_euler_scenario2.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _l2_error_unit_square(nodal, n2, k, t, gamma=1.4):
    """L2 error on [0, 1]^2 of the state on the n2 x n2 mesh of [0, 2]^2 (nodal values at the
    Gauss points, tensor Lagrange interpolation to (k+3)^2 Gauss points per cell)."""
    xg, _ = np.polynomial.legendre.leggauss(k + 1)
    xq, wq = np.polynomial.legendre.leggauss(k + 3)
    B = np.ones((k + 3, k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            if b != a:
                B[:, a] *= (xq - xg[b]) / (xg[a] - xg[b])
    nh, h = n2 // 2, 2.0 / n2
    U = np.asarray(nodal).reshape(4, n2, n2, k + 1, k + 1)[:, :nh, :nh]
    Uq = np.einsum("qb,pa,mijba->mijqp", B, B, U)  # [m][cy][cx][qy][qx]
    cy = np.arange(nh)[:, None, None, None]
    cx = np.arange(nh)[None, :, None, None]
    Y = (cy + 0.5 + 0.5 * xq[None, None, :, None]) * h
    X = (cx + 0.5 + 0.5 * xq[None, None, None, :]) * h
    rho = 0.99 * np.sin(np.pi * (X + Y - 2.0 * t)) + 1.0
    exact = [rho, rho, rho, 1.0 / (gamma - 1.0) + rho]  # m = rho w, E = p/(gamma-1) + rho |w|^2/2
    W = np.outer(wq, wq)[None, None] * (0.5 * h) ** 2
    return math.sqrt(sum(float(((Uq[c] - exact[c]) ** 2 * W).sum()) for c in range(4)))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_table3_on_the_gpu(k):
    from paper_2412_16002_gb300.solver import Solver

    tab = {1: "midpoint2", 2: "heun3", 3: "rk4"}[k]
    rows = [r for r in _rows() if int(r[0]) == k]
    errs = []
    for r in rows:
        nx, dt = int(r[1]), float(r[2])
        wl = inputs.scenario2(2 * nx, k)
        g = Solver.from_workload(wl)
        g.set_state(wl.state)
        t = 0.0
        for _ in range(int(round(0.1024 / dt))):
            info = g.step(dt, tab)
            assert info["restarts"] == 0
            t += dt
        assert g.margins().min() >= 0.0
        errs.append(_l2_error_unit_square(g.get_state(), 2 * nx, k, t))
    for i, r in enumerate(rows):
        printed = float(r[3])
        assert printed / 8.0 < errs[i] < printed * 1.5, (k, r, errs[i])
        if i:
            rate = math.log(errs[i - 1] / errs[i]) / math.log(2)
            assert abs(rate - float(r[4])) < 0.35 or abs(rate - (k + 1)) < 0.15, (k, rate)
