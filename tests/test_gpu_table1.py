"""Table 1 of the paper (Example 4.1) on the GPU: 1D linear advection u_t + u_x = 0 on [0, 1],
u = sin 2 pi (x - t) + 2, bounds [1, 3], to T = 0.1024 at the printed fixed time steps, with the
printed schemes: P^1 with the explicit midpoint rule (eq. cRKDG2), P^2 with Heun's method
(eq. cRKDG3), P^3 with the classic RK4 (eq. cRKDG4).  In 1D the P^k and Q^k spaces coincide.
The solution is 1-periodic, so periodic sides give the exact boundary data.

The L2 errors are taken with (k+3)-point Gauss quadrature per cell (reading C18) and held to
the band the oracle's own pin uses against the printed values (the paper does not state its
nodes, initial projection or error quadrature), the convergence rates to 0.2 of the printed
ones (or of k+1), and bounds [1, 3] hold on every S_K point at the end."""
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
    with open(os.path.join(GOLDEN, "table1_linear_advection.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _l2_error(nodal, nx, k, t):
    """L2 norm of u_h - u(t) on [0, 1] by (k+3)-point Gauss quadrature per cell, u_h the
    Lagrange interpolant of the nodal values at the k+1 Gauss points."""
    xg, _ = np.polynomial.legendre.leggauss(k + 1)
    xq, wq = np.polynomial.legendre.leggauss(k + 3)
    # Lagrange basis at the quadrature points: B[q, a] = l_a(xq[q])
    B = np.ones((k + 3, k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            if b != a:
                B[:, a] *= (xq - xg[b]) / (xg[a] - xg[b])
    u = np.asarray(nodal).reshape(nx, k + 1) @ B.T  # [cell][q]
    h = 1.0 / nx
    x = (np.arange(nx)[:, None] + 0.5 + 0.5 * xq[None, :]) * h
    err = u - (np.sin(2 * np.pi * (x - t)) + 2.0)
    return math.sqrt(float((err ** 2 * wq[None, :]).sum() * 0.5 * h))


def _run(k, nx, dt):
    from paper_2412_16002_gb300.solver import Solver

    g = Solver(1, nx, 1, k, (0.0, 1.0), "advection", velocity=(1.0, 0.0), bounds=(1.0, 3.0))
    X = inputs.node_coords(1, nx, 1, k, (0.0, 1.0))
    g.set_state((np.sin(2 * np.pi * X) + 2.0)[None])
    nsteps = int(round(0.1024 / dt))
    t, done, restarts = g.advance_fixed(nsteps, dt, 0.1024, {1: "midpoint2", 2: "heun3", 3: "rk4"}[k])
    assert done == nsteps and restarts == 0 and abs(t - 0.1024) < 1e-12
    assert g.margins().min() >= 0.0
    return _l2_error(g.get_state(), nx, k, t)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_table1_on_the_gpu(k):
    rows = [r for r in _rows() if int(r[0]) == k]
    errs = [_run(k, int(r[1]), float(r[2])) for r in rows]
    for i, r in enumerate(rows):
        printed = float(r[3])
        assert printed / 3.5 < errs[i] < printed * 1.5, (k, r, errs[i])
        if i:
            rate = math.log(errs[i - 1] / errs[i]) / math.log(2)
            assert abs(rate - float(r[4])) < 0.2 or abs(rate - (k + 1)) < 0.12, (k, rate)
