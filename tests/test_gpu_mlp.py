"""Learned troubled-cell indicator: the CUDA feature, forward, gradient and Adam kernels against
the FP64 reference MLP and the oracle's state; training on labels harvested from GPU runs.

Tolerances: the network runs in FP32, so forward probabilities are held to 2e-5 absolute,
gradients to 1e-3 of the largest gradient entry, features to 1e-5 absolute (they are
normalised to O(1))."""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import ORACLE_TABS
from oracle import Oracle, mlp
from paper_2412_16002_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16002_gb300 import _lib as L
    from paper_2412_16002_gb300 import build

    build()
    return L.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _ghost(o, avg, cx, cy, dx, dy, bc):
    """average at stencil position (cx+dx, cy+dy): outside the domain, the nearest in-domain
    cell's average with each crossed side's boundary state applied (outflow: a copy,
    reflect: the normal momentum negated)"""
    x, y = cx + dx, cy + dy
    sides = []
    if not 0 <= x < o.nx:
        if bc[0 if dx < 0 else 1] == "periodic":
            x %= o.nx
        else:
            sides.append(0 if dx < 0 else 1)
            x = cx
    if not 0 <= y < o.ny:
        if bc[2 if dy < 0 else 3] == "periodic":
            y %= o.ny
        else:
            sides.append(2 if dy < 0 else 3)
            y = cy
    v = avg[y, x].copy()
    for s in sides:
        assert bc[s] in ("outflow", "reflect")
        if bc[s] == "reflect":
            v[1 + s // 2] = -v[1 + s // 2]
    return v


def _expected_features(o, modal, bc, thr):
    """Features from the oracle's modal state: averages on the 3x3 stencil and the centre cell's
    first Legendre moments c_10 (x) and c_01 (y), through the FP64 reference feature map."""
    avg = o.averages(modal)  # [ny][nx][m]
    n, per = o.n, o.m * o.n * o.n
    out = np.zeros((o.ny * o.nx, 44))
    for cy in range(o.ny):
        for cx in range(o.nx):
            a3 = np.stack([_ghost(o, avg, cx, cy, dx, dy, bc) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=1)
            cell = cy * o.nx + cx
            sl = np.array([[modal[cell * per + c * n * n + 1], modal[cell * per + c * n * n + n]] for c in range(o.m)])
            out[cell] = mlp.features(a3, sl, thr)
    return out


@pytest.mark.parametrize("k", [2, 3])
def test_features_match_oracle_state(lib, k):
    """Features of the unlimited final stage (the state the indicator sees), 3 steps of a
    four-quadrant Riemann problem with outflow sides: GPU (FP64 features rounded to FP32)
    against the reference feature map on the oracle's state, and the plain flags exactly."""
    from paper_2412_16002_gb300.solver import Solver

    wl = inputs.riemann_quadrants(11, 12, k)
    g = Solver.from_workload(wl, indicator="tvb", tvb_M=1.0)
    o = Oracle(2, 12, 12, k, wl.domain, "euler", gamma=wl.gamma, eps=wl.eps, bc=wl.bc, indicator=True, tvb_M=1.0)
    g.set_state(wl.state)
    o.set_state(wl.state)
    g.set_harvest(True)
    t = 0.0
    for _ in range(3):
        dt = o.max_dt(wl.cfl)
        g.step(dt, wl.tableau)
        before = o.c.copy()
        rc, _ = o.step(dt, ORACLE_TABS[wl.tableau], t)
        assert rc == 0
        rc, us, _ = o.step_stages(dt, ORACLE_TABS[wl.tableau], t, modal=before)
        t += dt
        feat = g.last_features()
        ref = _expected_features(o, us[-1], wl.bc, 1.0 / 144.0)
        assert np.abs(feat - ref).max() < 1e-5
        assert np.array_equal(g.troubled_flags(), o.troubled(us[-1]))


def test_forward_matches_reference(lib):
    rng = np.random.default_rng(0)
    theta = mlp.init_params(3)
    X = rng.normal(size=(1000, 44))
    z, _ = mlp.forward(theta, X)
    ref = mlp.sigmoid(z)
    tp = torch.tensor(theta, dtype=torch.float32, device="cuda")
    tx = torch.tensor(X, dtype=torch.float32, device="cuda")
    pr = torch.empty(1000, dtype=torch.float32, device="cuda")
    assert lib.crkdg_mlp_forward(_ptr(tp), _ptr(tx), 1000, _ptr(pr), None) == 0
    torch.cuda.synchronize()
    assert np.abs(pr.cpu().numpy() - ref).max() < 2e-5


@pytest.mark.parametrize("n,scale", [(128, 1.0), (152 * 128 * 3 + 45, 1.0), (5000, 2.0)])
def test_tensor_core_forward_tiles(lib, n, scale):
    """The forward pass on the tensor cores (128-cell tiles, persistent CTAs walking several
    tiles with the next tile's features prefetched, a ragged last tile) against the FP64
    reference network: 2e-5 absolute on the probabilities, no wait ran out."""
    rng = np.random.default_rng(n)
    theta = mlp.init_params(7) * scale
    X = rng.normal(size=(n, 44)) * scale
    z, _ = mlp.forward(theta, X)
    ref = mlp.sigmoid(z)
    tp = torch.tensor(theta, dtype=torch.float32, device="cuda")
    tx = torch.tensor(X, dtype=torch.float32, device="cuda")
    pr = torch.full((n + 1,), -1.0, dtype=torch.float32, device="cuda")
    assert lib.crkdg_mlp_forward(_ptr(tp), _ptr(tx), n, _ptr(pr), None) == 0
    torch.cuda.synchronize()
    got = pr.cpu().numpy()
    assert got[n] == -1.0  # nothing written past the last row
    assert np.abs(got[:n] - ref).max() < 2e-5
    fault = C.c_int(-1)
    assert lib.crkdg_mlp_fault(C.byref(fault)) == 0 and fault.value == 0


def test_gradient_matches_reference(lib):
    rng = np.random.default_rng(1)
    theta = mlp.init_params(5)
    X = rng.normal(size=(300, 44))
    y = (rng.uniform(size=300) > 0.6).astype(float)
    gref = mlp.backward(theta, X, y)
    lref = mlp.loss(theta, X, y)
    tp = torch.tensor(theta, dtype=torch.float32, device="cuda")
    tx = torch.tensor(X, dtype=torch.float32, device="cuda")
    ty = torch.tensor(y, dtype=torch.float32, device="cuda")
    gr = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    ls = torch.zeros(1, dtype=torch.float32, device="cuda")
    assert lib.crkdg_mlp_grad(_ptr(tp), _ptr(tx), _ptr(ty), 300, _ptr(gr), _ptr(ls), None) == 0
    torch.cuda.synchronize()
    g = gr.cpu().numpy()
    assert np.abs(g - gref).max() <= 1e-3 * np.abs(gref).max()
    assert abs(float(ls.item()) - lref) < 1e-4 * max(1.0, lref)
    # one Adam step against the reference update
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    assert lib.crkdg_mlp_adam(_ptr(tp), _ptr(m), _ptr(v), _ptr(gr), 1, C.c_float(1e-3), None) == 0
    torch.cuda.synchronize()
    th_ref, _, _ = mlp.adam(theta, np.zeros_like(theta), np.zeros_like(theta), g.astype(np.float64), 1, lr=1e-3)
    assert np.abs(tp.cpu().numpy() - th_ref).max() < 1e-6


def _harvest(seeds, n=48, steps=12):
    from paper_2412_16002_gb300.solver import Solver

    X, Y = [], []
    for seed in seeds:
        wl = inputs.riemann_quadrants(seed, n, 2)
        g = Solver.from_workload(wl, indicator="tvb", tvb_M=1.0)
        g.set_state(wl.state)
        g.set_harvest(True)
        for _ in range(steps):
            g.step(g.max_dt(wl.cfl), wl.tableau)
            X.append(g.last_features())
            Y.append(g.troubled_flags().astype(np.float32))
    return np.concatenate(X), np.concatenate(Y)


def test_training_on_harvested_labels_learns_the_plain_indicator(lib):
    """Labels from the plain indicator on seeded Riemann runs (GPU), training with the project's
    own gradient and Adam kernels: the loss falls and held-out accuracy exceeds the trivial
    all-smooth classifier."""
    Xtr, Ytr = _harvest(range(1000, 1006))
    Xte, Yte = _harvest(range(2000, 2002))
    print(f"harvest: {len(Ytr)} cells, troubled fraction {Ytr.mean():.4f}")
    assert Ytr.sum() >= 100 and Ytr.mean() < 0.5
    theta = torch.tensor(mlp.init_params(7), dtype=torch.float32, device="cuda")
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    tx = torch.tensor(Xtr, device="cuda")
    ty = torch.tensor(Ytr, device="cuda")
    grad = torch.zeros_like(theta)
    loss = torch.zeros(1, device="cuda")
    n = tx.shape[0]
    bs = 8192
    first = None
    step = 0
    for epoch in range(30):
        perm = torch.randperm(n, device="cuda")
        for s0 in range(0, n, bs):
            idx = perm[s0:s0 + bs]
            xb = tx[idx].contiguous()
            yb = ty[idx].contiguous()
            grad.zero_()
            loss.zero_()
            assert lib.crkdg_mlp_grad(_ptr(theta), _ptr(xb), _ptr(yb), xb.shape[0], _ptr(grad), _ptr(loss), None) == 0
            step += 1
            assert lib.crkdg_mlp_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), step, C.c_float(2e-3), None) == 0
            if first is None:
                torch.cuda.synchronize()
                first = float(loss.item())
    grad.zero_()
    loss.zero_()
    assert lib.crkdg_mlp_grad(_ptr(theta), _ptr(tx), _ptr(ty), n, _ptr(grad), _ptr(loss), None) == 0
    torch.cuda.synchronize()
    last = float(loss.item())  # mean loss over the whole training set
    assert last < 0.5 * first
    te = torch.tensor(Xte, device="cuda")
    pr = torch.empty(te.shape[0], device="cuda")
    assert lib.crkdg_mlp_forward(_ptr(theta), _ptr(te), te.shape[0], _ptr(pr), None) == 0
    torch.cuda.synchronize()
    acc = float(((pr.cpu().numpy() > 0.5) == (Yte > 0.5)).mean())
    base = max(Yte.mean(), 1 - Yte.mean())
    print(f"held-out accuracy {acc:.4f} (all-smooth classifier {base:.4f}); loss {first:.4f} -> {last:.4f}")
    assert acc > base + 0.5 * (1 - base), (acc, base)
