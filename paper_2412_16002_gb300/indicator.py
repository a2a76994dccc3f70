"""Learned troubled-cell indicator: training data from GPU runs and training on the GPU.

The network (44 -> 64 -> 64 -> 1, ReLU, sigmoid, FP32) classifies a cell from the
normalised cell averages of its 3x3 neighbourhood and its two first Legendre moments
per component.  Its labels are the decisions of the plain TVB-minmod indicator on the
unlimited final-stage state of each step; both are harvested from seeded four-quadrant
Riemann runs through the solver's own step (features and flags never leave the
device).  Training runs the library's gradient and Adam kernels (crkdg_mlp_grad,
crkdg_mlp_adam); this module only orders the calls.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib as L
from . import inputs

NIN, NH = 44, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def init_params(seed=0, device="cuda"):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases; FP32 on the device."""
    import torch

    gen = torch.Generator().manual_seed(seed)
    parts = []
    for shape, fan_in in (((NH, NIN), NIN), ((NH,), 0), ((NH, NH), NH), ((NH,), 0), ((NH,), NH), ((1,), 0)):
        if fan_in:
            lim = math.sqrt(6.0 / fan_in)
            parts.append((torch.rand(shape, generator=gen, dtype=torch.float64) * 2.0 - 1.0).mul_(lim).reshape(-1))
        else:
            parts.append(torch.zeros(int(np.prod(shape)), dtype=torch.float64))
    theta = torch.cat(parts).to(device=device, dtype=torch.float32)
    assert theta.numel() == NPARAM
    return theta


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def harvest(seeds, n=256, k=2, steps=60, every=4, tvb_M=10.0, cfl=None, device="cuda"):
    """Labelled features from seeded Riemann runs: every `every`-th of `steps` steps of each
    seed contributes all n*n cells.  Returns (X [N,44] float32, Y [N] float32) on the device."""
    import torch

    from .solver import Solver

    X, Y = [], []
    for seed in seeds:
        wl = inputs.riemann_quadrants(seed, n, k)
        g = Solver.from_workload(wl, indicator="tvb", tvb_M=tvb_M)
        g.set_state(wl.state)
        g.set_harvest(True)
        flags = torch.empty(n * n, dtype=torch.int32, device=device)
        for s in range(steps):
            g.step(g.max_dt(cfl or wl.cfl), wl.tableau)
            if (s + 1) % every == 0:
                feat = torch.empty((n * n, NIN), dtype=torch.float32, device=device)
                g.last_features(feat)
                g._chk(g.lib.crkdg_troubled_flags(g.h, _ptr(flags), 1))
                X.append(feat)
                Y.append(flags.to(torch.float32))
        g.close()
    return torch.cat(X), torch.cat(Y)


def harvest_ensemble(seeds, n=256, k=2, steps=60, every=4, tvb_M=10.0, device="cuda"):
    """As harvest, from one ensemble run of the seeded Riemann problems (all n x n, degree k,
    plain TVB indicator, each problem at its own trial step): every `every`-th of `steps`
    ensemble steps contributes every cell of every problem.  The ensemble reproduces each
    problem's single-handle run bit for bit, so the labelled set is the same as harvest's."""
    import torch

    from .ensemble import Ensemble, riemann_problem

    probs = [riemann_problem(s, n, k) for s in seeds]
    for p in probs:
        p["t_end"] = 1e30
    ens = Ensemble(probs, indicator="tvb", tvb_M=tvb_M)
    for i, s in enumerate(seeds):
        ens.set_state(i, inputs.riemann_quadrants(s, n, k).state)
    ens.set_harvest(True)
    per_problem = [[] for _ in seeds]
    flags = torch.empty(n * n, dtype=torch.int32, device=device)
    for s in range(steps):
        ens.step()
        if (s + 1) % every == 0:
            for i in range(len(seeds)):
                feat = torch.empty((n * n, NIN), dtype=torch.float32, device=device)
                ens.last_features(i, feat)
                ens.troubled_flags(i, flags)
                per_problem[i].append((feat, flags.to(torch.float32)))
    ens.close()
    X = [f for rows in per_problem for f, _ in rows]  # problem by problem, as harvest orders them
    Y = [y for rows in per_problem for _, y in rows]
    return torch.cat(X), torch.cat(Y)


def loss_and_grad(lib, theta, X, Y, grad=None, loss=None):
    import torch

    grad = torch.zeros_like(theta) if grad is None else grad.zero_()
    loss = torch.zeros(1, dtype=torch.float32, device=theta.device) if loss is None else loss.zero_()
    st = lib.crkdg_mlp_grad(_ptr(theta), _ptr(X), _ptr(Y), X.shape[0], _ptr(grad), _ptr(loss),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != L.OK:
        raise L.CrkdgError(st, "crkdg_mlp_grad failed")
    return loss, grad


def predict(theta, X, lib=None):
    """Troubled probabilities of the rows of X (device)."""
    import torch

    lib = lib or L.load()
    prob = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    st = lib.crkdg_mlp_forward(_ptr(theta), _ptr(X), X.shape[0], _ptr(prob),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != L.OK:
        raise L.CrkdgError(st, "crkdg_mlp_forward failed")
    return prob


def train(X, Y, epochs=20, batch=8192, lr=2e-3, seed=0, theta=None):
    """Mini-batch Adam on the mean binary cross-entropy.  Returns (theta, losses per epoch),
    each loss the mean over the whole training set after that epoch."""
    import torch

    lib = L.load()
    theta = init_params(seed, X.device) if theta is None else theta.clone()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.zeros_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    gen = torch.Generator(device=X.device).manual_seed(seed)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    step = 0
    history = []
    n = X.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=gen)
        for s0 in range(0, n, batch):
            idx = perm[s0:s0 + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            loss_and_grad(lib, theta, xb, yb, grad, loss)
            step += 1
            st = lib.crkdg_mlp_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), step, C.c_float(lr), stream)
            if st != L.OK:
                raise L.CrkdgError(st, "crkdg_mlp_adam failed")
        full, _ = loss_and_grad(lib, theta, X, Y, grad, loss)
        history.append(float(full.item()))
    return theta, history


def confusion(theta, X, Y, lo=0.4, hi=0.6):
    """Agreement of the learned flags (the plain flag where lo <= p <= hi) with the plain
    flags Y: returns dict with accuracy, false positives/negatives and the undecided share."""
    p = predict(theta, X)
    undecided = (p >= lo) & (p <= hi)
    flag = (p > hi) | (undecided & (Y > 0.5))
    y = Y > 0.5
    return {
        "accuracy": float((flag == y).float().mean().item()),
        "false_pos": int((flag & ~y).sum().item()),
        "false_neg": int((~flag & y).sum().item()),
        "undecided": float(undecided.float().mean().item()),
        "positives": int(y.sum().item()),
        "cells": int(Y.numel()),
    }


def main():
    """Harvest labelled cells from seeded Riemann runs, train the network, save its parameters."""
    import argparse
    import time

    import torch

    from . import build

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--seeds", default="1000,1001,1002,1003")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--every", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--tvb-M", type=float, default=10.0)
    ap.add_argument("--out", default=None, help="write the FP32 parameters here (numpy .npy)")
    args = ap.parse_args()
    build()
    t0 = time.perf_counter()
    X, Y = harvest([int(s) for s in args.seeds.split(",")], n=args.n, steps=args.steps, every=args.every,
                   tvb_M=args.tvb_M)
    theta, hist = train(X, Y, epochs=args.epochs)
    conf = confusion(theta, X, Y)
    torch.cuda.synchronize()
    print({"cells": int(Y.numel()), "troubled_fraction": float(Y.mean().item()), "loss": hist,
           "agreement": conf["accuracy"], "seconds": time.perf_counter() - t0})
    if args.out:
        np.save(args.out, theta.cpu().numpy())


if __name__ == "__main__":
    main()
