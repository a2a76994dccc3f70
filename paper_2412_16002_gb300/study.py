"""Accuracy against cost of the cRKDG variants: L1 error of the cell averages against a finer
FP64 reference, and GPU time, on a sweep of grids; times compared at matched L1 error.

Variants (all bound-preserving, on the same seeded four-quadrant Riemann problem, Q^2,
Heun-3, CFL 0.178, outflow sides):
  fp64      the method as in the paper (scaling limiter only)
  tvb       plus the plain TVB indicator and shock limiter after the final stage
  mlp       plus the learned indicator (network trained by the library's kernels)
  mixed     split precision (FP64 averages, FP32 operators), scaling limiter only

The reference is the fp64 variant (or, with `ref_precision="mixed"`, the split-precision one,
whose errors agree with FP64's to four digits on this problem) on a grid `ref_factor` times
finer than the finest grid of the sweep; its cell averages are restricted (averaged) onto each
coarse grid.  The L1 error
is the sum over components of the mean absolute difference of the averages, divided by the
same sum for the reference's averages (a relative error over the domain).  Time is the
device time of the step kernels (inner, final, indicator) over the whole run.  Oscillation
measures (what an anti-oscillation indicator is for): the total variation of the density
averages relative to the restricted reference's, and the overshoot of the density averages
beyond the reference's range.

`matched_time(curve, target)`: the time a variant needs to reach the L1 error `target`,
interpolated log-linearly between the sweep's grids (None outside its range).
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import inputs

VARIANTS = ("fp64", "tvb", "mlp", "mixed")


def _solver(variant, seed, n, tvb_M, mlp):
    from .solver import Solver

    wl = inputs.riemann_quadrants(seed, n, 2)
    kw = {}
    if variant in ("tvb", "mlp"):
        kw = dict(indicator=variant, tvb_M=tvb_M)
    if variant == "mixed":
        kw = dict(precision="mixed")
    g = Solver.from_workload(wl, **kw)
    if variant == "mlp":
        g.set_mlp(mlp)
    g.set_state(wl.state)
    return g, wl


class RunFailed(RuntimeError):
    pass


def run(variant, seed, n, t_end, tvb_M=10.0, mlp=None):
    """Advance one variant to t_end; returns (cell averages [n][n][4], device ms, wall s, steps, troubled).
    Raises RunFailed (with the step, time, trial step and the bound margins before it) if a step
    cannot restore the bounds."""
    from ._lib import CrkdgError

    g, wl = _solver(variant, seed, n, tvb_M, mlp)
    g.set_profiling(True)
    t = 0.0
    steps = troubled = 0
    t0 = time.perf_counter()
    while t < t_end:
        dt = min(g.max_dt(wl.cfl), t_end - t)
        if t + dt == t:  # the remaining interval is below the resolution of t
            break
        try:
            info = g.step(dt, wl.tableau)
        except CrkdgError as err:
            raise RunFailed(f"{variant} n={n} step {steps} t={t!r} dt={dt!r} margins={g.margins().tolist()} "
                            f"averages min={g.averages().min(axis=(0, 1)).tolist()}: {err}") from err
        t += info["dt_taken"]
        steps += 1
        troubled += info["troubled"]
    wall = time.perf_counter() - t0
    ms, _ = g.kernel_times()
    avg = g.averages()
    g.close()
    return avg, ms["inner"] + ms["final"], wall, steps, troubled


def restrict(avg, factor):
    """Averages of factor x factor blocks of fine cell averages ([ny][nx][m])."""
    ny, nx, m = avg.shape
    return avg.reshape(ny // factor, factor, nx // factor, factor, m).mean(axis=(1, 3))


def l1_error(avg, ref):
    return float(np.abs(avg - ref).mean(axis=(0, 1)).sum() / np.abs(ref).mean(axis=(0, 1)).sum())


def total_variation(rho):
    """Mean absolute jump of the density averages between neighbouring cells (x and y)."""
    return float((np.abs(np.diff(rho, axis=0)).sum() + np.abs(np.diff(rho, axis=1)).sum()) / rho.size)


def overshoot(rho, ref):
    """How far the density averages leave the range of the (restricted) reference, relative to it."""
    lo, hi = ref.min(), ref.max()
    return float(max(0.0, rho.max() - hi, lo - rho.min()) / (hi - lo))


def matched_time(curve, target):
    """curve: list of (l1, ms) for increasing grids.  Log-linear interpolation of ms at l1 = target."""
    pts = sorted(curve, key=lambda p: -p[0])  # decreasing error
    for (e0, t0), (e1, t1) in zip(pts, pts[1:]):
        if e1 <= target <= e0 and e0 > e1:
            w = (math.log(e0) - math.log(target)) / (math.log(e0) - math.log(e1))
            return math.exp(math.log(t0) + w * (math.log(t1) - math.log(t0)))
    for e, t in pts:
        if e == target:
            return t
    return None


def study(seed=7, sizes=(64, 128, 256), ref_factor=2, t_end=0.1, tvb_M=10.0, variants=VARIANTS, mlp=None,
          train=None, ref_precision="fp64"):
    """Runs the sweep; returns a dict with per-variant curves and matched-L1 times."""
    ref_n = max(sizes) * ref_factor
    ref, ref_ms, _, ref_steps, _ = run("mixed" if ref_precision == "mixed" else "fp64", seed, ref_n, t_end)
    out = {"seed": seed, "t_end": t_end, "sizes": list(sizes), "reference": {"n": ref_n, "steps": ref_steps,
                                                                            "ms": ref_ms,
                                                                            "precision": ref_precision},
           "tvb_M": tvb_M, "training": train, "variants": {}}
    for v in variants:
        rows = []
        for n in sizes:
            try:
                avg, ms, wall, steps, troubled = run(v, seed, n, t_end, tvb_M, mlp)
            except RunFailed as err:
                rows.append({"n": n, "failed": str(err)})
                continue
            rr = restrict(ref, ref_n // n)
            err = l1_error(avg, rr)
            rows.append({"n": n, "l1": err, "ms": ms, "wall_s": wall, "steps": steps, "troubled": troubled,
                         "tv_ratio": total_variation(avg[..., 0]) / total_variation(rr[..., 0]),
                         "overshoot": overshoot(avg[..., 0], rr[..., 0])})
        out["variants"][v] = rows
    base = out["variants"]["fp64"]
    matched = {}
    for v, rows in out["variants"].items():
        curve = [(r["l1"], r["ms"]) for r in rows if "l1" in r]
        matched[v] = []
        for b in (r for r in base if "l1" in r):  # at the plain method's errors: time / time of fp64
            t = matched_time(curve, b["l1"])
            matched[v].append({"l1": b["l1"], "ms": t, "speedup_vs_fp64": (b["ms"] / t) if t else None})
    out["matched"] = matched
    return out


def main():
    import argparse

    import torch

    from . import build
    from . import indicator as ind

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--sizes", default="64,128,256")
    ap.add_argument("--t-end", type=float, default=0.1)
    ap.add_argument("--ref-factor", type=int, default=2)
    ap.add_argument("--tvb-M", type=float, default=10.0)
    ap.add_argument("--ref-precision", choices=("fp64", "mixed"), default="fp64")
    args = ap.parse_args()
    build()
    torch.cuda.init()
    t0 = time.perf_counter()
    X, Y = ind.harvest_ensemble(list(range(1000, 1004)), n=256, k=2, steps=800, every=200, tvb_M=args.tvb_M)
    theta, hist = ind.train(X, Y, epochs=8)
    conf = ind.confusion(theta, X, Y)
    train = {"cells": int(Y.numel()), "loss": hist[-1], "agreement": conf["accuracy"],
             "seconds": time.perf_counter() - t0}
    del X, Y
    res = study(args.seed, tuple(int(s) for s in args.sizes.split(",")), args.ref_factor, args.t_end, args.tvb_M,
                mlp=theta, train=train, ref_precision=args.ref_precision)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
