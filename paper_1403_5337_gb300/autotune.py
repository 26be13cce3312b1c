"""Choice of the leaf size and rank cap per front size by measurement.

The many fronts of one nested-dissection tree (the batched workload) come in
a few size classes.  For each class, one representative front is solved
(hodlr_build + gmres_solve to the target residual, as the batch does) for
every leaf size and rank cap of the search grid; the setting with the least
median device time that converges is kept.  The result maps a front size to
(leaf, rank_cap) and is stored as JSON so that later runs reuse it.  All
arithmetic runs in the library; this module only times calls and keeps the
best.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import hodlr as _h

LEAVES = (64, 128, 256, 512)
RANK_CAPS = (32, 64, 128, 256, 0)   # 0: no cap (1024)


def _time_solve(ctx, A, B, leaf, cap, tol, precision, gmres_tol, reps):
    ts = []
    ok = True
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        h = _h.hodlr_build(ctx, A, leaf, tol, "aca", precision=precision, rank_cap=cap)
        _, info = _h.gmres_solve(ctx, A, B, h, tol=gmres_tol, max_iter=400)
        e1.record()
        torch.cuda.synchronize()
        h.close()
        ok = ok and bool(info.converged and np.all(info.true_relres <= gmres_tol))
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), ok


def tune(ctx, samples, tol=1e-4, precision="fp32", gmres_tol=1e-12, reps=3, leaves=LEAVES, caps=RANK_CAPS):
    """samples: {front size n: (A (n x n CUDA tensor), B (s x n CUDA tensor))}.
    Returns {n: {"leaf", "rank_cap", "ms", "table"}}: the fastest converging
    setting of the grid (leaf sizes below n only; n itself when n <= the
    smallest leaf) and every measured setting."""
    out = {}
    for n, (A, B) in sorted(samples.items()):
        table = []
        cand_leaves = [l for l in leaves if l < n] or [n]
        for leaf in cand_leaves:
            for cap in caps:
                # warm the context's block cache for this shape, then time
                _time_solve(ctx, A, B, leaf, cap, tol, precision, gmres_tol, 1)
                ms, ok = _time_solve(ctx, A, B, leaf, cap, tol, precision, gmres_tol, reps)
                table.append({"leaf": leaf, "rank_cap": cap, "ms": ms, "converged": ok})
        good = [t for t in table if t["converged"]] or table
        best = min(good, key=lambda t: t["ms"])
        out[int(n)] = {"leaf": best["leaf"], "rank_cap": best["rank_cap"], "ms": best["ms"], "table": table}
    return out


def save(choice, path):
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump({str(k): v for k, v in choice.items()}, f, indent=1)
    os.replace(tmp, path)


def load(path):
    with open(path) as f:
        return {int(k): v for k, v in json.load(f).items()}


def lookup(choice, n):
    """(leaf, rank_cap) for a front of size n: the entry of the nearest tuned size."""
    k = min(choice, key=lambda m: abs(np.log2(max(m, 1)) - np.log2(max(n, 1))))
    return choice[k]["leaf"], choice[k]["rank_cap"]
