"""Estimator conservativeness diagnostic (evaluation section and the slack
appendix): for a target rank r, sample block subsets of increasing size
uniformly at random, and compare the predicted rank-r reconstruction error
of each estimator -- the max-norm (Weyl, Thm. 1), the residual-based
(Cor. 1) and the approximate incremental (plug-in, Cor. 2) -- with the true
optimal error E_r of the concatenation; the slack is
Delta = E~_r - E_r (absolute) and also reported relative to ||M||_F.

Every value comes from the library: the three estimates from csvd_bounds,
the true error from the incremental estimator run at full rank
min(m, sum k) (no truncation, so its spectrum is the concatenation's,
Lemma 1), summed over the discarded part sum_{j > r} sigma_j^2.
"""
from __future__ import annotations

import math

import numpy as np

from . import csvd

ESTIMATORS = ("weyl", "residual", "plugin")


def true_tail_sq(blocks, r):
    """E_r^2 = sum_{j > r} sigma_j^2(M) from an untruncated incremental SVD."""
    m = int(blocks[0].shape[0])
    full = min(m, sum(int(b.shape[1]) for b in blocks))
    st = csvd.IncrSVD(m, full, "plain")
    for b in blocks:
        st.append(b)
    s = np.asarray(st.sigma(), dtype=np.float64)
    st.close()
    return float(np.sum(s[r:] ** 2))


def slack(blocks, r, sizes, trials=10, seed=0):
    """One row per (size, trial): the sampled block indices (in sampled
    order), the energy, the true error and, per estimator, its prediction
    and slack (absolute and relative to ||M||_F)."""
    rng = np.random.default_rng(seed)
    rows = []
    for size in sizes:
        for t in range(trials):
            idx = [int(i) for i in rng.choice(len(blocks), size=size, replace=False)]
            sub = [blocks[i] for i in idx]
            b = csvd.bounds(sub, r)
            energy = b["energy"]
            true = math.sqrt(max(true_tail_sq(sub, r), 0.0))
            row = dict(size=size, trial=t, blocks=idx, energy=energy, true=true)
            norm = math.sqrt(energy) if energy > 0 else 1.0
            for name in ESTIMATORS:
                est = math.sqrt(max(b[name + "_sq"], 0.0))
                row[name] = est
                row["slack_" + name] = est - true
                row["rel_slack_" + name] = (est - true) / norm
            rows.append(row)
    return rows


def summary(rows):
    """Per cluster size and estimator: min / median / max relative slack."""
    out = {}
    for size in sorted({r["size"] for r in rows}):
        sel = [r for r in rows if r["size"] == size]
        out[size] = {name: (min(r["rel_slack_" + name] for r in sel),
                            float(np.median([r["rel_slack_" + name] for r in sel])),
                            max(r["rel_slack_" + name] for r in sel))
                     for name in ESTIMATORS}
    return out


def _main():
    import argparse
    import json
    import time

    import torch

    from . import synth
    ap = argparse.ArgumentParser(description="estimator slack on a synthetic collection")
    ap.add_argument("--recipe", choices=("c1", "c2"), default="c2")
    ap.add_argument("--n-blocks", type=int, default=64)
    ap.add_argument("--r", type=int, default=None)
    ap.add_argument("--sizes", type=int, nargs="+", default=[2, 4, 8, 16])
    ap.add_argument("--trials", type=int, default=10)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    col = synth.small_c1() if a.recipe == "c1" else synth.mid_c2(n_blocks=a.n_blocks)
    r = a.r or col.meta["r"]
    blocks = [b.cuda() for b in col.blocks]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows = slack(blocks, r, a.sizes, a.trials, a.seed)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s = summary(rows)
    neg = {name: sum(1 for row in rows if row["slack_" + name] < 0) for name in ESTIMATORS}
    print(json.dumps({"recipe": a.recipe, "m": int(col.m), "r": r, "trials": a.trials,
                      "sizes": a.sizes, "seconds": dt, "negative_slack_counts": neg,
                      "rel_slack_min_median_max": {str(k): v for k, v in s.items()}}))


if __name__ == "__main__":
    _main()
