"""Clustering on synthetic stand-ins with the shapes of the paper's four
datasets (evaluation section, dataset table): the number of blocks, their
size m x n_i, the target rank r and the error constraint eps are the
paper's; the contents are not (the datasets are not available).  The paper
says only that the datasets differ in spectral decay and in how well their
blocks align, so each stand-in is a latent-subspace mixture (synth.py) with
its own decay, subspace count and noise, stated in SHAPES.  The k = 1 shape
gets the least structure (many latent subspaces, heavy noise) and the
PDE-shaped one the most (few subspaces, fast decay).

``run`` clusters one stand-in with one algorithm and sort order, then
performs the final decomposition of every cluster (rank-r basis of the
cluster, csvd_reconstruct) and reports the clustering wall time, the
compression ratio, the number of clusters and the largest true relative
reconstruction error, which the max-norm and residual algorithms guarantee
to be at most eps.
"""
from __future__ import annotations

import math
import time

import torch

from . import csvd, synth

SHAPES = {
    # blocks, m, n_i, r, eps | latent subspaces (as a fraction of the blocks,
    # or a count), their dimension, decay per index, noise
    "qualcomm": dict(K=2468, m=12800, k=20, r=20, eps=0.05, sub=0.5, d=12, decay=0.85, noise=1e-3),
    "bigearthnet": dict(K=10000, m=1440, k=20, r=20, eps=0.05, sub=0.5, d=12, decay=0.85,
                        noise=1e-3),
    "pdebench": dict(K=5000, m=3072, k=67, r=67, eps=0.05, sub=32, d=48, decay=0.75, noise=1e-4),
    "smolvlm": dict(K=333760, m=768, k=1, r=32, eps=0.2, sub=1 / 64, d=24, decay=0.9, noise=5e-2),
}


def make(name, scale=1.0, seed=0, device="cuda"):
    """The stand-in's blocks (views into one pool, rows padded to 4 floats)."""
    p = SHAPES[name]
    K = max(2, int(round(p["K"] * scale)))
    n_sub = p["sub"] if isinstance(p["sub"], int) else max(1, int(round(K * p["sub"])))
    bases = synth.latent_bases(p["m"], p["d"], n_sub, seed)
    spec = [p["decay"] ** i for i in range(p["d"])]
    blocks, latent, pool = synth.latent_mixture(p["m"], [p["k"]] * K, bases, spec, p["noise"],
                                                seed + 1, w_max=0.3, device=device, ld_align=4)
    return blocks, pool


def make_config5(scale=1.0, seed=0, device="cuda"):
    """The differentiation + clustering collection (synth.grad_c5): 1024
    blocks of 2048 x 256 from 32 latent subspaces of dimension 48 with a
    spectral gap at r = 128, eps = 0.05; ``scale`` shrinks the block count."""
    n = max(8, int(round(1024 * scale)))
    w = synth.grad_c5(seed=seed, device=device, n_blocks=n)
    return w["blocks"], dict(K=n, m=w["m"], k=256, r=w["r"], eps=w["eps"]), w["latent"]


def run(name, algo="approx", sort_mode="frobenius", scale=1.0, precision="mixed", seed=0,
        decompose=True):
    latent = None
    if name == "config5":
        blocks, p, latent = make_config5(scale, seed)
    else:
        p = SHAPES[name]
        blocks, pool = make(name, scale, seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = csvd.cluster(blocks, p["r"], p["eps"], algo, sort_mode, precision)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = dict(shape=name, blocks=len(blocks), m=p["m"], k=p["k"], r=p["r"], eps=p["eps"],
               algo=algo, sort=sort_mode, precision=precision, cluster_seconds=wall,
               clusters=res["n_clusters"], compression_ratio=res["compression_ratio"])
    if latent is not None:
        # how many latent subspaces each cluster mixes (their blocks' primary ones)
        mix = {}
        for lab, c in zip(res["labels"], latent):
            mix.setdefault(lab, set()).add(c)
        out.update(max_subspaces_per_cluster=max(len(v) for v in mix.values()),
                   clusters_per_subspace=max(sum(1 for v in mix.values() if c in v)
                                             for c in set(latent)))
    if decompose:
        # the final decomposition uses the cluster's rank-r truncated SVD:
        # the incremental estimator at a working rank r + 16, refined by two
        # subspace-iteration sweeps, then the explicit residuals
        groups = {}
        for i, lab in enumerate(res["labels"]):
            groups.setdefault(lab, []).append(i)
        t1 = time.perf_counter()
        worst, num, den = 0.0, 0.0, 0.0
        for members in groups.values():
            sub = [blocks[i] for i in members]
            U = csvd.top_basis(sub, p["r"], p["r"] + 16, refine=2)
            d = csvd.reconstruct(U, [1.0] * U.shape[1], sub, want_v=False)
            worst = max(worst, d.rel_error)
            num += float(d.resid_sq.sum())
            den += float(d.energy.sum())
        torch.cuda.synchronize()
        out.update(decompose_seconds=time.perf_counter() - t1, max_cluster_rel_error=worst,
                   overall_rel_error=math.sqrt(num / den) if den > 0 else 0.0)
    return out


def _main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="clustering on paper-shaped stand-ins")
    ap.add_argument("--shape", choices=sorted(SHAPES) + ["config5"], default="qualcomm")
    ap.add_argument("--algo", choices=("weyl", "residual", "approx"), default="approx")
    ap.add_argument("--sort", choices=("frobenius", "residual"), default="frobenius")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--precision", choices=("plain", "mixed"), default="mixed")
    ap.add_argument("--no-decompose", action="store_true")
    a = ap.parse_args()
    print(json.dumps(run(a.shape, a.algo, a.sort, a.scale, a.precision,
                         decompose=not a.no_decompose)))


if __name__ == "__main__":
    _main()
