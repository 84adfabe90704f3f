"""Autotuner for the batched merge scoring.

The one launch parameter of the mixed form that changes speed but not the
arithmetic is where the eigen core's three launch classes meet: cores of
size n = r_t + k up to ``edge_small`` run four to an SM (4 warps each), up
to ``edge_medium`` two to an SM (8 warps), larger ones alone (16 warps).
Which split is fastest depends on the batch's core-size mix (it decides
how well each launch fills the SMs and how many tiles spill to the global
workspace).  ``autotune`` times csvd_score over a grid of edges on the
caller's own batch (CUDA events, after a warm-up call), installs the
fastest and, when ``CSVD_TUNE_CACHE`` names a file, records it under a key
of the device, m, the state ranks and the core-size histogram (buckets of
64), so that the next process with the same shape skips the search.
"""
from __future__ import annotations

import ctypes as C
import json
import os

DEFAULT = (192, 320)
SMALL = (128, 160, 192, 224, 256, 288)
MEDIUM = (256, 288, 320, 384, 448, 480)


def key(device_name, m, ranks, core_sizes):
    """Cache key: device, m, the distinct state ranks and the histogram of
    core sizes in buckets of 64 (fractions rounded to 1/16)."""
    hist = {}
    for n in core_sizes:
        hist[n // 64] = hist.get(n // 64, 0) + 1
    tot = max(1, len(core_sizes))
    h = ",".join(f"{b}:{round(16 * c / tot)}" for b, c in sorted(hist.items()))
    return f"{device_name}|m={m}|r={','.join(str(r) for r in sorted(set(ranks)))}|n={h}"


def load_cache(path=None):
    """The cache as a dict (empty when the file is missing or unreadable)."""
    path = path or os.environ.get("CSVD_TUNE_CACHE")
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
        return {k: tuple(v) for k, v in data.items()
                if isinstance(v, (list, tuple)) and len(v) == 2}
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=None):
    path = path or os.environ.get("CSVD_TUNE_CACHE")
    if not path:
        return False
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({k: list(v) for k, v in cache.items()}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return True


def get():
    from . import csvd
    a, b = C.c_int32(), C.c_int32()
    csvd._check(csvd.lib(False).csvd_tune_get(C.byref(a), C.byref(b)))
    return a.value, b.value


def set_edges(edges):
    from . import csvd
    csvd._check(csvd.lib(False).csvd_tune_set(int(edges[0]), int(edges[1])))


def candidates(core_sizes):
    """Edge pairs worth timing: the default, and every grid pair whose
    classes each receive some cores or that moves a populated boundary."""
    out = [DEFAULT]
    for a in SMALL:
        for b in MEDIUM:
            if a < b and (a, b) not in out:
                out.append((a, b))
    return out


def autotune(batch, core_sizes, m, ranks, steps=2, cache_path=None, grid=None):
    """Time ``batch`` (a csvd.ScoreBatch) under each candidate edge pair and
    install the fastest.  Returns dict(edges, ms, default_ms, tried, cached)."""
    import torch
    from . import csvd
    dev = torch.cuda.get_device_name()
    k = key(dev, m, ranks, core_sizes)
    cache = load_cache(cache_path)
    if k in cache:
        set_edges(cache[k])
        return dict(edges=tuple(cache[k]), ms=None, default_ms=None, tried=0, cached=True, key=k)
    stream = torch.cuda.current_stream()
    times = {}
    for edges in (grid or candidates(core_sizes)):
        set_edges(edges)
        batch.run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            batch.run()
        e1.record(stream)
        e1.synchronize()
        times[edges] = e0.elapsed_time(e1) / steps
    best = min(times, key=lambda e: (times[e], e != DEFAULT))
    set_edges(best)
    cache[k] = best
    save_cache(cache, cache_path)
    return dict(edges=best, ms=times[best], default_ms=times.get(DEFAULT), tried=len(times),
                cached=False, key=k)
