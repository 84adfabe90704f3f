"""Benchmark: merge evaluations/s of batched uneven merge scoring on GB300.

Workload (one step = one pass of the whole hot path over one batch): 64
cluster states (m = 2048, rank r = 64, each built from 8 appends, not timed)
and 4096 candidate blocks of widths uniform in [16, 512]; every candidate is
scored against its state: projection, Gram / residual, core spectrum,
truncation, tail estimate and accept flag (Alg. 3 step 3).  Inputs (8.9 GB)
exceed the 129 MB L2, so no flush is needed between steps.

Reported: device-resident throughput (``value``), the same through the
public API with host<->device copies (``e2e``), the plain FP32 form of the
same evaluations, the dominant kernel's roofline from CUDA events recorded
around its launches, SM clocks sampled during the timed region, and the
FP64 oracle on a bounded sample on the host cores (``cpu_baseline``).

``--impl reference`` times the oracle alone on the same workload (a bounded
sample per step) and prints its own line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "merge evaluations/s (incremental rank-r SVD) vs plain FP32 at <=1e-4 rel err"
UNIT = "merge evals/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(ms_local, units_local, world):
    """Whole-job throughput of a weakly scaled run: every rank processes
    ``units_local`` units (its own shard, no exchange on the data path) in
    ``ms_local`` ms; the job takes as long as its slowest rank.  Returns
    (units per second over all ranks, slowest rank's ms).  With world > 1
    the caller has initialised torch.distributed (NCCL on GPUs, gloo on CPU)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t)
    return world * units_local / (ms / 1000.0), ms


def _work_per_candidate(m, rt, k):
    """Algorithmic work of one mixed-form merge evaluation."""
    n = rt + k
    return dict(
        gram_flops=2.0 * m * rt * k + 1.0 * m * k * (k + 1),
        gram_bytes=4.0 * m * k + 4.0 * m * rt,
        core_flops=(4.0 / 3.0) * n ** 3,
    )


def _tc_issued_flops(m, rt, k, tile=128, kstep=32, parts=6):
    """bf16 tensor-core flops the Gram kernel issues for one candidate: every
    128 x 128 output tile (P tiles over U's rt columns, the upper tiles of
    A^T A) runs M = 128, N = its valid columns rounded up to 16, over the m
    rows rounded up to the 32-row stage, six MMAs per product."""
    mp = -(-m // kstep) * kstep
    f = 0.0
    for c0 in range(0, k, tile):
        nfit = min(tile, -(-(k - c0) // 16) * 16)
        rows = (-(-rt // tile)) + (c0 // tile + 1)  # P row tiles + G row tiles at or above c0
        f += rows * 2.0 * tile * nfit * mp * parts
    return f


def _time_form(csvd, states, cand_state, cands, eps, form, steps, stream, ref):
    """CUDA-event time of ``steps`` csvd_score calls in one form after one
    untimed call; with ``ref`` (a ScoreBatch of the same candidates), the
    largest relative difference of E~ and whether the accept flags agree."""
    import torch
    b = csvd.ScoreBatch(states, cand_state, cands, eps, form)
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.run()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"value": len(cands) / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms, "steps": steps}
    if ref is not None:
        out["max_tail_rel_diff_vs_mixed"] = float(((b.tail.sqrt() - ref.tail.sqrt()).abs()
                                                   / ref.tail.sqrt().clamp_min(1e-300)).max())
        out["accept_agree"] = bool((b.accept == ref.accept).all())
    del b
    return out


def rank_legs(csvd, synth, ranks, rank, steps):
    """The batched-scoring workload at other state ranks: mixed form against
    the same-algorithm FP32 comparator, device-resident inputs."""
    import torch
    out = {}
    for r in ranks:
        w = synth.scoring_c4(r=r, seed=rank, device="cuda")
        states = []
        for blocks in w["states"]:
            st = csvd.IncrSVD(w["m"], r)
            for b in blocks:
                st.append(b)
            states.append(st)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        mixed = _time_form(csvd, states, w["cand_state"], w["candidates"], w["eps"], "mixed",
                           steps, stream, None)
        ref = csvd.ScoreBatch(states, w["cand_state"], w["candidates"], w["eps"], "mixed").run()
        fp32 = _time_form(csvd, states, w["cand_state"], w["candidates"], w["eps"], "gram_fp32",
                          steps, stream, ref)
        out[f"r{r}"] = {"mixed": mixed["value"], "mixed_ms_per_step": mixed["ms_per_step"],
                        "plain_fp32": fp32["value"], "plain_fp32_ms_per_step": fp32["ms_per_step"],
                        "speedup": mixed["value"] / fp32["value"],
                        "max_tail_rel_diff": fp32["max_tail_rel_diff_vs_mixed"],
                        "accept_agree": fp32["accept_agree"], "steps": steps,
                        "n_candidates": len(w["candidates"])}
        del ref
        for st in states:
            st.close()
        del w, states
        torch.cuda.empty_cache()
    return out


def c2_leg(csvd, synth, steps, oracle_samples):
    """The mid-size recipe (256 blocks 1024 x 128, 16 latent subspaces, r = 64)
    at eps in {0.02, 0.05, 0.1}: 16 states (blocks c, c + 16, c + 32 of
    subspace c), every other block scored against its own subspace's state
    and the next one's; mixed form against the same-algorithm FP32
    comparator and the residual + Jacobi form; accept counts per eps and
    the oracle's E~ on a sample that includes same-subspace merges."""
    import numpy as np
    import torch
    from oracle import incremental as oinc
    col = synth.mid_c2(device="cuda")
    m, r = col.m, col.meta["r"]
    groups = [[c, c + 16, c + 32] for c in range(16)]
    states = []
    for g in groups:
        st = csvd.IncrSVD(m, r)
        for j in g:
            st.append(col.blocks[j])
        states.append(st)
    rest = [j for j in range(48, len(col.blocks))]
    cands, cs = [], []
    for j in rest:
        c = j % 16
        cands += [col.blocks[j], col.blocks[j]]
        cs += [c, (c + 1) % 16]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    out = {"workload": f"{len(states)} states (3 blocks each) x {len(cands)} evaluations, m={m}, "
                       f"k=128, r={r}", "n_candidates": len(cands)}
    ref = csvd.ScoreBatch(states, cs, cands, 0.05, "mixed").run()
    forms = {}
    for form in ("mixed", "gram_fp32", "plain"):
        forms[form] = _time_form(csvd, states, cs, cands, 0.05, form, steps, stream,
                                 None if form == "mixed" else ref)
    out["mixed"] = forms["mixed"]["value"]
    out["plain_fp32"] = forms["gram_fp32"]["value"]
    out["plain_fp32_jacobi"] = forms["plain"]["value"]
    out["speedup"] = forms["mixed"]["value"] / forms["gram_fp32"]["value"]
    out["speedup_vs_jacobi"] = forms["mixed"]["value"] / forms["plain"]["value"]
    tails = ref.tail.cpu().numpy()
    energies = []
    per_eps = {}
    # oracle sample: same-subspace merges (small tails) and cross-subspace ones
    rng = np.random.default_rng(5)
    idx = sorted(set([int(i) for i in rng.choice(len(cands), oracle_samples, replace=False)] +
                     list(range(0, 2 * oracle_samples, 2))))
    cache, worst, rels = {}, 0.0, {}
    for i in idx:
        s_ = cs[i]
        if s_ not in cache:
            st = states[s_]
            te = st.tail_error()
            cache[s_] = oinc.IncrementalSVD(m, r, st.basis().double().cpu().numpy(),
                                            st.sigma().astype(np.float64), te["energy"],
                                            te["tail_sq"])
        s_o, t_o, a_o, nxt = cache[s_].evaluate(cands[i].cpu(), 0.05)
        worst = max(worst, abs(math.sqrt(tails[i]) - math.sqrt(nxt[3])) / math.sqrt(nxt[3]))
        rels[i] = math.sqrt(nxt[3] / nxt[2])
    for eps in (0.02, 0.05, 0.1):
        b = csvd.ScoreBatch(states, cs, cands, eps, "mixed").run()
        acc = b.accept.cpu().numpy()
        agree = sum(int(bool(acc[i]) == (rels[i] <= eps)) for i in idx
                    if abs(rels[i] - eps) > 1e-3 * eps)
        boundary = [i for i in idx if abs(rels[i] - eps) <= 1e-3 * eps]
        per_eps[str(eps)] = {"accepted": int(acc.sum()), "sampled_accept_agree": agree,
                             "sampled_boundary": boundary}
        del b
    out["per_eps"] = per_eps
    out["sampled"] = len(idx)
    out["sampled_rel_tail_range"] = [min(rels.values()), max(rels.values())]
    out["max_tail_rel_err"] = worst
    del ref
    for st in states:
        st.close()
    return out


def cpu_baseline(w, eps, budget_s=15.0, max_evals=64):
    """Oracle (FP64 numpy) merge evaluations on a bounded sample of the same
    workload: the states of the first candidates are rebuilt on the CPU
    (untimed), then evaluations are timed until the budget is spent."""
    import torch
    from oracle import incremental as oinc

    m, r = w["m"], w["r"]
    need = sorted(set(w["cand_state"][:max_evals]))
    states = {}
    for s in need[:2]:
        st = oinc.IncrementalSVD(m, r)
        for b in w["states"][s]:
            st.append(b.cpu())
        states[s] = st
    idx = [i for i in range(min(max_evals, len(w["candidates"]))) if w["cand_state"][i] in states]
    blocks = {i: w["candidates"][i].cpu().double().numpy() for i in idx}
    t0 = time.perf_counter()
    done = 0
    for i in idx:
        states[w["cand_state"][i]].evaluate(blocks[i], eps)
        done += 1
        if time.perf_counter() - t0 > budget_s and done >= 4:
            break
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max((p.get("num_threads", 1) for p in threadpool_info()), default=os.cpu_count())
    except Exception:
        cores = os.cpu_count()
    ks = [w["candidates"][i].shape[1] for i in idx[:done]]
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} merge evaluations (m=2048, r={r}, k in {min(ks)}..{max(ks)}) "
                      f"against 2 rebuilt states, FP64 numpy, {dt:.1f} s"}


def run_reference(args):
    """The oracle timed as it stands on the host cores, same workload."""
    import torch
    from paper_2601_11626_gb300 import synth
    from oracle import incremental as oinc

    w = synth.scoring_c4(r=args.r, n_states=args.n_states, per_state=args.per_state, device="cpu")
    m, r, eps = w["m"], w["r"], w["eps"]
    st = oinc.IncrementalSVD(m, r)
    for b in w["states"][0]:
        st.append(b)
    cands = [i for i in range(len(w["candidates"])) if w["cand_state"][i] == 0]
    blocks = [w["candidates"][i].double().numpy() for i in cands]
    per_step = max(1, args.ref_sample)
    k = 0
    for _ in range(args.warmup):
        st.evaluate(blocks[k % len(blocks)], eps)
        k += 1
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        for _ in range(per_step):
            st.evaluate(blocks[k % len(blocks)], eps)
            k += 1
            n += 1
    dt = time.perf_counter() - t0
    v = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched uneven merge scoring (oracle sample)", "m": m, "r": r,
                       "k_range": [16, 512], "sample_per_step": per_step},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": v, "unit": UNIT,
                             "sample": f"{per_step} evaluations per step against one state"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


K1_SHAPE = dict(n_states=256, per_state=256)


def _k1_work(m, rt, r_new):
    """Algorithmic work of one one-column evaluation: p = U^T a (2 m r_t),
    ||a||^2 (2 m) and r_new roots of the arrowhead's secular equation at 4
    evaluations each (a fast-converging zero finder), 6 flops per term of the
    O(r_t) secular sum and its derivative; bytes: the candidate and its
    outputs."""
    return dict(flops=2.0 * m * rt + 2.0 * m + 4.0 * r_new * 6.0 * rt,
                bytes=4.0 * m + 17.0 + 4.0 * r_new)


def run_reference_k1(args):
    """The oracle on one-column candidates, timed on the host cores."""
    from paper_2601_11626_gb300 import synth
    from oracle import incremental as oinc

    w = synth.scoring_k1(n_states=2, per_state=64, device="cpu")
    m, r, eps = w["m"], w["r"], w["eps"]
    st = oinc.IncrementalSVD(m, r)
    st.append(w["states"][0][0])
    rows = [w["Xt"][j].double().numpy().reshape(m, 1) for j in range(64)]
    per_step = max(1, args.ref_sample) * 8
    k = 0
    for _ in range(args.warmup):
        st.evaluate(rows[k % len(rows)], eps)
        k += 1
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        for _ in range(per_step):
            st.evaluate(rows[k % len(rows)], eps)
            k += 1
            n += 1
    dt = time.perf_counter() - t0
    v = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "one-column merge scoring (oracle sample)", "m": m, "r": r,
                       "k": 1, "sample_per_step": per_step},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": v, "unit": UNIT,
                             "sample": f"{per_step} one-column evaluations per step, one state"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_k1(args, world, rank, local):
    """One-column (k = 1) merge scoring: 256 states (m = 768, r = 32, each
    built from one 768 x 64 block, not timed) and 65,536 candidate vectors,
    the rows of one matrix, 256 adjacent rows per state; one step scores all
    of them through csvd_score_columns.  Inputs (201 MB) exceed L2."""
    import numpy as np
    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import __graft_entry__
    if local == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2601_11626_gb300 import csvd, synth

    dev = torch.cuda.current_device()
    w = synth.scoring_k1(seed=rank, device="cuda", **K1_SHAPE)
    m, r, eps = w["m"], w["r"], w["eps"]
    states = []
    for blocks in w["states"]:
        st = csvd.IncrSVD(m, r)
        for b in blocks:
            st.append(b)
        states.append(st)
    torch.cuda.synchronize()
    Xt = w["Xt"]
    n = Xt.shape[0]
    cs = w["cand_state"]
    batch = csvd.ScoreColumns(states, cs, Xt, eps)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        batch.run()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        csvd.profile(True)
        l0 = csvd.launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            batch.run()
        e1.record(stream)
        e1.synchronize()
        launches = csvd.launch_count() - l0
        prof = csvd.profile_report()
        csvd.profile(False)
    ms = e0.elapsed_time(e1)
    barrier()
    value, ms = job_throughput(ms, n * args.steps, world)

    peaks, _ = _peaks()
    ranks = [s.rank for s in states]
    work = [_k1_work(m, ranks[cs[j]], min(r, ranks[cs[j]] + 1)) for j in range(n)]
    flops = sum(x["flops"] for x in work)
    nl, tms = prof.get("core_arrow", (0, float("nan")))
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = flops * args.steps / (tms / 1000.0) / 1e12
    roof = {"kernel": "core_arrow", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
            "peak_note": f"FP32 SIMT: {n_sm} SMs x 128 lanes x 2 flop x max SM clock",
            "hbm_gbs": sum(x["bytes"] for x in work) * args.steps / (tms / 1000.0) / 1e9,
            "kernels": {k: {"launches": v[0], "ms": v[1],
                            "share": v[1] / sum(x[1] for x in prof.values())}
                        for k, v in prof.items()}}

    # plain FP32 form on the first 4096 candidates, for context
    plain = None
    if args.plain_steps > 0:
        sub = 4096
        pb = csvd.ScoreBatch(states, cs[:sub], [Xt[j].view(m, 1) for j in range(sub)], eps,
                             "plain")
        pb.run()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.plain_steps):
            pb.run()
        p1.record(stream)
        p1.synchronize()
        pms = p0.elapsed_time(p1) / args.plain_steps
        plain = {"value": world * sub / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms,
                 "candidates": sub,
                 "max_tail_rel_diff_vs_mixed": float(((pb.tail.sqrt() - batch.tail[:sub].sqrt()).abs()
                                                      / batch.tail[:sub].sqrt().clamp_min(1e-300)).max()),
                 "accept_agree": bool((pb.accept == batch.accept[:sub]).all())}
        del pb

    # end to end: each step copies Xt from pinned host memory (second
    # stream, double-buffered) and reads tail, accept and sigma back
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty(Xt.shape, dtype=Xt.dtype, pin_memory=True)
        host.copy_(Xt)
        bufs = [Xt, torch.empty_like(Xt)]
        batches = [batch, csvd.ScoreColumns(states, cs, bufs[1], eps)]
        outs = [(torch.empty(batch.tail.shape, dtype=batch.tail.dtype, pin_memory=True),
                 torch.empty(batch.accept.shape, dtype=batch.accept.dtype, pin_memory=True),
                 torch.empty(batch.sigma.shape, dtype=batch.sigma.dtype, pin_memory=True))
                for _ in range(2)]
        out_bytes = batch.tail.numel() * 8 + batch.accept.numel() + batch.sigma.numel() * 4
        copy_stream = torch.cuda.Stream()
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for e in done:
            e.record(stream)
        for i in range(args.e2e_steps):
            b = i % 2
            copy_stream.wait_event(done[b])
            with torch.cuda.stream(copy_stream):
                bufs[b].copy_(host, non_blocking=True)
                ready[b].record(copy_stream)
            stream.wait_event(ready[b])
            batches[b].run()
            for o, src in zip(outs[b], (batches[b].tail, batches[b].accept, batches[b].sigma)):
                o.copy_(src, non_blocking=True)
            done[b].record(stream)
        q1.record(stream)
        q1.synchronize()
        qms = q0.elapsed_time(q1) / args.e2e_steps
        e2e_value, qms = job_throughput(qms, n, world)
        in_bytes = Xt.numel() * Xt.element_size()
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": out_bytes, "ms_per_step": qms, "steps": args.e2e_steps,
               "overlap": "inputs of step i copied on a second stream while step i-1 is scored"}
        del batches, bufs

    parity = None
    if rank == 0 and args.parity_samples > 0:
        from oracle import incremental as oinc
        rng = np.random.default_rng(7)
        idx = sorted(int(i) for i in rng.choice(n, args.parity_samples * 4, replace=False))
        sig_d = batch.sigma.cpu().double().numpy()
        tail_d = batch.tail.cpu().numpy()
        acc_d = batch.accept.cpu().numpy()
        worst_t, worst_s, flags, cache = 0.0, 0.0, 0, {}
        for j in idx:
            s_ = cs[j]
            if s_ not in cache:
                st = states[s_]
                te = st.tail_error()
                cache[s_] = oinc.IncrementalSVD(m, r, st.basis().double().cpu().numpy(),
                                                st.sigma().astype(np.float64), te["energy"],
                                                te["tail_sq"])
            s_o, t_o, a_o, nxt = cache[s_].evaluate(Xt[j].reshape(m, 1).cpu(), eps)
            worst_t = max(worst_t, abs(math.sqrt(tail_d[j]) - math.sqrt(nxt[3])) / math.sqrt(nxt[3]))
            worst_s = max(worst_s, float(np.max(np.abs(sig_d[j, :len(s_o)] - s_o) / s_o[0])))
            flags += int(bool(acc_d[j]) == a_o)
        parity = {"sampled": len(idx), "max_tail_rel_err": worst_t,
                  "max_sigma_err_rel_sigma1": worst_s, "accept_agree": flags,
                  "reference": "FP64 oracle from the exported GPU states"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import incremental as oinc
        st0 = oinc.IncrementalSVD(m, r)
        st0.append(w["states"][0][0].cpu())
        rows = [Xt[j].reshape(m, 1).cpu().double().numpy() for j in range(256)]
        t0 = time.perf_counter()
        done_n = 0
        while time.perf_counter() - t0 < 10.0 and done_n < 4096:
            st0.evaluate(rows[done_n % len(rows)], eps)
            done_n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": done_n / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done_n} one-column evaluations against one rebuilt state "
                         f"(m={m}, r={r}), FP64 numpy, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": f"one-column merge scoring (k = 1 dataset shape): {len(states)} states "
                            f"x {K1_SHAPE['per_state']} candidate vectors per GPU, m={m}, r={r}",
                "m": m, "r": r, "k": 1, "n_candidates": n, "precision_form": "mixed", "eps": eps,
                "l2": "inputs (%.2f GB) larger than L2, no flush" % (Xt.numel() * 4 / 1e9),
                "parallelism": f"dp{world} (candidates sharded, no collective on the data path)"},
            "plain_fp32": plain, "parity": parity, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk.summary(), "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    for st in states:
        st.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--r", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "plain", "gram_fp32"])
    ap.add_argument("--n-states", type=int, default=64)
    ap.add_argument("--per-state", type=int, default=64)
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--jacobi-candidates", type=int, default=512,
                    help="candidates timed in the residual + Jacobi form (0: skip)")
    ap.add_argument("--no-legs", dest="legs", action="store_false",
                    help="skip the other-rank and mid-size legs")
    ap.add_argument("--leg-ranks", default="32,128")
    ap.add_argument("--leg-steps", type=int, default=3)
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="keep the hand-set launch classes of the eigen core")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="skip the CUDA-graph replay of the step")
    ap.add_argument("--e2e-steps", type=int, default=20,
                    help="end-to-end steps; the first copy cannot overlap a step, so more "
                         "steps weigh the pipeline fill less")
    ap.add_argument("--ref-sample", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--parity-samples", type=int, default=8)
    ap.add_argument("--k1", action="store_true",
                    help="one-column candidates (the k = 1 dataset shape) through "
                         "csvd_score_columns instead of the uneven-width batch")
    args = ap.parse_args()

    world, rank, local = _dist()
    if args.impl == "reference":
        if rank == 0:
            run_reference_k1(args) if args.k1 else run_reference(args)
        return
    if args.k1:
        run_k1(args, world, rank, local)
        return

    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import __graft_entry__
    # one build per node: the other ranks wait for it, then load the library
    if local == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2601_11626_gb300 import csvd, synth

    dev = torch.cuda.current_device()
    w = synth.scoring_c4(r=args.r, seed=rank, n_states=args.n_states, per_state=args.per_state,
                         device="cuda")
    m, r, eps = w["m"], w["r"], w["eps"]
    states = []
    for blocks in w["states"]:
        st = csvd.IncrSVD(m, r)
        for b in blocks:
            st.append(b)
        states.append(st)
    torch.cuda.synchronize()
    ranks = [s.rank for s in states]
    cands = w["candidates"]
    n = len(cands)
    k_mean = sum(c.shape[1] for c in cands) / n
    pool_bytes = w["pools"][1].numel() * 4
    n_states = len(states)
    batch = csvd.ScoreBatch(states, w["cand_state"], cands, eps, args.precision)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # launch-class edges of the eigen core for this batch (untimed)
    tuning = None
    if args.tune and args.precision != "plain":
        from paper_2601_11626_gb300 import tune
        tuning = tune.autotune(batch, [ranks[w["cand_state"][i]] + cands[i].shape[1]
                                       for i in range(n)], m, ranks, steps=2)
        tuning["edges"] = list(tuning["edges"])
    # the step as a prepared plan (csvd_score_plan): descriptors, tile lists
    # and workspace built once after the tuning; every step then launches
    # the same kernels on the resident candidates
    batch.plan()
    for _ in range(args.warmup):
        batch.launch()
    batch.check()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        csvd.profile(True)
        l0 = csvd.launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            batch.launch()
        e1.record(stream)
        e1.synchronize()
        launches = csvd.launch_count() - l0
        prof = csvd.profile_report()
        csvd.profile(False)
    batch.check()
    ms = e0.elapsed_time(e1)
    barrier()
    value, ms = job_throughput(ms, n * args.steps, world)

    # the same step captured once into a CUDA graph and replayed
    graph = None
    if args.graph:
        g = batch.graph()
        for _ in range(args.warmup):
            g.replay()
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            g.replay()
        g1.record(stream)
        g1.synchronize()
        batch.check()
        gv, gms = job_throughput(g0.elapsed_time(g1), n * args.steps, world)
        graph = {"value": gv, "unit": UNIT, "ms_per_step": gms / args.steps, "steps": args.steps,
                 "kernels_per_step": launches // max(args.steps, 1)}
        del g

    # dominant kernel roofline
    peaks, peak_src = _peaks()
    work = [_work_per_candidate(m, ranks[w["cand_state"][i]], cands[i].shape[1]) for i in range(n)]
    gram_flops = sum(x["gram_flops"] for x in work)
    gram_bytes = sum(x["gram_bytes"] for x in work)
    core_flops = sum(x["core_flops"] for x in work)
    # launch classes of one kernel ("core_tridiag.large", ...) count together
    groups = {}
    for k, (nl_k, ms_k) in prof.items():
        g = groups.setdefault(k.split(".")[0], [0, 0.0])
        g[0] += nl_k
        g[1] += ms_k
    name, (nl, tms) = max(groups.items(), key=lambda kv: kv[1][1])
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if name.startswith("core"):
        achieved = core_flops * args.steps / (tms / 1000.0) / 1e12
        roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                "peak_note": f"FP32 SIMT: {n_sm} SMs x 128 lanes x 2 flop x max SM clock"}
    else:
        achieved = gram_bytes * args.steps / (tms / 1000.0) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_note": f"{peak_src} copy bandwidth"}
    roof["kernels"] = {k: {"launches": v[0], "ms": v[1], "share": v[1] / sum(x[1] for x in prof.values())}
                       for k, v in prof.items()}
    if "tc_gram" in groups:
        g_ms = groups["tc_gram"][1]
        issued = sum(_tc_issued_flops(m, ranks[w["cand_state"][i]], cands[i].shape[1])
                     for i in range(n))
        roof["tc_gram"] = {
            "ms_per_step": g_ms / args.steps,
            "hbm_gbs": gram_bytes * args.steps / (g_ms / 1000.0) / 1e9,
            "hbm_frac": gram_bytes * args.steps / (g_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
            "tensor_tflops": issued * args.steps / (g_ms / 1000.0) / 1e12,
            "tensor_frac": issued * args.steps / (g_ms / 1000.0) / 1e12 / peaks["bf16_tflops"],
            "note": f"algorithmic bytes (A once, U once per candidate) over the kernel's CUDA-event "
                    f"time; issued bf16 MMA flops (six per product, padded tiles) against the "
                    f"{peak_src} bf16 peak"}

    # the plain FP32 comparator of the metric: the same Gram route with FP32
    # SIMT products, on every candidate; and the residual + Jacobi route (the
    # step as Lemma 1 states it) on a bounded subset
    plain = None
    if args.plain_steps > 0 and args.precision == "mixed":
        plain = _time_form(csvd, states, w["cand_state"], cands, eps, "gram_fp32", args.plain_steps,
                           stream, batch)
        plain["form"] = "Gram route with FP32 SIMT products (same algorithm as the mixed form)"
        plain["value"] *= world
        plain["speedup_of_mixed"] = value / plain["value"]
    jacobi = None
    if args.jacobi_candidates > 0 and args.precision == "mixed":
        sub = min(n, args.jacobi_candidates)
        jacobi = _time_form(csvd, states, w["cand_state"][:sub], cands[:sub], eps, "plain",
                            args.plain_steps, stream, None)
        jacobi["form"] = "residual, Householder QR and one-sided Jacobi on K, FP32 SIMT"
        jacobi["candidates"] = sub
        jacobi["value"] *= world

    # end to end through the public API: every step copies its inputs from
    # pinned host memory and reads its results back; the copy of step i runs
    # on a second stream into the other of two device pools while step i - 1
    # is scored (double buffering)
    e2e = None
    if args.e2e_steps > 0:
        pool = w["pools"][1]
        host = torch.empty(pool.shape, dtype=pool.dtype, pin_memory=True)
        host.copy_(pool)
        pools = [pool, torch.empty_like(pool)]

        def views(p):
            out = []
            for c in cands:
                off = (c.data_ptr() - pool.data_ptr()) // pool.element_size()
                ld = c.stride(0)
                out.append(p[off:off + m * ld].view(m, ld)[:, :c.shape[1]])
            return out

        batches = [batch, csvd.ScoreBatch(states, w["cand_state"], views(pools[1]), eps,
                                          args.precision).plan()]
        out_bytes = batch.tail.numel() * 8 + batch.accept.numel() + batch.sigma.numel() * 4
        outs = [(torch.empty(batch.tail.shape, dtype=batch.tail.dtype, pin_memory=True),
                 torch.empty(batch.accept.shape, dtype=batch.accept.dtype, pin_memory=True),
                 torch.empty(batch.sigma.shape, dtype=batch.sigma.dtype, pin_memory=True))
                for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        # one copy with nothing else running, for reference
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(copy_stream):
            a0.record(copy_stream)
            pools[1].copy_(host, non_blocking=True)
            a1.record(copy_stream)
        a1.synchronize()
        alone_ms = a0.elapsed_time(a1)
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        c0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
        c1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
        barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for e in done:
            e.record(stream)
        for i in range(args.e2e_steps):
            b = i % 2
            copy_stream.wait_event(done[b])
            with torch.cuda.stream(copy_stream):
                c0[i].record(copy_stream)
                pools[b].copy_(host, non_blocking=True)
                c1[i].record(copy_stream)
                ready[b].record(copy_stream)
            stream.wait_event(ready[b])
            batches[b].launch()
            for o, src in zip(outs[b], (batches[b].tail, batches[b].accept, batches[b].sigma)):
                o.copy_(src, non_blocking=True)
            done[b].record(stream)
        q1.record(stream)
        q1.synchronize()
        for bt in batches:
            bt.check()
        qms = q0.elapsed_time(q1) / args.e2e_steps
        h2d_ms = sum(a.elapsed_time(z) for a, z in zip(c0, c1)) / args.e2e_steps
        e2e_value, qms = job_throughput(qms, n, world)
        in_bytes = pool.numel() * pool.element_size()
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
               "ms_per_step": qms, "steps": args.e2e_steps,
               "h2d_gbs": in_bytes / (h2d_ms / 1000.0) / 1e9,
               "h2d_gbs_alone": in_bytes / (alone_ms / 1000.0) / 1e9,
               "h2d_ms_each": [round(a.elapsed_time(z), 2) for a, z in zip(c0, c1)],
               "overlap": "inputs of step i copied on a second stream while step i-1 is scored"}
        batches[1].close()
        del batches, pools

    # sampled parity against the FP64 oracle from the states the GPU used
    parity = None
    if rank == 0 and args.parity_samples > 0:
        import numpy as np
        from oracle import incremental as oinc
        rng = np.random.default_rng(123)
        idx = sorted(int(i) for i in rng.choice(n, args.parity_samples, replace=False))
        sig_d = batch.sigma.cpu().double().numpy()
        tail_d = batch.tail.cpu().numpy()
        acc_d = batch.accept.cpu().numpy()
        worst_t, worst_s, flags = 0.0, 0.0, 0
        cache = {}
        for i in idx:
            s_ = w["cand_state"][i]
            if s_ not in cache:
                st = states[s_]
                te = st.tail_error()
                cache[s_] = oinc.IncrementalSVD(m, r, st.basis().double().cpu().numpy(),
                                                st.sigma().astype(np.float64), te["energy"],
                                                te["tail_sq"])
            s_o, t_o, a_o, nxt = cache[s_].evaluate(cands[i].cpu(), eps)
            worst_t = max(worst_t, abs(math.sqrt(tail_d[i]) - math.sqrt(nxt[3])) / math.sqrt(nxt[3]))
            worst_s = max(worst_s, float(np.max(np.abs(sig_d[i, :len(s_o)] - s_o) / s_o[0])))
            flags += int(bool(acc_d[i]) == a_o)
        parity = {"sampled": len(idx), "max_tail_rel_err": worst_t,
                  "max_sigma_err_rel_sigma1": worst_s, "accept_agree": flags,
                  "reference": "FP64 oracle from the exported GPU states"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, eps)

    # other state ranks and the mid-size recipe (free the main workload first)
    legs = None
    if args.legs and args.precision == "mixed":
        ranks_ = [int(x) for x in args.leg_ranks.split(",") if x]
        del batch
        for st in states:
            st.close()
        states = []
        del w, cands
        torch.cuda.empty_cache()
        legs = {"ranks": rank_legs(csvd, synth, ranks_, rank, args.leg_steps),
                "c2": c2_leg(csvd, synth, max(args.leg_steps, 3), 12)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": f"batched uneven merge scoring: {n_states} states x {args.per_state} "
                            f"candidates per GPU, m={m}, k~U[16,512], r={r}",
                "m": m, "r": r, "n_candidates": n, "k_mean": k_mean, "k_range": [16, 512],
                "precision_form": args.precision, "eps": eps,
                "l2": "inputs (%.1f GB) larger than L2, no flush" % (pool_bytes / 1e9),
                "parallelism": f"dp{world} (candidates sharded, no collective on the data path)"},
            "graph": graph,
            "plain_fp32": plain, "plain_fp32_jacobi": jacobi, "parity": parity, "e2e": e2e,
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": launches, "legs": legs, "tuning": tuning,
        }
        print(json.dumps(line), flush=True)
    for st in states:
        st.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
