"""Prepared batched evaluation (csvd_score_plan / csvd_plan_launch) and its
capture into a CUDA graph, against csvd_score on the same candidates.

The plan runs the same kernels on the same descriptors, so its outputs
equal csvd_score's up to the order of the atomic sums (column energies,
the eigen core's p = G v accumulations): the comparison uses the parity
tests' tolerances.  A plan reads the candidate blocks when it runs, so new
contents written into the same buffers are scored by the next launch."""
import numpy as np
import pytest
import torch

from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def csvd(cuda_lib):
    from paper_2601_11626_gb300 import csvd as mod
    return mod


def _workload(csvd, precision="mixed"):
    """Three states (r = 32) and candidates of widths 1 (the arrowhead
    core), 16..400 (every launch class of the eigen core)."""
    w = synth.scoring_c4(r=32, n_states=3, appends=3, per_state=5, m=512, k_lo=16, k_hi=400,
                         device="cuda")
    states = []
    for blocks in w["states"]:
        st = csvd.IncrSVD(w["m"], w["r"], precision="plain")
        for b in blocks:
            st.append(b)
        states.append(st)
    cands = list(w["candidates"])
    cs = list(w["cand_state"])
    cols = synth.random_blocks(w["m"], [1, 1, 1], seed=4, device="cuda")
    cands += [c.contiguous() for c in cols]
    cs += [0, 1, 2]
    return w, states, cands, cs


def _same(csvd, a, b, energies, rmax):
    """Outputs of two evaluations of the same candidates (sigma, tail, accept)."""
    sa, ta, aa = a.sigma.cpu().double().numpy(), a.tail.cpu().numpy(), a.accept.cpu().numpy()
    sb, tb, ab = b.sigma.cpu().double().numpy(), b.tail.cpu().numpy(), b.accept.cpu().numpy()
    ok = (np.abs(sa - sb) <= 1e-5 * np.abs(sb) + 2e-6 * np.abs(sb[:, :1])) | \
        (np.abs(sa ** 2 - sb ** 2) <= 2e-5 * sb ** 2 + 8 * U * sb[:, :1] ** 2)
    assert np.all(ok)
    assert np.all(np.abs(ta - tb) <= 2e-4 * np.abs(tb) + 4 * U * energies)
    tight = np.abs(np.sqrt(tb / energies) - a.eps) <= 1e-3 * a.eps
    assert np.all((aa == ab) | tight)


def _energies(states, cands, cs):
    e = [s.tail_error()["energy"] for s in states]
    return np.array([e[cs[i]] + float((c.double() ** 2).sum()) for i, c in enumerate(cands)])


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_plan_launch_matches_score(csvd, precision):
    w, states, cands, cs = _workload(csvd)
    eps = 0.2
    ref = csvd.ScoreBatch(states, cs, cands, eps, precision).run()
    b = csvd.ScoreBatch(states, cs, cands, eps, precision).plan()
    for _ in range(3):  # repeated launches reuse the workspace
        b.sigma.zero_()
        b.tail.zero_()
        b.launch()
    b.check()
    torch.cuda.synchronize()
    _same(csvd, b, ref, _energies(states, cands, cs), w["r"])
    b.close()


def test_plan_reads_the_blocks_when_it_runs(csvd):
    w, states, cands, cs = _workload(csvd)
    eps = 0.2
    b = csvd.ScoreBatch(states, cs, cands, eps, "mixed").plan()
    b.launch().check()
    first = b.tail.clone()
    # new contents in the same buffers: the next launch scores them
    fresh = synth.random_blocks(w["m"], [c.shape[1] for c in cands], seed=21, device="cuda")
    for c, f in zip(cands, fresh):
        c.copy_(f)
    b.launch().check()
    ref = csvd.ScoreBatch(states, cs, cands, eps, "mixed").run()
    torch.cuda.synchronize()
    _same(csvd, b, ref, _energies(states, cands, cs), w["r"])
    assert not torch.allclose(first, b.tail)
    b.close()


def test_plan_in_a_cuda_graph(csvd):
    w, states, cands, cs = _workload(csvd)
    eps = 0.2
    ref = csvd.ScoreBatch(states, cs, cands, eps, "mixed").run()
    b = csvd.ScoreBatch(states, cs, cands, eps, "mixed")
    g = b.graph()
    for _ in range(2):
        b.sigma.zero_()
        b.tail.zero_()
        b.accept.zero_()
        g.replay()
    torch.cuda.synchronize()
    b.check()
    _same(csvd, b, ref, _energies(states, cands, cs), w["r"])
    b.close()


def test_plan_reports_device_failures(csvd):
    """A bisection cap of one iteration makes the eigen core report
    CSVD_ERR_NOT_CONVERGED through the plan's status word."""
    w, states, cands, cs = _workload(csvd)
    b = csvd.ScoreBatch(states, cs, cands, 0.2, "mixed").plan()
    try:
        csvd.debug_limits(solver_iters=1)
        b.launch()
        with pytest.raises(csvd.CsvdError) as ei:
            b.check()
        assert ei.value.status == csvd.Status.ERR_NOT_CONVERGED
    finally:
        csvd.debug_limits()
    b.launch().check()  # the status word was cleared by the read
    b.close()
