"""Parity at the benchmark's full size and launch configuration.

The batched-scoring workload of bench.py (64 states of rank 64 at m = 2048,
4096 candidates with widths uniform in [16, 512]) is scored in one call per
form.  Sampled candidates are re-evaluated by the FP64 oracle from the
state the GPU used (exported through the C ABI); every candidate is
cross-checked between the mixed form, the plain form and the Gram route
with FP32 SIMT products.
"""
import math

import numpy as np
import pytest
import torch

from oracle import incremental as oinc
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload(cuda_lib):
    from paper_2601_11626_gb300 import csvd
    w = synth.scoring_c4(r=64, device="cuda")
    states = []
    for blocks in w["states"]:
        st = csvd.IncrSVD(w["m"], w["r"])
        for b in blocks:
            st.append(b)
        states.append(st)
    torch.cuda.synchronize()
    out = {}
    for form in ("mixed", "plain", "gram_fp32"):
        b = csvd.ScoreBatch(states, w["cand_state"], w["candidates"], w["eps"], form).run()
        torch.cuda.synchronize()
        out[form] = (b.sigma.cpu().double().numpy(), b.tail.cpu().numpy(), b.accept.cpu().numpy())
    return csvd, w, states, out


def _oracle_from(st, m, r):
    U = st.basis().double().cpu().numpy()
    te = st.tail_error()
    return oinc.IncrementalSVD(m, r, U, st.sigma().astype(np.float64), te["energy"], te["tail_sq"])


def test_states_stay_orthonormal(workload):
    csvd, w, states, _ = workload
    for st in states[:8]:
        U = st.basis().double().cpu().numpy()
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 5e-6


def test_sampled_candidates_match_oracle(workload):
    csvd, w, states, out = workload
    m, r, eps = w["m"], w["r"], w["eps"]
    ks = np.array([c.shape[1] for c in w["candidates"]])
    rng = np.random.default_rng(1)
    sample = list(rng.choice(len(ks), 16, replace=False))
    sample += [int(np.argmax(ks)), int(np.argmin(ks))]
    oracles = {}
    for i in sample:
        s = w["cand_state"][i]
        if s not in oracles:
            oracles[s] = _oracle_from(states[s], m, r)
        s_o, t_o, a_o, nxt = oracles[s].evaluate(w["candidates"][i].cpu(), eps)
        for form in ("mixed", "plain", "gram_fp32"):
            sig, tail, acc = out[form]
            g, wt = math.sqrt(tail[i]), math.sqrt(nxt[3])
            assert abs(g - wt) <= 1e-4 * wt, (form, i, ks[i], g, wt)
            g_s = sig[i, :len(s_o)]
            ok = np.abs(g_s - s_o) <= 1e-5 * s_o + 2e-6 * s_o[0]
            if form != "plain":  # Gram eigenvalues: the normwise floor sits on sigma^2
                ok |= np.abs(g_s ** 2 - s_o ** 2) <= 2e-5 * s_o ** 2 + 8 * 2.0 ** -24 * s_o[0] ** 2
            assert np.all(ok), (form, i)
            if abs(math.sqrt(t_o / nxt[2]) - eps) > 1e-3 * eps:
                assert bool(acc[i]) == a_o


@pytest.mark.parametrize("other", ["plain", "gram_fp32"])
def test_plain_and_mixed_agree_on_every_candidate(workload, other):
    _, w, _, out = workload
    tm, tp = np.sqrt(out["mixed"][1]), np.sqrt(out[other][1])
    rel = np.abs(tm - tp) / tp
    assert rel.max() <= 1e-4, (int(rel.argmax()), float(rel.max()))
    assert np.array_equal(out["mixed"][2], out[other][2])
