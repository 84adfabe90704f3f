"""The allocation-free merge evaluation against csvd_score.

csvd_score_one_noalloc serves callers that cannot allocate device memory
when they score a merge (GPU memory wholly owned by another allocator, or
loops that cannot afford cudaMalloc / cudaFree): its intermediates live in
a fixed device array inside the library.  Two calls in a row must each
reproduce csvd_score's mixed-form results for the same candidates, with
the tolerances of the parity tests.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_score_on_two_calls_in_a_row(cuda_lib):
    from paper_2601_11626_gb300 import csvd
    w = synth.scoring_c4(r=64, n_states=1, appends=3, per_state=6, device="cuda")
    st = csvd.IncrSVD(w["m"], w["r"])
    for b in w["states"][0]:
        st.append(b)
    eps = 0.25
    cands = w["candidates"]
    ks = [c.shape[1] for c in cands]
    # both eigen-core classes, including one that spills to the scratch workspace
    extra = synth.pack_blocks(synth.random_blocks(w["m"], [40, 500], seed=9, decay=0.97,
                                                  device="cuda"), ld_align=4)[0]
    cands = list(cands) + list(extra)
    ref_sig, ref_tail, ref_paper, ref_acc = csvd.score([st], [0] * len(cands), cands, eps, "mixed")
    ref_sig, ref_tail = ref_sig.cpu().double().numpy(), ref_tail.cpu().numpy()
    ref_acc = ref_acc.cpu().numpy()
    e_state = st.tail_error()["energy"]
    for call in range(2):
        for i, c in enumerate(cands):
            sig, tail, paper, acc = csvd.score_one_noalloc(st, c, eps)
            torch.cuda.synchronize()
            rn = min(st.r, st.rank + c.shape[1])
            s = sig.cpu().double().numpy()[:rn]
            want = ref_sig[i, :rn]
            assert np.all(np.abs(s ** 2 - want ** 2) <= 1e-4 * want ** 2 + 2e-6 * want[0] ** 2), (call, i)
            # the tail is tr(T) - sum of the top eigenvalues, both sums of
            # FP32-rounded terms as large as the total energy ||M||^2, and the
            # two paths differ by the order of FP32 atomics: relative part
            # plus a small multiple of the energy
            g, wt = float(tail[0]), float(ref_tail[i])
            energy = e_state + float((c.double() ** 2).sum())
            assert abs(g - wt) <= 1e-4 * wt + 1e-6 * energy, (call, i, g, wt, energy)
            assert int(acc[0]) == int(ref_acc[i])
    assert max(ks + [500]) + st.rank > 288  # the spilling class was exercised
