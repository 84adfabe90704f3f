"""The allocation-free merge evaluation against csvd_score.

csvd_score_one_noalloc serves callers that cannot allocate device memory
when they score a merge (GPU memory wholly owned by another allocator, or
loops that cannot afford cudaMalloc / cudaFree): its intermediates live in
a fixed device array inside the library.  Two calls in a row must each
reproduce csvd_score's mixed-form results for the same candidates, with
the tolerances of the parity tests.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import incremental as oinc
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
            # sigma~ from Gram eigenvalues: 1e-5 relative, or the normwise
            # FP32 floor of a Gram, 8 u sigma_1^2 on sigma^2
            ok = (np.abs(s - want) <= 1e-5 * want + 2e-6 * want[0]) | \
                (np.abs(s ** 2 - want ** 2) <= 2e-5 * want ** 2 + 8 * 2.0 ** -24 * want[0] ** 2)
            assert np.all(ok), (call, i)
            # same kernels, same data: the two paths differ only by the order
            # of the FP64 atomics that sum the column energies
            g, wt = float(tail[0]), float(ref_tail[i])
            energy = e_state + float((c.double() ** 2).sum())
            assert abs(g - wt) <= 2e-4 * wt + 4 * 2.0 ** -24 * energy, (call, i, g, wt, energy)
            assert int(acc[0]) == int(ref_acc[i])
    assert max(ks + [500]) + st.rank > 288  # the spilling class was exercised


def test_noalloc_empty_state_matches_score_and_oracle(cuda_lib):
    """A state with no columns yet (r_t = 0: no projection tiles, U unused)
    scored without allocation: the same result as csvd_score and as the
    oracle's first append (the rank-r SVD of the block)."""
    from paper_2601_11626_gb300 import csvd
    m, r = 256, 16
    blocks = synth.pack_blocks(synth.random_blocks(m, [40, 128], seed=12, decay=0.9, noise=1e-2,
                                                   device="cuda"), ld_align=4)[0]
    st = csvd.IncrSVD(m, r)
    assert st.rank == 0
    ref_sig, ref_tail, _, _ = csvd.score([st], [0, 0], blocks, 0.1, "mixed")
    for call in range(2):
        for i, b in enumerate(blocks):
            sig, tail, paper, acc = csvd.score_one_noalloc(st, b, 0.1)
            torch.cuda.synchronize()
            s_o, t_o, a_o, nxt = oinc.IncrementalSVD(m, r).evaluate(b.cpu(), 0.1)
            got = sig.cpu().double().numpy()[:len(s_o)]
            ok = (np.abs(got - s_o) <= 1e-5 * s_o + 2e-6 * s_o[0]) | \
                (np.abs(got ** 2 - s_o ** 2) <= 2e-5 * s_o ** 2 + 8 * 2.0 ** -24 * s_o[0] ** 2)
            assert np.all(ok), (call, i)
            assert abs(float(tail[0]) - nxt[3]) <= 2e-4 * nxt[3] + 4 * 2.0 ** -24 * nxt[2]
            assert abs(float(tail[0]) - float(ref_tail[i])) <= 2e-4 * float(ref_tail[i]) + \
                4 * 2.0 ** -24 * nxt[2]
            ref = ref_sig[i, :len(s_o)].cpu().double().numpy()
            assert np.all((np.abs(got - ref) <= 1e-5 * s_o + 2e-6 * s_o[0]) |
                          (np.abs(got ** 2 - ref ** 2) <= 2e-5 * s_o ** 2 +
                           8 * 2.0 ** -24 * s_o[0] ** 2))
            assert bool(acc[0]) == a_o


def test_noalloc_limits_rejected_before_any_launch(cuda_lib):
    """Sizes beyond the scratch array's limits return CSVD_ERR_SHAPE (and a
    misaligned block CSVD_ERR_ARG) without launching a kernel, and the state
    stays usable."""
    from paper_2601_11626_gb300 import csvd
    lib = csvd.lib()
    m = 256
    outs = [torch.zeros(160, device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda"),
            torch.zeros(1, dtype=torch.float64, device="cuda"),
            torch.zeros(1, dtype=torch.uint8, device="cuda")]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]

    def call(st, blk):
        b = csvd.block(blk, m)
        before = csvd.launch_count()
        rc = lib.csvd_score_one_noalloc(st.handle, ctypes.byref(b), 0.1, *ptrs)
        return rc, csvd.launch_count() - before

    st = csvd.IncrSVD(m, 16)
    wide = torch.zeros(m, 516, device="cuda")
    rc, n = call(st, wide[:, :513])            # k = 513 > 512
    assert rc == csvd.Status.ERR_SHAPE and n == 0
    rc, n = call(st, wide[:, 1:33])             # base not 16-byte aligned
    assert rc == csvd.Status.ERR_ARG and n == 0
    big = csvd.IncrSVD(m, 160)                  # rank above 128
    big.append(torch.randn(m, 140, device="cuda"))
    assert big.rank == 140
    rc, n = call(big, wide[:, :32])
    assert rc == csvd.Status.ERR_SHAPE and n == 0
    odd = csvd.IncrSVD(m, 18)                   # rank cap not divisible by 4
    odd.append(torch.randn(m, 8, device="cuda"))
    rc, n = call(odd, wide[:, :32])
    assert rc == csvd.Status.ERR_SHAPE and n == 0
    # the states still work
    sig, tail, _, _ = csvd.score_one_noalloc(st, wide[:, :32], 0.1)
    torch.cuda.synchronize()
    assert float(tail[0]) == 0.0
