"""The wide regime (weight-matrix-shaped config, reduced size): square bf16
blocks W_i = B C_i + E_i (shared low-rank basis plus a power-law residual)
with r + k > m, so the merge's core keeps k' = m - r_t new directions
(Lemma 1 / Cor. 3).  Four 1024 x 1024 matrices at r = 256: the state of the
first three is built by the FP64 oracle and loaded; the fourth (and the
first, already inside the span) are scored in the mixed form from bf16
storage (products on the FP32 SIMT path, cores of size 1280) and compared
with the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import incremental as oinc
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


def test_wide_regime_reduced_size(cuda_lib):
    from paper_2601_11626_gb300 import csvd
    w = synth.weights_c3(n_mats=4, m=1024, shared_rank=128)
    m, r = w["m"], 256
    blocks = w["blocks"]
    ost = oinc.IncrementalSVD(m, r)
    for b in blocks[:3]:
        ost.append(b.float())
    ost.Q = ost.Q.astype(np.float32).astype(np.float64)
    ost.s = ost.s.astype(np.float32).astype(np.float64)
    st = csvd.IncrSVD(m, r)
    st.load(torch.tensor(ost.Q, dtype=torch.float32, device="cuda"), ost.s.astype(np.float32),
            ost.energy, ost.discarded)
    cands = [blocks[3].cuda(), blocks[0].cuda()]
    for form in ("mixed", "gram_fp32"):
        sig, tail, _, acc = csvd.score([st], [0, 0], cands, 0.3, form)
        sig, tail = sig.cpu().double().numpy(), tail.cpu().numpy()
        for i, b in enumerate((blocks[3], blocks[0])):
            s_o, t_o, a_o, nxt = ost.evaluate(b.float(), 0.3)
            g = sig[i, :len(s_o)]
            ok = (np.abs(g - s_o) <= 1e-5 * s_o + 2e-6 * s_o[0]) | \
                (np.abs(g ** 2 - s_o ** 2) <= 2e-5 * s_o ** 2 + 8 * 2.0 ** -24 * s_o[0] ** 2)
            assert np.all(ok), (form, i, np.nonzero(~ok)[0][:8])
            assert abs(tail[i] - nxt[3]) <= 2e-4 * nxt[3] + 4 * 2.0 ** -24 * nxt[2], \
                (form, i, tail[i], nxt[3])
            assert bool(acc[i].item()) == a_o or abs(math.sqrt(t_o / nxt[2]) - 0.3) <= 3e-4
