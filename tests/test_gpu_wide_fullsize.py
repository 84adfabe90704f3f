"""The wide regime at full size (weight-matrix-shaped config): two 4096 x
4096 bf16 matrices W_i = B C_i + E_i at r = 256 and r = 512.  The state of
the first is built by the FP64 oracle (one exact rank-r truncation) and
loaded; the second is scored in the mixed form from bf16 storage, a merge
whose core has n = r + k = 4352 or 4608 (Lemma 1 / Cor. 3 with
k' = m - r_t new directions), and compared with the oracle's evaluation of
the same merge."""
import math
import time

import numpy as np
import pytest
import torch

from oracle import incremental as oinc
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r", [256, 512])
def test_wide_regime_full_size_one_merge(cuda_lib, r):
    from paper_2601_11626_gb300 import csvd
    w = synth.weights_c3(n_mats=2, device="cuda")
    m = w["m"]
    a0, a1 = (b.cpu() for b in w["blocks"])
    ost = oinc.IncrementalSVD(m, r)
    ost.append(a0.float())
    ost.Q = ost.Q.astype(np.float32).astype(np.float64)
    ost.s = ost.s.astype(np.float32).astype(np.float64)
    st = csvd.IncrSVD(m, r)
    st.load(torch.tensor(ost.Q, dtype=torch.float32, device="cuda"), ost.s.astype(np.float32),
            ost.energy, ost.discarded)
    cand = w["blocks"][1]
    eps = 0.5
    csvd.score([st], [0], [cand], eps, "mixed")  # first call: workspace and attributes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sig, tail, _, acc = csvd.score([st], [0], [cand], eps, "mixed")
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t0
    sig, tail = sig.cpu().double().numpy()[0], float(tail.cpu()[0])
    s_o, t_o, a_o, nxt = ost.evaluate(a1.float(), eps)
    g = sig[:len(s_o)]
    ok = (np.abs(g - s_o) <= 1e-5 * s_o + 2e-6 * s_o[0]) | \
        (np.abs(g ** 2 - s_o ** 2) <= 2e-5 * s_o ** 2 + 8 * 2.0 ** -24 * s_o[0] ** 2)
    assert np.all(ok), np.nonzero(~ok)[0][:8]
    assert abs(tail - nxt[3]) <= 2e-4 * nxt[3] + 4 * 2.0 ** -24 * nxt[2], (tail, nxt[3])
    assert bool(acc[0].item()) == a_o or abs(math.sqrt(t_o / nxt[2]) - eps) <= 1e-3 * eps
    print(f"\nfull-size wide merge (core n = {r + m}): {gpu_s:.2f} s on the GPU, "
          f"tail rel. err {abs(tail - nxt[3]) / nxt[3]:.2e}, relative tail "
          f"{math.sqrt(nxt[3] / nxt[2]):.3f}")
