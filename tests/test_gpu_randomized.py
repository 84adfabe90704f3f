"""The randomized range-finder estimator on the GPU (csvd_randomized_tail)
against the FP64 oracle with the same test matrices: the small recipe at
r = 32 (all 32 latent directions, a wide gap to the noise) with l = 40 and
one power iteration, a rank-deficient case (exact zero), and the
certificate property E~_rand >= E_r on both."""
import numpy as np
import pytest
import torch

from oracle import exact
from oracle import randomized as ornd
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("power_iters", [0, 1, 2])
def test_randomized_tail_matches_oracle(cuda_lib, power_iters):
    from paper_2601_11626_gb300 import csvd
    col = synth.small_c1()
    r, l = 32, 40
    blocks = col.blocks
    om = ornd.gaussian_omegas([b.shape[1] for b in blocks], l, 17)
    want = ornd.tail_sq(blocks, om, r, power_iters)
    got, U = csvd.randomized_tail([b.cuda() for b in blocks], [torch.from_numpy(o).cuda() for o in om],
                                  r, power_iters, want_basis=True)
    energy = exact.energy(blocks)
    assert abs(got - want) <= 2e-4 * want + 4 * 2.0 ** -24 * energy, (got, want)
    ex = exact.tail_sq(blocks, r)
    assert got >= ex * (1 - 2e-4) - 4 * 2.0 ** -24 * energy
    Ud = U.double().cpu().numpy()
    assert np.abs(Ud.T @ Ud - np.eye(r)).max() < 1e-5


def test_randomized_tail_rank_deficient_is_zero(cuda_lib):
    from paper_2601_11626_gb300 import csvd
    blocks = synth.random_blocks(64, [10, 12, 9], seed=8, rank=2)   # rank <= 6
    r, l = 6, 10
    om = ornd.gaussian_omegas([b.shape[1] for b in blocks], l, 2)
    got = csvd.randomized_tail([b.cuda() for b in blocks], [torch.from_numpy(o).cuda() for o in om],
                               r, 1)
    assert got <= 8 * 2.0 ** -24 * exact.energy(blocks)
