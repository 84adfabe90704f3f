"""The seeded input generators shared by the oracle and the CUDA path (CPU):
determinism and the recipe properties their docstrings state."""
import numpy as np
import torch

from paper_2601_11626_gb300 import synth


def test_latent_bases_orthonormal_and_seeded():
    a = synth.latent_bases(40, 5, 3, seed=7)
    b = synth.latent_bases(40, 5, 3, seed=7)
    c = synth.latent_bases(40, 5, 3, seed=8)
    for q, q2, q3 in zip(a, b, c):
        np.testing.assert_allclose(q.T @ q, np.eye(5), atol=1e-12)
        assert torch.equal(q, q2) and not torch.equal(q, q3)


def test_latent_mixture_rank_and_padding():
    bases = synth.latent_bases(30, 4, 2, seed=1)
    spec = [0.5 ** i for i in range(4)]
    blocks, latent, pool = synth.latent_mixture(30, [3, 7, 9], bases, spec, 0.0, 2, ld_align=8)
    assert latent == [0, 1, 0]
    for b in blocks:
        assert b.stride(0) % 8 == 0 and b.stride(1) == 1
        s = np.linalg.svd(b.double().numpy(), compute_uv=False)
        assert np.sum(s > 1e-6 * s[0]) <= 4          # noise-free: inside one 4-dim subspace
    again, _, _ = synth.latent_mixture(30, [3, 7, 9], bases, spec, 0.0, 2, ld_align=8)
    assert all(torch.equal(x, y) for x, y in zip(blocks, again))


def test_scoring_c4_recipe():
    w = synth.scoring_c4(r=16, n_states=4, appends=2, per_state=3, m=128, k_lo=5, k_hi=20)
    assert w["m"] == 128 and w["r"] == 16 and len(w["states"]) == 4
    assert all(len(s) == 2 for s in w["states"])
    n = 12
    assert len(w["candidates"]) == n
    assert w["cand_state"] == [i // 3 for i in range(n)]
    assert w["cand_latent"] == [i % 4 for i in range(n)]
    for c in w["candidates"]:
        assert 5 <= c.shape[1] <= 20 and c.shape[0] == 128 and c.stride(0) % 8 == 0
    w2 = synth.scoring_c4(r=16, n_states=4, appends=2, per_state=3, m=128, k_lo=5, k_hi=20)
    assert all(torch.equal(x, y) for x, y in zip(w["candidates"], w2["candidates"]))


def test_scoring_k1_recipe():
    w = synth.scoring_k1(n_states=6, per_state=5, m=64, r=8, build=16, d=4)
    Xt = w["Xt"]
    assert Xt.shape == (30, 64) and Xt.stride(1) == 1
    assert w["cand_state"] == [j // 5 for j in range(30)]            # rows of a state adjacent
    assert w["cand_latent"] == [j % 6 for j in range(30)]
    assert len(w["states"]) == 6 and w["states"][0][0].shape == (64, 16)
    w2 = synth.scoring_k1(n_states=6, per_state=5, m=64, r=8, build=16, d=4)
    assert torch.equal(Xt, w2["Xt"])
    w3 = synth.scoring_k1(seed=1, n_states=6, per_state=5, m=64, r=8, build=16, d=4)
    assert not torch.equal(Xt, w3["Xt"])
