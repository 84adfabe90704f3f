"""GPU parity of the final per-cluster decomposition (csvd_reconstruct)
against the FP64 oracle on the same basis.

Tolerances (FP32 products of length m): coefficient blocks within 2e-5 of
their largest entry (times the sigma_1 / sigma_j amplification of the
inverse scaling); residual energies (explicit residuals, no cancellation)
within 1e-3 relative plus 1e-6 of the block energy; block energies within
1e-6 relative.
"""
import numpy as np
import pytest
import torch

from oracle import decomp, exact
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csvd(cuda_lib):
    from paper_2601_11626_gb300 import csvd as mod
    return mod


def _check(d, U, s, blocks):
    Ut_o, V_o, res_o, en_o = decomp.decompose(U.double().cpu().numpy(), np.asarray(s, dtype=np.float64),
                                              [b.cpu() for b in blocks])
    s = np.asarray(s, dtype=np.float64)
    amp = s[0] / np.maximum(s, s[0] * 1e-3)
    for v_g, v_o in zip(d.V, V_o):
        v_g = v_g.double().cpu().numpy()
        tol = 2e-5 * np.abs(v_o).max() * amp[None, :] + 1e-12
        assert np.all(np.abs(v_g - v_o) <= tol), np.abs(v_g - v_o).max()
    assert np.allclose(d.Ut.double().cpu().numpy(), Ut_o, rtol=1e-6, atol=1e-6 * np.abs(Ut_o).max())
    assert np.allclose(d.energy, en_o, rtol=1e-6)
    assert np.all(np.abs(d.resid_sq - res_o) <= 1e-3 * res_o + 1e-6 * en_o), (d.resid_sq, res_o)
    assert d.rel_error == pytest.approx(decomp.rel_error(res_o, en_o), rel=1e-3)


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_decompose_incremental_cluster(csvd, precision):
    col = synth.mid_c2(n_blocks=12)
    m, r = col.m, col.meta["r"]
    blocks = [b.cuda() for b in col.blocks[:8]]
    st = csvd.IncrSVD(m, r, precision)
    for b in blocks:
        st.append(b)
    d = st.decompose(blocks)
    U = st.basis()
    _check(d, U, st.sigma()[: U.shape[1]], blocks)
    assert d.memory == decomp.memory(m, U.shape[1], [b.shape[1] for b in blocks])
    # the true error of the estimated basis is at least the optimum (Thm. 4)
    assert d.rel_error >= exact.rel_error([b.cpu() for b in blocks], r) * (1 - 1e-4)
    st.close()


def test_decompose_exact_basis_gives_the_optimal_tail(csvd):
    """With the exact top-r SVD (FP64, rounded to FP32) the GPU residuals sum
    to the Eckart-Young tail and the stacked V has orthonormal columns."""
    col = synth.small_c1()
    r = col.meta["r"]
    blocks = [b.cuda() for b in col.blocks[:10]]
    M = np.hstack([b.double().numpy() for b in col.blocks[:10]])
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    Ug = torch.tensor(U[:, :r], dtype=torch.float32, device="cuda")
    d = csvd.reconstruct(Ug, s[:r], blocks)
    _check(d, Ug, s[:r].astype(np.float32), blocks)
    tail = exact.tail_sq([b.cpu() for b in col.blocks[:10]], r)
    assert d.resid_sq.sum() == pytest.approx(tail, rel=2e-3)
    Vc = np.vstack([v.double().cpu().numpy() for v in d.V])
    assert np.allclose(Vc.T @ Vc, np.eye(r), atol=1e-3)


def test_decompose_argument_errors(csvd):
    """The library rejects what the binding passes through: bf16 blocks (the
    decomposition takes f32)."""
    U = torch.zeros(16, 4, device="cuda")
    with pytest.raises(csvd.CsvdError):
        csvd.reconstruct(U, [1.0, 1.0, 1.0, 1.0], [torch.zeros(16, 3, device="cuda", dtype=torch.bfloat16)])
