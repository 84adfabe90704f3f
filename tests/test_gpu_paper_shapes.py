"""The paper-shaped stand-in runner end to end at a tiny scale: cluster,
decompose every cluster, and check each cluster's true relative error
against the constraint (guaranteed for the max-norm algorithm, observed for
the approximate one)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["weyl", "approx"])
def test_pdebench_shaped_tiny(cuda_lib, algo):
    from paper_2601_11626_gb300 import paper_shapes
    out = paper_shapes.run("pdebench", algo=algo, scale=0.006, precision="mixed")
    assert out["blocks"] == 30
    assert 1 <= out["clusters"] <= 30
    assert out["compression_ratio"] >= 1.0
    assert out["max_cluster_rel_error"] <= out["eps"] * (1 + 1e-3)
