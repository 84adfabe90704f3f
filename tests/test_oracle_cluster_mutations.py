"""Plant plausible mistakes in the oracle's clustering (on the CPU) and
check that the clustering pins catch each one."""
import inspect
import types

import pytest

import oracle
from oracle import cluster as ocluster
from tests import test_oracle_cluster as pins

PINS = [pins.test_weyl_head_hand_derived, pins.test_approx_recovers_exact_subspaces,
        pins.test_residual_merges_orthogonal_growth_only_up_to_rank,
        pins.test_c1_approx_groups_latent_pairs, pins.test_exhaustive_tiny,
        pins.test_compression_ratio_closed_form, pins.test_frobenius_scan_repeats_until_nothing_joins]


def _mutant(old, new):
    src = inspect.getsource(ocluster)
    assert old in src, old
    mod = types.ModuleType("oracle.cluster")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new", [
    ("key=lambda j: (-norms[j], j)", "key=lambda j: (norms[j], j)"),            # smallest anchor
    ("order = sorted(remaining, key=lambda j: (norms[j], j))",
     "order = sorted(remaining, key=lambda j: (-norms[j], j))"),                 # descending scan
    ("    e2 = eps * eps\n    if sort_mode", "    e2 = eps\n    if sort_mode"),  # eps not squared
    ("if width + widths[j] > r:", "if width + widths[j] >= r:"),                  # head one short
    ("if not accepted_any or not remaining:", "if True:"),                        # one pass only
    ("stored += min(m * n_c, r_eff * (m + n_c))", "stored += r_eff * (m + n_c)"),  # no raw cap
])
def test_cluster_pins_catch_planted_mistakes(old, new, monkeypatch):
    monkeypatch.setattr(pins, "cluster", _mutant(old, new))
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"no clustering pin caught the mutant {new!r}"
