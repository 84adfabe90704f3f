"""Plant plausible mistakes in the oracle's bounds (Thm. 1, Cor. 1) on the
CPU and check that the bound pins catch each one."""
import inspect
import types

import pytest

from oracle import bounds as obounds
from tests import test_oracle_core as pins

PINS = [pins.test_bounds_are_upper_bounds_random, pins.test_weyl_rank_one_example,
        pins.test_residual_bound_exact_under_orthogonal_growth,
        pins.test_residual_bound_degenerate_under_nesting,
        pins.test_residual_mu_is_union_and_monotone,
        pins.test_thm2_individual_inequality_fails_but_cor1_holds]


def _mutant(old, new):
    src = inspect.getsource(obounds)
    assert old in src, old
    mod = types.ModuleType("oracle.bounds")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new", [
    ("top = max(top_r_energy(b, r) for b in blocks)",
     "top = min(top_r_energy(b, r) for b in blocks)"),                     # Weyl: min block
    ("return float(np.sum(s[:r] ** 2))", "return float(np.sum(s[:r + 1] ** 2))"),  # top r+1
    ("return max(0.0, energy - float(np.sum(mu[:r] ** 2)))",
     "return max(0.0, energy - float(np.sum(mu[:r + 1] ** 2)))"),           # mu r+1
    ("Q = np.hstack([self.Q, u[:, keep]])", "Q = self.Q"),                   # basis not grown
    ("energy = self.energy + float(np.sum(A * A))", "energy = float(np.sum(A * A))"),
])
def test_bound_pins_catch_planted_mistakes(old, new, monkeypatch):
    monkeypatch.setattr(pins, "bounds", _mutant(old, new))
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"no bound pin caught the mutant {new!r}"
