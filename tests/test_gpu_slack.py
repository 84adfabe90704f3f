"""GPU slack diagnostic (estimator conservativeness) against the FP64
oracle on the same sampled subsets, and the signs the theorems fix:
the Weyl and residual bounds never undershoot the true error (Thm. 1,
Cor. 1) and neither does the plug-in estimate (the retained Gram is
dominated by the exact one; see the oracle pins)."""
import math

import numpy as np
import pytest

from oracle import bounds as obounds
from oracle import exact
from paper_2601_11626_gb300 import synth

pytestmark = pytest.mark.gpu


def test_slack_matches_the_oracle_and_is_nonnegative(cuda_lib):
    from paper_2601_11626_gb300 import diagnostics
    col = synth.small_c1()
    r = col.meta["r"]
    blocks = [b.cuda() for b in col.blocks]
    rows = diagnostics.slack(blocks, r, sizes=(2, 4, 8), trials=4, seed=3)
    assert len(rows) == 12
    for row in rows:
        sub = [col.blocks[i] for i in row["blocks"]]
        w, res, plug, energy = obounds.all_bounds(sub, r)
        true = math.sqrt(exact.tail_sq(sub, r))
        norm = math.sqrt(energy)
        assert row["energy"] == pytest.approx(energy, rel=1e-6)
        # E within 1e-4 relative, plus a floor of 8 u ||M||^2 on E^2 (the
        # rounding of FP32 data of energy ||M||^2, through a few appends)
        floor_sq = 8 * 2.0 ** -24 * energy

        def close(got, want_sq):
            want_sq = max(want_sq, 0.0)
            return abs(got * got - want_sq) <= 2e-4 * want_sq + floor_sq

        assert close(row["true"], true * true), (row["true"], true)
        for name, want in (("weyl", w), ("residual", res), ("plugin", plug)):
            assert close(row[name], want), (name, row[name], math.sqrt(max(want, 0.0)))
            # the estimators never undershoot the true error (beyond rounding)
            assert row[name] ** 2 >= true * true - floor_sq - 2e-4 * true * true, (name, row)
    s = diagnostics.summary(rows)
    assert sorted(s) == [2, 4, 8]
