"""Host side of the learned order: the training target (how cheap checking a
constraint is, optionally plus what it removes) and the arrays built from the
pipeline's logs."""
import math

import numpy as np
import pytest

from paper_1912_08453_gb300 import ordering


def rec(ms_search, ms_lcc, before, after, f0=0.0):
    return {"ms_search": ms_search, "ms_lcc": ms_lcc, "bits_before": before, "bits_after": after,
            "features": [f0] + [0.0] * 15}


def test_target_is_minus_log_microseconds():
    assert ordering.target(rec(0.0, 0.0, 10, 10)) == 0.0
    assert ordering.target(rec(0.003, 0.004, 10, 10)) == pytest.approx(-math.log2(8.0))
    # cheaper constraints score higher
    assert ordering.target(rec(0.001, 0.0, 5, 5)) > ordering.target(rec(0.1, 0.0, 5, 5))


def test_target_benefit_term():
    r = rec(0.0, 0.001, 100, 37)
    assert ordering.target(r, benefit_weight=0.5) == pytest.approx(0.5 * math.log2(64.0) - 1.0)
    # bits never come back: a negative difference counts as nothing removed
    assert ordering.target(rec(0.0, 0.0, 5, 9), benefit_weight=1.0) == 0.0


def test_targets_from_shapes():
    recs = [rec(0.001 * i, 0.0, 10, 5, f0=float(i)) for i in range(7)]
    X, y = ordering.targets_from(recs)
    assert X.shape == (7, 16) and X.dtype == np.float32
    assert y.shape == (7,) and y.dtype == np.float32
    assert np.array_equal(X[:, 0], np.arange(7, dtype=np.float32))
    assert np.all(np.diff(y) < 0)
