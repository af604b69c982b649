"""Detection thresholds and F2 (Sec. 5.3): the library's host functions and
the oracle against closed forms and invariants (no GPU: host arithmetic)."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_12134_gb300 import _abi, build


@pytest.fixture(scope="module")
def api():
    build.build()
    _abi.load()
    from paper_2404_12134_gb300 import api as a
    return a


def test_thresholds_closed_form(api):
    """Scores 1..5: mean 3, std sqrt(2); quartiles 2 and 4 (positions 1 and 3);
    boxplot 4 + 1.5 * 2 = 7.  Scores 1..4: quartiles at positions 0.75 and 2.25,
    i.e. 1.75 and 3.25, boxplot 3.25 + 2.25 = 5.5."""
    for impl in (api.thresholds, oracle.thresholds):
        ts, bp = impl(np.array([5, 1, 4, 2, 3], np.float32))
        assert abs(ts - (3 + 2 * math.sqrt(2))) < 1e-12 and bp == 7.0
        ts, bp = impl(np.array([4, 3, 2, 1], np.float32))
        assert bp == 5.5
        ts, bp = impl(np.array([2.5], np.float32))
        assert ts == 2.5 and bp == 2.5


def test_thresholds_equivariance_and_agreement(api):
    """thr(a x + b) = a thr(x) + b for a > 0; library = oracle on random sets."""
    rng = np.random.default_rng(60)
    for n in (2, 3, 10, 101, 1000):
        x = rng.gamma(2.0, 1.0, size=n).astype(np.float32)
        ts, bp = api.thresholds(x)
        ots, obp = oracle.thresholds(x)
        assert abs(ts - ots) <= 1e-12 * max(1, abs(ots)) and abs(bp - obp) <= 1e-12 * max(1, abs(obp))
        y = (x.astype(np.float64) * 4 + 3).astype(np.float32)      # exact in float for these magnitudes? compare loosely
        ts2, bp2 = api.thresholds(y)
        assert abs(ts2 - (4 * ts + 3)) <= 1e-5 * abs(ts2) and abs(bp2 - (4 * bp + 3)) <= 1e-5 * abs(bp2)


def test_f2_counts(api):
    scores = np.array([0.1, 0.9, 0.5, 0.95, 0.2, 0.7], np.float32)
    labels = np.array([0, 1, 0, 1, 1, 0], np.int8)
    for impl in (api.f2_score, oracle.f2):
        r = impl(scores, labels, 0.6)          # flags: 0.9, 0.95, 0.7
        assert (r["tp"], r["fp"], r["fn"]) == (2, 1, 1)
        assert abs(r["f2"] - 10 / (10 + 4 + 1)) < 1e-12
        assert impl(scores, labels, 0.15)["f2"] == 15 / (15 + 2)     # tp 3, fp 2, fn 0
        assert impl(scores, np.zeros(6, np.int8), 2.0)["f2"] == 0.0  # nothing to find, nothing flagged
        perfect = impl(scores, (scores > 0.6).astype(np.int8), 0.6)
        assert perfect["f2"] == 1.0


def test_thresholds_reject_bad_input(api):
    with pytest.raises(Exception):
        api.thresholds(np.array([1.0, np.nan], np.float32))
    with pytest.raises(Exception):
        api.thresholds(np.zeros(0, np.float32))
