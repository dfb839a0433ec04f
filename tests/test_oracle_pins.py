"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import datagen
import oracle
import pins


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(orc, check):
    check(orc)


def test_unsound_combinations_are_the_expected_ones(orc):
    """Eq. 1 fails exactly for the paper's binary count encoding and for the
    Hamming-only types (occurrence halved, position) under Levenshtein."""
    res = pins.check_bound_sweep(orc)
    bad = sorted({(t, gray, metric) for (t, w, b, p, gray, metric), v in res.items() if v})
    assert bad == [("count", False, "ham"), ("count", False, "lev"), ("occh", True, "lev"),
                   ("pos", True, "lev")]


def test_filter_is_pure_speedup_uniform10k(orc):
    """Full 10,000-word / 1,000-query workload, occ16 common: the paper's filter
    + verify gives exactly the brute-force match lists, for both metrics."""
    w = datagen.uniform10k()
    m, _, _ = orc.symbol_map(w.dictionary.chars, "common", 16)
    for metric, Q in w.queries.items():
        rp0, idx0 = orc.match(w.dictionary, Q, 1, metric)
        rp1, idx1 = orc.match(w.dictionary, Q, 1, metric, prune=False)
        assert np.array_equal(rp0, rp1) and np.array_equal(idx0, idx1)
        rp, idx, pairs, surv = orc.filter_match(w.dictionary, Q, 1, metric, m, "occ", 16)
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)
        assert pairs == oracle.eligible_pairs(w.dictionary, Q, 1, metric)
        # the mutated half of the queries come from dictionary words within one edit
        assert (np.diff(rp0) > 0).sum() >= 450
