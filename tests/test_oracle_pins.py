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


def test_weight_difference_bounds_fd(orc):
    """popc(a ^ b) >= sum over the parts of |popc(a_part) - popc(b_part)|, for
    one part (the whole word) and for the three parts of the weight cells
    (W = 32: bits 21..31, 10..20, 0..9; W = 16: 10..15, 5..9, 0..4), on the
    oracle's own fingerprints: a pair whose cells are more than 2k apart fails
    Eq. 1, which is what lets the GPU path skip it."""
    w = datagen.english1m(3000, 400)
    for t, width in (("occ", 32), ("count", 32), ("occ", 16), ("occh", 16)):
        m, _, _ = orc.symbol_map(w.dictionary.chars, "common", oracle.layout(t, width)["sigma"])
        a = orc.fingerprints(w.dictionary, m, t, width).astype(np.uint64)
        b = orc.fingerprints(w.queries["ham"], m, t, width).astype(np.uint64)
        x = a[None, :] ^ b[:, None]
        fdx = np.zeros(x.shape, dtype=np.int64)
        for s in range(32):
            fdx += ((x >> np.uint64(s)) & np.uint64(1)).astype(np.int64)
        bits = [width // 3 + (1 if i < width % 3 else 0) for i in range(3)]
        shifts = [bits[1] + bits[2], bits[2], 0]
        for parts in ([(0, width)], list(zip(shifts, bits))):
            dw = np.zeros(x.shape, dtype=np.int64)
            for sh, nb in parts:
                mask = np.uint64((1 << nb) - 1)
                pa = np.array([bin(int(v)).count("1") for v in (a >> np.uint64(sh)) & mask])
                pb = np.array([bin(int(v)).count("1") for v in (b >> np.uint64(sh)) & mask])
                dw += np.abs(pa[None, :] - pb[:, None])
            assert (fdx >= dw).all()
            assert (fdx == dw).any() and (fdx > dw).any()  # both cases occur
