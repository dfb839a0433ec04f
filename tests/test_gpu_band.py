"""Weight bands (needs a GPU).

The buckets are ordered by weight cell (the population counts of three parts
of the fingerprint) and every query tile tests only the runs of cells whose L1
distance to the tile's box of cells is at most 2k: the parts' weight
differences add up to at most popc(a ^ b), so the skipped pairs fail Eq. 1
(pinned on the CPU in test_oracle_pins.py).  Here: the match lists and the
survivor count stay the oracle's, and the number of pairs the filter tested
equals the count of a plain re-statement of the band rule on the oracle's
fingerprints.
"""
import numpy as np
import pytest

import datagen
import oracle
from band_rule import expected_tested, popc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1711_08475_gb300 import build
    build.build()
    import paper_1711_08475_gb300 as m
    return m


@pytest.mark.parametrize("t,width", [("occ", 32), ("count", 32), ("occ", 16), ("occh", 16)])
@pytest.mark.parametrize("metric,k", [("ham", 1), ("lev", 1), ("lev", 2), ("ham", 0)])
@pytest.mark.parametrize("tq", [256, 24])
def test_band_counts_and_results(fp, t, width, metric, k, tq):
    if metric == "lev" and t == "occh":
        pytest.skip("occurrence-halved fingerprints bound only the Hamming distance")
    w = datagen.english1m(20000, 1500)
    d, q = w.dictionary, w.queries[metric]
    ix = fp.fp_build(d, fp_type=t, width=width)
    m = ix.symbol_map()
    r = fp.fp_query_ex(ix, q, k=k, metric=metric, tile_queries=tq)
    rp, idx = r.csr()
    st = r.stats()
    rp0, idx0 = oracle.match(d, q, k, metric)
    assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)
    _, _, pairs, surv = oracle.filter_match(d, q, k, metric, m, t, width, gray=True)
    assert st["pairs"] == pairs and st["survivors"] == surv
    assert st["pairs_tested"] == expected_tested(d, q, k, metric, m, t, width, tq)
    assert st["pairs_tested"] < st["pairs"]


def test_plain_scan_and_position_fingerprints_test_every_pair(fp):
    w = datagen.english1m(20000, 800)
    d, q = w.dictionary, w.queries["ham"]
    ix = fp.fp_build(d, fp_type="occ", width=32)
    st = fp.fp_query_ex(ix, q, k=1, metric="ham", mode="plain").stats()
    assert st["pairs_tested"] == st["pairs"] > 0
    ixp = fp.fp_build(d, fp_type="pos", width=32)
    r = fp.fp_query_ex(ixp, q, k=1, metric="ham")
    st = r.stats()
    assert st["pairs_tested"] == st["pairs"] > 0
    rp0, idx0 = oracle.match(d, q, 1, "ham")
    rp, idx = r.csr()
    assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)


@pytest.mark.parametrize("mode,variant", [("fused", 0), ("tiled", 2), ("tiled", 1)])
def test_band_other_forms(fp, mode, variant):
    w = datagen.english1m(30000, 2000)
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    for metric, k in (("lev", 1), ("ham", 2), ("lev", 3)):
        q = w.queries[metric]
        r = fp.fp_query_ex(ix, q, k=k, metric=metric, mode=mode, variant=variant)
        rp0, idx0 = oracle.match(w.dictionary, q, k, metric)
        rp, idx = r.csr()
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (mode, variant, metric, k)
        st = r.stats()
        assert st["pairs_tested"] <= st["pairs"]


def test_band_after_new_symbol_map(fp):
    """A new map changes every weight: the index is re-ordered and its table rebuilt."""
    w = datagen.english1m(20000, 1000)
    d, q = w.dictionary, w.queries["lev"]
    ix = fp.fp_build(d, fp_type="occ", width=16)
    m2 = oracle.map_from_order(b"zyxwvutsrqponmlk")  # 16 fields, rarely used letters first
    ix.set_symbol_map(m2)
    r = fp.fp_query_ex(ix, q, k=1, metric="lev")
    rp0, idx0 = oracle.match(d, q, 1, "lev")
    rp, idx = r.csr()
    assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)
    st = r.stats()
    assert st["pairs_tested"] == expected_tested(d, q, 1, "lev", ix.symbol_map(), "occ", 16, 64)  # default tile
    _, _, _, surv = oracle.filter_match(d, q, 1, "lev", ix.symbol_map(), "occ", 16, gray=True)
    assert st["survivors"] == surv


@pytest.mark.parametrize("metric", ["ham", "lev"])
def test_band_at_scale(fp, metric):
    """Bins with many tiles (8,000 patterns): the bands skip a large share of the pairs."""
    w = datagen.english1m(50000, 8000)
    d, q = w.dictionary, w.queries[metric]
    ix = fp.fp_build(d, fp_type="count", width=32)
    m = ix.symbol_map()
    for tq in (128, 64):
        r = fp.fp_query_ex(ix, q, k=1, metric=metric, tile_queries=tq)
        st = r.stats()
        rp0, idx0 = oracle.match(d, q, 1, metric)
        rp, idx = r.csr()
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)
        assert st["pairs_tested"] == expected_tested(d, q, 1, metric, m, "count", 32, tq)
        assert st["pairs_tested"] < 0.95 * st["pairs"]


def test_batched_plan_falls_back_to_whole_buckets(fp):
    """The batched pipeline's planner scratch holds n / 32 + bins tiles (bins:
    256 per (k, metric) group the run may hold, 32 groups); 12,000 patterns at
    one pattern per tile need more, so the device plans whole buckets instead:
    every eligible pair is tested, the answers stay the oracle's.  With 64 per
    tile the bands apply."""
    w = datagen.english1m(20000, 6000)
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    parts, spec = [], []
    for metric, k, n in (("lev", 1, 5000), ("ham", 1, 5000), ("lev", 2, 2000)):
        parts.append(w.queries[metric].subset(np.arange(n)))
        spec.append((n, k, metric))
    Q = datagen.Strings.concat(parts)
    for tq, banded in ((1, False), (64, True)):
        res = fp.fp_query_batched(ix, Q, batches=spec, tile_queries=tq)
        st = res.stats()
        if banded:
            assert st["pairs_tested"] < st["pairs"]
        else:
            assert st["pairs_tested"] == st["pairs"]
        rp, idx = res.csr()
        base = 0
        for (n, k, metric) in spec:
            sub = Q.subset(np.arange(base, base + n))
            rp0, idx0 = oracle.match(w.dictionary, sub, k, metric)
            assert np.array_equal(rp[base:base + n + 1] - rp[base], rp0), (tq, n, k, metric)
            assert np.array_equal(idx[rp[base]:rp[base + n]], idx0), (tq, n, k, metric)
            base += n


def short_words_twenty_letters():
    """Every word of length 1..3 over twenty letters (8,420 words) and, as
    patterns, every 23rd word of length 2..3 (366, deterministic, no draw).  The
    count fingerprint tracks 16 of the letters, the occurrence fingerprint all
    twenty, so the second check has letters of its own to reject on."""
    import itertools
    words = [bytes(t) for n in range(1, 4) for t in itertools.product(b"etaoinshrdlucmfwypvg", repeat=n)]
    d = datagen.Strings.from_list(words)
    rows = np.nonzero(d.lengths() >= 2)[0][::23]
    return d, d.subset(rows)


@pytest.mark.parametrize("mode", ["tiled", "fused"])
def test_combined_types_dense_batches(fp, mode):
    """Combined types where most pairs pass the first fingerprint: short words
    have fingerprints of few bits, so at k = 2 about 60 % of the eligible pairs
    pass count32 alone and most 32-pattern batches hold more passing (lane,
    pattern) cells than the hit queue; they take the one-pattern-at-a-time path,
    which checks the second fingerprints there.  Match lists equal the oracle's
    and the survivors are exactly the pairs whose two fingerprints both pass
    Eq. 1."""
    d, q = short_words_twenty_letters()
    ix = fp.fp_build(d, fp_type="count", width=32, combined=True)
    plain = fp.fp_build(d, fp_type="count", width=32)
    mc = ix.symbol_map()
    mo, _, _ = oracle.default().symbol_map(d.chars, "common", 32)
    fd = (oracle.fingerprints(d, mc, "count", 32).astype(np.uint64), oracle.fingerprints(d, mo, "occ", 32).astype(np.uint64))
    fq = (oracle.fingerprints(q, mc, "count", 32).astype(np.uint64), oracle.fingerprints(q, mo, "occ", 32).astype(np.uint64))
    for metric, k in (("lev", 2), ("ham", 2), ("lev", 1)):
        r = fp.fp_query_ex(ix, q, k=k, metric=metric, mode=mode)
        rp0, idx0 = oracle.match(d, q, k, metric)
        rp, idx = r.csr()
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (mode, metric, k)
        st = r.stats()
        assert st["survivors"] == pair_survivors(d, q, k, metric, fd, fq), (mode, metric, k)
        # dense: most eligible pairs pass the count fingerprint alone
        st1 = fp.fp_query_ex(plain, q, k=k, metric=metric, mode=mode).stats()
        assert st1["survivors"] == pair_survivors(d, q, k, metric, fd[:1], fq[:1])
        if k == 2:
            assert st1["survivors"] > 0.5 * st1["pairs"], (metric, st1)
        assert st["survivors"] < st1["survivors"]


def test_combined_types_dense_plan(fp):
    """The same dense workload through one captured plan with (k, metric) groups
    mixed, replayed once: every group's rows are the oracle's."""
    d, q = short_words_twenty_letters()
    ix = fp.fp_build(d, fp_type="count", width=32, combined=True)
    n = len(q)
    cut = [0, n // 3, 2 * n // 3, n]
    spec = [(cut[1] - cut[0], 2, "lev"), (cut[2] - cut[1], 1, "ham"), (cut[3] - cut[2], 2, "ham")]
    plan = fp.Plan(ix, n, len(q.chars), len(spec))
    for _ in range(2):  # capture, then replay
        rp, idx = plan.run(q, batches=spec).csr()
        for (m, k, metric), lo in zip(spec, cut):
            rp0, idx0 = oracle.match(d, q.subset(np.arange(lo, lo + m)), k, metric)
            assert np.array_equal(rp[lo:lo + m + 1] - rp[lo], rp0), (k, metric)
            assert np.array_equal(idx[rp[lo]:rp[lo + m]], idx0), (k, metric)
    plan.free()


def pair_survivors(d, q, k, metric, fps_d, fps_q):
    """Eligible pairs whose every fingerprint pair passes Eq. 1 (popc(x) <= 2k)."""
    ld, lq = d.lengths(), q.lengths()
    total = 0
    for i in range(len(q)):
        sel = (ld == lq[i]) if metric == "ham" else (np.abs(ld.astype(np.int64) - int(lq[i])) <= k)
        ok = np.ones(int(sel.sum()), dtype=bool)
        for fd_, fq_ in zip(fps_d, fps_q):
            ok &= popc(fd_[sel] ^ fq_[i]) <= 2 * k
        total += int(ok.sum())
    return total


@pytest.mark.parametrize("mode,variant", [("tiled", 0), ("fused", 0), ("tiled", 2), ("plain", 0)])
def test_combined_types(fp, mode, variant):
    """Combined types (occurrence + count): a pair survives only if its count32
    and its occ32 (32 most frequent symbols) fingerprints both pass Eq. 1; the
    match lists stay the oracle's and the survivors are exactly those pairs."""
    w = datagen.english1m(20000, 600)
    d = w.dictionary
    ix = fp.fp_build(d, fp_type="count", width=32, combined=True)
    plain = fp.fp_build(d, fp_type="count", width=32)
    mc = ix.symbol_map()
    mo, _, _ = oracle.default().symbol_map(d.chars, "common", 32)
    fd_c = oracle.fingerprints(d, mc, "count", 32).astype(np.uint64)
    fd_o = oracle.fingerprints(d, mo, "occ", 32).astype(np.uint64)
    for metric, k in (("ham", 1), ("lev", 1), ("lev", 2)):
        q = w.queries[metric]
        r = fp.fp_query_ex(ix, q, k=k, metric=metric, mode=mode, variant=variant)
        rp0, idx0 = oracle.match(d, q, k, metric)
        rp, idx = r.csr()
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (mode, variant, metric, k)
        st = r.stats()
        fq_c = oracle.fingerprints(q, mc, "count", 32).astype(np.uint64)
        fq_o = oracle.fingerprints(q, mo, "occ", 32).astype(np.uint64)
        assert st["survivors"] == pair_survivors(d, q, k, metric, (fd_c, fd_o), (fq_c, fq_o))
        st1 = fp.fp_query_ex(plain, q, k=k, metric=metric, mode=mode, variant=variant).stats()
        assert st["survivors"] < st1["survivors"] and st["pairs"] == st1["pairs"]
