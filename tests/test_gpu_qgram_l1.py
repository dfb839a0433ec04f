"""q-gram fingerprints (Sec. 5, future work) and count fingerprints compared by
the L1 distance of their binary-coded counts (Sec. 3.3 remark after Eq. 1):
the CUDA path against the CPU oracle, through the C ABI (needs a GPU).

Exact integer checks: the q-grams the GPU selects, every fingerprint it
builds, the match lists, and the number of pairs that pass the bound
(F_D <= 2qk for q-grams, Eq. 1 on the L1 distance for counts) all equal the
oracle's.
"""
import numpy as np
import pytest

import datagen
import oracle

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


@pytest.fixture(scope="module")
def english():
    return datagen.english1m(20000, 500)


@pytest.fixture(scope="module")
def urls():
    return datagen.url2m(6000, 200)


def same(res, rp0, idx0):
    rp, idx = res.csr()
    return np.array_equal(rp, rp0) and np.array_equal(idx, idx0)


def any_bytes(n, seed=3):
    law = datagen.StringLaw(np.arange(0, 256, dtype=np.uint8), np.ones(256), datagen.LengthLaw("uniform", 0, 255))
    return law.draw(seed, "qgram-any-bytes", n)


# ---------------------------------------------------------------------------
# q-gram fingerprints
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("width", [16, 32])
def test_qgram_map_and_fingerprints(fp, english, urls, q, width):
    for d in (english.dictionary, urls.dictionary):
        ix = fp.fp_build(d, fp_type="qgram", width=width, qgram=q)
        grams0, _ = oracle.qgram_map(d, q, width)
        assert np.array_equal(ix.qgrams(), grams0), (q, width)
        info = ix.info()
        assert info["qgram"] == q and info["sigma"] == width
        for strings in (d.subset(np.arange(0, len(d), 7)), any_bytes(2000),
                        datagen.Strings.from_list([b"", b"a", b"ab", b"abc", b"the", b"ththth"])):
            got = ix.fingerprint(strings)
            want = oracle.qgram_fingerprints(strings, grams0)
            assert np.array_equal(got, want), (q, width, np.nonzero(got != want)[0][:5])


def test_qgram_one_is_occurrence(fp, english):
    """With q = 1 the fields are the most frequent symbols: the fingerprints of
    the q-gram index equal those of the occurrence index (Sec. 3.2)."""
    d = english.dictionary
    a = fp.fp_build(d, fp_type="qgram", width=32, qgram=1)
    b = fp.fp_build(d, fp_type="occ", width=32)
    S = any_bytes(1500, 5)
    assert np.array_equal(a.fingerprint(S), b.fingerprint(S))


@pytest.mark.parametrize("mode", ["tiled", "fused", "plain"])
@pytest.mark.parametrize("q", [2, 3])
def test_qgram_parity(fp, english, urls, q, mode):
    for w in (english, urls):
        d = w.dictionary
        ix = fp.fp_build(d, fp_type="qgram", width=32, qgram=q)
        grams0, _ = oracle.qgram_map(d, q, 32)
        dfp = oracle.qgram_fingerprints(d, grams0)
        for metric in ("ham", "lev"):
            Q = w.queries[metric]
            qfp = oracle.qgram_fingerprints(Q, grams0)
            for k in (0, 1, 2):
                rp0, idx0, pairs, surv = oracle.filter_match_fps(d, Q, k, metric, dfp, qfp, "weight", 32, q=q)
                res = fp.fp_query_ex(ix, Q, k=k, metric=metric, mode=mode)
                assert same(res, rp0, idx0), (w.name, q, metric, k, mode)
                st = res.stats()
                assert (st["pairs"], st["survivors"]) == (pairs, surv), (w.name, q, metric, k, mode)


def test_qgram_batched_plan(fp, english):
    """Mixed (k, metric) batches through one captured plan: the per-group
    threshold 2qk reaches the fused kernel and the banded planner."""
    d = english.dictionary
    ix = fp.fp_build(d, fp_type="qgram", width=32, qgram=2)
    parts = [(english.queries["ham"].subset(np.arange(0, 150)), 1, "ham"),
             (english.queries["lev"].subset(np.arange(0, 200)), 2, "lev"),
             (english.queries["lev"].subset(np.arange(200, 320)), 1, "lev")]
    allq = datagen.Strings.concat([p[0] for p in parts])
    plan = fp.Plan(ix, len(allq), len(allq.chars), len(parts))
    for _ in range(2):  # capture, then replay
        rp, idx = plan.run(allq, batches=[(len(p[0]), p[1], p[2]) for p in parts]).csr()
        lo = 0
        for Q, k, metric in parts:
            rp0, idx0 = oracle.match(d, Q, k, metric)
            hi = lo + len(Q)
            assert np.array_equal(rp[lo:hi + 1] - rp[lo], rp0) and np.array_equal(idx[rp[lo]:rp[hi]], idx0)
            lo = hi
    plan.free()


def test_qgram_rejects_other_sets_and_maps(fp, english):
    from paper_1711_08475_gb300 import native
    d = english.dictionary.subset(np.arange(300))
    with pytest.raises(fp.FpError) as e:
        fp.fp_build(d, fp_type="qgram", width=32, qgram=2, symbol_set="rare")
    assert e.value.code == native.FP_E_UNSUPPORTED
    with pytest.raises(fp.FpError) as e:
        fp.fp_build(d, fp_type="qgram", width=32, qgram=4)
    assert e.value.code == native.FP_E_UNSUPPORTED
    ix = fp.fp_build(d, fp_type="qgram", width=32, qgram=2)
    with pytest.raises(fp.FpError) as e:
        ix.set_symbol_map(np.full(256, -1, np.int8))
    assert e.value.code == native.FP_E_UNSUPPORTED


# ---------------------------------------------------------------------------
# count fingerprints, binary code, L1 distance
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("width", [16, 32])
def test_count_l1_fingerprints(fp, english, width):
    d = english.dictionary
    ix = fp.fp_build(d, fp_type="count_l1", width=width)
    m = ix.symbol_map()
    m0, _, _ = oracle.symbol_map(d.chars, "common", width // 2)
    assert np.array_equal(m, m0)
    for strings in (d.subset(np.arange(0, len(d), 5)), any_bytes(2000, 7)):
        got = ix.fingerprint(strings)
        want = oracle.fingerprints(strings, m, "count", width, gray=False)
        assert np.array_equal(got, want), (width, np.nonzero(got != want)[0][:5])


@pytest.mark.parametrize("mode", ["tiled", "fused", "plain"])
@pytest.mark.parametrize("width", [16, 32])
def test_count_l1_parity(fp, english, urls, width, mode):
    for w in (english, urls):
        d = w.dictionary
        ix = fp.fp_build(d, fp_type="count_l1", width=width)
        m = ix.symbol_map()
        dfp = oracle.fingerprints(d, m, "count", width, gray=False)
        gray_ix = fp.fp_build(d, fp_type="count", width=width)
        for metric in ("ham", "lev"):
            Q = w.queries[metric]
            qfp = oracle.fingerprints(Q, m, "count", width, gray=False)
            for k in (0, 1, 2):
                rp0, idx0, pairs, surv = oracle.filter_match_fps(d, Q, k, metric, dfp, qfp, "count_l1", width)
                res = fp.fp_query_ex(ix, Q, k=k, metric=metric, mode=mode)
                assert same(res, rp0, idx0), (w.name, width, metric, k, mode)
                st = res.stats()
                assert (st["pairs"], st["survivors"]) == (pairs, surv), (w.name, width, metric, k, mode)
                # never more survivors than the Gray-coded count distance lets through
                assert st["survivors"] <= fp.fp_query(gray_ix, Q, k=k, metric=metric).stats()["survivors"]


# ---------------------------------------------------------------------------
# full sizes: the bench's workloads, sampled
# ---------------------------------------------------------------------------


def full_sampled(fp, d, Q, ix, k, metric, dfp, qfp_of, kind, q, n_sample, seed):
    """The whole batch through the bench's launch configuration: properties that
    hold at any size, the match lists of sampled patterns against brute force,
    and the sampled patterns' pairs passing the bound against the oracle's."""
    res = fp.fp_query_ex(ix, Q, k=k, metric=metric)
    rp, idx = res.csr()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(idx)
    assert res.stats()["pairs"] == oracle.eligible_pairs(d, Q, k, metric)
    sel = np.sort(datagen.permutation(datagen.stream_key(seed, "sample"), len(Q))[:n_sample])
    sub = Q.subset(sel)
    rp0, idx0, pairs0, surv0 = oracle.filter_match_fps(d, sub, k, metric, dfp, qfp_of(sub), kind, 32, q=q)
    for j, qi in enumerate(sel):
        assert np.array_equal(idx[rp[qi]:rp[qi + 1]], idx0[rp0[j]:rp0[j + 1]]), qi
    st = fp.fp_query_ex(ix, sub, k=k, metric=metric).stats()
    assert (st["pairs"], st["survivors"]) == (pairs0, surv0)


def test_qgram_url2m_full_sampled(fp):
    w = datagen.url2m()
    d = w.dictionary
    ix = fp.fp_build(d, fp_type="qgram", width=32, qgram=2)
    grams, _ = oracle.qgram_map(d, 2, 32)
    assert np.array_equal(ix.qgrams(), grams)
    dfp = oracle.qgram_fingerprints(d, grams)
    for metric in ("ham", "lev"):
        full_sampled(fp, d, w.queries[metric], ix, 1, metric, dfp, lambda S: oracle.qgram_fingerprints(S, grams),
                     "weight", 2, 40, 5)


def test_count_l1_english1m_full_sampled(fp):
    w = datagen.english1m()
    d = w.dictionary
    ix = fp.fp_build(d, fp_type="count_l1", width=32)
    m = ix.symbol_map()
    dfp = oracle.fingerprints(d, m, "count", 32, gray=False)
    for metric in ("ham", "lev"):
        full_sampled(fp, d, w.queries[metric], ix, 1, metric, dfp,
                     lambda S: oracle.fingerprints(S, m, "count", 32, gray=False), "count_l1", 1, 60, 6)
