"""The tensor-core filter (variant 2: F_D from FP8 dot products of +-1
fingerprint vectors) against the CPU oracle, through the C ABI (needs a GPU).

Its decisions must be exactly those of Eq. 1: the same survivor count as the
oracle's filter with the same map and encoding, and bit-identical match lists.
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


def check(fp, ix, d, q, k, metric, t, width, mode="tiled", survivors=True):
    res = fp.fp_query_ex(ix, q, k=k, metric=metric, mode=mode, variant=2)
    rp, idx = res.csr()
    rp0, idx0 = oracle.match(d, q, k, metric)
    assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (t, width, metric, k, mode)
    if survivors:
        _, _, pairs, surv = oracle.filter_match(d, q, k, metric, ix.symbol_map(), t, width, gray=True)
        st = res.stats()
        assert (st["pairs"], st["survivors"]) == (pairs, surv), (t, width, metric, k, mode)


@pytest.mark.parametrize("mode", ["tiled", "fused"])
@pytest.mark.parametrize("metric", ["ham", "lev"])
def test_uniform10k_full(fp, metric, mode):
    w = datagen.uniform10k()
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=16)
    check(fp, ix, w.dictionary, w.queries[metric], 1, metric, "occ", 16, mode)


@pytest.fixture(scope="module")
def english_small():
    return datagen.english1m(20000, 600)


@pytest.mark.parametrize("t,width", [("occ", 16), ("occ", 32), ("count", 16), ("count", 32), ("occh", 16),
                                     ("occh", 32)])
def test_types_widths_all_k(fp, english_small, t, width):
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type=t, width=width)
    for metric in ("ham", "lev"):
        if metric == "lev" and t == "occh":
            continue
        # k >= W/4 makes the threshold W - 4k <= 0: every pair passes Eq. 1
        for k in (0, 1, 2, 3, 4, 8, 15):
            check(fp, ix, w.dictionary, w.queries[metric], k, metric, t, width)


def test_fused_and_position_fallback(fp, english_small):
    w = english_small
    for t, width in (("count", 32), ("occ", 16)):
        ix = fp.fp_build(w.dictionary, fp_type=t, width=width)
        for metric, k in (("ham", 1), ("lev", 2)):
            check(fp, ix, w.dictionary, w.queries[metric], k, metric, t, width, mode="fused")
    # position fingerprints have no dot-product form: the population-count kernel runs
    ix = fp.fp_build(w.dictionary, fp_type="pos", width=32)
    check(fp, ix, w.dictionary, w.queries["ham"], 1, "ham", "pos", 32)


def test_ragged_tiles_and_edges(fp):
    """Buckets straddling the 128-pattern and 1024-word tile edges, duplicates,
    empty and 255-byte strings."""
    law = datagen.StringLaw(np.frombuffer(b"abcdefgh", np.uint8), np.ones(8), datagen.LengthLaw("uniform", 5, 7))
    base = law.draw(8, "rag", 3100)
    d = datagen.Strings.concat([base, base.subset(np.arange(0, 3100, 3))])
    q = datagen.Strings.concat([law.draw(8, "ragq", 257), d.subset(np.arange(0, 4000, 29))])
    for t, width in (("occ", 32), ("occ", 16), ("count", 32)):
        ix = fp.fp_build(d, fp_type=t, width=width)
        for metric in ("ham", "lev"):
            check(fp, ix, d, q, 1, metric, t, width)
    S = datagen.Strings.from_list
    d = S([b"", b"a", b"ab", b"ab", b"\x00\xff", b"x" * 255, b"x" * 254 + b"y", b"abc", b"", b"ba"])
    q = S([b"", b"a", b"ab", b"b", b"\x00\x00", b"x" * 255, b"zzz", b"ab" * 100, b"abcd", b"x" * 253])
    for t, width in (("occ", 32), ("count", 32), ("occ", 16)):
        ix = fp.fp_build(d, fp_type=t, width=width)
        for metric in ("ham", "lev"):
            for k in (0, 1, 2, 4, 15):
                check(fp, ix, d, q, k, metric, t, width, survivors=False)


def test_english1m_full_sampled(fp):
    """The benchmark's workload and launch configuration, sampled against the oracle."""
    w = datagen.english1m()
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    for metric in ("ham", "lev"):
        Q = w.queries[metric]
        r2 = fp.fp_query_ex(ix, Q, k=1, metric=metric, variant=2)
        r0 = fp.fp_query_ex(ix, Q, k=1, metric=metric, variant=0)
        rp, idx = r2.csr()
        rpb, idxb = r0.csr()
        assert np.array_equal(rp, rpb) and np.array_equal(idx, idxb)
        s2, s0 = r2.stats(), r0.stats()
        assert (s2["pairs"], s2["survivors"]) == (s0["pairs"], s0["survivors"])
        sel = np.sort(datagen.permutation(datagen.stream_key(5, "mma"), len(Q))[:120])
        rp0, idx0 = oracle.match(w.dictionary, Q.subset(sel), 1, metric)
        for j, qi in enumerate(sel):
            assert np.array_equal(idx[rp[qi]:rp[qi + 1]], idx0[rp0[j]:rp0[j + 1]])


def test_plan_and_server(fp, english_small):
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    qh, ql = w.queries["ham"], w.queries["lev"]
    both = datagen.Strings.concat([qh, ql])
    spec = [(len(qh), 1, "ham"), (len(ql), 2, "lev")]
    plan = fp.Plan(ix, len(both), len(both.chars), 2, variant=2)
    rp, idx = plan.run(both, batches=spec).csr()
    plan.free()
    srv = fp.Server(ix, lanes=2, variant=2)
    got = [srv.wait(srv.submit(qh, k=1, metric="ham"), 60).csr(), srv.wait(srv.submit(ql, k=2, metric="lev"), 60).csr()]
    srv.free()
    for (q, k, m), lo, g in ((spec[0] + (), 0, got[0]), (spec[1] + (), len(qh), got[1])):
        Q = qh if m == "ham" else ql
        rp0, idx0 = oracle.match(w.dictionary, Q, k, m)
        n = len(Q)
        assert np.array_equal(rp[lo:lo + n + 1] - rp[lo], rp0) and np.array_equal(idx[rp[lo]:rp[lo + n]], idx0)
        assert np.array_equal(g[0], rp0) and np.array_equal(g[1], idx0)
