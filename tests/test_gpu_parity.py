"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Match lists must be bit-identical (integer work).  The survivor count of the
filter must equal the oracle's count under Eq. 1 with the same map and
encoding, and every fingerprint the GPU builds must equal the oracle's.
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


def assert_same(res, rp0, idx0, what=""):
    rp, idx = res.csr()
    assert rp.shape == rp0.shape, what
    if not (np.array_equal(rp, rp0) and np.array_equal(idx, idx0)):
        bad = np.nonzero(np.diff(rp) != np.diff(rp0))[0][:5]
        raise AssertionError(f"{what}: match lists differ (first rows with different counts: {bad})")


def oracle_survivors(d, q, k, metric, m, t, width, b=2, p=3):
    _, _, pairs, surv = oracle.filter_match(d, q, k, metric, m, t, width, b=b, p=p, gray=True)
    return pairs, surv


# ---------------------------------------------------------------------------
# the smallest workload in full: 10,000 words / 1,000 queries, occ16, k = 1
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("mode", ["tiled", "plain", "fused"])
@pytest.mark.parametrize("metric", ["ham", "lev"])
def test_uniform10k_full(fp, metric, mode):
    w = datagen.uniform10k()
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=16)
    Q = w.queries[metric]
    res = fp.fp_query_ex(ix, Q, k=1, metric=metric, mode=mode)
    rp0, idx0 = oracle.match(w.dictionary, Q, 1, metric)
    assert_same(res, rp0, idx0, f"uniform10k {metric} {mode}")
    st = res.stats()
    m = ix.symbol_map()
    pairs, surv = oracle_survivors(w.dictionary, Q, 1, metric, m, "occ", 16)
    assert st["pairs"] == pairs == oracle.eligible_pairs(w.dictionary, Q, 1, metric)
    assert st["survivors"] == surv
    assert st["matches"] == len(idx0)


# ---------------------------------------------------------------------------
# every fingerprint type and width, several k, both metrics where Eq. 1 holds
# ---------------------------------------------------------------------------

TYPE_CASES = [("occ", 16), ("occ", 32), ("count", 16), ("count", 32), ("occh", 16), ("occh", 32),
              ("pos", 16), ("pos", 32)]


@pytest.fixture(scope="module")
def english_small():
    return datagen.english1m(20000, 600)


@pytest.mark.parametrize("t,width", TYPE_CASES)
def test_types_widths_english(fp, english_small, t, width):
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type=t, width=width)
    m = ix.symbol_map()
    m0, _, _ = oracle.symbol_map(w.dictionary.chars, "common", oracle.layout(t, width)["sigma"])
    assert np.array_equal(m, m0), "symbol map differs from the oracle's"
    for metric in ("ham", "lev"):
        if metric == "lev" and t in ("occh", "pos"):
            continue
        Q = w.queries[metric]
        for k in (0, 1, 2, 3):
            res = fp.fp_query(ix, Q, k=k, metric=metric)
            rp0, idx0 = oracle.match(w.dictionary, Q, k, metric)
            assert_same(res, rp0, idx0, f"{t}{width} {metric} k={k}")
            pairs, surv = oracle_survivors(w.dictionary, Q, k, metric, m, t, width)
            st = res.stats()
            assert (st["pairs"], st["survivors"]) == (pairs, surv), (t, width, metric, k)


def test_hamming_only_types_reject_levenshtein(fp, english_small):
    from paper_1711_08475_gb300 import native
    for t in ("occh", "pos"):
        ix = fp.fp_build(english_small.dictionary.subset(np.arange(500)), fp_type=t, width=32)
        with pytest.raises(fp.FpError) as e:
            fp.fp_query(ix, english_small.queries["lev"].subset(np.arange(10)), k=1, metric="lev")
        assert e.value.code == native.FP_E_UNSUPPORTED


@pytest.mark.parametrize("symbol_set", ["common", "rare", "mixed"])
def test_symbol_sets(fp, english_small, symbol_set):
    w = english_small
    for t, width in (("occ", 32), ("count", 16), ("pos", 16)):
        ix = fp.fp_build(w.dictionary, fp_type=t, width=width, symbol_set=symbol_set)
        m0, _, _ = oracle.symbol_map(w.dictionary.chars, symbol_set, oracle.layout(t, width)["sigma"])
        assert np.array_equal(ix.symbol_map(), m0), (symbol_set, t, width)
        Q = w.queries["ham"]
        res = fp.fp_query(ix, Q, k=1, metric="ham")
        rp0, idx0 = oracle.match(w.dictionary, Q, 1, "ham")
        assert_same(res, rp0, idx0, f"{symbol_set} {t}{width}")


def test_url_long_strings(fp):
    w = datagen.url2m(8000, 300)
    for t in ("occ", "pos"):
        ix = fp.fp_build(w.dictionary, fp_type=t, width=32)
        for metric in ("ham", "lev"):
            if metric == "lev" and t == "pos":
                continue
            for k in (1, 2, 5):
                Q = w.queries[metric]
                res = fp.fp_query(ix, Q, k=k, metric=metric)
                rp0, idx0 = oracle.match(w.dictionary, Q, k, metric)
                assert_same(res, rp0, idx0, f"url {t} {metric} k={k}")


# ---------------------------------------------------------------------------
# fingerprints themselves
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("t,width", TYPE_CASES)
def test_fingerprint_arrays(fp, t, width):
    law = datagen.StringLaw(np.arange(0, 256, dtype=np.uint8), np.ones(256), datagen.LengthLaw("uniform", 0, 255))
    S = law.draw(3, "fp-any-bytes", 3000)
    eng = datagen.english1m(5000, 10).dictionary
    ix = fp.fp_build(eng, fp_type=t, width=width)
    m = ix.symbol_map()
    for strings in (S, eng):
        got = ix.fingerprint(strings)
        want = oracle.fingerprints(strings, m, t, width)
        assert np.array_equal(got, want), (t, width, np.nonzero(got != want)[0][:5])
    inst = datagen.Strings.from_list([b"instance"])
    order = b"etaoinshrdlcumwf"[: oracle.layout(t, 16)["sigma"]]
    if width == 16:
        ix2 = fp.fp_build(eng, fp_type=t, width=16, custom_map=oracle.map_from_order(order))
        want = {"occ": 0x0877, "occh": 0x1D26, "count": 0x1D15, "pos": 0x8F1F}[t]
        assert int(ix2.fingerprint(inst)[0]) == want  # Sec. 3.1 worked example (count Gray-coded)


def test_custom_and_learned_style_maps(fp, english_small):
    """Any many-to-one map keeps the bound sound (occ, count): results stay exact."""
    w = english_small
    r = datagen.randint(datagen.stream_key(9, "map"), 256, -1, 31)
    m = np.full(256, -1, np.int8)
    for c in range(ord("a"), ord("z") + 1):
        m[c] = r[c]
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32, custom_map=m)
    for metric in ("ham", "lev"):
        Q = w.queries[metric]
        rp0, idx0 = oracle.match(w.dictionary, Q, 1, metric)
        assert_same(fp.fp_query(ix, Q, k=1, metric=metric), rp0, idx0, "custom map")
        pairs, surv = oracle_survivors(w.dictionary, Q, 1, metric, m, "occ", 32)
        assert fp.fp_query(ix, Q, k=1, metric=metric).stats()["survivors"] == surv
    # replace the map in place: fingerprints are rebuilt on the device
    m2 = np.where(m >= 0, (m.astype(np.int32) * 7) % 32, -1).astype(np.int8)
    ix.set_symbol_map(m2)
    assert np.array_equal(ix.symbol_map(), m2)
    Q = w.queries["lev"]
    rp0, idx0 = oracle.match(w.dictionary, Q, 2, "lev")
    assert_same(fp.fp_query(ix, Q, k=2, metric="lev"), rp0, idx0, "after set_symbol_map")
    pairs, surv = oracle_survivors(w.dictionary, Q, 2, "lev", m2, "occ", 32)
    assert fp.fp_query(ix, Q, k=2, metric="lev").stats()["survivors"] == surv


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------


def test_edge_cases(fp):
    S = datagen.Strings.from_list
    d = S([b"", b"a", b"ab", b"ab", b"\x00\xff", b"x" * 255, b"x" * 254 + b"y", b"abc", b"", b"ba"])
    q = S([b"", b"a", b"ab", b"b", b"\x00\x00", b"x" * 255, b"zzz", b"ab" * 100, b"abcd", b"x" * 253])
    for t, width in (("occ", 32), ("count", 32), ("occ", 16), ("pos", 32), ("occh", 16)):
        ix = fp.fp_build(d, fp_type=t, width=width)
        for metric in ("ham", "lev"):
            if metric == "lev" and t in ("occh", "pos"):
                continue
            for k in (0, 1, 2, 4, 15):
                res = fp.fp_query(ix, q, k=k, metric=metric)
                rp0, idx0 = oracle.match(d, q, k, metric)
                assert_same(res, rp0, idx0, f"edge {t}{width} {metric} k={k}")
    ix = fp.fp_build(d, fp_type="occ", width=32)
    # zero queries
    r = fp.fp_query(ix, S([]), k=1, metric="lev")
    rp, idx = r.csr()
    assert list(rp) == [0] and len(idx) == 0
    # empty dictionary
    e = fp.fp_build(S([]), fp_type="occ", width=32)
    rp, idx = fp.fp_query(e, q, k=3, metric="lev").csr()
    assert np.all(rp == 0)
    # invalid arguments
    from paper_1711_08475_gb300 import native
    with pytest.raises(fp.FpError) as ex:
        fp.fp_query(ix, q, k=16, metric="lev")
    assert ex.value.code == native.FP_E_INVAL
    bad = datagen.Strings(np.zeros(300, np.uint8), np.array([0, 300], np.int64))
    with pytest.raises(fp.FpError) as ex:
        fp.fp_query(ix, bad, k=1, metric="ham")
    assert ex.value.code == native.FP_E_INVAL
    with pytest.raises(fp.FpError) as ex:
        fp.fp_build(bad, fp_type="occ", width=32)
    assert ex.value.code == native.FP_E_INVAL


def test_ragged_tiles_and_duplicates(fp):
    """Bucket sizes straddling tile boundaries, many queries per bucket, duplicate words."""
    law = datagen.StringLaw(np.frombuffer(b"abcdefgh", np.uint8), np.ones(8), datagen.LengthLaw("uniform", 5, 7))
    base = law.draw(4, "rag", 6000)
    d = datagen.Strings.concat([base, base.subset(np.arange(0, 6000, 3))])  # duplicates
    q = datagen.Strings.concat([law.draw(4, "ragq", 900), d.subset(np.arange(0, 8000, 17))])
    for tq in (1, 7, 64, 256):
        for wpt in (4, 8):
            for t, width in (("occ", 32), ("occ", 16)):
                ix = fp.fp_build(d, fp_type=t, width=width)
                for metric in ("ham", "lev"):
                    res = fp.fp_query_ex(ix, q, k=1, metric=metric, tile_queries=tq, words_per_thread=wpt)
                    rp0, idx0 = oracle.match(d, q, 1, metric)
                    assert_same(res, rp0, idx0, f"ragged tq={tq} v={wpt} {t}{width} {metric}")


def test_device_resident_inputs(fp):
    import torch
    w = datagen.uniform10k(4000, 300)
    dc = torch.from_numpy(w.dictionary.chars).cuda()
    do = torch.from_numpy(w.dictionary.offsets).cuda()
    ix = fp.fp_build(dc, do, fp_type="occ", width=16)
    Q = w.queries["lev"]
    res = fp.fp_query(ix, torch.from_numpy(Q.chars).cuda(), torch.from_numpy(Q.offsets).cuda(), k=1, metric="lev")
    rp0, idx0 = oracle.match(w.dictionary, Q, 1, "lev")
    assert_same(res, rp0, idx0, "device inputs")


# ---------------------------------------------------------------------------
# full sizes, in the benchmark's launch configuration: sampled queries
# ---------------------------------------------------------------------------


def sampled_check(fp, d, Q, ix, k, metric, n_sample, seed, **kw):
    res = fp.fp_query_ex(ix, Q, k=k, metric=metric, **kw)
    rp, idx = res.csr()
    # properties that hold at any size
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(idx)
    for qi in range(0, len(Q), max(1, len(Q) // 2000)):
        row = idx[rp[qi]:rp[qi + 1]]
        assert np.all(np.diff(row) > 0)
    sel = np.sort(datagen.permutation(datagen.stream_key(seed, "sample"), len(Q))[:n_sample])
    sub = Q.subset(sel)
    rp0, idx0 = oracle.match(d, sub, k, metric)
    for j, qi in enumerate(sel):
        got = idx[rp[qi]:rp[qi + 1]]
        want = idx0[rp0[j]:rp0[j + 1]]
        assert np.array_equal(got, want), f"query {qi}: {got[:8]} vs {want[:8]}"
    st = res.stats()
    assert st["pairs"] == oracle.eligible_pairs(d, Q, k, metric)
    return st


def test_english1m_full_sampled(fp):
    w = datagen.english1m()
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    for metric in ("ham", "lev"):
        st = sampled_check(fp, w.dictionary, w.queries[metric], ix, 1, metric, 150, 1)
        assert st["survivors"] < st["pairs"]
    ix2 = fp.fp_build(w.dictionary, fp_type="occh", width=32)
    sampled_check(fp, w.dictionary, w.queries["ham"], ix2, 1, "ham", 150, 2)


def test_url2m_full_sampled(fp):
    w = datagen.url2m()
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    for metric in ("ham", "lev"):
        sampled_check(fp, w.dictionary, w.queries[metric], ix, 1, metric, 60, 3)
    ix2 = fp.fp_build(w.dictionary, fp_type="pos", width=32)
    sampled_check(fp, w.dictionary, w.queries["ham"], ix2, 1, "ham", 60, 4)


# ---------------------------------------------------------------------------
# the fused form (filter and verification in one persistent kernel)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("t,width", [("occ", 32), ("count", 32), ("pos", 32), ("occ", 16), ("occh", 16)])
def test_fused_form(fp, english_small, t, width):
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type=t, width=width)
    m = ix.symbol_map()
    for metric in ("ham", "lev"):
        if metric == "lev" and t in ("occh", "pos"):
            continue
        Q = w.queries[metric]
        for k in (0, 1, 2, 4, 7):
            res = fp.fp_query_ex(ix, Q, k=k, metric=metric, mode="fused")
            rp0, idx0 = oracle.match(w.dictionary, Q, k, metric)
            assert_same(res, rp0, idx0, f"fused {t}{width} {metric} k={k}")
            pairs, surv = oracle_survivors(w.dictionary, Q, k, metric, m, t, width)
            st = res.stats()
            assert (st["pairs"], st["survivors"], st["matches"]) == (pairs, surv, len(idx0))


def test_fused_long_strings_and_edges(fp):
    w = datagen.url2m(6000, 200)
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    for k in (1, 3, 15):
        Q = w.queries["lev"]
        rp0, idx0 = oracle.match(w.dictionary, Q, k, "lev")
        assert_same(fp.fp_query_ex(ix, Q, k=k, metric="lev", mode="fused"), rp0, idx0, f"fused url k={k}")
    S = datagen.Strings.from_list
    d = S([b"", b"a", b"ab", b"ab", b"\x00\xff", b"x" * 255, b"abc", b"ba"])
    q = S([b"", b"a", b"ab", b"b", b"\x00\x00", b"x" * 255, b"zzz", b"abcd"])
    ix2 = fp.fp_build(d, fp_type="occ", width=32)
    for metric in ("ham", "lev"):
        for k in (0, 1, 2, 15):
            rp0, idx0 = oracle.match(d, q, k, metric)
            assert_same(fp.fp_query_ex(ix2, q, k=k, metric=metric, mode="fused"), rp0, idx0, f"fused edge {metric} {k}")


# ---------------------------------------------------------------------------
# batched queries (mixed k and metric in one pass) and captured plans
# ---------------------------------------------------------------------------


def mixed_batches(w, sizes, seed):
    """Consecutive batches drawn from both query sets with assorted (k, metric)."""
    parts, spec = [], []
    r = datagen.randint(datagen.stream_key(seed, "mix"), 2 * len(sizes), 0, 7)
    for i, n in enumerate(sizes):
        metric = ("ham", "lev")[int(r[2 * i]) % 2]
        k = int(r[2 * i + 1]) % 4
        Q = w.queries[metric]
        start = (i * 97) % max(1, len(Q) - n)
        parts.append(Q.subset(np.arange(start, start + n)))
        spec.append((n, k, metric))
    return datagen.Strings.concat(parts), spec


def check_batched(res, w, Q, spec):
    rp, idx = res.csr()
    base = 0
    for (n, k, metric) in spec:
        sub = Q.subset(np.arange(base, base + n))
        rp0, idx0 = oracle.match(w.dictionary, sub, k, metric)
        got_rp = rp[base:base + n + 1] - rp[base]
        assert np.array_equal(got_rp, rp0), (n, k, metric)
        assert np.array_equal(idx[rp[base]:rp[base + n]], idx0), (n, k, metric)
        base += n


def test_batched_mixed(fp, english_small):
    w = english_small
    Q, spec = mixed_batches(w, [1, 37, 150, 0, 64, 5, 200, 3], 21)
    for t, width in (("occ", 32), ("count", 32), ("occ", 16)):
        ix = fp.fp_build(w.dictionary, fp_type=t, width=width)
        res = fp.fp_query_batched(ix, Q, batches=spec)
        check_batched(res, w, Q, spec)


def test_plan_graph_replay(fp, english_small):
    import torch
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    Q1, spec1 = mixed_batches(w, [100, 7, 250, 31], 5)
    Q2, spec2 = mixed_batches(w, [300, 1, 12], 6)
    plan = fp.Plan(ix, max_queries=1000, max_chars=20000, max_batches=16)
    launches = []
    for rep in range(3):  # capture, then two replays of the same shape
        before = fp.fp_launch_count()
        check_batched(plan.run(Q1, batches=spec1), w, Q1, spec1)
        launches.append(fp.fp_launch_count() - before)
    assert launches[1] == launches[2] > 0
    check_batched(plan.run(Q2, batches=spec2), w, Q2, spec2)  # another shape: captured again
    dc, do = torch.from_numpy(Q1.chars).cuda(), torch.from_numpy(Q1.offsets).cuda()
    check_batched(plan.run(dc, do, batches=spec1), w, Q1, spec1)  # device inputs, replayed
    # a batch set larger than the plan is rejected
    with pytest.raises(fp.FpError):
        plan.run(*mixed_batches(w, [600, 600], 7)[:1], batches=[(600, 1, "ham"), (600, 1, "lev")])


def test_autotuner(fp, english_small, tmp_path, monkeypatch):
    w = english_small
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    best, allr = fp.fp_autotune(ix, w.queries["lev"], k=1, metric="lev", mode="tiled", reps=1)
    assert len(allr) == 16 and best["ms"] == min(r["ms"] for r in allr)
    assert best["tile_queries"] in (32, 64, 128, 256) and best["words_per_thread"] in (4, 8)
    best_f, allf = fp.fp_autotune(ix, w.queries["ham"], k=2, metric="ham", mode="fused", reps=1)
    assert len(allf) == 4 and all(r["words_per_thread"] == 4 for r in allf)
    from paper_1711_08475_gb300 import tune
    monkeypatch.setenv("FPMATCH_TUNE_CACHE", str(tmp_path / "tune.json"))
    o1 = tune.tuned_opts(ix, w.queries["lev"], k=1, metric="lev")
    o2 = tune.tuned_opts(ix, w.queries["lev"], k=1, metric="lev")  # from the cache
    assert o1 == o2 and (tmp_path / "tune.json").exists()
    rp0, idx0 = oracle.match(w.dictionary, w.queries["lev"], 1, "lev")
    res = fp.fp_query_ex(ix, w.queries["lev"], k=1, metric="lev", tile_queries=o1["tile_queries"],
                         words_per_thread=o1["words_per_thread"], variant=o1["variant"])
    assert_same(res, rp0, idx0, "tuned shape")


# ---------------------------------------------------------------------------
# the batched and the serving workloads at full size, sampled
# ---------------------------------------------------------------------------


def test_batched10m_full_sampled(fp):
    """10,000,000 words, 256 uneven batches (k in {1, 2}, Ham and Lev) in one
    captured plan with the autotuned tile, as the benchmark runs it; sampled
    patterns of every (k, metric) pair against the oracle."""
    from paper_1711_08475_gb300 import tune
    w, batches = datagen.batched10m()
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    allq = datagen.Strings.concat([b.queries for b in batches])
    spec = [(len(b.queries), b.k, b.metric) for b in batches]
    sample = datagen.Strings.concat([b.queries for b in batches if (b.k, b.metric) == (1, "lev")])
    opts = tune.tuned_opts(ix, sample.subset(np.arange(min(len(sample), 20000))), k=1, metric="lev", mode="fused",
                           reps=1)
    plan = fp.Plan(ix, len(allq), len(allq.chars), len(spec), tile_queries=opts["tile_queries"],
                   variant=opts["variant"])
    r = plan.run(allq, batches=spec)
    rp, idx = r.csr()
    st = r.stats()
    plan.free()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(idx) == st["matches"]
    base, picks = 0, {}
    for n, k, metric in spec:
        sel = picks.setdefault((k, metric), [])
        if n and len(sel) < 12:
            sel.extend(sorted({base, base + n // 2, base + n - 1}))
        base += n
    for (k, metric), rows in picks.items():
        rows = np.array(sorted(set(rows)), np.int64)
        rp0, idx0 = oracle.match(w.dictionary, allq.subset(rows), k, metric)
        for j, q in enumerate(rows):
            assert np.array_equal(idx[rp[q]:rp[q + 1]], idx0[rp0[j]:rp0[j + 1]]), (k, metric, q)


def test_serving5m_full_sampled(fp):
    """5,000,000 URL-like strings with a learned map, the Poisson request stream
    replayed against the server (arrival times compressed to 1 s); sampled
    patterns against the oracle, and the same rows as the frequency index."""
    w, reqs = datagen.serving5m()
    freq = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    train = datagen.make_queries(w.dictionary, w.law, w.seed, "train/lev", 20000, 0.5, "lev")
    s = fp.fp_sample_pairs(freq, train, k=1, metric="lev", n_samples=400000, seed=11)
    mp, _, _ = fp.fp_learn_map(32, s["masks"], s["match"], k=1, seed=3)
    lrn = fp.fp_build(w.dictionary, fp_type="occ", width=32, custom_map=mp)
    allq = datagen.Strings.concat([r.queries for r in reqs])
    sizes = [len(r.queries) for r in reqs]
    last = max(r.arrival_s for r in reqs) or 1.0
    arrive = np.array([int(r.arrival_s / last * 1e6) for r in reqs], np.int64)
    srv = fp.Server(lrn, lanes=4)
    res, lat = srv.replay(allq, request_sizes=sizes, arrival_us=arrive, k=1, metric="lev")
    srv.free()
    rp, idx = res.csr()
    rpf, idxf = fp.fp_query(freq, allq, k=1, metric="lev").csr()
    assert np.array_equal(rp, rpf) and np.array_equal(idx, idxf)
    pick = np.arange(0, len(allq), max(1, len(allq) // 40))
    rp0, idx0 = oracle.match(w.dictionary, allq.subset(pick), 1, "lev")
    for j, q in enumerate(pick):
        assert np.array_equal(idx[rp[q]:rp[q + 1]], idx0[rp0[j]:rp0[j + 1]])
    assert (lat > 0).all()


def test_levenshtein_one_exhaustive(fp):
    """Every pair of strings over {a, b, c} up to length 4, plus longer strings
    around the 4- and 16-byte word and row edges, at k = 1 and k = 0 (the
    direct Lev <= 1 test and the strip recurrence must agree with the DP)."""
    import itertools
    small = [b""] + [bytes(t) for n in range(1, 5) for t in itertools.product(b"abc", repeat=n)]
    law = datagen.StringLaw(np.frombuffer(b"ab", np.uint8), np.ones(2), datagen.LengthLaw("uniform", 14, 36))
    long = law.draw(12, "edge", 300).to_list()
    muts = datagen.make_queries(datagen.Strings.from_list(long), law, 12, "edge/q", 300, 1.0, "lev").to_list()
    d = datagen.Strings.from_list(small + long)
    q = datagen.Strings.from_list(small + muts)
    for t, width in (("occ", 16), ("count", 32)):
        ix = fp.fp_build(d, fp_type=t, width=width)
        for k in (0, 1):
            for mode in ("tiled", "fused"):
                res = fp.fp_query_ex(ix, q, k=k, metric="lev", mode=mode)
                rp0, idx0 = oracle.match(d, q, k, "lev")
                assert_same(res, rp0, idx0, f"lev k={k} {t}{width} {mode}")
