"""Serving loop (continuous batching) on the GPU: each request's match lists
are the same alone and merged with others, launches overlap, admission keeps
to the memory budget, and waits are bounded."""
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
def served(fp):
    """200,000 URL-like strings, occ32; 40 requests of 1..600 patterns (Lev mutations + random)."""
    w, reqs = datagen.serving5m(200000, duration_s=1.0, rate_qps=20000.0, max_request=600)
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    reqs = reqs[:40]
    return w, ix, reqs


def rows(rp, idx, lo, hi):
    return [idx[rp[i]:rp[i + 1]] for i in range(lo, hi)]


def alone(fp, ix, q, k, metric):
    r = fp.fp_query(ix, q, k=k, metric=metric)
    return r.csr()


def test_replay_equals_each_request_alone(fp, served):
    w, ix, reqs = served
    allq = datagen.Strings.concat([r.queries for r in reqs])
    sizes = [len(r.queries) for r in reqs]
    srv = fp.Server(ix, lanes=4, max_requests=8)
    # a burst: everything arrives within 2 ms, so launches merge requests and overlap
    arrival = np.linspace(0, 2000, len(reqs)).astype(np.int64)
    res, lat = srv.replay(allq, request_sizes=sizes, arrival_us=arrival, k=1, metric="lev")
    st = srv.stats()
    srv.free()
    rp, idx = res.csr()
    assert st["completed"] == len(reqs) and st["queries"] == sum(sizes)
    assert st["max_requests_per_launch"] > 1, st
    assert st["max_lanes_busy"] > 1, st
    assert (lat > 0).all() and st["p99_ms"] >= st["p50_ms"] > 0
    q0 = 0
    for r in reqs:
        arp, aidx = alone(fp, ix, r.queries, 1, "lev")
        got = rows(rp, idx, q0, q0 + len(r.queries))
        want = rows(arp, aidx, 0, len(r.queries))
        assert all(np.array_equal(a, b) for a, b in zip(got, want))
        q0 += len(r.queries)
    # and the oracle on a sample of the patterns
    pick = np.arange(0, len(allq), 97)
    orp, oidx = oracle.match(w.dictionary, allq.subset(pick), 1, "lev")
    for j, i in enumerate(pick):
        assert np.array_equal(idx[rp[i]:rp[i + 1]], oidx[orp[j]:orp[j + 1]])


def test_mixed_k_and_metric_requests_in_one_launch(fp, served):
    w, ix, reqs = served
    srv = fp.Server(ix, lanes=2, max_requests=16)
    kinds = [(1, "lev"), (0, "ham"), (2, "lev"), (1, "ham"), (3, "ham"), (0, "lev")]
    ids = []
    for i, r in enumerate(reqs[:12]):
        k, m = kinds[i % len(kinds)]
        ids.append((srv.submit(r.queries, k=k, metric=m), r.queries, k, m))
    for rid, q, k, m in ids:
        res = srv.wait(rid, timeout_s=120)
        got = res.csr()
        want = alone(fp, ix, q, k, m)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (k, m)
    st = srv.stats()
    srv.free()
    assert st["completed"] == 12 and st["max_requests_per_launch"] > 1


def test_memory_budget_serialises_launches(fp, served):
    w, ix, reqs = served
    allq = datagen.Strings.concat([r.queries for r in reqs])
    chunks = [allq.subset(np.arange(300 * i, 300 * (i + 1))) for i in range(10)]  # equal-size requests
    seq = fp.Server(ix, lanes=1, max_requests=1, max_queries=300)
    outs = [seq.wait(seq.submit(c, k=1, metric="lev"), timeout_s=120).csr() for c in chunks]
    one = seq.stats()["peak_bytes"]  # the largest single launch
    seq.free()
    # room for one of these launches, not two
    budget = int(1.5 * one)
    srv = fp.Server(ix, lanes=4, max_requests=1, max_queries=300, memory_budget=budget)
    ids = [srv.submit(c, k=1, metric="lev") for c in chunks]
    got = [srv.wait(i, timeout_s=120).csr() for i in ids]
    st = srv.stats()
    assert st["peak_bytes"] <= budget and st["in_use_bytes"] == 0
    assert st["max_lanes_busy"] == 1, st
    for c, g, o in zip(chunks, got, outs):
        want = alone(fp, ix, c, 1, "lev")
        assert np.array_equal(g[0], want[0]) and np.array_equal(g[1], want[1])
        assert np.array_equal(o[0], want[0]) and np.array_equal(o[1], want[1])
    srv.free()
    # a request that could never fit is refused at once
    srv2 = fp.Server(ix, lanes=1, max_queries=len(allq), memory_budget=budget)
    with pytest.raises(fp.FpError) as e:
        srv2.submit(allq, k=1, metric="lev")
    assert e.value.code == -3  # FP_E_NOMEM
    srv2.free()


def test_bounded_wait_and_errors(fp, served):
    w, ix, reqs = served
    srv = fp.Server(ix, lanes=1)
    big = datagen.Strings.concat([r.queries for r in reqs[:20]])
    rid = srv.submit(big, k=1, metric="lev")
    with pytest.raises(fp.FpError) as e:
        srv.wait(rid, timeout_s=0)  # nothing finishes between the two calls
    assert e.value.code == -5  # FP_E_TIMEOUT
    res = srv.wait(rid, timeout_s=120)  # still pending: wait again
    want = alone(fp, ix, big, 1, "lev")
    got = res.csr()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    with pytest.raises(fp.FpError):
        srv.wait(rid, timeout_s=1)  # taken already
    with pytest.raises(fp.FpError):
        srv.submit(big, k=16, metric="lev")
    srv.free()
    pos = fp.fp_build(w.dictionary, fp_type="pos", width=32)
    srv = fp.Server(pos, lanes=1)
    with pytest.raises(fp.FpError) as e:
        srv.submit(reqs[0].queries, k=1, metric="lev")
    assert e.value.code == -2  # FP_E_UNSUPPORTED
    r = srv.wait(srv.submit(reqs[0].queries, k=1, metric="ham"), timeout_s=60)
    want = alone(fp, pos, reqs[0].queries, 1, "ham")
    assert np.array_equal(r.csr()[1], want[1])
    srv.free()


def test_empty_and_tiny_inputs(fp, served):
    w, ix, reqs = served
    S = datagen.Strings.from_list
    # a plan run with no patterns, then with empty and one-byte patterns
    plan = fp.Plan(ix, 8, 64, 2)
    rp, idx = plan.run(S([]), batches=[(0, 1, "lev")]).csr()
    assert list(rp) == [0] and len(idx) == 0
    q = S([b"", b"a", b"", b"/"])
    rp, idx = plan.run(q, batches=[(2, 1, "lev"), (2, 0, "ham")]).csr()
    plan.free()
    for lo, hi, k, m in ((0, 2, 1, "lev"), (2, 4, 0, "ham")):
        rp0, idx0 = oracle.match(w.dictionary, q.subset(np.arange(lo, hi)), k, m)
        assert np.array_equal(rp[lo:hi + 1] - rp[lo], rp0) and np.array_equal(idx[rp[lo]:rp[hi]], idx0)
    # the server takes a request of empty and one-byte patterns
    srv = fp.Server(ix, lanes=1)
    got = srv.wait(srv.submit(q, k=1, metric="lev"), timeout_s=60).csr()
    srv.free()
    rp0, idx0 = oracle.match(w.dictionary, q, 1, "lev")
    assert np.array_equal(got[0], rp0) and np.array_equal(got[1], idx0)
    with pytest.raises(fp.FpError):
        fp.Server(ix, lanes=1).submit(S([]), k=1, metric="lev")  # a request needs at least one pattern
