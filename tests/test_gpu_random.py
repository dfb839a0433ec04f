"""Randomised cross-checks against the oracle (needs a GPU): many small seeded
dictionaries and pattern sets with skewed alphabets, lengths from 0 to 255,
duplicates and k from 0 to 15, through every fingerprint type, width, form and
filter variant, and a server fed by several submitting threads at once."""
import threading

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


def random_case(seed):
    """A dictionary and patterns drawn from a small random alphabet and length law."""
    key = datagen.stream_key(seed, "case")
    r = datagen.uniform(key, 16)
    sigma = 2 + int(r[0] * 30)
    alphabet = np.unique(datagen.randint(datagen.stream_key(seed, "alpha"), sigma, 0, 255).astype(np.uint8))
    weights = np.exp(-np.arange(len(alphabet)) * (0.05 + r[1]))
    lo = int(r[2] * 8)
    hi = lo + 1 + int(r[3] * (40 if r[4] < 0.8 else 255 - lo - 1))
    hi = min(hi, 255)
    law = datagen.StringLaw(alphabet, weights, datagen.LengthLaw("uniform", lo, hi))
    long_strings = hi > 40
    n_words = 50 + int(r[5] * (400 if long_strings else 3000))
    d = law.draw(seed, "dict", n_words)
    if r[6] < 0.5:  # duplicates
        d = datagen.Strings.concat([d, d.subset(np.arange(0, n_words, 7))])
    metric = "ham" if r[7] < 0.5 else "lev"
    n_q = 20 + int(r[8] * (60 if long_strings else 300))
    q = datagen.make_queries(d, law, seed, "q", n_q, 0.5, metric)
    k = int(r[9] * 4) if r[10] < 0.8 else int(r[9] * 16)
    return d, q, metric, k


CASES = [(t, w) for t in ("occ", "count", "occh", "pos") for w in (16, 32)]


@pytest.mark.parametrize("seed", range(64))
def test_random_against_oracle(fp, seed):
    d, q, metric, k = random_case(seed)
    rp0, idx0 = oracle.match(d, q, k, metric)
    t, width = CASES[seed % len(CASES)]
    if metric == "lev" and t in ("occh", "pos"):
        t = "count" if t == "occh" else "occ"
    ix = fp.fp_build(d, fp_type=t, width=width, symbol_set=("common", "rare", "mixed")[seed % 3])
    for mode, variant in (("tiled", 0), ("tiled", 1), ("fused", 0), ("tiled", 2), ("plain", 0)):
        r = fp.fp_query_ex(ix, q, k=k, metric=metric, mode=mode, variant=variant)
        rp, idx = r.csr()
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (seed, t, width, metric, k, mode, variant)


def test_server_with_concurrent_submitters(fp):
    w = datagen.english1m(50000, 3000)
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    srv = fp.Server(ix, lanes=3, max_requests=6)
    jobs = []
    for i in range(24):
        Q = w.queries["lev" if i % 2 else "ham"]
        lo = (i * 113) % (len(Q) - 200)
        jobs.append((Q.subset(np.arange(lo, lo + 40 + 7 * i)), 1 + (i % 3 == 0), "lev" if i % 2 else "ham"))
    got = [None] * len(jobs)
    errors = []

    def worker(t):
        try:
            for j in range(t, len(jobs), 4):
                q, k, m = jobs[j]
                got[j] = srv.wait(srv.submit(q, k=k, metric=m), timeout_s=120).csr()
        except Exception as e:  # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    st = srv.stats()
    srv.free()
    assert not errors, errors
    assert st["completed"] == len(jobs)
    for (q, k, m), (rp, idx) in zip(jobs, got):
        rp0, idx0 = oracle.match(w.dictionary, q, k, m)
        assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0)
