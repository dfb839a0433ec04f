"""Seeded generators: determinism and the workload shapes."""
import numpy as np

import datagen
import oracle


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: first outputs of the published generator
    out = datagen.draws(np.uint64(0), 3)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_determinism_and_shapes():
    a = datagen.uniform10k(3000, 300)
    b = datagen.uniform10k(3000, 300)
    assert np.array_equal(a.dictionary.chars, b.dictionary.chars)
    assert np.array_equal(a.queries["lev"].offsets, b.queries["lev"].offsets)
    L = a.dictionary.lengths()
    assert L.min() >= 4 and L.max() <= 12
    assert set(np.unique(a.dictionary.chars)) <= set(range(ord("a"), ord("z") + 1))


def test_mutations_are_one_edit_away():
    w = datagen.english1m(5000, 400)
    d = w.dictionary.to_list()
    for metric, Q in w.queries.items():
        n_close = 0
        for q in Q.to_list()[:120]:
            best = min((oracle.lev(q, x) if metric == "lev" else (oracle.ham(q, x) or 99)) for x in d
                       if abs(len(x) - len(q)) <= 1)
            n_close += best <= 1
        assert n_close >= 0.5 * 120


def test_english_law_mean_and_range():
    law = datagen.english_law(24)
    L = law.lengths.sample(datagen.stream_key(1, "t"), 200000)
    assert L.min() >= 2 and L.max() <= 24 and abs(L.mean() - 8.0) < 0.05
    sym, w, rho = datagen.english_table()
    assert abs(w[0] - 0.12) < 1e-9 and bytes(sym[:16]) == b"etaoinshrdlcumwf"


def test_url_prefix_sharing():
    w = datagen.url2m(20000, 100)
    L = w.dictionary.lengths()
    assert L.min() >= 15 and L.max() <= 120
    s = w.dictionary.to_list()
    pf = datagen.url_law(w.seed).prefixes.to_list()
    shared = sum(any(x.startswith(p[:min(len(p), len(x))]) for p in pf) for x in s[:2000])
    assert 0.35 * 2000 < shared < 0.5 * 2000
