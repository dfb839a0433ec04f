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


def popc(x):
    x = np.asarray(x, dtype=np.uint64)
    return np.array([bin(int(v)).count("1") for v in x], dtype=np.int64)


def part_bits(width):
    """Bits of the three parts, most significant part first (W = 32: 11, 11, 10)."""
    return [width // 3 + (1 if i < width % 3 else 0) for i in range(3)]


def cells(f, width):
    b0, b1, b2 = part_bits(width)
    f = np.asarray(f, dtype=np.uint64)
    x = popc(f >> np.uint64(b1 + b2))
    y = popc((f >> np.uint64(b2)) & np.uint64((1 << b1) - 1))
    z = popc(f & np.uint64((1 << b2) - 1))
    return (x * (b1 + 1) + y) * (b2 + 1) + z


def expected_tested(d, q, k, metric, m, t, width, tq):
    """Pairs a banded plan tests.  Per length bin the patterns sorted by cell
    are cut into tiles of tq.  With (x1, y1, z1), (x2, y2, z2) the cells of a
    tile's first and last pattern, its box is x in [x1, x2], y in [y1, y2] if
    x1 = x2 (else everything), z in [z1, z2] if also y1 = y2 (else
    everything).  In every dictionary bucket of an admissible length, for
    every (x', y') whose L1 distance to the box's x and y ranges is at most
    2k, the tile tests the words of cells (x', y', z') with z' within the
    remaining distance of the z range: one run of slots, started at the
    bucket's 8-slot boundary below its first word; runs that then touch or
    overlap are merged."""
    b0, b1, b2 = part_bits(width)
    R1, R2 = b1 + 1, b2 + 1
    cq = cells(oracle.fingerprints(q, m, t, width), width)
    cd = cells(oracle.fingerprints(d, m, t, width), width)
    lq, ld = q.lengths(), d.lengths()
    by_len = {L: np.sort(cd[ld == L]) for L in np.unique(ld)}
    dist = lambda v, lo, hi: max(lo - v, 0, v - hi)
    total = 0
    for n in np.unique(lq):
        cs = np.sort(cq[lq == n])
        lens = [n] if metric == "ham" else range(max(0, n - k), min(255, n + k) + 1)
        for s in range(0, len(cs), tq):
            tile = cs[s:s + tq]
            f, l = int(tile[0]), int(tile[-1])
            xa, xb = f // (R1 * R2), l // (R1 * R2)
            y1, y2, z1, z2 = f // R2 % R1, l // R2 % R1, f % R2, l % R2
            ya, yb = (y1, y2) if xa == xb else (0, b1)
            za, zb = (z1, z2) if xa == xb and y1 == y2 else (0, b2)
            for L in lens:
                if L not in by_len:
                    continue
                b = by_len[L]
                runs = []
                for x in range(max(0, xa - 2 * k), min(b0, xb + 2 * k) + 1):
                    r1 = 2 * k - dist(x, xa, xb)
                    for y in range(max(0, ya - r1), min(b1, yb + r1) + 1):
                        r2 = r1 - dist(y, ya, yb)
                        zlo, zhi = max(0, za - r2), min(b2, zb + r2)
                        c = (x * R1 + y) * R2
                        first = int(np.searchsorted(b, c + zlo, side="left"))
                        end = int(np.searchsorted(b, c + zhi + 1, side="left"))
                        if end <= first:
                            continue
                        s8 = first & ~7
                        if runs and s8 <= runs[-1][1]:
                            runs[-1][1] = max(runs[-1][1], end)
                        else:
                            runs.append([s8, end])
                total += len(tile) * sum(e - a for a, e in runs)
    return total


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
