"""The weight-band rule on the CPU: every word that some pattern of a tile can
pass by the cell bound lies inside the runs the tile tests (so the bands never
skip a pair Eq. 1 could pass), for occ32, count32, occ16 and occh16, at several
tile sizes and k.  The rule is the one the GPU tests compare the kernels' tested
pair counts with."""
import numpy as np
import pytest

import datagen
import oracle
from band_rule import cells, part_bits, tile_runs


def parts(c, width):
    b0, b1, b2 = part_bits(width)
    R1, R2 = b1 + 1, b2 + 1
    c = np.asarray(c, dtype=np.int64)
    return np.stack([c // (R1 * R2), c // R2 % R1, c % R2], 1)


@pytest.mark.parametrize("t,width", [("occ", 32), ("count", 32), ("occ", 16), ("occh", 16)])
@pytest.mark.parametrize("k,tq", [(1, 64), (1, 7), (2, 32), (0, 128)])
def test_runs_cover_every_word_within_the_bound(t, width, k, tq):
    w = datagen.english1m(4000, 600)
    d, q = w.dictionary, w.queries["lev"]
    m, _, _ = oracle.default().symbol_map(d.chars, "common", oracle.layout(t, width)["sigma"])
    cq = cells(oracle.fingerprints(q, m, t, width), width)
    cd = cells(oracle.fingerprints(d, m, t, width), width)
    lq, ld = q.lengths(), d.lengths()
    checked = skipped = 0
    for n in np.unique(lq):
        cs = np.sort(cq[lq == n])
        for L in range(max(0, n - k), n + k + 1):
            b = np.sort(cd[ld == L])
            if len(b) == 0:
                continue
            pb = parts(b, width)
            for s in range(0, len(cs), tq):
                tile = cs[s:s + tq]
                covered = np.zeros(len(b), dtype=bool)
                for a, e in tile_runs(tile, b, k, width):
                    covered[a:e] = True
                # L1 distance of every word's cell to every pattern's cell
                l1 = np.abs(parts(tile, width)[:, None, :] - pb[None, :, :]).sum(2)
                need = (l1 <= 2 * k).any(0)
                assert not (need & ~covered).any(), (n, L, s)
                checked += int(need.sum())
                skipped += int((~covered).sum())
    assert checked > 0 and skipped > 0  # the bound binds, and the bands skip words
