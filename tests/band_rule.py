"""The weight-band rule, restated in plain Python from its definition (the
planner's, in csrc/planner.cu): cells, a tile's box from its first and last
pattern, and the runs of a dictionary bucket a tile tests.  Used by the GPU
tests (tested-pair counts) and by a CPU test of the rule's soundness."""
import numpy as np

import oracle


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


def tile_runs(tile, bucket, k, width):
    """Runs [start, end) of positions in a bucket (cells sorted ascending) that a
    tile (cells sorted ascending) tests.  With (x1, y1, z1), (x2, y2, z2) the
    cells of the tile's first and last pattern, its box is x in [x1, x2], y in
    [y1, y2] if x1 = x2 (else everything), z in [z1, z2] if also y1 = y2 (else
    everything); for every (x', y') whose L1 distance to the box's x and y
    ranges is at most 2k the tile tests the words of cells (x', y', z') with z'
    within the remaining distance of the z range: one run, started at the
    8-slot boundary below its first word; runs that then touch or overlap are
    merged."""
    b0, b1, b2 = part_bits(width)
    R1, R2 = b1 + 1, b2 + 1
    dist = lambda v, lo, hi: max(lo - v, 0, v - hi)
    f, l = int(tile[0]), int(tile[-1])
    xa, xb = f // (R1 * R2), l // (R1 * R2)
    y1, y2, z1, z2 = f // R2 % R1, l // R2 % R1, f % R2, l % R2
    ya, yb = (y1, y2) if xa == xb else (0, b1)
    za, zb = (z1, z2) if xa == xb and y1 == y2 else (0, b2)
    runs = []
    for x in range(max(0, xa - 2 * k), min(b0, xb + 2 * k) + 1):
        r1 = 2 * k - dist(x, xa, xb)
        for y in range(max(0, ya - r1), min(b1, yb + r1) + 1):
            r2 = r1 - dist(y, ya, yb)
            zlo, zhi = max(0, za - r2), min(b2, zb + r2)
            c = (x * R1 + y) * R2
            first = int(np.searchsorted(bucket, c + zlo, side="left"))
            end = int(np.searchsorted(bucket, c + zhi + 1, side="left"))
            if end <= first:
                continue
            s8 = first & ~7
            if runs and s8 <= runs[-1][1]:
                runs[-1][1] = max(runs[-1][1], end)
            else:
                runs.append([s8, end])
    return runs


def expected_tested(d, q, k, metric, m, t, width, tq):
    """Pairs a banded plan tests: per length bin the patterns sorted by cell are
    cut into tiles of tq; each tile tests tile_runs of every dictionary bucket
    of an admissible length."""
    cq = cells(oracle.fingerprints(q, m, t, width), width)
    cd = cells(oracle.fingerprints(d, m, t, width), width)
    lq, ld = q.lengths(), d.lengths()
    by_len = {L: np.sort(cd[ld == L]) for L in np.unique(ld)}
    total = 0
    for n in np.unique(lq):
        cs = np.sort(cq[lq == n])
        lens = [n] if metric == "ham" else range(max(0, n - k), min(255, n + k) + 1)
        for s in range(0, len(cs), tq):
            tile = cs[s:s + tq]
            for L in lens:
                if L in by_len:
                    total += len(tile) * sum(e - a for a, e in tile_runs(tile, by_len[L], k, width))
    return total
