"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Each ``check_*`` takes an ``oracle.Oracle`` (a compiled copy of oracle.c) and
raises AssertionError when the copy disagrees with a value the paper prints,
a hand-derived value of a definition in the paper, a brute-force enumeration,
or a mathematical identity.  ``test_oracle_pins.py`` runs them on the real
oracle; ``test_oracle_mutants.py`` runs them on copies with planted mistakes
and requires each mistake to be caught.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import datagen
from oracle import layout, map_from_order

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out: dict = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("box", "value"):
                out.setdefault(parts[0], {})[parts[1]] = parts[2]
            else:
                out[parts[0]] = parts[1:] if len(parts) > 2 else parts[1]
    return out


# ---------------------------------------------------------------------------
# Printed form of a fingerprint, as the boxes of Sec. 3.1 show it
# ---------------------------------------------------------------------------


def printed(fp: int, type_name: str, width: int = 16, b: int = 2, p: int = 3, gray: bool = False) -> str:
    lay = layout(type_name, width, b, p)
    if type_name == "occ":
        return "".join(str((fp >> q) & 1) for q in range(width))
    if type_name == "occh":
        return "".join(f"{(fp >> (2 * q)) & 1}{(fp >> (2 * q + 1)) & 1}" for q in range(width // 2))
    if type_name == "count":
        out = []
        for q in range(width // b):
            v = (fp >> (b * q)) & ((1 << b) - 1)
            if gray:  # Gray -> binary
                x, s = v, v >> 1
                while s:
                    x ^= s
                    s >>= 1
                v = x
            out.append(format(v, f"0{b}b"))
        return "".join(out)
    n_pos = lay["n_pos"]
    fields = "".join(format((fp >> (p * j)) & ((1 << p) - 1), f"0{p}b") for j in range(n_pos))
    occ = "".join(str((fp >> (p * n_pos + t)) & 1) for t in range(width - p * n_pos))
    return fields + occ


def _trim(order: bytes, type_name: str, width: int = 16) -> np.ndarray:
    return map_from_order(order[: layout(type_name, width)["sigma"]])


# ---------------------------------------------------------------------------
# Sec. 3.1 worked example and Sec. 3.3 run/ran
# ---------------------------------------------------------------------------


def check_instance_example(orc):
    g = read_golden("instance.txt")
    word, order = g["word"].encode(), g["order"].encode()
    for t in ("occ", "occh", "pos"):
        fp = orc.fingerprint(word, _trim(order, t), t, 16)
        assert printed(fp, t) == g["box"][t], (t, printed(fp, t), g["box"][t])
        assert fp == int(g["value"][t], 16), (t, hex(fp))
    fb = orc.fingerprint(word, _trim(order, "count"), "count", 16, gray=False)
    fg = orc.fingerprint(word, _trim(order, "count"), "count", 16, gray=True)
    assert printed(fb, "count") == g["box"]["count"], printed(fb, "count")
    assert printed(fg, "count", gray=True) == g["box"]["count"]
    assert fb == int(g["value"]["count_binary"], 16), hex(fb)
    assert fg == int(g["value"]["count_gray"], 16), hex(fg)


def check_run_ran(orc):
    g = read_golden("run_ran.txt")
    a, b = (x.encode() for x in g["pair"])
    m = map_from_order(read_golden("instance.txt")["order"].encode())
    f = orc.fd(orc.fingerprint(a, m, "occ", 16), orc.fingerprint(b, m, "occ", 16), "occ", 16)
    assert f == int(g["fd_occ16"]), f
    assert orc.ham(a, b) == int(g["ham"])
    assert orc.lev(a, b) == int(g["lev"])
    # Eq. 1 decision: reject iff ceil(F_D / 2) > k
    assert not (f + 1) // 2 > 1
    assert (f + 1) // 2 > 0


def check_repeated_symbols(orc):
    """Sec. 3.3: strings made of one repeated symbol each have F_D <= 2 (0 when
    neither symbol is tracked) while the Hamming distance is n."""
    m = map_from_order(b"ab")
    for n in range(1, 9):
        s, t = b"a" * n, b"b" * n
        f = orc.fd(orc.fingerprint(s, m, "occ", 16), orc.fingerprint(t, m, "occ", 16), "occ", 16)
        assert f == 2 and orc.ham(s, t) == n
        u, v = b"x" * n, b"y" * n
        f0 = orc.fd(orc.fingerprint(u, m, "occ", 16), orc.fingerprint(v, m, "occ", 16), "occ", 16)
        assert f0 == 0


# ---------------------------------------------------------------------------
# Hand-derived values of the Sec. 3 / Sec. 3.2 definitions
# ---------------------------------------------------------------------------


def check_halves(orc):
    """Occurrence halved: S[1, floor(n/2)] and S[floor(n/2)+1, n] (Sec. 3)."""
    m = map_from_order(b"abcde")
    # n = 5: first half "ab", second half "cde": bits 0, 2, 5, 7, 9
    assert orc.fingerprint(b"abcde", m, "occh", 16) == (1 | 4 | 32 | 128 | 512)
    # n = 1: the first half is empty, so 'a' is in the second half: bit 1
    assert orc.fingerprint(b"a", m, "occh", 16) == 2
    # n = 2: "a" | "a"
    assert orc.fingerprint(b"aa", m, "occh", 16) == 3
    # n = 4: "ab" | "ba"
    assert orc.fingerprint(b"abba", m, "occh", 16) == (1 | 2 | 4 | 8)
    assert orc.fingerprint(b"", m, "occh", 16) == 0


def check_count_saturation(orc):
    """Count in [0, 2^b - 1], where 2^b - 1 means 2^b - 1 or more (Sec. 3)."""
    m = map_from_order(b"nq")
    cases = {1: (1, 1), 2: (2, 3), 3: (3, 2), 5: (3, 2)}  # n -> (binary, gray), b = 2
    for n, (vb, vg) in cases.items():
        assert orc.fingerprint(b"n" * n, m, "count", 16, b=2, gray=False) == vb
        assert orc.fingerprint(b"n" * n, m, "count", 16, b=2, gray=True) == vg
    # b = 3: nine copies saturate at 7 (binary 111, Gray 100); field 1 holds 'q'
    assert orc.fingerprint(b"n" * 9 + b"qq", m, "count", 16, b=3, gray=False) == 7 | (2 << 3)
    assert orc.fingerprint(b"n" * 9 + b"qq", m, "count", 16, b=3, gray=True) == 4 | (3 << 3)
    # symbols outside the map leave the fingerprint unchanged (Theorem 1, case ii)
    assert orc.fingerprint(b"zzzz", m, "count", 16) == 0


def check_positions(orc):
    """First 0-indexed position, all ones for 'at 2^p - 1 or later, or absent'."""
    m = map_from_order(b"hab")  # p = 3, width 16: fields h, a, b, (unused), (unused)
    sat = 7
    f = orc.fingerprint(b"abcdefgh", m, "pos", 16)
    assert f & 7 == sat  # h at index 7 -> saturated
    assert (f >> 3) & 7 == 0  # a at index 0
    assert (f >> 6) & 7 == 1  # b at index 1
    f = orc.fingerprint(b"bcdefaha", m, "pos", 16)
    assert f & 7 == 6 and (f >> 3) & 7 == 5 and (f >> 6) & 7 == 0
    # first occurrence beyond 2^p - 1 (index 9) also reads as all ones
    f = orc.fingerprint(b"zzzzzzzzzhab", m, "pos", 16)
    assert f & 7 == sat and (f >> 3) & 7 == sat and (f >> 6) & 7 == sat and (f >> 9) == 0x3F
    # p = 2 saturates at 3: positions 2 -> 2, 3 -> 3, absent -> 3
    m2 = map_from_order(b"xyz")
    f = orc.fingerprint(b"abxy", m2, "pos", 8, p=2)
    assert f & 3 == 2 and (f >> 2) & 3 == 3 and (f >> 4) & 3 == 3
    f = orc.fingerprint(b"abcdzyx", m2, "pos", 8, p=2)
    assert f == 0xFF
    # occurrence bits: width 8, p = 2 -> 4 position fields, 0 occurrence bits;
    # width 16, p = 3 -> 5 fields + 1 occurrence bit for the 6th symbol
    m6 = map_from_order(b"abcdeq")
    assert orc.fingerprint(b"q", m6, "pos", 16) >> 15 == 1
    assert orc.fingerprint(b"", m6, "pos", 16) == 0x7FFF


def check_fd_fields(orc):
    """F_D for pos counts mismatching p-bit fields, not bits (Sec. 3.3)."""
    assert orc.fd(0, 0b011, "pos", 16) == 1
    assert orc.fd(0, 0b011001, "pos", 16) == 2
    assert orc.fd(0, 1 << 15, "pos", 16) == 1
    assert orc.fd(0b111 << 12, 0, "pos", 16) == 1
    assert orc.fd(0, 0b011, "occ", 16) == 2
    assert orc.fd(0xFFFF, 0, "count", 16) == 16
    assert orc.fd(0xFFFFFFFF, 0, "occ", 32) == 32


def check_symbol_sets(orc):
    """Common, rare and mixed sets from occurrence counts (Sec. 3)."""
    chars = np.frombuffer(b"aaaabbbccde", dtype=np.uint8)  # a4 b3 c2 d1 e1
    m, c, used = orc.symbol_map(chars, "common", 3)
    assert used == 3 and m[ord("a")] == 0 and m[ord("b")] == 1 and m[ord("c")] == 2
    assert m[ord("d")] == -1 and c[ord("a")] == 4 and c[ord("e")] == 1
    m, _, _ = orc.symbol_map(chars, "rare", 3)
    assert m[ord("d")] == 0 and m[ord("e")] == 1 and m[ord("c")] == 2 and m[ord("a")] == -1
    m, _, _ = orc.symbol_map(chars, "mixed", 3)
    assert m[ord("a")] == 0 and m[ord("b")] == 1 and m[ord("d")] == 2 and m[ord("e")] == -1
    m, _, used = orc.symbol_map(np.frombuffer(b"ab", dtype=np.uint8), "common", 4)
    assert used == 2 and m[ord("a")] == 0 and m[ord("b")] == 1 and (m >= 0).sum() == 2


# ---------------------------------------------------------------------------
# Distances: textbook values and brute-force edit-ball enumeration
# ---------------------------------------------------------------------------


def all_strings(alphabet: bytes, max_len: int):
    out = []
    for n in range(max_len + 1):
        out += [bytes(t) for t in itertools.product(alphabet, repeat=n)]
    return out


def edit_ball(p: bytes, k: int, alphabet: bytes, substitutions_only: bool = False):
    """Every string reachable from p by at most k single-symbol edits."""
    seen = {p}
    frontier = {p}
    for _ in range(k):
        nxt = set()
        for s in frontier:
            for i in range(len(s)):
                for c in alphabet:
                    nxt.add(s[:i] + bytes([c]) + s[i + 1:])
                if not substitutions_only:
                    nxt.add(s[:i] + s[i + 1:])
            if not substitutions_only:
                for i in range(len(s) + 1):
                    for c in alphabet:
                        nxt.add(s[:i] + bytes([c]) + s[i:])
        nxt -= seen
        seen |= nxt
        frontier = nxt
    return seen


def check_textbook_distances(orc):
    assert orc.lev(b"kitten", b"sitting") == 3
    assert orc.lev(b"flaw", b"lawn") == 2
    assert orc.lev(b"", b"") == 0
    assert orc.lev(b"abc", b"") == 3 and orc.lev(b"", b"abcd") == 4
    assert orc.ham(b"karolin", b"kathrin") == 3
    assert orc.ham(b"1011101", b"1001001") == 2
    assert orc.ham(b"abc", b"ab") is None
    assert orc.ham(b"", b"") == 0


def check_edit_ball(orc, max_pat: int = 4, kmax: int = 2, alphabet: bytes = b"abc"):
    """{S : Lev(P, S) <= k} equals the set reachable by <= k edits, and
    {S : Ham(P, S) <= k} the set reachable by <= k substitutions."""
    pats = all_strings(alphabet, max_pat)
    universe = all_strings(alphabet, max_pat + kmax)
    D = datagen.Strings.from_list(universe)
    Q = datagen.Strings.from_list(pats)
    for k in range(kmax + 1):
        for metric in ("lev", "ham"):
            rp, idx = orc.match(D, Q, k, metric, prune=False)
            for qi, p in enumerate(pats):
                got = {universe[i] for i in idx[rp[qi]:rp[qi + 1]]}
                want = edit_ball(p, k, alphabet, substitutions_only=(metric == "ham"))
                assert got == want, (metric, k, p, sorted(got ^ want)[:5])
                assert list(idx[rp[qi]:rp[qi + 1]]) == sorted(idx[rp[qi]:rp[qi + 1]])


def check_distance_identities(orc, seed: int = 7):
    key = datagen.stream_key(seed, "identities")
    law = datagen.StringLaw(np.frombuffer(b"abcd", np.uint8), np.ones(4), datagen.LengthLaw("uniform", 0, 9))
    S = law.draw(seed, "identities", 300).to_list()
    r = datagen.randint(key, 600, 0, len(S) - 1)
    for t in range(200):
        x, y, z = S[r[3 * t % 600]], S[r[(3 * t + 1) % 600]], S[r[(3 * t + 2) % 600]]
        dxy, dyx = orc.lev(x, y), orc.lev(y, x)
        assert dxy == dyx
        assert orc.lev(x, x) == 0
        assert abs(len(x) - len(y)) <= dxy <= max(len(x), len(y))
        assert orc.lev(x, z) <= dxy + orc.lev(y, z)
        if len(x) == len(y):
            h = orc.ham(x, y)
            assert dxy <= h
            if h <= 1:
                assert dxy == h


def check_verifiers(orc, alphabet: bytes = b"ab", max_len: int = 5):
    """The paper's verification loops (Sec. 4) decide D <= k exactly."""
    S = all_strings(alphabet, max_len)
    for a in S:
        for b in S:
            if abs(len(a) - len(b)) > 3:
                continue
            d = orc.lev(a, b)
            h = orc.ham(a, b)
            for k in range(4):
                assert orc.lev_within(a, b, k) == (d <= k), (a, b, k)
                assert orc.ham_within(a, b, k) == (h is not None and h <= k), (a, b, k)


def check_match_against_pairs(orc, seed: int = 11):
    """The threaded matcher lists exactly the pairs the scalar distance admits."""
    law = datagen.StringLaw(np.frombuffer(b"abcde", np.uint8), np.ones(5), datagen.LengthLaw("uniform", 0, 7))
    D = law.draw(seed, "d", 400)
    Q = datagen.Strings.concat([law.draw(seed, "q", 60), D.subset(np.arange(0, 400, 37))])
    dl, ql = D.to_list(), Q.to_list()
    dist = {"lev": [[orc.lev(q, w) for w in dl] for q in ql],
            "ham": [[orc.ham(q, w) for w in dl] for q in ql]}
    for metric in ("ham", "lev"):
        for k in (0, 1, 2):
            for prune in (True, False):
                rp, idx = orc.match(D, Q, k, metric, prune=prune, threads=3)
                for qi in range(len(ql)):
                    want = [i for i, d in enumerate(dist[metric][qi]) if d is not None and d <= k]
                    assert list(idx[rp[qi]:rp[qi + 1]]) == want, (metric, k, qi)


# ---------------------------------------------------------------------------
# Eq. 1 / Theorems 1 and 2: exhaustive soundness sweep
# ---------------------------------------------------------------------------


def random_maps(seed: int, n: int, symbols: bytes, fields: int):
    """Many-to-one symbol -> field maps, some symbols untracked (-1)."""
    out = []
    for t in range(n):
        r = datagen.randint(datagen.stream_key(seed, f"map{t}"), len(symbols), -1, fields - 1)
        m = np.full(256, -1, dtype=np.int8)
        for s, q in zip(symbols, r):
            m[s] = q
        out.append(m)
    return out


SWEEP_ALPHABET = b"abcx"


def sweep_cases():
    """(type, width, b, p, gray, metric, sound) combinations for the sweep."""
    cases = []
    for metric in ("ham", "lev"):
        cases.append(("occ", 8, 2, 3, True, metric, True))
        cases.append(("count", 8, 2, 3, True, metric, True))
        cases.append(("count", 9, 3, 3, True, metric, True))
        cases.append(("count", 8, 1, 3, True, metric, True))
        cases.append(("count", 8, 2, 3, False, metric, False))  # the paper's binary counts
        cases.append(("occh", 8, 2, 3, True, metric, metric == "ham"))
        cases.append(("pos", 8, 2, 2, True, metric, metric == "ham"))
        cases.append(("pos", 11, 2, 3, True, metric, metric == "ham"))
    return cases


def check_bound_sweep(orc, max_len: int = 5, n_random_maps: int = 3, seed: int = 5):
    S = datagen.Strings.from_list(all_strings(SWEEP_ALPHABET, max_len))
    small = datagen.Strings.from_list(all_strings(SWEEP_ALPHABET, min(max_len, 4)))
    results = {}
    for (t, width, b, p, gray, metric, sound) in sweep_cases():
        sigma = layout(t, width, b, p)["sigma"]
        maps = [map_from_order(SWEEP_ALPHABET[:sigma]), map_from_order(SWEEP_ALPHABET[:3][:sigma])]
        viol = 0
        for m in maps:
            r = orc.bound_violations(S, m, t, width, metric, b=b, p=p, gray=gray)
            assert r["pairs"] > 0
            viol += r["violations"]
        for m in random_maps(seed, n_random_maps, SWEEP_ALPHABET, sigma):
            r = orc.bound_violations(small, m, t, width, metric, b=b, p=p, gray=gray)
            viol += r["violations"]
        results[(t, width, b, p, gray, metric)] = viol
        if sound:
            assert viol == 0, (t, width, b, p, gray, metric, viol)
        else:
            assert viol > 0, ("sweep cannot bite", t, width, b, p, gray, metric)
    return results


def check_counterexamples(orc):
    """The specific pairs where the unsound combinations reject a true match."""
    m = map_from_order(b"ab")
    fa = orc.fingerprint(b"aa", m, "count", 16, gray=False)
    fb = orc.fingerprint(b"ab", m, "count", 16, gray=False)
    assert orc.fd(fa, fb, "count", 16) == 3 and orc.lev(b"aa", b"ab") == 1
    fa = orc.fingerprint(b"aab", m, "count", 16, gray=False)
    fb = orc.fingerprint(b"abb", m, "count", 16, gray=False)
    assert orc.fd(fa, fb, "count", 16) == 4 and orc.ham(b"aab", b"abb") == 1
    ga = orc.fingerprint(b"aa", m, "count", 16, gray=True)
    gb = orc.fingerprint(b"ab", m, "count", 16, gray=True)
    assert orc.fd(ga, gb, "count", 16) == 2
    fa = orc.fingerprint(b"a", m, "occh", 16)
    fb = orc.fingerprint(b"ab", m, "occh", 16)
    assert orc.fd(fa, fb, "occh", 16) == 3 and orc.lev(b"a", b"ab") == 1
    mc = map_from_order(b"abc")
    fa = orc.fingerprint(b"ab", mc, "pos", 16)
    fb = orc.fingerprint(b"cab", mc, "pos", 16)
    assert orc.fd(fa, fb, "pos", 16) == 3 and orc.lev(b"ab", b"cab") == 1


# ---------------------------------------------------------------------------
# The filter is a pure speedup (Sec. 3: fingerprints only reject)
# ---------------------------------------------------------------------------


def check_filter_is_speedup(orc, w=None, types=(("occ", 16), ("count", 16), ("occh", 16), ("pos", 16))):
    if w is None:
        w = datagen.uniform10k(2000, 200)
    for metric, Q in w.queries.items():
        rp0, idx0 = orc.match(w.dictionary, Q, 1, metric)
        for (t, width) in types:
            if metric == "lev" and t in ("occh", "pos"):
                continue
            m, _, _ = orc.symbol_map(w.dictionary.chars, "common", layout(t, width)["sigma"])
            rp, idx, pairs, surv = orc.filter_match(w.dictionary, Q, 1, metric, m, t, width)
            assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (metric, t)
            assert 0 <= surv <= pairs
            assert rp0[-1] <= surv


def check_filter_decision(orc):
    """Eq. 1 decides on ceil(F_D / 2) > k: F_D = 2 passes at k = 1, F_D = 3 and
    F_D = 4 are rejected, and at k = 0 any nonzero F_D is rejected."""
    m = map_from_order(b"abcdefgh")
    D = datagen.Strings.from_list([b"abc", b"acd", b"ccd", b"efg", b"abd"])
    Q = datagen.Strings.from_list([b"aab"])  # occ {a, b}
    # F_D per word: abc {a,b,c} 1, acd {a,c,d} 3, ccd {c,d} 4, efg 5, abd 1
    fds = [orc.fd(orc.fingerprint(w, m, "occ", 16), orc.fingerprint(b"aab", m, "occ", 16), "occ", 16)
           for w in D.to_list()]
    assert fds == [1, 3, 4, 5, 1], fds
    _, _, pairs, surv = orc.filter_match(D, Q, 1, "ham", m, "occ", 16)
    assert (pairs, surv) == (5, 2)
    _, _, pairs, surv = orc.filter_match(D, Q, 0, "ham", m, "occ", 16)
    assert (pairs, surv) == (5, 0)
    D2 = datagen.Strings.from_list([b"abc", b"abd", b"ade"])
    _, _, pairs, surv = orc.filter_match(D2, datagen.Strings.from_list([b"abc"]), 1, "ham", m, "occ", 16)
    assert (pairs, surv) == (3, 2)  # F_D 0, 2, 4
    _, _, pairs, surv = orc.filter_match(D2, datagen.Strings.from_list([b"abc"]), 2, "lev", m, "occ", 16)
    assert (pairs, surv) == (3, 3)


# ---------------------------------------------------------------------------
# Count fingerprints compared by the L1 distance of the counts (Sec. 3.3)
# ---------------------------------------------------------------------------


def _unary(fields, bits):
    """Thermometer code of saturating counts: value v of a field as v ones in
    2^bits - 1 bit positions (popc of the XOR of two codes = |v1 - v2|)."""
    width = (1 << bits) - 1
    u = 0
    for i, v in enumerate(fields):
        u |= ((1 << v) - 1) << (width * i)
    return u


def _pack(fields, bits):
    return sum(v << (bits * i) for i, v in enumerate(fields))


def check_count_l1(orc):
    # the remark after Eq. 1: a count of 3 (11) against a count of 1 (01)
    # differs by 2, where the Hamming weight of the XOR gives 1
    assert orc.fd_count_l1(0b11, 0b01, 2, 2) == 2
    assert orc.fd(0b11, 0b01, "count", 2) == 1
    # hand values over several fields (field 0 in the low bits)
    assert orc.fd_count_l1(_pack([0, 3, 1, 2], 2), _pack([3, 0, 2, 1], 2), 8, 2) == 8
    assert orc.fd_count_l1(_pack([7, 0, 5], 3), _pack([0, 7, 5], 3), 9, 3) == 14
    assert orc.fd_count_l1(_pack([1] * 16, 2), _pack([1] * 16, 2), 32, 2) == 0
    # fields above the width do not count
    assert orc.fd_count_l1(0b1100, 0, 2, 2) == 0
    # from strings: aaab -> counts (3, 1), ab -> (1, 1) in the binary code
    m = map_from_order(b"ab")
    fa = orc.fingerprint(b"aaab", m, "count", 16, gray=False)
    fb = orc.fingerprint(b"ab", m, "count", 16, gray=False)
    assert orc.fd_count_l1(fa, fb, 16, 2) == 2 and orc.lev(b"aaab", b"ab") == 2
    # against the thermometer code on random count vectors (a different
    # computation of the same distance), and never below the Gray-code
    # distance, equal to it unless some field differs by 3
    r = datagen.randint(datagen.stream_key(3, "l1"), 2 * 16 * 300, 0, 3).reshape(300, 2, 16)
    for a, b in r:
        la = orc.fd_count_l1(_pack(a, 2), _pack(b, 2), 32, 2)
        assert la == bin(_unary(a, 2) ^ _unary(b, 2)).count("1")
        ga = _pack([v ^ (v >> 1) for v in a], 2)
        gb = _pack([v ^ (v >> 1) for v in b], 2)
        gray = bin(ga ^ gb).count("1")
        assert la >= gray
        assert (la == gray) == (not np.any(np.abs(a.astype(int) - b.astype(int)) == 3))


def check_count_l1_sweep(orc, max_len: int = 5, n_random_maps: int = 3, seed: int = 5):
    """Eq. 1 with the L1 count distance on the paper's binary code: zero
    violations (b = 1, 2, 3), where the Hamming weight of the same binary
    fingerprints has violations (check_bound_sweep)."""
    S = datagen.Strings.from_list(all_strings(SWEEP_ALPHABET, max_len))
    small = datagen.Strings.from_list(all_strings(SWEEP_ALPHABET, min(max_len, 4)))
    for metric in ("ham", "lev"):
        for b, width in ((2, 8), (3, 9), (1, 8)):
            sigma = width // b
            maps = [map_from_order(SWEEP_ALPHABET[:sigma]), map_from_order(SWEEP_ALPHABET[:3][:sigma])]
            runs = [(S, m) for m in maps] + [(small, m) for m in random_maps(seed, n_random_maps, SWEEP_ALPHABET,
                                                                              sigma)]
            for strs, m in runs:
                fp = orc.fingerprints(strs, m, "count", width, b=b, gray=False)
                r = orc.bound_violations_fps(strs, fp, "count_l1", width, metric, bits=b)
                assert r["pairs"] > 0 and r["violations"] == 0, (metric, b, r)


# ---------------------------------------------------------------------------
# q-gram fingerprints (Sec. 5): occurrence of the most frequent q-grams
# ---------------------------------------------------------------------------


def check_qgram_fingerprints(orc):
    S = datagen.Strings.from_list([b"abab", b"abc"])
    grams, counts = orc.qgram_map(S, 2, 32)
    # bigram occurrences: ab 3 (abab twice, abc once), ba 1, bc 1; ba before bc
    assert [bytes(g) for g in grams] == [b"ab", b"ba", b"bc"] and list(counts) == [3, 1, 1]
    fps = [orc.qgram_fingerprint(s, grams) for s in (b"abab", b"abc", b"cab", b"bcab", b"b", b"")]
    assert fps == [0b011, 0b101, 0b001, 0b101, 0, 0], fps
    # ties go to the smaller q-gram in byte order, whatever the order of appearance
    g2, _ = orc.qgram_map(datagen.Strings.from_list([b"ba", b"ab"]), 2, 32)
    assert [bytes(g) for g in g2] == [b"ab", b"ba"]
    # sigma caps the fields; trigrams
    g3, c3 = orc.qgram_map(datagen.Strings.from_list([b"abcd", b"xbcd"]), 3, 2)
    assert [bytes(g) for g in g3] == [b"bcd", b"abc"] and list(c3) == [2, 1]
    assert orc.qgram_fingerprint(b"abcd", g3) == 0b11 and orc.qgram_fingerprint(b"abc", g3) == 0b10
    # q = 1 is the occurrence fingerprint over the common symbols (Sec. 3.2)
    w = datagen.english1m(2000, 10)
    g1, _ = orc.qgram_map(w.dictionary, 1, 16)
    m, _, _ = orc.symbol_map(w.dictionary.chars, "common", 16)
    assert all(m[g[0]] == f for f, g in enumerate(g1)) and (m >= 0).sum() == len(g1)
    assert np.array_equal(orc.qgram_fingerprints(w.dictionary, g1), orc.fingerprints(w.dictionary, m, "occ", 16))


def check_qgram_sweep(orc, max_len: int = 5, seed: int = 9):
    """One edit changes the q-gram fingerprint by at most 2q bits, so
    D >= ceil(F_D / 2q): zero violations over every string of length <= 5 on
    {a, b, c, x} (q = 2, 3; the collection's own q-grams and random sets);
    the Eq. 1 bound (2 in place of 2q) has violations, so the sweep bites."""
    S = datagen.Strings.from_list(all_strings(SWEEP_ALPHABET, max_len))
    for q in (2, 3):
        sets = [orc.qgram_map(S, q, 12)[0]]
        every = list(itertools.product(SWEEP_ALPHABET, repeat=q))
        for t in range(2):  # random sets of 12 distinct q-grams (each q-gram owns at most one bit)
            pick = datagen.permutation(datagen.stream_key(seed, f"grams{q}/{t}"), len(every))[:12]
            sets.append(np.array([every[i] for i in pick], dtype=np.uint8))
        loose = 0
        for grams in sets:
            fp = orc.qgram_fingerprints(S, grams)
            for metric in ("ham", "lev"):
                r = orc.bound_violations_fps(S, fp, "weight", 32, metric, q=q)
                assert r["pairs"] > 0 and r["violations"] == 0, (q, metric, r)
                loose += orc.bound_violations_fps(S, fp, "weight", 32, metric, q=1)["violations"]
        assert loose > 0, ("sweep cannot bite", q)


def check_fps_filter_is_speedup(orc):
    """The Sec. 4 method on q-gram fingerprints (bound 2qk) and on binary counts
    compared by L1 gives the brute-force match lists; L1 lets no more pairs
    through than the Gray-code Hamming weight does."""
    w = datagen.english1m(3000, 300)
    for metric, Q in w.queries.items():
        for k in (1, 2):
            rp0, idx0 = orc.match(w.dictionary, Q, k, metric)
            for q in (2, 3):
                grams, _ = orc.qgram_map(w.dictionary, q, 32)
                rp, idx, pairs, surv = orc.filter_match_fps(w.dictionary, Q, k, metric,
                                                            orc.qgram_fingerprints(w.dictionary, grams),
                                                            orc.qgram_fingerprints(Q, grams), "weight", 32, q=q)
                assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (metric, k, q)
                assert rp0[-1] <= surv <= pairs
            m, _, _ = orc.symbol_map(w.dictionary.chars, "common", 16)
            rp, idx, pairs, surv = orc.filter_match_fps(
                w.dictionary, Q, k, metric, orc.fingerprints(w.dictionary, m, "count", 32, gray=False),
                orc.fingerprints(Q, m, "count", 32, gray=False), "count_l1", 32)
            assert np.array_equal(rp, rp0) and np.array_equal(idx, idx0), (metric, k, "l1")
            _, _, pairs_g, surv_g = orc.filter_match(w.dictionary, Q, k, metric, m, "count", 32)
            assert pairs == pairs_g and rp0[-1] <= surv <= surv_g


ALL_CHECKS = [
    check_instance_example, check_run_ran, check_repeated_symbols, check_halves,
    check_count_saturation, check_positions, check_fd_fields, check_symbol_sets,
    check_textbook_distances, check_edit_ball, check_distance_identities, check_verifiers,
    check_match_against_pairs, check_counterexamples, check_filter_decision, check_bound_sweep,
    check_filter_is_speedup, check_count_l1, check_count_l1_sweep, check_qgram_fingerprints, check_qgram_sweep,
    check_fps_filter_is_speedup,
]
