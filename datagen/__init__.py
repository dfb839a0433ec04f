"""Seeded synthetic workloads for fingerprint-filtered keyword matching.

This module only produces inputs: dictionaries of byte strings, query batches,
batch schedules and request arrivals.  It holds none of the matching method's
arithmetic (no fingerprints, no distances, no filter), so both the CPU oracle
and the CUDA path can take their inputs from here without sharing any of the
method.

Every random number comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: draw ``i`` of a stream with key ``s`` is the
``(i+1)``-th SplitMix64 output from seed ``s``, i.e. the 64-bit finaliser
applied to ``s + (i+1) * 0x9E3779B97F4A7C15``.  Stream keys are derived from a
config seed and a text label with FNV-1a (64-bit) followed by the same
finaliser, so every workload is reproducible from ``(seed, label)`` alone.

The paper's data sets (an English word list, a URL crawl, a synthetic English
file) are not available; the generators below stand in for them with the
shapes the matching method cares about: the length distribution (equal-length
buckets for Hamming, neighbouring lengths for Levenshtein), a skewed symbol
distribution (fingerprints track the most frequent symbols, Sec. 3) and, for
URL-like data, shared prefixes (Sec. 4.1 explains the URL speedups by them).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# ---------------------------------------------------------------------------
# SplitMix64, counter-based
# ---------------------------------------------------------------------------


def mix64(z):
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _fnv1a64(label: str) -> int:
    h = 0xCBF29CE484222325
    for b in label.encode():
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def stream_key(seed: int, label: str) -> np.uint64:
    """Key of the stream named ``label`` under config seed ``seed``."""
    s = np.array([(int(seed) & 0xFFFFFFFFFFFFFFFF) ^ _fnv1a64(label)], dtype=np.uint64)
    return mix64(s)[0]


def draws(key, n: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+n-1`` of the stream with key ``key`` (uint64)."""
    i = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (i + np.uint64(1)) * GOLDEN)


def uniform(key, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws(key, n, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def randint(key, n: int, lo, hi) -> np.ndarray:
    """Integers uniform on the closed range [lo, hi] (elementwise bounds allowed)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    span = (hi - lo + 1).astype(np.float64)
    return lo + np.minimum(np.floor(uniform(key, n) * span).astype(np.int64), (hi - lo))


def normal(key, n: int) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniforms."""
    u1 = uniform(key, n, 0)
    u2 = uniform(key, n, n)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 is in (0, 1]
    return r * np.cos(2.0 * math.pi * u2)


def categorical(key, n: int, weights: np.ndarray, chunk: int = 1 << 24) -> np.ndarray:
    """Indices drawn with probability proportional to ``weights``."""
    cdf = np.cumsum(np.asarray(weights, dtype=np.float64))
    cdf /= cdf[-1]
    out = np.empty(n, dtype=np.int64)
    # searchsorted(cdf, u, "right") through a 4096-cell guide table: start at the
    # count of cdf entries <= the cell's left edge, then step over the few
    # entries inside the cell (same result as a full binary search, faster)
    T = 4096
    guide = np.searchsorted(cdf, np.arange(T, dtype=np.float64) / T, side="right")
    last = len(cdf) - 1
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        u = uniform(key, e - s, s)
        r = guide[(u * T).astype(np.int64)]
        while True:
            step = cdf[np.minimum(r, last)] <= u
            step &= r <= last
            if not step.any():
                break
            r += step
        out[s:e] = r
    np.minimum(out, last, out=out)
    return out


def permutation(key, n: int) -> np.ndarray:
    """A uniformly shuffled order of ``0..n-1`` (argsort of draws)."""
    return np.argsort(draws(key, n), kind="stable")


# ---------------------------------------------------------------------------
# String sets
# ---------------------------------------------------------------------------


@dataclass
class Strings:
    """A list of byte strings in CSR form: string i is chars[offsets[i]:offsets[i+1]]."""

    chars: np.ndarray  # uint8
    offsets: np.ndarray  # int64, len n+1

    def __post_init__(self):
        self.chars = np.ascontiguousarray(self.chars, dtype=np.uint8)
        self.offsets = np.ascontiguousarray(self.offsets, dtype=np.int64)

    def __len__(self) -> int:
        return len(self.offsets) - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def get(self, i: int) -> bytes:
        return self.chars[self.offsets[i]:self.offsets[i + 1]].tobytes()

    def subset(self, idx) -> "Strings":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths()[idx]
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        pos = np.repeat(self.offsets[idx] - off[:-1], lens) + np.arange(off[-1], dtype=np.int64)
        return Strings(self.chars[pos], off)

    @staticmethod
    def from_list(items) -> "Strings":
        bs = [x.encode() if isinstance(x, str) else bytes(x) for x in items]
        off = np.zeros(len(bs) + 1, dtype=np.int64)
        np.cumsum([len(b) for b in bs], out=off[1:])
        return Strings(np.frombuffer(b"".join(bs), dtype=np.uint8).copy(), off)

    @staticmethod
    def concat(parts) -> "Strings":
        chars = np.concatenate([p.chars for p in parts]) if parts else np.zeros(0, np.uint8)
        lens = np.concatenate([p.lengths() for p in parts]) if parts else np.zeros(0, np.int64)
        off = np.zeros(len(lens) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        return Strings(chars, off)

    def to_list(self):
        return [self.get(i) for i in range(len(self))]


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


# ---------------------------------------------------------------------------
# Symbol tables (all synthetic; none is a published frequency table)
# ---------------------------------------------------------------------------

# The paper prints only the rank order of the 16 most common English letters
# (Sec. 3.1).  The remaining ten letters follow in alphabetical order, an
# arbitrary choice.
ENGLISH_ORDER = b"etaoinshrdlcumwf" + b"bgjkpqvxyz"
ENGLISH_TOP_MASS = 0.12


def _solve_rho(top_mass: float, n: int) -> float:
    """rho with (1-rho)/(1-rho**n) == top_mass (the first of n geometric weights)."""
    lo, hi = 1e-9, 1.0 - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        w0 = (1.0 - mid) / (1.0 - mid ** n)
        if w0 > top_mass:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def english_table():
    """(symbols uint8[26], weights float64[26], rho): geometric weights w_r ~ rho**r."""
    rho = _solve_rho(ENGLISH_TOP_MASS, 26)
    w = rho ** np.arange(26, dtype=np.float64)
    w /= w.sum()
    return np.frombuffer(ENGLISH_ORDER, dtype=np.uint8).copy(), w, rho


def uniform_az_table():
    sym = np.arange(ord("a"), ord("z") + 1, dtype=np.uint8)
    return sym, np.full(26, 1.0 / 26.0)


def url_table():
    """Printable ASCII 0x20..0x7E (95 symbols) with URL-like weights.

    Lower case letters carry 0.68 of the mass (split by the English-like
    geometric table), '/', '.', '-', ':' carry 0.07, 0.05, 0.03, 0.01, the ten
    digits 0.08 and the upper case letters 0.05 (uniformly), and the other 29
    printable symbols share the remaining 0.03.
    """
    sym = np.arange(0x20, 0x7F, dtype=np.uint8)
    w = np.zeros(95)
    esym, ew, _ = english_table()
    for s, x in zip(esym, ew):
        w[s - 0x20] += 0.68 * x
    for ch, m in ((b"/", 0.07), (b".", 0.05), (b"-", 0.03), (b":", 0.01)):
        w[ch[0] - 0x20] += m
    digits = [c - 0x20 for c in range(ord("0"), ord("9") + 1)]
    upper = [c - 0x20 for c in range(ord("A"), ord("Z") + 1)]
    w[digits] += 0.08 / 10
    w[upper] += 0.05 / 26
    rest = [i for i in range(95) if w[i] == 0.0]
    assert len(rest) == 29
    w[rest] += 0.03 / 29
    w /= w.sum()
    return sym, w


# ---------------------------------------------------------------------------
# Length laws
# ---------------------------------------------------------------------------


def _phi(x: float) -> float:
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


def lognormal_round_pmf(mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    """P(L = l) for L = clamp(round(exp(mu + sigma Z)), lo, hi), l = lo..hi."""
    p = np.zeros(hi - lo + 1)
    for l in range(lo, hi + 1):
        a = -math.inf if l == lo else (math.log(l - 0.5) - mu) / sigma
        b = math.inf if l == hi else (math.log(l + 0.5) - mu) / sigma
        p[l - lo] = (1.0 if b == math.inf else _phi(b)) - (0.0 if a == -math.inf else _phi(a))
    return p


def fit_lognormal_mu(target_mean: float, sigma: float, lo: int, hi: int) -> float:
    """mu such that the discretised, clamped lognormal has mean ``target_mean``."""
    a, b = math.log(lo) - 2.0, math.log(hi) + 2.0
    ls = np.arange(lo, hi + 1)
    for _ in range(200):
        mid = 0.5 * (a + b)
        m = float((lognormal_round_pmf(mid, sigma, lo, hi) * ls).sum())
        if m < target_mean:
            a = mid
        else:
            b = mid
    return 0.5 * (a + b)


@dataclass
class LengthLaw:
    kind: str  # "uniform" | "lognormal"
    lo: int
    hi: int
    mu: float = 0.0
    sigma: float = 0.0

    def sample(self, key, n: int) -> np.ndarray:
        if self.kind == "uniform":
            return randint(key, n, self.lo, self.hi)
        z = normal(key, n)
        x = np.rint(np.exp(self.mu + self.sigma * z))
        return np.clip(x, self.lo, self.hi).astype(np.int64)


ENGLISH_SIGMA = 0.35
ENGLISH_MEAN = 8.0


def english_length_law(hi: int = 24) -> LengthLaw:
    # mu is fitted once on the 2..24 law (mean 8) and reused for wider clamps.
    mu = fit_lognormal_mu(ENGLISH_MEAN, ENGLISH_SIGMA, 2, 24)
    return LengthLaw("lognormal", 2, hi, mu=mu, sigma=ENGLISH_SIGMA)


def url_length_law() -> LengthLaw:
    return LengthLaw("lognormal", 15, 120, mu=math.log(45.0), sigma=0.4)


# ---------------------------------------------------------------------------
# Dictionaries
# ---------------------------------------------------------------------------


@dataclass
class StringLaw:
    """How to draw one collection: symbol table, length law and shared prefixes."""

    symbols: np.ndarray
    weights: np.ndarray
    lengths: LengthLaw
    n_prefixes: int = 0
    prefix_frac: float = 0.0
    prefix_len: tuple = (10, 30)
    prefixes: Strings | None = None

    def draw(self, seed: int, label: str, n: int) -> Strings:
        lens = self.lengths.sample(stream_key(seed, label + "/len"), n)
        off = _offsets(lens)
        idx = categorical(stream_key(seed, label + "/sym"), int(off[-1]), self.weights)
        chars = self.symbols[idx]
        if self.prefixes is not None and self.prefix_frac > 0.0 and n > 0:
            use = uniform(stream_key(seed, label + "/usepfx"), n) < self.prefix_frac
            which = randint(stream_key(seed, label + "/pfx"), n, 0, len(self.prefixes) - 1)
            rows = np.nonzero(use)[0]
            plen = np.minimum(self.prefixes.lengths()[which[rows]], lens[rows])
            if len(rows):
                dst = np.repeat(off[rows], plen) + _ranges(plen)
                src = np.repeat(self.prefixes.offsets[which[rows]], plen) + _ranges(plen)
                chars[dst] = self.prefixes.chars[src]
        return Strings(chars, off)


def _ranges(lens: np.ndarray) -> np.ndarray:
    """Concatenation of arange(l) for each l in lens."""
    lens = np.asarray(lens, dtype=np.int64)
    total = int(lens.sum())
    if total == 0:
        return np.zeros(0, dtype=np.int64)
    starts = np.repeat(_offsets(lens)[:-1], lens)
    return np.arange(total, dtype=np.int64) - starts


def uniform_law() -> StringLaw:
    s, w = uniform_az_table()
    return StringLaw(s, w, LengthLaw("uniform", 4, 12))


def english_law(hi: int = 24) -> StringLaw:
    s, w, _ = english_table()
    return StringLaw(s, w, english_length_law(hi))


def url_law(seed: int) -> StringLaw:
    s, w = url_table()
    law = StringLaw(s, w, url_length_law(), n_prefixes=64, prefix_frac=0.40)
    plaw = StringLaw(s, w, LengthLaw("uniform", 10, 30))
    law.prefixes = plaw.draw(seed, "prefixes", 64)
    return law


# ---------------------------------------------------------------------------
# Queries: one-edit mutations of dictionary words plus fresh random strings
# ---------------------------------------------------------------------------

SUB, INS, DEL = 0, 1, 2


def mutate(dictionary: Strings, law: StringLaw, seed: int, label: str, n: int, metric: str) -> Strings:
    """``n`` one-edit mutations of uniformly chosen dictionary words.

    Hamming: a substitution at a uniform position by a different symbol drawn
    from the law's symbol distribution.  Levenshtein: substitution, insertion
    or deletion with probability 1/3 each; an insertion position is uniform in
    [0, len]; a deletion needs len > 1 (else it becomes a substitution); an
    empty source word gets an insertion.
    """
    if n == 0:
        return Strings(np.zeros(0, np.uint8), np.zeros(1, np.int64))
    base = randint(stream_key(seed, label + "/base"), n, 0, len(dictionary) - 1)
    src_len = dictionary.lengths()[base]
    if metric == "ham":
        op = np.full(n, SUB, dtype=np.int64)
    elif metric == "lev":
        op = randint(stream_key(seed, label + "/op"), n, 0, 2)
        op[(op == DEL) & (src_len <= 1)] = SUB
    else:
        raise ValueError(metric)
    op[src_len == 0] = INS
    hi = np.where(op == INS, src_len, src_len - 1)
    pos = randint(stream_key(seed, label + "/pos"), n, 0, np.maximum(hi, 0))
    old = np.zeros(n, dtype=np.uint8)
    has_old = op != INS
    old[has_old] = dictionary.chars[dictionary.offsets[base[has_old]] + pos[has_old]]
    sym = law.symbols[categorical(stream_key(seed, label + "/sym0"), n, law.weights)]
    need = (op == SUB) & (sym == old)
    rnd = 1
    while need.any():
        if rnd > 256:
            raise RuntimeError("symbol table cannot provide a different symbol")
        rows = np.nonzero(need)[0]
        sym[rows] = law.symbols[categorical(stream_key(seed, f"{label}/sym{rnd}"), n, law.weights)[rows]]
        need = (op == SUB) & (sym == old)
        rnd += 1
    new_len = src_len + (op == INS) - (op == DEL)
    off = _offsets(new_len)
    q = np.repeat(np.arange(n, dtype=np.int64), new_len)
    j = _ranges(new_len)
    p = pos[q]
    o = op[q]
    src_j = j.copy()
    src_j[(o == INS) & (j > p)] -= 1
    src_j[(o == DEL) & (j >= p)] += 1
    fresh = ((o == SUB) | (o == INS)) & (j == p)
    src_j[fresh] = 0
    chars = np.zeros(len(j), dtype=np.uint8)
    keep = ~fresh
    chars[keep] = dictionary.chars[dictionary.offsets[base[q[keep]]] + src_j[keep]]
    chars[fresh] = sym[q[fresh]]
    return Strings(chars, off)


def make_queries(dictionary: Strings, law: StringLaw, seed: int, label: str, n: int,
                 mut_frac: float, metric: str) -> Strings:
    n_mut = int(round(mut_frac * n))
    m = mutate(dictionary, law, seed, label + "/mut", n_mut, metric)
    r = law.draw(seed, label + "/rand", n - n_mut)
    both = Strings.concat([m, r])
    order = permutation(stream_key(seed, label + "/shuffle"), n)
    return both.subset(order)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    seed: int
    dictionary: Strings
    queries: dict = field(default_factory=dict)  # metric -> Strings
    fp_types: list = field(default_factory=list)  # [(type_name, width, metrics)]
    k: int = 1
    info: dict = field(default_factory=dict)
    law: StringLaw | None = None


WORKLOADS = ("uniform10k", "english1m", "url2m", "batched10m", "serving5m")
SEEDS = {name: 1711 + i + 1 for i, name in enumerate(WORKLOADS)}


def uniform10k(n_words: int = 10_000, n_queries: int = 1_000, seed: int | None = None) -> Workload:
    """10,000 words over 'a'..'z' (iid uniform letters, lengths uniform 4..12);
    1,000 queries per metric, half one-edit mutations, half fresh; k=1; occ16."""
    seed = SEEDS["uniform10k"] if seed is None else seed
    law = uniform_law()
    d = law.draw(seed, "dict", n_words)
    qs = {m: make_queries(d, law, seed, "q/" + m, n_queries, 0.5, m) for m in ("ham", "lev")}
    return Workload("uniform10k", seed, d, qs, [("occ", 16, ("ham", "lev"))], 1, {}, law)


def english1m(n_words: int = 1_000_000, n_queries: int = 100_000, seed: int | None = None) -> Workload:
    """1,000,000 English-like words (lognormal lengths, mean 8, 2..24); 100,000
    queries per metric (60% one-edit mutations); k=1; count32 (Ham, Lev) and
    occh32 (Ham only)."""
    seed = SEEDS["english1m"] if seed is None else seed
    law = english_law(24)
    d = law.draw(seed, "dict", n_words)
    qs = {m: make_queries(d, law, seed, "q/" + m, n_queries, 0.6, m) for m in ("ham", "lev")}
    _, _, rho = english_table()
    info = {"lognormal_mu": law.lengths.mu, "lognormal_sigma": law.lengths.sigma, "rho": rho}
    return Workload("english1m", seed, d, qs, [("count", 32, ("ham", "lev")), ("occh", 32, ("ham",))],
                    1, info, law)


def url2m(n_words: int = 2_000_000, n_queries: int = 100_000, seed: int | None = None) -> Workload:
    """2,000,000 URL-like strings (printable ASCII, lognormal lengths median 45,
    15..120, 40% with one of 64 shared prefixes); 100,000 queries per metric
    (50% mutations); k=1; occ32 (Ham, Lev) and pos32 (Ham only)."""
    seed = SEEDS["url2m"] if seed is None else seed
    law = url_law(seed)
    d = law.draw(seed, "dict", n_words)
    qs = {m: make_queries(d, law, seed, "q/" + m, n_queries, 0.5, m) for m in ("ham", "lev")}
    return Workload("url2m", seed, d, qs, [("occ", 32, ("ham", "lev")), ("pos", 32, ("ham",))], 1, {}, law)


@dataclass
class Batch:
    k: int
    metric: str
    queries: Strings


def batched10m(n_words: int = 10_000_000, n_batches: int = 256, max_batch: int = 50_000,
               seed: int | None = None) -> tuple[Workload, list]:
    """10,000,000 English-like words (lengths 2..64); ``n_batches`` query batches
    with sizes floor(exp(U(0, ln max_batch))); per batch k in {1, 2} and the
    metric drawn by seed; 60% one-edit mutations per batch."""
    seed = SEEDS["batched10m"] if seed is None else seed
    law = english_law(64)
    d = law.draw(seed, "dict", n_words)
    u = uniform(stream_key(seed, "batch/size"), n_batches)
    sizes = np.maximum(1, np.floor(np.exp(u * math.log(max_batch))).astype(np.int64))
    ks = randint(stream_key(seed, "batch/k"), n_batches, 1, 2)
    ms = randint(stream_key(seed, "batch/metric"), n_batches, 0, 1)
    batches = []
    for b in range(n_batches):
        metric = ("ham", "lev")[int(ms[b])]
        q = make_queries(d, law, seed, f"batch/{b}", int(sizes[b]), 0.6, metric)
        batches.append(Batch(int(ks[b]), metric, q))
    w = Workload("batched10m", seed, d, {}, [("occ", 32, ("ham", "lev")), ("count", 32, ("ham", "lev"))],
                 0, {"batch_sizes": sizes.tolist()}, law)
    return w, batches


@dataclass
class Request:
    arrival_s: float
    queries: Strings


def poisson_requests(d: Strings, law: StringLaw, seed: int, duration_s: float, rate_qps: float,
                     max_request: int = 4096, label: str = "req", n_requests: int | None = None):
    """Requests with sizes U{1..max_request} (50% one-edit Lev mutations of
    dictionary words) arriving as a Poisson process whose mean pattern rate is
    ``rate_qps``: every request that arrives within ``duration_s``, or exactly
    ``n_requests`` requests when that is given."""
    mean_size = (1 + max_request) / 2.0
    lam = rate_qps / mean_size
    n_draw = n_requests if n_requests is not None else max(1, int(math.ceil(duration_s * lam * 1.5)) + 8)
    gaps = -np.log1p(-uniform(stream_key(seed, f"{label}/gap"), n_draw)) / lam
    t = np.cumsum(gaps)
    n_req = n_requests if n_requests is not None else (int(np.searchsorted(t, duration_s, side="right")) or 1)
    sizes = randint(stream_key(seed, f"{label}/size"), n_req, 1, max_request)
    pool = make_queries(d, law, seed, f"{label}/pool", int(sizes.sum()), 0.5, "lev")
    off = _offsets(sizes)
    reqs = [Request(float(t[i]), pool.subset(np.arange(off[i], off[i + 1]))) for i in range(n_req)]
    return reqs, pool


def serving5m(n_words: int = 5_000_000, duration_s: float = 10.0, rate_qps: float = 5000.0,
              max_request: int = 4096, seed: int | None = None, n_requests: int | None = None
              ) -> tuple[Workload, list]:
    """5,000,000 URL-like strings; requests with sizes U{1..max_request} arriving
    as a Poisson process whose mean query rate is ``rate_qps``; k=1 Lev."""
    seed = SEEDS["serving5m"] if seed is None else seed
    law = url_law(seed)
    d = law.draw(seed, "dict", n_words)
    reqs, pool = poisson_requests(d, law, seed, duration_s, rate_qps, max_request, "req", n_requests)
    w = Workload("serving5m", seed, d, {"lev": pool}, [("occ", 32, ("lev",))], 1,
                 {"rate_qps": rate_qps, "n_requests": len(reqs)}, law)
    return w, reqs
