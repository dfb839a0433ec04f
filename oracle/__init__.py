"""CPU oracle for fingerprint-filtered keyword matching (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never calls it and shares no
code with it.  ``oracle.c`` holds the matching definitions (Sec. 1, Sec. 3,
Sec. 3.3, Eq. 1, Sec. 4 of arXiv 1711.08475); ``learned.py`` holds the fp64
reference of the learned symbol-to-bit map's loss and gradients.  This module
compiles ``oracle.c`` with the host C compiler and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

HAM, LEV = 0, 1
OCC, OCCH, COUNT, POS = 0, 1, 2, 3
TYPES = {"occ": OCC, "occh": OCCH, "count": COUNT, "pos": POS}
METRICS = {"ham": HAM, "lev": LEV}
FD_KINDS = {"weight": 0, "count_l1": 1}  # distance of orc_filter_match_fps / orc_bound_violations_fps
SET_COMMON, SET_RARE, SET_MIXED = 0, 1, 2
SETS = {"common": SET_COMMON, "rare": SET_RARE, "mixed": SET_MIXED}

_lock = threading.Lock()
_default = None


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile oracle.c (or another copy of it) into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-pthread", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _bind(path: str):
    L = ctypes.CDLL(path)
    u8p, i64p, i32p, u32p, i8p = (ctypes.POINTER(t) for t in (
        ctypes.c_uint8, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int8))
    i64, i32 = ctypes.c_int64, ctypes.c_int
    L.orc_ham.argtypes = [u8p, i64, u8p, i64]
    L.orc_ham.restype = i64
    L.orc_lev.argtypes = [u8p, i64, u8p, i64]
    L.orc_lev.restype = i64
    L.orc_ham_within.argtypes = [u8p, i64, u8p, i64, i32]
    L.orc_ham_within.restype = i32
    L.orc_lev_within.argtypes = [u8p, i64, u8p, i64, i32]
    L.orc_lev_within.restype = i32
    L.orc_fingerprint.argtypes = [u8p, i64, i8p, i32, i32, i32, i32, i32]
    L.orc_fingerprint.restype = ctypes.c_uint32
    L.orc_fingerprint_many.argtypes = [u8p, i64p, i64, i8p, i32, i32, i32, i32, i32, u32p]
    L.orc_fingerprint_many.restype = None
    L.orc_fd.argtypes = [ctypes.c_uint32, ctypes.c_uint32, i32, i32, i32, i32]
    L.orc_fd.restype = i32
    L.orc_symbol_map.argtypes = [u8p, i64, i32, i32, i8p, i64p]
    L.orc_symbol_map.restype = i32
    L.orc_match.argtypes = [u8p, i64p, i64, u8p, i64p, i64, i32, i32, i32, i32, i64p,
                            ctypes.POINTER(i32p)]
    L.orc_match.restype = i32
    L.orc_filter_match.argtypes = [u8p, i64p, i64, u8p, i64p, i64, i32, i32, i32, i32, i32,
                                   i32, i32, i8p, i32, i64p, ctypes.POINTER(i32p), i64p]
    L.orc_filter_match.restype = i32
    L.orc_bound_violations.argtypes = [u8p, i64p, i64, i8p, i32, i32, i32, i32, i32, i32, i64p]
    L.orc_bound_violations.restype = None
    L.orc_fd_count_l1.argtypes = [ctypes.c_uint32, ctypes.c_uint32, i32, i32]
    L.orc_fd_count_l1.restype = i32
    L.orc_qgram_map.argtypes = [u8p, i64p, i64, i32, i32, u8p, i64p]
    L.orc_qgram_map.restype = i32
    L.orc_fp_qgram.argtypes = [u8p, i64, u8p, i32, i32]
    L.orc_fp_qgram.restype = ctypes.c_uint32
    L.orc_fp_qgram_many.argtypes = [u8p, i64p, i64, u8p, i32, i32, u32p]
    L.orc_fp_qgram_many.restype = None
    L.orc_filter_match_fps.argtypes = [u8p, i64p, i64, u8p, i64p, i64, i32, i32, u32p, u32p, i32, i32, i32,
                                       i32, i32, i64p, ctypes.POINTER(i32p), i64p]
    L.orc_filter_match_fps.restype = i32
    L.orc_bound_violations_fps.argtypes = [u8p, i64p, i64, u32p, i32, i32, i32, i32, i32, i64p]
    L.orc_bound_violations_fps.restype = None
    L.orc_free.argtypes = [ctypes.c_void_p]
    L.orc_free.restype = None
    return L


def lib():
    return default().L


def default() -> "Oracle":
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _bytes(s) -> np.ndarray:
    if isinstance(s, str):
        s = s.encode()
    return np.frombuffer(bytes(s), dtype=np.uint8) if len(s) else np.zeros(1, np.uint8)


def layout(type_name: str, width: int, b: int = 2, p: int = 3) -> dict:
    """Number of tracked symbols for a fingerprint type and width.

    Sec. 4 fixes 16-bit fingerprints with b = 2 and p = 3: 16 occurrence
    symbols, 8 occurrence-halved or count symbols, and 5 position symbols plus
    1 occurrence bit.  Wider fingerprints follow the same rule: floor(W/p)
    position fields and the W mod p leftover bits as occurrence bits.
    """
    if type_name == "occ":
        return {"sigma": width, "n_pos": 0}
    if type_name == "occh":
        return {"sigma": width // 2, "n_pos": 0}
    if type_name == "count":
        return {"sigma": width // b, "n_pos": 0}
    if type_name == "pos":
        n_pos = width // p
        return {"sigma": n_pos + (width - p * n_pos), "n_pos": n_pos}
    raise ValueError(type_name)


def map_from_order(order: bytes) -> np.ndarray:
    """Map giving field q to the q-th symbol of ``order`` (-1 elsewhere)."""
    m = np.full(256, -1, dtype=np.int8)
    for q, ch in enumerate(order):
        m[ch] = q
    return m


def _nz(a: np.ndarray) -> np.ndarray:
    return a if a.size else np.zeros(1, a.dtype)


class Oracle:
    """ctypes view of one compiled copy of oracle.c."""

    def __init__(self, path: str):
        self.path = path
        self.L = _bind(path)

    # -- distances ---------------------------------------------------------
    def ham(self, a, b):
        """Hamming distance (Sec. 1); None when the lengths differ (infinite)."""
        A, B = _bytes(a), _bytes(b)
        d = self.L.orc_ham(_p(A, ctypes.c_uint8), len(a), _p(B, ctypes.c_uint8), len(b))
        return None if d < 0 else int(d)

    def lev(self, a, b) -> int:
        """Levenshtein distance (Sec. 1), full Wagner-Fischer."""
        A, B = _bytes(a), _bytes(b)
        return int(self.L.orc_lev(_p(A, ctypes.c_uint8), len(a), _p(B, ctypes.c_uint8), len(b)))

    def ham_within(self, a, b, k: int) -> bool:
        A, B = _bytes(a), _bytes(b)
        return bool(self.L.orc_ham_within(_p(A, ctypes.c_uint8), len(a), _p(B, ctypes.c_uint8),
                                          len(b), k))

    def lev_within(self, a, b, k: int) -> bool:
        A, B = _bytes(a), _bytes(b)
        return bool(self.L.orc_lev_within(_p(A, ctypes.c_uint8), len(a), _p(B, ctypes.c_uint8),
                                          len(b), k))

    # -- fingerprints ------------------------------------------------------
    def symbol_map(self, chars: np.ndarray, set_name: str, sigma: int):
        """(map int8[256], counts int64[256], fields used) for a collection."""
        chars = np.ascontiguousarray(chars, dtype=np.uint8)
        m = np.full(256, -1, dtype=np.int8)
        c = np.zeros(256, dtype=np.int64)
        used = self.L.orc_symbol_map(_p(_nz(chars), ctypes.c_uint8), chars.size, SETS[set_name],
                                     sigma, _p(m, ctypes.c_int8), _p(c, ctypes.c_int64))
        return m, c, used

    def fingerprint(self, s, map_: np.ndarray, type_name: str, width: int = 16, b: int = 2,
                    p: int = 3, gray: bool = True) -> int:
        S = _bytes(s)
        lay = layout(type_name, width, b, p)
        m = np.ascontiguousarray(map_, dtype=np.int8)
        return int(self.L.orc_fingerprint(_p(S, ctypes.c_uint8), len(s), _p(m, ctypes.c_int8),
                                          TYPES[type_name], b, p, lay["n_pos"], int(gray)))

    def fingerprints(self, strings, map_: np.ndarray, type_name: str, width: int, b: int = 2,
                     p: int = 3, gray: bool = True) -> np.ndarray:
        lay = layout(type_name, width, b, p)
        n = len(strings)
        out = np.zeros(max(n, 1), dtype=np.uint32)
        m = np.ascontiguousarray(map_, dtype=np.int8)
        self.L.orc_fingerprint_many(_p(_nz(strings.chars), ctypes.c_uint8),
                                    _p(strings.offsets, ctypes.c_int64), n, _p(m, ctypes.c_int8),
                                    TYPES[type_name], b, p, lay["n_pos"], int(gray),
                                    _p(out, ctypes.c_uint32))
        return out[:n]

    def fd(self, a: int, b: int, type_name: str, width: int, p: int = 3) -> int:
        lay = layout(type_name, width, 2, p)
        return int(self.L.orc_fd(a, b, TYPES[type_name], width, p, lay["n_pos"]))

    def fd_count_l1(self, a: int, b: int, width: int, bits: int = 2) -> int:
        """Sum over count fields of |c1 - c2| (binary-coded counts, Sec. 3.3 remark)."""
        return int(self.L.orc_fd_count_l1(a, b, width, bits))

    def qgram_map(self, strings, q: int, sigma: int = 32):
        """(grams uint8[used, q], counts int64[used]): the sigma most frequent q-grams."""
        g = np.zeros(max(sigma * q, 1), dtype=np.uint8)
        c = np.zeros(max(sigma, 1), dtype=np.int64)
        used = self.L.orc_qgram_map(_p(_nz(strings.chars), ctypes.c_uint8), _p(strings.offsets, ctypes.c_int64),
                                    len(strings), q, sigma, _p(g, ctypes.c_uint8), _p(c, ctypes.c_int64))
        if used < 0:
            raise ValueError("q must be 1..3")
        return g[:used * q].reshape(used, q), c[:used]

    def qgram_fingerprint(self, s, grams: np.ndarray) -> int:
        S = _bytes(s)
        g = np.ascontiguousarray(grams, dtype=np.uint8)
        return int(self.L.orc_fp_qgram(_p(S, ctypes.c_uint8), len(s), _p(_nz(g.reshape(-1)), ctypes.c_uint8),
                                       g.shape[0], g.shape[1] if g.ndim == 2 else 1))

    def qgram_fingerprints(self, strings, grams: np.ndarray) -> np.ndarray:
        g = np.ascontiguousarray(grams, dtype=np.uint8)
        out = np.zeros(max(len(strings), 1), dtype=np.uint32)
        self.L.orc_fp_qgram_many(_p(_nz(strings.chars), ctypes.c_uint8), _p(strings.offsets, ctypes.c_int64),
                                 len(strings), _p(_nz(g.reshape(-1)), ctypes.c_uint8), g.shape[0], g.shape[1],
                                 _p(out, ctypes.c_uint32))
        return out[:len(strings)]

    # -- matchers ----------------------------------------------------------
    def _collect(self, rc, row_ptr, idx_p):
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        n = int(row_ptr[-1])
        idx = np.ctypeslib.as_array(idx_p, shape=(max(n, 1),))[:n].copy()
        self.L.orc_free(ctypes.cast(idx_p, ctypes.c_void_p))
        return row_ptr, idx

    def match(self, dictionary, queries, k: int, metric: str, prune: bool = True, threads: int = 0):
        """Brute-force match lists as CSR (row_ptr int64[q+1], idx int32)."""
        d, q = dictionary, queries
        row_ptr = np.zeros(len(q) + 1, dtype=np.int64)
        idx_p = ctypes.POINTER(ctypes.c_int32)()
        rc = self.L.orc_match(_p(_nz(d.chars), ctypes.c_uint8), _p(d.offsets, ctypes.c_int64), len(d),
                              _p(_nz(q.chars), ctypes.c_uint8), _p(q.offsets, ctypes.c_int64), len(q),
                              k, METRICS[metric], int(prune), threads, _p(row_ptr, ctypes.c_int64),
                              ctypes.byref(idx_p))
        return self._collect(rc, row_ptr, idx_p)

    def filter_match(self, dictionary, queries, k: int, metric: str, map_: np.ndarray,
                     type_name: str, width: int, b: int = 2, p: int = 3, gray: bool = True,
                     threads: int = 0):
        """The paper's filter + verify method: (row_ptr, idx, pairs, survivors)."""
        d, q = dictionary, queries
        row_ptr = np.zeros(len(q) + 1, dtype=np.int64)
        stats = np.zeros(2, dtype=np.int64)
        idx_p = ctypes.POINTER(ctypes.c_int32)()
        m = np.ascontiguousarray(map_, dtype=np.int8)
        rc = self.L.orc_filter_match(_p(_nz(d.chars), ctypes.c_uint8), _p(d.offsets, ctypes.c_int64),
                                     len(d), _p(_nz(q.chars), ctypes.c_uint8),
                                     _p(q.offsets, ctypes.c_int64), len(q), k, METRICS[metric],
                                     TYPES[type_name], width, b, p, int(gray), _p(m, ctypes.c_int8),
                                     threads, _p(row_ptr, ctypes.c_int64), ctypes.byref(idx_p),
                                     _p(stats, ctypes.c_int64))
        rp, idx = self._collect(rc, row_ptr, idx_p)
        return rp, idx, int(stats[0]), int(stats[1])

    def filter_match_fps(self, dictionary, queries, k: int, metric: str, dfp: np.ndarray, qfp: np.ndarray,
                         kind: str = "weight", width: int = 32, bits: int = 2, q: int = 1, threads: int = 0):
        """The Sec. 4 method on given fingerprints, bound D >= ceil(F_D / 2q): (row_ptr, idx, pairs, survivors)."""
        d, qs = dictionary, queries
        row_ptr = np.zeros(len(qs) + 1, dtype=np.int64)
        stats = np.zeros(2, dtype=np.int64)
        idx_p = ctypes.POINTER(ctypes.c_int32)()
        df = np.ascontiguousarray(_nz(np.asarray(dfp, dtype=np.uint32)))
        qf = np.ascontiguousarray(_nz(np.asarray(qfp, dtype=np.uint32)))
        rc = self.L.orc_filter_match_fps(_p(_nz(d.chars), ctypes.c_uint8), _p(d.offsets, ctypes.c_int64), len(d),
                                         _p(_nz(qs.chars), ctypes.c_uint8), _p(qs.offsets, ctypes.c_int64), len(qs),
                                         k, METRICS[metric], _p(df, ctypes.c_uint32), _p(qf, ctypes.c_uint32),
                                         FD_KINDS[kind], width, bits, q, threads, _p(row_ptr, ctypes.c_int64),
                                         ctypes.byref(idx_p), _p(stats, ctypes.c_int64))
        rp, idx = self._collect(rc, row_ptr, idx_p)
        return rp, idx, int(stats[0]), int(stats[1])

    def bound_violations_fps(self, strings, fp: np.ndarray, kind: str, width: int, metric: str, bits: int = 2,
                             q: int = 1) -> dict:
        """Exhaustive check of D >= ceil(F_D / 2q) over all pairs of strings with lengths within 1."""
        out = np.zeros(4, dtype=np.int64)
        f = np.ascontiguousarray(_nz(np.asarray(fp, dtype=np.uint32)))
        self.L.orc_bound_violations_fps(_p(_nz(strings.chars), ctypes.c_uint8), _p(strings.offsets, ctypes.c_int64),
                                        len(strings), _p(f, ctypes.c_uint32), FD_KINDS[kind], width, bits, q,
                                        METRICS[metric], _p(out, ctypes.c_int64))
        return {"pairs": int(out[0]), "violations": int(out[1]),
                "example": (int(out[2]), int(out[3])) if out[1] else None}

    def bound_violations(self, strings, map_: np.ndarray, type_name: str, width: int, metric: str,
                         b: int = 2, p: int = 3, gray: bool = True) -> dict:
        """Exhaustive Eq. 1 check over all pairs of ``strings`` whose lengths differ by <= 1."""
        out = np.zeros(4, dtype=np.int64)
        m = np.ascontiguousarray(map_, dtype=np.int8)
        self.L.orc_bound_violations(_p(_nz(strings.chars), ctypes.c_uint8),
                                    _p(strings.offsets, ctypes.c_int64), len(strings),
                                    _p(m, ctypes.c_int8), TYPES[type_name], width, b, p, int(gray),
                                    METRICS[metric], _p(out, ctypes.c_int64))
        return {"pairs": int(out[0]), "violations": int(out[1]),
                "example": (int(out[2]), int(out[3])) if out[1] else None}


def eligible_pairs(dictionary, queries, k: int, metric: str) -> int:
    """Number of (query, word) pairs with equal lengths (Ham) or lengths within k (Lev)."""
    dl = np.bincount(dictionary.lengths(), minlength=1).astype(np.int64)
    csum = np.concatenate([[0], np.cumsum(dl)])
    n = queries.lengths()
    if metric == "ham":
        ok = n < len(dl)
        return int(dl[n[ok]].sum())
    lo = np.clip(n - k, 0, len(dl))
    hi = np.clip(n + k + 1, 0, len(dl))
    return int((csum[hi] - csum[lo]).sum())


# module-level shortcuts to the default build
def ham(a, b):
    return default().ham(a, b)


def lev(a, b):
    return default().lev(a, b)


def ham_within(a, b, k):
    return default().ham_within(a, b, k)


def lev_within(a, b, k):
    return default().lev_within(a, b, k)


def symbol_map(chars, set_name, sigma):
    return default().symbol_map(chars, set_name, sigma)


def fingerprint(s, map_, type_name, width=16, b=2, p=3, gray=True):
    return default().fingerprint(s, map_, type_name, width, b, p, gray)


def fingerprints(strings, map_, type_name, width, b=2, p=3, gray=True):
    return default().fingerprints(strings, map_, type_name, width, b, p, gray)


def fd(a, b, type_name, width, p=3):
    return default().fd(a, b, type_name, width, p)


def match(dictionary, queries, k, metric, prune=True, threads=0):
    return default().match(dictionary, queries, k, metric, prune, threads)


def filter_match(dictionary, queries, k, metric, map_, type_name, width, b=2, p=3, gray=True,
                 threads=0):
    return default().filter_match(dictionary, queries, k, metric, map_, type_name, width, b, p, gray,
                                  threads)


def bound_violations(strings, map_, type_name, width, metric, b=2, p=3, gray=True):
    return default().bound_violations(strings, map_, type_name, width, metric, b, p, gray)


def fd_count_l1(a, b, width, bits=2):
    return default().fd_count_l1(a, b, width, bits)


def qgram_map(strings, q, sigma=32):
    return default().qgram_map(strings, q, sigma)


def qgram_fingerprints(strings, grams):
    return default().qgram_fingerprints(strings, grams)


def filter_match_fps(dictionary, queries, k, metric, dfp, qfp, kind="weight", width=32, bits=2, q=1, threads=0):
    return default().filter_match_fps(dictionary, queries, k, metric, dfp, qfp, kind, width, bits, q, threads)


def bound_violations_fps(strings, fp, kind, width, metric, bits=2, q=1):
    return default().bound_violations_fps(strings, fp, kind, width, metric, bits, q)
