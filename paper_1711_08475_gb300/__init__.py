"""GB300-native fingerprint-filtered approximate keyword matching.

Method: Cislak and Grabowski, arXiv 1711.08475.  The names below mirror the
C ABI in include/fp.h one to one; this layer only turns numpy arrays / torch
tensors into pointers and handles into objects.  All computation happens in
libfpmatch.so (CUDA, sm_103a).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import (FP_COUNT, FP_HAM, FP_LEV, FP_MODE_FUSED, FP_MODE_PLAIN, FP_MODE_TILED, FP_OCC,
                     FP_OCC_HALVED, FP_POS, FP_SET_COMMON, FP_SET_CUSTOM, FP_SET_MIXED, FP_SET_RARE, FpError,
                     check, load)

TYPES = {"occ": FP_OCC, "occh": FP_OCC_HALVED, "count": FP_COUNT, "pos": FP_POS, "qgram": native.FP_QGRAM,
         "count_l1": native.FP_COUNT_L1}
METRICS = {"ham": FP_HAM, "lev": FP_LEV}
SETS = {"common": FP_SET_COMMON, "rare": FP_SET_RARE, "mixed": FP_SET_MIXED, "custom": FP_SET_CUSTOM}
MODES = {"tiled": FP_MODE_TILED, "plain": FP_MODE_PLAIN, "fused": FP_MODE_FUSED}

__all__ = ["fp_build", "fp_query", "fp_query_ex", "Index", "Result", "Plan", "Server", "fp_launch_count", "fp_version",
           "fp_probe", "FpError", "TYPES", "METRICS", "SETS", "MODES"]


def _ptr(a):
    """(pointer, keep-alive) for a numpy array or torch tensor (host or device)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return (a.ctypes.data if a.size else None), a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        return (a.data_ptr() if a.numel() else None), a
    raise TypeError(f"expected numpy array or torch tensor, got {type(a)}")


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _strings(chars, offsets):
    if offsets is None and hasattr(chars, "chars") and hasattr(chars, "offsets"):
        chars, offsets = chars.chars, chars.offsets
    n = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
    if isinstance(chars, np.ndarray):
        chars = np.ascontiguousarray(chars, dtype=np.uint8)
        if chars.size == 0:
            chars = np.zeros(16, np.uint8)
    if isinstance(offsets, np.ndarray):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    return chars, offsets, n


class Result:
    """Per-query match lists (CSR) of one fp_query call."""

    def __init__(self, handle: int, n_queries: int):
        self._h = handle
        self.n_queries = n_queries

    def csr(self, copy: bool = True):
        """Host match lists: (row_ptr int64[n+1], idx int32[row_ptr[n]]).

        copy=False returns views of the library's host buffers instead of
        copies; they keep this result alive and stay valid until free()."""
        L = load()
        rp, ix = ctypes.c_void_p(), ctypes.c_void_p()
        check(L.fp_result_csr(self._h, ctypes.byref(rp), ctypes.byref(ix), 0), "fp_result_csr")
        rbuf = (ctypes.c_int64 * (self.n_queries + 1)).from_address(rp.value)
        rbuf._owner = self
        row_ptr = np.frombuffer(rbuf, dtype=np.int64)
        n = int(row_ptr[-1])
        if n:
            ibuf = (ctypes.c_int32 * n).from_address(ix.value)
            ibuf._owner = self
            idx = np.frombuffer(ibuf, dtype=np.int32)
        else:
            idx = np.zeros(0, np.int32)
        return (row_ptr.copy(), idx.copy()) if copy else (row_ptr, idx)

    def device_csr(self):
        """Device pointers (row_ptr, idx) owned by this result."""
        L = load()
        rp, ix = ctypes.c_void_p(), ctypes.c_void_p()
        check(L.fp_result_csr(self._h, ctypes.byref(rp), ctypes.byref(ix), 1), "fp_result_csr")
        return rp.value, ix.value

    def stats(self) -> dict:
        s = native.fp_stats()
        check(load().fp_result_stats(self._h, ctypes.byref(s)), "fp_result_stats")
        return s.as_dict()

    def free(self):
        if self._h:
            load().fp_result_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Index:
    """A dictionary resident on the GPU with one fingerprint per word."""

    def __init__(self, handle: int):
        self._h = handle

    def info(self) -> dict:
        i = native.fp_index_info()
        check(load().fp_index_info_get(self._h, ctypes.byref(i)), "fp_index_info_get")
        d = {n: getattr(i, n) for n, _ in i._fields_ if n != "bucket_count"}
        d["bucket_count"] = np.array(i.bucket_count[:], dtype=np.int64)
        return d

    def symbol_map(self) -> np.ndarray:
        m = np.zeros(256, dtype=np.int8)
        check(load().fp_index_map(self._h, m.ctypes.data), "fp_index_map")
        return m

    def qgrams(self) -> np.ndarray:
        """The q-grams of a q-gram index in field order, uint8[fields, q] (fp_index_qgrams)."""
        L = load()
        buf = np.zeros(96, dtype=np.uint8)
        n, q = ctypes.c_int32(0), ctypes.c_int32(0)
        check(L.fp_index_qgrams(self._h, buf.ctypes.data, ctypes.byref(n), ctypes.byref(q)), "fp_index_qgrams")
        return buf[:n.value * q.value].reshape(n.value, q.value)

    def set_symbol_map(self, m):
        m = np.ascontiguousarray(m, dtype=np.int8)
        assert m.shape == (256,)
        check(load().fp_set_symbol_map(self._h, m.ctypes.data), "fp_set_symbol_map")

    def fingerprint(self, chars, offsets=None, stream=None) -> np.ndarray:
        chars, offsets, n = _strings(chars, offsets)
        out = np.zeros(max(n, 1), dtype=np.uint32)
        cp, k1 = _ptr(chars)
        op, k2 = _ptr(offsets)
        check(load().fp_fingerprint(self._h, cp, op, n, out.ctypes.data, _stream(stream)), "fp_fingerprint")
        return out[:n]

    def query(self, chars, offsets=None, k: int = 1, metric: str = "ham", **kw) -> Result:
        return fp_query_ex(self, chars, offsets, k, metric, **kw)

    def free(self):
        if self._h:
            load().fp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fp_build(chars, offsets=None, fp_type: str = "occ", width: int = 32, symbol_set: str = "common",
             count_bits: int = 2, pos_bits: int = 3, custom_map=None, stream=None, combined: bool = False,
             qgram: int = 0) -> Index:
    """Builds the resident index (fp_build in include/fp.h)."""
    L = load()
    chars, offsets, n = _strings(chars, offsets)
    o = native.fp_build_opts()
    o.set = SETS[symbol_set] if custom_map is None else FP_SET_CUSTOM
    o.count_bits = count_bits
    o.pos_bits = pos_bits
    o.combined = 1 if combined else 0
    o.qgram = qgram
    keep = None
    if custom_map is not None:
        keep = np.ascontiguousarray(custom_map, dtype=np.int8)
        o.custom_map = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    cp, k1 = _ptr(chars)
    op, k2 = _ptr(offsets)
    h = ctypes.c_void_p()
    check(L.fp_build(cp, op, n, TYPES[fp_type], width, ctypes.byref(o), _stream(stream), ctypes.byref(h)),
          "fp_build")
    return Index(h.value)


def fp_query_ex(index: Index, chars, offsets=None, k: int = 1, metric: str = "ham", mode: str = "tiled",
                tile_queries: int = 0, words_per_thread: int = 0, variant: int = 0, stream=None) -> Result:
    """Match lists of a pattern batch (fp_query_ex in include/fp.h)."""
    L = load()
    chars, offsets, n = _strings(chars, offsets)
    o = native.fp_query_opts()
    o.mode = MODES[mode]
    o.tile_queries = tile_queries
    o.words_per_thread = words_per_thread
    o.variant = variant
    cp, k1 = _ptr(chars)
    op, k2 = _ptr(offsets)
    h = ctypes.c_void_p()
    check(L.fp_query_ex(index._h, cp, op, n, k, METRICS[metric], ctypes.byref(o), _stream(stream),
                        ctypes.byref(h)), "fp_query_ex")
    return Result(h.value, n)


def fp_query(index: Index, chars, offsets=None, k: int = 1, metric: str = "ham", stream=None) -> Result:
    return fp_query_ex(index, chars, offsets, k, metric, stream=stream)


def _batches(batches):
    """[(n_queries, k, metric), ...] -> ctypes array of fp_batch."""
    arr = (native.fp_batch * len(batches))()
    for i, (n, k, metric) in enumerate(batches):
        arr[i].n_queries = int(n)
        arr[i].k = int(k)
        arr[i].metric = METRICS[metric] if isinstance(metric, str) else int(metric)
    return arr


def fp_query_batched(index: Index, chars, offsets=None, batches=(), tile_queries: int = 0, variant: int = 0,
                     stream=None) -> Result:
    """Many batches with their own (k, metric) in one pass (fp_query_batched)."""
    L = load()
    chars, offsets, n = _strings(chars, offsets)
    o = native.fp_query_opts()
    o.tile_queries = tile_queries
    o.variant = variant
    b = _batches(batches)
    cp, k1 = _ptr(chars)
    op, k2 = _ptr(offsets)
    h = ctypes.c_void_p()
    check(L.fp_query_batched(index._h, cp, op, n, ctypes.cast(b, ctypes.c_void_p), len(b), ctypes.byref(o),
                             _stream(stream), ctypes.byref(h)), "fp_query_batched")
    return Result(h.value, n)


class Plan:
    """Buffers and a captured CUDA graph for repeated batched queries (fp_plan_*)."""

    def __init__(self, index: Index, max_queries: int, max_chars: int, max_batches: int, tile_queries: int = 0,
                 variant: int = 0, graph: bool = True):
        o = native.fp_query_opts()
        o.mode = FP_MODE_FUSED
        o.flags = 0 if graph else native.FP_OPT_NO_GRAPH
        o.tile_queries = tile_queries
        o.variant = variant
        h = ctypes.c_void_p()
        check(load().fp_plan_create(index._h, max_queries, max_chars, max_batches, ctypes.byref(o), ctypes.byref(h)),
              "fp_plan_create")
        self._h = h.value
        self.index = index

    def run(self, chars, offsets=None, batches=(), stream=None) -> Result:
        chars, offsets, n = _strings(chars, offsets)
        b = _batches(batches)
        cp, k1 = _ptr(chars)
        op, k2 = _ptr(offsets)
        h = ctypes.c_void_p()
        check(load().fp_plan_run(self._h, cp, op, n, ctypes.cast(b, ctypes.c_void_p), len(b), _stream(stream),
                                 ctypes.byref(h)), "fp_plan_run")
        return Result(h.value, n)

    def free(self):
        if self._h:
            load().fp_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over a resident index (fp_server_*).

    submit() copies a request and returns its id at once; wait() blocks (with
    the GIL released) until the request's match lists are ready."""

    def __init__(self, index: Index, lanes: int = 0, max_requests: int = 0, max_queries: int = 0,
                 max_chars: int = 0, memory_budget: int = 0, tile_queries: int = 0, variant: int = 0):
        o = native.fp_server_opts()
        o.lanes, o.max_requests, o.max_queries, o.max_chars = lanes, max_requests, max_queries, max_chars
        o.memory_budget, o.tile_queries, o.variant = memory_budget, tile_queries, variant
        h = ctypes.c_void_p()
        check(load().fp_server_create(index._h, ctypes.byref(o), ctypes.byref(h)), "fp_server_create")
        self._h = h.value
        self.index = index

    def submit(self, chars, offsets=None, k: int = 1, metric: str = "lev") -> int:
        chars, offsets, n = _strings(chars, offsets)
        cp, k1 = _ptr(chars)
        op, k2 = _ptr(offsets)
        rid = ctypes.c_int64()
        check(load().fp_server_submit(self._h, cp, op, n, k, METRICS[metric], ctypes.byref(rid)), "fp_server_submit")
        return rid.value

    def wait(self, request_id: int, timeout_s: float = 60.0) -> Result:
        h = ctypes.c_void_p()
        rc = load().fp_server_wait(self._h, request_id, int(timeout_s * 1e6), ctypes.byref(h))
        check(rc, "fp_server_wait")
        s = native.fp_stats()
        check(load().fp_result_stats(h.value, ctypes.byref(s)), "fp_result_stats")
        return Result(h.value, int(s.n_queries))

    def stats(self) -> dict:
        s = native.fp_server_stats()
        check(load().fp_server_stats_get(self._h, ctypes.byref(s)), "fp_server_stats_get")
        return s.as_dict()

    def replay(self, chars, offsets=None, request_sizes=(), arrival_us=(), k: int = 1, metric: str = "lev",
               timeout_s: float = 600.0):
        """Submits request r at arrival_us[r] after the call starts, waits for all:
        (Result over all patterns in order, latency ms per request)."""
        chars, offsets, n = _strings(chars, offsets)
        sizes = np.ascontiguousarray(request_sizes, dtype=np.int64)
        arr = np.ascontiguousarray(arrival_us, dtype=np.int64)
        lat = np.zeros(len(sizes), np.float64)
        cp, k1 = _ptr(chars)
        op, k2 = _ptr(offsets)
        h = ctypes.c_void_p()
        check(load().fp_server_replay(self._h, cp, op, sizes.ctypes.data, arr.ctypes.data, len(sizes), k,
                                      METRICS[metric], int(timeout_s * 1e6), lat.ctypes.data, ctypes.byref(h)),
              "fp_server_replay")
        return Result(h.value, int(sizes.sum())), lat

    def free(self):
        if self._h:
            load().fp_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fp_launch_count() -> int:
    return int(load().fp_launch_count())


def fp_version() -> str:
    return load().fp_version().decode()


def fp_probe(kind: int, iters: int = 2000, stream=None) -> dict:
    r = native.fp_probe_result()
    check(load().fp_probe(kind, iters, _stream(stream), ctypes.byref(r)), "fp_probe")
    return r.as_dict()


def fp_autotune(index: Index, chars, offsets=None, k: int = 1, metric: str = "ham", mode: str = "tiled",
                reps: int = 2, stream=None):
    """Times every tile shape on a pattern sample (fp_autotune); returns (best, all)."""
    L = load()
    chars, offsets, n = _strings(chars, offsets)
    best = native.fp_tune_result()
    allr = (native.fp_tune_result * 32)()
    cnt = ctypes.c_int32(0)
    cp, k1 = _ptr(chars)
    op, k2 = _ptr(offsets)
    check(L.fp_autotune(index._h, cp, op, n, k, METRICS[metric], MODES[mode], reps, _stream(stream),
                        ctypes.byref(best), ctypes.cast(allr, ctypes.c_void_p), 32, ctypes.byref(cnt)), "fp_autotune")
    return best.as_dict(), [allr[i].as_dict() for i in range(cnt.value)]


def fp_sample_pairs(index: Index, chars, offsets=None, k: int = 1, metric: str = "lev", n_samples: int = 100000,
                    seed: int = 1711, stream=None) -> dict:
    """Method-generated (pattern, word, passed, match, symbol masks) samples (fp_sample_pairs)."""
    L = load()
    chars, offsets, n = _strings(chars, offsets)
    out = {"q": np.zeros(n_samples, np.int32), "w": np.zeros(n_samples, np.int32),
           "passed": np.zeros(n_samples, np.uint8), "match": np.zeros(n_samples, np.uint8),
           "masks": np.zeros((n_samples, 4), np.uint64)}
    cp, k1 = _ptr(chars)
    op, k2 = _ptr(offsets)
    check(L.fp_sample_pairs(index._h, cp, op, n, k, METRICS[metric], n_samples, seed, _stream(stream),
                            out["q"].ctypes.data, out["w"].ctypes.data, out["passed"].ctypes.data,
                            out["match"].ctypes.data, out["masks"].ctypes.data), "fp_sample_pairs")
    return out


def fp_mlp_param_count() -> int:
    return int(load().fp_mlp_param_count())


def fp_mlp_loss_grad(params, fields: int, tau: float, beta: float, k: int, masks, match, stream=None):
    """One GPU forward + backward: (summed loss, non-matching samples, mean gradient)."""
    L = load()
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(masks, dtype=np.uint64)
    mt = np.ascontiguousarray(match, dtype=np.uint8)
    g = np.zeros(fp_mlp_param_count(), np.float32)
    loss = ctypes.c_double(0.0)
    used = ctypes.c_int64(0)
    check(L.fp_mlp_loss_grad(p.ctypes.data, fields, tau, beta, k, m.ctypes.data, mt.ctypes.data, len(mt),
                             _stream(stream), ctypes.byref(loss), ctypes.byref(used), g.ctypes.data),
          "fp_mlp_loss_grad")
    return loss.value, used.value, g


def fp_learn_map(fields: int, masks, match, k: int = 1, epochs: int = 0, batch: int = 0, lr: float = 0.0,
                 tau0: float = 0.0, tau1: float = 0.0, beta: float = 0.0, seed: int = 0, stream=None,
                 init_params=None):
    """Trains the map on the GPU: (map int8[256], params float32, loss per epoch)."""
    L = load()
    o = native.fp_learn_opts()
    o.epochs, o.batch, o.lr, o.tau0, o.tau1, o.beta, o.seed = epochs, batch, lr, tau0, tau1, beta, seed
    init = None
    if init_params is not None:
        init = np.ascontiguousarray(init_params, dtype=np.float32)
        assert init.size == fp_mlp_param_count()
        o.init_params = init.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    m = np.ascontiguousarray(masks, dtype=np.uint64)
    mt = np.ascontiguousarray(match, dtype=np.uint8)
    mp = np.zeros(256, np.int8)
    params = np.zeros(fp_mlp_param_count(), np.float32)
    curve = np.zeros(max(epochs, 12) if epochs else 12, np.float32)
    check(L.fp_learn_map(fields, m.ctypes.data, mt.ctypes.data, len(mt), k, ctypes.byref(o), _stream(stream),
                         params.ctypes.data, mp.ctypes.data, curve.ctypes.data), "fp_learn_map")
    return mp, params, curve[: (epochs or 12)]
