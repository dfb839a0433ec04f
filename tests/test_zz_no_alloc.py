"""fp_query_noalloc: the query entry point that allocates no device memory.

Some callers cannot allocate device memory once they are serving (their
device memory is carved up in advance by their own allocator, or an
allocation's possible device-wide synchronisation is not acceptable in their
loop).  For them the library offers fp_query_noalloc, which works inside a
fixed scratch array compiled into the library.  This test calls it through
the C ABI on device inputs and checks that its match lists equal those of
fp_query on the same inputs, exactly (integer results), on two calls in a
row -- the scratch keeps the previous call's contents, so the second call
also checks that everything that must start at zero is cleared.

It also checks the point of the entry point: across warm calls (after the
first call on the device has looked up the scratch array and loaded the
kernels) neither the device's free memory nor the device's stream-ordered
pool changes -- no reserved bytes, no used bytes, and no allocation between
the calls that was freed again (the pool's high-water mark is reset before
them and read after them).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


def patterns(w, metric, k):
    """The workload's patterns; at k = 2 the first 300 (the whole batch would let
    more than FP_NOALLOC_MAX_CANDIDATES pairs through the filter)."""
    Q = w.queries[metric]
    return Q if k < 2 else Q.subset(np.arange(300))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1711_08475_gb300 import build
    build.build()
    import paper_1711_08475_gb300 as fp
    from paper_1711_08475_gb300 import native
    return fp, native, native.load(), torch


class DevBuffers:
    """Device inputs and outputs of one call, allocated before any memory is measured."""

    def __init__(self, env, Q, capacity):
        fp, native, L, torch = env
        self.n = len(Q)
        self.chars = torch.from_numpy(Q.chars if Q.chars.size else np.zeros(16, np.uint8)).cuda()
        self.offsets = torch.from_numpy(Q.offsets).cuda()
        self.row_ptr = torch.empty((len(Q) + 1,), dtype=torch.int64, device="cuda")
        self.idx = torch.empty((max(capacity, 1),), dtype=torch.int32, device="cuda")
        self.capacity = capacity
        torch.cuda.synchronize()


def call(env, ix, B, k, metric):
    fp, native, L, torch = env
    B.row_ptr.fill_(-7)
    B.idx.fill_(-7)
    torch.cuda.synchronize()
    n = ctypes.c_int64(-1)
    rc = L.fp_query_noalloc(ix._h, B.chars.data_ptr(), B.offsets.data_ptr(), B.n, k, fp.METRICS[metric],
                            B.row_ptr.data_ptr(), B.idx.data_ptr(), B.capacity, ctypes.byref(n), None)
    torch.cuda.synchronize()
    return rc, n.value


def result(B, n):
    return B.row_ptr.cpu().numpy(), B.idx.cpu().numpy()[: max(n, 0)]


def noalloc_query(env, ix, Q, k, metric, capacity):
    B = DevBuffers(env, Q, capacity)
    rc, n = call(env, ix, B, k, metric)
    rp, idx = result(B, n)
    return rc, rp, idx, n


class DevicePool:
    """Reads the current device's default stream-ordered pool (the one the
    library's other entry points allocate from) through the CUDA driver API."""

    RESERVED_CURRENT, USED_CURRENT, USED_HIGH = 5, 7, 8  # CUmemPool_attribute

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(-1)
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(z)) == 0

    def snapshot(self):
        return {"reserved": self.get(self.RESERVED_CURRENT), "used": self.get(self.USED_CURRENT)}


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("fp_type,width", [("count", 32), ("occ", 16)])
def test_noalloc_matches_fp_query_twice(env, fp_type, width, k):
    fp, native, L, torch = env
    w = datagen.english1m(30000, 3000)
    ix = fp.fp_build(w.dictionary, fp_type=fp_type, width=width)
    for metric in ("ham", "lev"):
        Q = patterns(w, metric, k)
        ref_rp, ref_idx = fp.fp_query(ix, Q, k=k, metric=metric).csr()
        B = DevBuffers(env, Q, max(200000, len(ref_idx)))
        for c in range(2):
            rc, n = call(env, ix, B, k, metric)
            assert rc == native.FP_OK, L.fp_last_error()
            rp, idx = result(B, n)
            assert n == len(ref_idx)
            assert np.array_equal(rp, ref_rp), (metric, k, c)
            assert np.array_equal(idx, ref_idx), (metric, k, c)


def test_noalloc_allocates_nothing(env):
    """Warm calls leave the device's free memory and its stream-ordered pool as
    they found them; the results stay equal to fp_query's."""
    fp, native, L, torch = env
    w = datagen.english1m(30000, 3000)
    ix = fp.fp_build(w.dictionary, fp_type="count", width=32)
    refs, bufs = {}, {}
    for metric in ("ham", "lev"):
        for k in (0, 1, 2):
            Q = patterns(w, metric, k)
            refs[metric, k] = fp.fp_query(ix, Q, k=k, metric=metric).csr()
            bufs[metric, k] = DevBuffers(env, Q, max(200000, len(refs[metric, k][1])))
    for key, B in bufs.items():  # first calls: symbol look-up and kernel loading happen here
        assert call(env, ix, B, key[1], key[0])[0] == native.FP_OK, L.fp_last_error()
    torch.cuda.synchronize()
    pool = DevicePool()
    before_free, _ = torch.cuda.mem_get_info()
    before = pool.snapshot()
    pool.reset_high()
    for _ in range(2):
        for key, B in bufs.items():
            rc, n = call(env, ix, B, key[1], key[0])
            assert rc == native.FP_OK, L.fp_last_error()
            rp, idx = result(B, n)
            assert np.array_equal(rp, refs[key][0]) and np.array_equal(idx, refs[key][1]), key
    torch.cuda.synchronize()
    after_free, _ = torch.cuda.mem_get_info()
    after = pool.snapshot()
    assert after == before, (before, after)
    assert pool.get(pool.USED_HIGH) <= before["used"], "an allocation was made and freed between the calls"
    assert after_free == before_free, (before_free, after_free)


def test_noalloc_limits(env):
    fp, native, L, torch = env
    w = datagen.english1m(5000, 10)
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    big = datagen.english_law(24).draw(5, "big", 4097)
    rc, _, _, _ = noalloc_query(env, ix, big, 1, "ham", 1000)
    assert rc == native.FP_E_INVAL
    # too little room for the match list: an overflow error with the needed count
    Q = datagen.Strings.concat([w.dictionary.subset(np.arange(200))] * 3)
    ref_rp, ref_idx = fp.fp_query(ix, Q, k=1, metric="lev").csr()
    assert len(ref_idx) > 10
    rc, _, _, n = noalloc_query(env, ix, Q, 1, "lev", 10)
    assert rc == native.FP_E_OVERFLOW and n == len(ref_idx)
    # and the same call with room succeeds afterwards
    rc, rp, idx, n = noalloc_query(env, ix, Q, 1, "lev", len(ref_idx))
    assert rc == native.FP_OK and np.array_equal(rp, ref_rp) and np.array_equal(idx, ref_idx)
