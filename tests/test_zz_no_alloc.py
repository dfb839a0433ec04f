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

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


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


def noalloc_query(env, ix, Q, k, metric, capacity):
    fp, native, L, torch = env
    chars = torch.from_numpy(Q.chars if Q.chars.size else np.zeros(16, np.uint8)).cuda()
    offsets = torch.from_numpy(Q.offsets).cuda()
    row_ptr = torch.full((len(Q) + 1,), -7, dtype=torch.int64, device="cuda")
    idx = torch.full((max(capacity, 1),), -7, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    rc = L.fp_query_noalloc(ix._h, chars.data_ptr(), offsets.data_ptr(), len(Q), k, fp.METRICS[metric],
                            row_ptr.data_ptr(), idx.data_ptr(), capacity, ctypes.byref(n), None)
    torch.cuda.synchronize()
    return rc, row_ptr.cpu().numpy(), idx.cpu().numpy()[: max(n.value, 0)], n.value


@pytest.mark.parametrize("fp_type,width", [("count", 32), ("occ", 16)])
def test_noalloc_matches_fp_query_twice(env, fp_type, width):
    fp, native, L, torch = env
    w = datagen.english1m(30000, 3000)
    ix = fp.fp_build(w.dictionary, fp_type=fp_type, width=width)
    for metric in ("ham", "lev"):
        Q = w.queries[metric]
        ref_rp, ref_idx = fp.fp_query(ix, Q, k=1, metric=metric).csr()
        for call in range(2):
            rc, rp, idx, n = noalloc_query(env, ix, Q, 1, metric, 200000)
            assert rc == native.FP_OK, L.fp_last_error()
            assert n == len(ref_idx)
            assert np.array_equal(rp, ref_rp), (metric, call)
            assert np.array_equal(idx, ref_idx), (metric, call)


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
