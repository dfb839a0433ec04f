"""Learned symbol-to-bit map on the GPU: gradients against the fp64 reference,
the pair sampler against the oracle, and the rejection gain at exact results."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import learned

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


def sample_set(seed, n, alphabet=95):
    law = datagen.StringLaw(np.arange(0x20, 0x20 + alphabet, dtype=np.uint8), np.ones(alphabet),
                            datagen.LengthLaw("uniform", 1, 30))
    S = law.draw(seed, "s", 2 * n).to_list()
    M = learned.masks_of(S)
    masks = np.concatenate([M[0::2], M[1::2]], axis=1)
    match = (datagen.uniform(datagen.stream_key(seed, "m"), n) < 0.15).astype(np.uint8)
    return masks, match


@pytest.mark.parametrize("fields,tau,k", [(32, 0.8, 1), (16, 0.5, 2), (7, 1.3, 0)])
def test_gpu_gradients_match_fp64(fp, fields, tau, k):
    p = (datagen.uniform(datagen.stream_key(fields, "p"), learned.NPARAM) * 2 - 1) * 0.6
    masks, match = sample_set(11 + fields, 400)
    beta = 2.0
    l_gpu, used_gpu, g_gpu = fp.fp_mlp_loss_grad(p.astype(np.float32), fields, tau, beta, k, masks, match)
    l_cpu, used_cpu, g_cpu = learned.loss_and_grad(p.astype(np.float32).astype(np.float64), fields, tau, beta, k,
                                                   masks, match)
    assert used_gpu == used_cpu == int((match == 0).sum())
    assert abs(l_gpu - l_cpu) <= 1e-5 * abs(l_cpu)
    err = np.linalg.norm(g_gpu - g_cpu) / np.linalg.norm(g_cpu)
    assert err <= 1e-4, err


def test_gpu_adam_steps_match_fp64(fp):
    """Two epochs of one full batch each are two Adam steps (beta1 0.9, beta2
    0.999, eps 1e-8, bias-corrected; tau0 in the first epoch, tau1 in the
    second).  From the same starting parameters, the library's result must
    equal the same two steps taken in fp64 on the fp64 reference gradients.
    Adam divides each update by the gradient's magnitude, so a component is
    compared tightly only where both steps' gradients are well above the
    FP32 summation noise (relative 1e-3 of the largest); the rest may differ by
    the few step sizes Adam's normalisation allows, and rows of fields past
    `fields` (zero gradient) must not move at all."""
    fields, k, beta, lr, tau0, tau1 = 24, 1, 2.0, 3e-3, 1.0, 0.5
    p0 = ((datagen.uniform(datagen.stream_key(5, "adam/p"), learned.NPARAM) * 2 - 1) * 0.4).astype(np.float32)
    masks, match = sample_set(31, 600)
    _, p_gpu, _ = fp.fp_learn_map(fields, masks, match, k=k, epochs=2, batch=600, lr=lr, tau0=tau0, tau1=tau1,
                                  beta=beta, init_params=p0)
    p = p0.astype(np.float64)
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    firm = np.ones(p.size, dtype=bool)
    for step, tau in ((1, tau0), (2, tau1)):
        _, _, g = learned.loss_and_grad(p, fields, tau, beta, k, masks, match)
        firm &= np.abs(g) > 1e-3 * np.abs(g).max()
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        p = p - lr * (m1 / (1 - 0.9 ** step)) / (np.sqrt(m2 / (1 - 0.999 ** step)) + 1e-8)
    d_gpu, d_ref = p_gpu.astype(np.float64) - p0, p - p0
    assert firm.mean() > 0.2, firm.mean()
    assert np.abs(d_gpu - d_ref)[firm].max() <= 1e-3 * lr
    assert np.abs(d_gpu - d_ref).max() <= 4 * lr
    W2, b2 = learned.unpack(p_gpu.astype(np.float64))[2:4]
    W2_0, b2_0 = learned.unpack(p0.astype(np.float64))[2:4]
    assert np.array_equal(W2[fields:], W2_0[fields:]) and np.array_equal(b2[fields:], b2_0[fields:])
    assert np.abs(d_gpu).max() > 0.5 * lr  # the parameters did move


@pytest.fixture(scope="module")
def url_small():
    return datagen.url2m(200000, 6000)


def test_sampler_agrees_with_oracle(fp, url_small):
    w = url_small
    ix = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    m = ix.symbol_map()
    Q = w.queries["lev"]
    s = fp.fp_sample_pairs(ix, Q, k=1, metric="lev", n_samples=3000, seed=5)
    assert (s["q"] >= 0).all() and (s["w"] >= 0).all()
    ql, dl = Q.to_list(), w.dictionary.to_list()
    qfp = oracle.fingerprints(Q, m, "occ", 32)
    for i in range(3000):
        a, b = ql[s["q"][i]], dl[s["w"][i]]
        assert abs(len(a) - len(b)) <= 1
        f = oracle.fd(int(qfp[s["q"][i]]), oracle.fingerprint(b, m, "occ", 32), "occ", 32)
        assert s["passed"][i] == (f <= 2)
        assert s["match"][i] == (oracle.lev(a, b) <= 1)
        assert tuple(s["masks"][i]) == tuple(learned.masks_of([a])[0]) + tuple(learned.masks_of([b])[0])


def test_learned_map_rejects_more_at_identical_results(fp, url_small):
    w = url_small
    freq = fp.fp_build(w.dictionary, fp_type="occ", width=32)
    s = fp.fp_sample_pairs(freq, w.queries["lev"], k=1, metric="lev", n_samples=400000, seed=7)
    mp, params, curve = fp.fp_learn_map(32, s["masks"], s["match"], k=1, epochs=12, seed=3)
    assert curve[-1] < curve[0]
    assert (mp[0x20:0x7F] >= 0).all() and (mp[:0x20] == -1).all()
    lrn = fp.fp_build(w.dictionary, fp_type="occ", width=32, custom_map=mp)
    # held-out patterns: other mutations of the same dictionary, other random strings
    held = datagen.make_queries(w.dictionary, w.law, w.seed, "held/lev", 2000, 0.5, "lev")
    r_f = fp.fp_query(freq, held, k=1, metric="lev")
    r_l = fp.fp_query(lrn, held, k=1, metric="lev")
    rp_f, idx_f = r_f.csr()
    rp_l, idx_l = r_l.csr()
    assert np.array_equal(rp_f, rp_l) and np.array_equal(idx_f, idx_l)
    sf, sl = r_f.stats(), r_l.stats()
    assert sf["pairs"] == sl["pairs"]
    assert sf["matches"] >= 1000
    # the learned map lets 25-35 % fewer pairs through than the frequency map of
    # Sec. 3 on these strings (0.65 - 0.74 of its survivors over six training
    # samples); 0.8 leaves room for the spread between samples
    assert sl["survivors"] < 0.8 * sf["survivors"], (sl["survivors"], sf["survivors"])
    sub = held.subset(np.arange(0, 2000, 40))
    rp0, idx0 = oracle.match(w.dictionary, sub, 1, "lev")
    rows = [idx_l[rp_l[i]:rp_l[i + 1]] for i in range(0, 2000, 40)]
    assert all(np.array_equal(r, idx0[rp0[j]:rp0[j + 1]]) for j, r in enumerate(rows))
