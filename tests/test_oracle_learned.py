"""Pins of the fp64 learned-map reference (no GPU)."""
import numpy as np

import datagen
import oracle
from oracle import learned


def rand_params(seed, scale=0.6):
    r = datagen.uniform(datagen.stream_key(seed, "prm"), learned.NPARAM) * 2 - 1
    return r * scale


def printable_strings(seed, n, lo=1, hi=12, alphabet=48):
    law = datagen.StringLaw(np.arange(0x20, 0x20 + alphabet, dtype=np.uint8), np.ones(alphabet),
                            datagen.LengthLaw("uniform", lo, hi))
    return law.draw(seed, "s", n).to_list()


def test_onehot_soft_fd_is_integer_fd():
    """With one-hot assignments the soft F_D is the F_D of occurrence fingerprints (Sec. 3.3)."""
    fields = 32
    r = datagen.randint(datagen.stream_key(3, "map"), learned.NSYM, 0, fields - 1)
    A = np.zeros((learned.NSYM, fields))
    A[np.arange(learned.NSYM), r] = 1.0
    bmap = np.full(256, -1, np.int8)
    bmap[0x20:0x20 + learned.NSYM] = r
    S = printable_strings(4, 200, alphabet=95)
    fps = [oracle.fingerprint(s, bmap, "occ", 32) for s in S]
    M = learned.masks_of(S)
    for i in range(0, 200, 2):
        f = learned.soft_fd(A, learned.symbols(M[i]), learned.symbols(M[i + 1]))
        assert f == oracle.fd(fps[i], fps[i + 1], "occ", 32)


def test_forward_closed_forms():
    p = np.zeros(learned.NPARAM)
    _, _, A = learned.forward(p, 20, 0.7)
    assert np.allclose(A, 1.0 / 20)  # zero logits: uniform assignment
    p[learned.P_B2 + 5] = 40.0
    _, _, A = learned.forward(p, 20, 1.0)
    assert np.all(A.argmax(axis=1) == 5) and A[:, 5].min() > 1 - 1e-12
    p = rand_params(2)
    H, Z, A = learned.forward(p, 32, 0.5)
    assert np.all(H >= 0) and np.allclose(A.sum(axis=1), 1.0)


def sample_set(seed, n):
    S = printable_strings(seed, 2 * n)
    M = learned.masks_of(S)
    masks = np.concatenate([M[0::2], M[1::2]], axis=1)
    match = (datagen.uniform(datagen.stream_key(seed, "m"), n) < 0.2).astype(np.uint8)
    return masks, match


def test_gradient_matches_finite_differences():
    p = rand_params(7)
    masks, match = sample_set(8, 24)
    fields, tau, beta, k = 32, 0.8, 2.0, 1
    _, used, g = learned.loss_and_grad(p, fields, tau, beta, k, masks, match)
    assert used == int((match == 0).sum())
    idx = datagen.randint(datagen.stream_key(9, "pick"), 60, 0, learned.NPARAM - 1)
    # W2/b2 rows past `fields` do not reach the loss: their gradient is exactly zero
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp = learned.loss_only(q, fields, tau, beta, k, masks, match)
        q[i] -= 2 * h
        lm = learned.loss_only(q, fields, tau, beta, k, masks, match)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    F = 12
    _, _, g12 = learned.loss_and_grad(p, F, tau, beta, k, masks, match)
    assert np.all(g12[learned.P_W2 + F * learned.HID:learned.P_B2] == 0)


def test_soft_fd_is_expected_fd_by_enumeration():
    """Soft F_D is the expectation of the occurrence-fingerprint F_D (Sec. 3.3)
    over independent random symbol-to-field assignments: enumerate every
    assignment of a few symbols to a few fields and weight it by its probability."""
    import itertools
    fields = 3
    rng = datagen.uniform(datagen.stream_key(21, "A"), learned.NSYM * fields).reshape(learned.NSYM, fields) + 0.05
    A = rng / rng.sum(axis=1, keepdims=True)
    cases = [([0, 1, 2], [1, 2, 3]), ([4], [5]), ([6, 7], [6, 7]), ([8, 9, 10], []), ([11, 12], [13, 12, 14])]
    for P, W in cases:
        syms = sorted(set(P) | set(W))
        exp = 0.0
        for assign in itertools.product(range(fields), repeat=len(syms)):
            pr = 1.0
            for c, b in zip(syms, assign):
                pr *= A[c, b]
            at = dict(zip(syms, assign))
            fp_p = 0
            for c in set(P):
                fp_p |= 1 << at[c]
            fp_w = 0
            for c in set(W):
                fp_w |= 1 << at[c]
            exp += pr * bin(fp_p ^ fp_w).count("1")
        assert abs(learned.soft_fd(A, P, W) - exp) <= 1e-12, (P, W)
