"""fp64 reference of the learned symbol-to-bit map's model, loss and gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper has no learned
map: Sec. 3.2 takes "a mapping c -> q" and Sec. 3 fills it with the most
frequent symbols.  This module states, plainly and in double precision, the
model the CUDA library trains, so that the library's FP32 forward and
backward kernels can be checked against it:

  printable symbol c (byte 0x20 + c, c < 95), one-hot input
  h_c  = relu(W1[:, c] + b1)                 W1: 64 x 95, b1: 64
  z_c  = W2[:F] h_c + b2[:F]                 W2: 32 x 64, b2: 32 (first F rows used)
  A_c  = softmax(z_c / tau)                  symbol c lands on field b with probability A_c,b
  F_D  = expected Hamming weight of the XOR of the two occurrence fingerprints
         (Sec. 3.3) when every symbol lands independently.  With I = P & W,
         P' = P - W, W' = W - P, field b differs iff no symbol of I lands on it
         and exactly one of P', W' has a symbol landing on it:
         F_D = sum_b prod_{c in I} (1 - A_c,b) (p_b + q_b - 2 p_b q_b),
         p_b = 1 - prod_{c in P'} (1 - A_c,b), q_b the same over W'
  loss = mean over non-matching pairs of softplus(beta (2k + 1 - F_D)) / beta

Pins (tests/test_oracle_learned.py): with one-hot assignments the soft F_D is
the integer F_D of the oracle's occurrence fingerprints (Sec. 3.3), and the
analytic gradient agrees with central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

NSYM, HID, MAXF = 95, 64, 32
P_W1, P_B1 = 0, HID * NSYM
P_W2 = P_B1 + HID
P_B2 = P_W2 + MAXF * HID
NPARAM = P_B2 + MAXF


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    W1 = p[P_W1:P_B1].reshape(HID, NSYM)
    b1 = p[P_B1:P_W2]
    W2 = p[P_W2:P_B2].reshape(MAXF, HID)
    b2 = p[P_B2:NPARAM]
    return W1, b1, W2, b2


def forward(params, fields: int, tau: float):
    """(H [95, 64], Z [95, F], A [95, F])."""
    W1, b1, W2, b2 = unpack(params)
    H = np.maximum(W1.T + b1[None, :], 0.0)  # row c = relu(W1[:, c] + b1)
    Z = H @ W2[:fields].T + b2[:fields][None, :]
    E = np.exp(Z / tau - (Z / tau).max(axis=1, keepdims=True))
    A = E / E.sum(axis=1, keepdims=True)
    return H, Z, A


def symbols(mask2) -> list:
    """Printable-symbol indices c set in a 2-word mask."""
    lo, hi = int(mask2[0]), int(mask2[1])
    return [c for c in range(64) if (lo >> c) & 1] + [64 + c for c in range(31) if (hi >> c) & 1]


def none_lands(A, syms):
    """prod_{c in syms} (1 - A_c): per field, the probability that no symbol of syms lands on it."""
    s = np.ones(A.shape[1])
    for c in syms:
        s = s * (1.0 - A[c])
    return s


def split(syms_p, syms_w):
    """(shared, pattern only, word only) symbol lists."""
    sp, sw = set(syms_p), set(syms_w)
    return sorted(sp & sw), sorted(sp - sw), sorted(sw - sp)


def soft_fd_fields(A, syms_p, syms_w):
    I, Pd, Wd = split(syms_p, syms_w)
    nI = none_lands(A, I)
    p, q = 1.0 - none_lands(A, Pd), 1.0 - none_lands(A, Wd)
    return nI * (p + q - 2.0 * p * q)


def soft_fd(A, syms_p, syms_w) -> float:
    return float(soft_fd_fields(A, syms_p, syms_w).sum())


def loss_and_grad(params, fields: int, tau: float, beta: float, k: int, masks, match):
    """(summed loss, number of non-matching samples, mean gradient over them)."""
    W1, b1, W2, b2 = unpack(params)
    H, Z, A = forward(params, fields, tau)
    T = 2.0 * k + 1.0
    dA = np.zeros_like(A)
    total, used = 0.0, 0
    for i in range(len(match)):
        if match[i]:
            continue
        I, Pd, Wd = split(symbols(masks[i][0:2]), symbols(masks[i][2:4]))
        nI = none_lands(A, I)
        p, q = 1.0 - none_lands(A, Pd), 1.0 - none_lands(A, Wd)
        F = float((nI * (p + q - 2.0 * p * q)).sum())
        t = beta * (T - F)
        total += np.logaddexp(0.0, t) / beta  # softplus(t) / beta
        used += 1
        dLdF = -1.0 / (1.0 + np.exp(-t))
        # each derivative is a product over the other symbols of the same group
        for c in I:
            dA[c] += dLdF * -none_lands(A, [x for x in I if x != c]) * (p + q - 2.0 * p * q)
        for c in Pd:
            dA[c] += dLdF * nI * (1.0 - 2.0 * q) * none_lands(A, [x for x in Pd if x != c])
        for c in Wd:
            dA[c] += dLdF * nI * (1.0 - 2.0 * p) * none_lands(A, [x for x in Wd if x != c])
    grad = np.zeros(NPARAM)
    if used == 0:
        return total, used, grad
    dA /= used
    # softmax: dz_j = A_j (dA_j - sum_i A_i dA_i) / tau
    dZ = A * (dA - (A * dA).sum(axis=1, keepdims=True)) / tau
    gW2 = np.zeros((MAXF, HID))
    gW2[:fields] = dZ.T @ H
    gb2 = np.zeros(MAXF)
    gb2[:fields] = dZ.sum(axis=0)
    dH = dZ @ W2[:fields]
    dH = dH * (H > 0)
    gW1 = dH.T  # [HID, NSYM]: the input is one-hot, so column c gets row c of dH
    gb1 = dH.sum(axis=0)
    grad[P_W1:P_B1] = gW1.reshape(-1)
    grad[P_B1:P_W2] = gb1
    grad[P_W2:P_B2] = gW2.reshape(-1)
    grad[P_B2:NPARAM] = gb2
    return total, used, grad


def loss_only(params, fields, tau, beta, k, masks, match) -> float:
    _, _, A = forward(params, fields, tau)
    T = 2.0 * k + 1.0
    total, used = 0.0, 0
    for i in range(len(match)):
        if match[i]:
            continue
        F = soft_fd(A, symbols(masks[i][0:2]), symbols(masks[i][2:4]))
        total += np.logaddexp(0.0, beta * (T - F)) / beta
        used += 1
    return total / max(used, 1)


def masks_of(strings) -> np.ndarray:
    """[n, 4] uint64 symbol masks (pattern layout of one string in words 0-1)."""
    out = np.zeros((len(strings), 2), dtype=np.uint64)
    for i, s in enumerate(strings):
        lo = hi = 0
        for b in s:
            c = b - 0x20
            if 0 <= c < 64:
                lo |= 1 << c
            elif 64 <= c < NSYM:
                hi |= 1 << (c - 64)
        out[i] = (lo, hi)
    return out
