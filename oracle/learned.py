"""fp64 reference of the learned symbol-to-bit map's model, loss and gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper has no learned
map: Sec. 3.2 takes "a mapping c -> q" and Sec. 3 fills it with the most
frequent symbols.  This module states, plainly and in double precision, the
model the CUDA library trains, so that the library's FP32 forward and
backward kernels can be checked against it:

  printable symbol c (byte 0x20 + c, c < 95), one-hot input
  h_c  = relu(W1[:, c] + b1)                 W1: 64 x 95, b1: 64
  z_c  = W2[:F] h_c + b2[:F]                 W2: 32 x 64, b2: 32 (first F rows used)
  A_c  = softmax(z_c / tau)
  s(S) = 1 - prod_{c in S} (1 - A_c)         soft occurrence fingerprint of symbol set S
  F_D  = sum_b s_b(P) + s_b(W) - 2 s_b(P) s_b(W)
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


def soft_fp(A, syms):
    s = np.ones(A.shape[1])
    for c in syms:
        s = s * (1.0 - A[c])
    return 1.0 - s


def soft_fd(A, syms_p, syms_w) -> float:
    sp, sw = soft_fp(A, syms_p), soft_fp(A, syms_w)
    return float((sp + sw - 2.0 * sp * sw).sum())


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
        P, W = symbols(masks[i][0:2]), symbols(masks[i][2:4])
        sp, sw = soft_fp(A, P), soft_fp(A, W)
        F = float((sp + sw - 2.0 * sp * sw).sum())
        t = beta * (T - F)
        total += np.logaddexp(0.0, t) / beta  # softplus(t) / beta
        used += 1
        dLdF = -1.0 / (1.0 + np.exp(-t))
        gP = dLdF * (1.0 - 2.0 * sw)  # dLoss / ds(P)
        gW = dLdF * (1.0 - 2.0 * sp)
        # ds_b(S) / dA_c,b = prod over the other symbols of S of (1 - A_c',b)
        for c in P:
            others = np.ones(fields)
            for c2 in P:
                if c2 != c:
                    others = others * (1.0 - A[c2])
            dA[c] += gP * others
        for c in W:
            others = np.ones(fields)
            for c2 in W:
                if c2 != c:
                    others = others * (1.0 - A[c2])
            dA[c] += gW * others
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
