"""FP64 numpy oracle of the learned initial-h predictor -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; it shares no code with the CUDA package.

The paper (Theuns et al. 2015) has no learned component: its h iteration (Sec. 2,
Newton on N_w(h) = N_ngb) starts from whatever h the particle had.  The library
may start it from a small MLP's guess instead; this module writes that model out
by definition, so the CUDA kernels can be compared with it:

* :func:`features` -- the six per-particle inputs, from the state after a cell
  build (uniform grid: the particle's cell; the arrays are in cell order).
* :func:`forward` -- 6 -> 64 -> 64 -> 1 MLP with SiLU on normalised features,
  output log(h0 / h_prev) after de-normalisation and clamping.  ``bf16=True``
  rounds what the inference path rounds to bfloat16 (weights, normalised
  inputs, first hidden layer), in the same precision it is computed in (FP32).
* :func:`loss_and_grad` -- mean squared error of the normalised target and its
  gradient by reverse-mode differentiation written out by hand.
* :func:`adam_steps` -- Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on
  sequential batches of 16384 samples.

Parameter vector layout (as the library's FP32 training state): W1[64][6],
b1[64], W2[64][64] (row = output unit), b2[64], W3[64], b3.  Normalisation:
feature means[6], feature sds[6], target mean, target sd.

Pins (``tests/test_oracle_hpredict.py``): finite-difference gradients, closed
forms of degenerate networks, the first Adam step, SiLU identities, and the
features of a uniform lattice.
"""
from __future__ import annotations

import numpy as np

NF, NH = 6, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + NH * NF
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAM = OFF_B3 + 1
BATCH = 16384
LOG_LO, LOG_HI = float(np.log(np.float32(0.5))), float(np.log(np.float32(1.2)))


def unpack(P):
    P = np.asarray(P, np.float64)
    return (P[OFF_W1:OFF_B1].reshape(NH, NF), P[OFF_B1:OFF_W2], P[OFF_W2:OFF_B2].reshape(NH, NH),
            P[OFF_B2:OFF_W3], P[OFF_W3:OFF_B3], P[OFF_B3])


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returns float32."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def bf16_bits(x):
    """bfloat16 bit patterns (uint16) of float32 values, rounded to nearest even."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, np.uint32) << 16).view(np.float32)


def silu(x):
    return x / (1.0 + np.exp(-x))


def silu_grad(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def normalise(X, norm):
    """(f - mean) / sd in FP32, as the inference path computes it (times 1/sd)."""
    X = np.asarray(X, np.float32)
    m = np.asarray(norm[:NF], np.float32)
    inv = (np.float32(1.0) / np.asarray(norm[NF:2 * NF], np.float32)).astype(np.float32)
    return ((X - m) * inv).astype(np.float32)


def forward(P, norm, X, bf16=False, clamp=True):
    """log(h0 / h_prev) for the feature rows X (n x 6)."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    Z = normalise(X, norm).astype(np.float64)
    if bf16:
        Z = bf16_round(Z).astype(np.float64)
        W1 = bf16_round(W1).astype(np.float64)
        W2 = bf16_round(W2).astype(np.float64)
        W3 = bf16_round(W3).astype(np.float64)
    H1 = silu(Z @ W1.T + b1)
    if bf16:
        H1 = bf16_round(H1).astype(np.float64)
    H2 = silu(H1 @ W2.T + b2)
    y = H2 @ W3 + b3
    out = y * float(norm[2 * NF + 1]) + float(norm[2 * NF])
    return np.clip(out, LOG_LO, LOG_HI) if clamp else out


def loss_and_grad(P, norm, X, Y):
    """Mean squared error of the normalised target over the rows, and dL/dP."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    Z = (np.asarray(X, np.float64) - np.asarray(norm[:NF], np.float64)) / np.asarray(norm[NF:2 * NF], np.float64)
    T = (np.asarray(Y, np.float64) - float(norm[2 * NF])) / float(norm[2 * NF + 1])
    A1 = Z @ W1.T + b1
    H1 = silu(A1)
    A2 = H1 @ W2.T + b2
    H2 = silu(A2)
    y = H2 @ W3 + b3
    r = y - T
    n = r.size
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3 = H2.T @ dy
    gb3 = dy.sum()
    D2 = np.outer(dy, W3) * silu_grad(A2)
    gW2 = D2.T @ H1
    gb2 = D2.sum(axis=0)
    D1 = (D2 @ W2) * silu_grad(A1)
    gW1 = D1.T @ Z
    gb1 = D1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def adam_steps(P, norm, X, Y, steps, lr, batch=BATCH):
    """`steps` Adam steps; step s takes rows (s*batch + k) mod n, k < batch."""
    P = np.asarray(P, np.float64).copy()
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    n = len(Y)
    b1, b2, eps = 0.9, 0.999, 1e-8
    losses = []
    for s in range(steps):
        idx = (s * batch + np.arange(batch)) % n
        loss, g = loss_and_grad(P, norm, X[idx], Y[idx])
        losses.append(loss)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        t = s + 1
        P = P - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return P, losses


def features(h, divv, n_ngb, vsig, cell_count, side, dt, n_ngb_target=48.0):
    """The six inputs per particle; cell_count and side are those of its cell."""
    h = np.asarray(h, np.float64)
    N = float(n_ngb_target)
    cnt = np.asarray(cell_count, np.float64)
    hc = np.cbrt(3.0 * N / (4.0 * np.pi * cnt)) * side
    return np.stack([dt * np.asarray(divv, np.float64),
                     np.log(np.maximum(np.asarray(n_ngb, np.float64), 1.0) / N),
                     np.log(hc / h),
                     np.log(cnt / N),
                     np.log(h / side),
                     dt * np.asarray(vsig, np.float64) / h], axis=1)


def glorot(seed):
    """A random parameter vector (for tests): Glorot-uniform weights, small biases."""
    rng = np.random.default_rng(seed)
    P = np.zeros(NPARAM)
    P[OFF_W1:OFF_B1] = rng.uniform(-1, 1, NH * NF) * np.sqrt(6.0 / (NF + NH))
    P[OFF_B1:OFF_W2] = rng.uniform(-0.1, 0.1, NH)
    P[OFF_W2:OFF_B2] = rng.uniform(-1, 1, NH * NH) * np.sqrt(6.0 / (2 * NH))
    P[OFF_B2:OFF_W3] = rng.uniform(-0.1, 0.1, NH)
    P[OFF_W3:OFF_B3] = rng.uniform(-1, 1, NH) * np.sqrt(6.0 / (NH + 1))
    P[OFF_B3] = 0.05
    return P


def to_library(P, norm):
    """(bf16 weight bits, f32 floats) in the library's load/save layout; the
    weights are rounded to bfloat16."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    w = np.concatenate([bf16_bits(W1.ravel()), bf16_bits(W2.ravel()), bf16_bits(W3)])
    f = np.concatenate([b1, b2, [b3], np.asarray(norm, np.float64)]).astype(np.float32)
    return w, f


def from_library(w, f):
    """Parameter vector (FP64 of the bfloat16 weights) and normalisation."""
    w = np.asarray(w, np.uint16)
    f = np.asarray(f, np.float32).astype(np.float64)
    W1 = from_bf16_bits(w[:NH * NF]).astype(np.float64)
    W2 = from_bf16_bits(w[NH * NF:NH * NF + NH * NH]).astype(np.float64)
    W3 = from_bf16_bits(w[NH * NF + NH * NH:]).astype(np.float64)
    P = np.concatenate([W1, f[:NH], W2, f[NH:2 * NH], W3, [f[2 * NH]]])
    return P, f[2 * NH + 1:]
