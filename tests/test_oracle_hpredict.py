"""Pins of the learned-h oracle (oracle/hpredict.py) against facts that do not come
from the oracle itself: finite differences, closed forms of degenerate networks,
the closed form of Adam's first step, Taylor expansions of SiLU, PyTorch's own
bfloat16 conversion, and the features of a uniform lattice."""
import numpy as np
import pytest

from oracle import hpredict as hp


def _norm():
    return np.array([0.0, 0.1, -0.2, 0.3, 0.0, 0.05, 1.0, 0.5, 0.7, 1.3, 0.9, 0.2, 0.01, 0.05])


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 6)) * np.array([1.0, 0.5, 0.7, 1.3, 0.9, 0.2]) + _norm()[:6]
    Y = 0.01 + 0.05 * np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.01 * rng.normal(size=n)
    return X, Y


def test_gradient_matches_finite_differences():
    P = hp.glorot(3)
    X, Y = _data(9, 4)
    _, g = hp.loss_and_grad(P, _norm(), X, Y)
    rng = np.random.default_rng(5)
    # every block of the parameter vector, several coordinates each
    idx = np.concatenate([rng.choice(np.arange(a, b), size=min(8, b - a), replace=False)
                          for a, b in ((hp.OFF_W1, hp.OFF_B1), (hp.OFF_B1, hp.OFF_W2), (hp.OFF_W2, hp.OFF_B2),
                                       (hp.OFF_B2, hp.OFF_W3), (hp.OFF_W3, hp.OFF_B3), (hp.OFF_B3, hp.NPARAM))])
    eps = 1e-6
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += eps
        Pm[k] -= eps
        fd = (hp.loss_and_grad(Pp, _norm(), X, Y)[0] - hp.loss_and_grad(Pm, _norm(), X, Y)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_degenerate_networks_closed_form():
    X, _ = _data(50, 6)
    norm = _norm()
    P = hp.glorot(7)
    # no output weights: y = b3 for every row
    P0 = P.copy()
    P0[hp.OFF_W3:hp.OFF_B3] = 0.0
    P0[hp.OFF_B3] = 0.4
    out = hp.forward(P0, norm, X, clamp=False)
    assert np.allclose(out, 0.4 * norm[13] + norm[12], rtol=0, atol=1e-15)
    # no second-layer weights or biases: H2 = silu(0) = 0, again y = b3
    P1 = P.copy()
    P1[hp.OFF_W2:hp.OFF_W3] = 0.0
    P1[hp.OFF_B3] = -0.3
    assert np.allclose(hp.forward(P1, norm, X, clamp=False), -0.3 * norm[13] + norm[12], atol=1e-15)
    # one hidden path: y = w3 silu(w2 silu(w1 . z + b1) + b2) + b3, by hand
    P2 = np.zeros(hp.NPARAM)
    P2[hp.OFF_W1 + 0 * 6 + 2] = 0.7          # unit 0 reads feature 2
    P2[hp.OFF_B1 + 0] = 0.1
    P2[hp.OFF_W2 + 5 * 64 + 0] = -1.2         # unit 5 of layer 2 reads unit 0
    P2[hp.OFF_B2 + 5] = 0.2
    P2[hp.OFF_W3 + 5] = 0.9
    P2[hp.OFF_B3] = 0.05
    z2 = (X[:, 2] - norm[2]) / norm[8]
    s = lambda v: v / (1 + np.exp(-v))
    y = 0.9 * s(-1.2 * s(0.7 * z2 + 0.1) + 0.2) + 0.05
    # (the oracle normalises in FP32, like the inference path: ~1e-9 absolute here)
    assert np.allclose(hp.forward(P2, norm, X, clamp=False), y * norm[13] + norm[12], rtol=1e-6, atol=1e-8)
    # the clamp bounds the log-ratio to [log 1/2, log 1.2]
    P3 = P0.copy()
    P3[hp.OFF_B3] = 1e3
    assert np.allclose(hp.forward(P3, norm, X), np.log(np.float32(1.2)), atol=1e-7)


def test_silu_taylor_and_derivative():
    x = np.array([-1e-3, -1e-4, 1e-4, 1e-3])
    # silu(x) = x/2 + x^2/4 - x^4/48 + ...
    assert np.allclose(hp.silu(x), x / 2 + x * x / 4, rtol=0, atol=1e-13)
    xs = np.linspace(-6, 6, 41)
    fd = (hp.silu(xs + 1e-6) - hp.silu(xs - 1e-6)) / 2e-6
    assert np.allclose(hp.silu_grad(xs), fd, atol=1e-8)
    assert hp.silu_grad(0.0) == 0.5


def test_first_adam_step_closed_form():
    P = hp.glorot(8)
    X, Y = _data(hp.BATCH, 9)
    lr = 1e-3
    _, g = hp.loss_and_grad(P, _norm(), X, Y)
    P1, _ = hp.adam_steps(P, _norm(), X, Y, 1, lr)
    # first step: m_hat = g, v_hat = g^2  ->  P - lr g / (|g| + eps)
    assert np.allclose(P1, P - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_adam_reduces_loss_on_learnable_target():
    X, Y = _data(4096, 10)
    P, losses = hp.adam_steps(hp.glorot(11), _norm(), X, Y, 60, 3e-3, batch=1024)
    assert losses[-1] < 0.2 * losses[0]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.normal(size=2000).astype(np.float32),
                        np.float32([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, 3.0e38, 1e-40])])
    ours = hp.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    # ties go to the even mantissa
    assert hp.bf16_round(np.float32([1 + 2 ** -8]))[0] == 1.0
    assert hp.bf16_round(np.float32([1 + 3 * 2 ** -8]))[0] == np.float32(1 + 2 ** -6)


def test_library_layout_roundtrip():
    P = hp.glorot(13)
    w, f = hp.to_library(P, _norm())
    assert w.size == 4544 and f.size == 143
    P2, norm2 = hp.from_library(w, f)
    W = slice(hp.OFF_W1, hp.OFF_B1)
    assert np.array_equal(P2[W], hp.bf16_round(P[W]).astype(np.float64))
    assert np.allclose(P2[hp.OFF_B1:hp.OFF_W2], P[hp.OFF_B1:hp.OFF_W2], rtol=1e-7)
    assert np.allclose(norm2, _norm(), rtol=1e-7)


def test_features_of_a_uniform_lattice():
    """n_side^3 lattice, grid of nc^3 cells: every cell holds (n_side/nc)^3
    particles, so h_cell is the h of the uniform density n_side^3 and, with h set
    to it, f2 = 0; f3 and f4 follow from the counts."""
    n_side, nc = 24, 6
    cnt = (n_side // nc) ** 3
    side = 1.0 / nc
    h_uni = np.cbrt(3 * 48 / (4 * np.pi * n_side ** 3))
    n = n_side ** 3
    f = hp.features(np.full(n, h_uni), np.full(n, 0.5), np.full(n, 48), np.full(n, 2.0),
                    np.full(n, cnt), side, dt=0.01)
    assert np.allclose(f[:, 0], 0.005)
    assert np.allclose(f[:, 1], 0.0)
    assert np.allclose(f[:, 2], 0.0, atol=1e-12)
    assert np.allclose(f[:, 3], np.log(cnt / 48))
    assert np.allclose(f[:, 4], np.log(h_uni / side))
    assert np.allclose(f[:, 5], 0.02 / h_uni)
