"""Learned initial h on the GPU (tensor-core inference, training, features, steps)
against the numpy oracle of oracle/hpredict.py.

Tolerances (from the arithmetic):
  inference   the oracle rounds what the kernel rounds to bfloat16 (unit roundoff
              2^-9); left are FP32 accumulation order and __expf (~1e-7 relative)
              and, rarely, a hidden activation that lands on the other side of a
              bfloat16 rounding boundary (one 2^-8 step of one of 64 inputs):
              99.9% of outputs within 1e-6, all within 1e-4 (outputs ~0.05)
  training    FP32 gradients (~1e-6 relative) through two Adam steps: 99% of the
              parameters within 1e-3 lr of the FP64 oracle
  features    FP32 logs and roots: 1e-5 absolute
"""
import numpy as np
import pytest

import oracle
from oracle import hpredict as hp
from paper_1508_00115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _norm():
    return np.array([0.0, 0.1, -0.2, 0.3, 0.0, 0.05, 1.0, 0.5, 0.7, 1.3, 0.9, 0.2, 0.01, 0.05])


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = (rng.normal(size=(n, 6)) * np.array([1.0, 0.5, 0.7, 1.3, 0.9, 0.2]) + _norm()[:6]).astype(np.float32)
    Y = (0.01 + 0.05 * np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.01 * rng.normal(size=n)).astype(np.float32)
    return X, Y


def _ctx(n=1000, **kw):
    from paper_1508_00115_gb300 import binding
    return binding.Context(n, **kw)


def test_hp_inference_matches_oracle():
    ctx = _ctx()
    w, f = hp.to_library(hp.glorot(21), _norm())
    ctx.hp_load(w, f)
    P, norm = hp.from_library(w, f)
    X, _ = _data(100003, 22)
    out = ctx.hp_eval(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = hp.forward(P, norm, X, bf16=True)
    err = np.abs(out - ref)
    assert np.quantile(err, 0.999) <= 1e-6, np.quantile(err, 0.999)
    assert err.max() <= 1e-4, err.max()
    # the saved weights are the loaded ones
    w2, f2 = ctx.hp_save()
    assert np.array_equal(w2, w) and np.array_equal(f2, f)


def test_hp_training_matches_oracle():
    ctx = _ctx()
    w, f = hp.to_library(hp.glorot(23), _norm())
    ctx.hp_load(w, f)
    P0, norm = hp.from_library(w, f)
    X, Y = _data(2 * hp.BATCH, 24)
    lr = 1e-3
    loss = ctx.hp_train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=1, lr=lr, seed=0)
    P_gpu = ctx.hp_params().astype(np.float64)
    P_ref, losses = hp.adam_steps(P0, norm, X.astype(np.float64), Y.astype(np.float64), 2, lr)
    d = np.abs(P_gpu - P_ref)
    assert np.quantile(d, 0.99) <= 1e-3 * lr, np.quantile(d, 0.99)
    assert abs(loss - losses[-1]) <= 1e-4 * losses[-1]
    # the BF16 inference copy is the rounding of the FP32 state
    w2, _ = ctx.hp_save()
    W = np.concatenate([P_gpu[hp.OFF_W1:hp.OFF_B1], P_gpu[hp.OFF_W2:hp.OFF_B2], P_gpu[hp.OFF_W3:hp.OFF_B3]])
    assert np.array_equal(w2, hp.bf16_bits(W.astype(np.float32)))


def test_hp_normalisation_from_training_data():
    ctx = _ctx()
    X, Y = _data(50000, 25)
    ctx.hp_init(7)
    ctx.hp_train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=0, lr=1e-3)
    _, f = ctx.hp_save()
    norm = f[129:]
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    assert np.allclose(norm[:6], X64.mean(axis=0), rtol=1e-6, atol=1e-7)
    assert np.allclose(norm[6:12], X64.std(axis=0), rtol=1e-5)
    assert np.isclose(norm[12], Y64.mean(), rtol=1e-5)
    assert np.isclose(norm[13], Y64.std(), rtol=1e-5)


def _uniform_moving(n, seed):
    d = inputs.uniform(n, seed=seed)
    d = inputs.random_velocities(d, 0.3, seed + 100)
    rng = np.random.default_rng(seed + 200)
    d["u"] = rng.uniform(0.5, 2.0, n)
    return d


def test_hp_features_match_oracle():
    from paper_1508_00115_gb300 import binding
    n = 20000
    d = _uniform_moving(n, 26)
    ctx = binding.Context(n)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    g0 = parts.numpy()
    p0 = ctx.permutation()
    # move the particles a little so that the next build permutes them
    dd = parts.numpy()
    rng = np.random.default_rng(27)
    for k in ("x", "y", "z"):
        dd[k] = dd[k] + rng.normal(scale=0.01, size=n)
    parts2 = binding.Particles(dd)
    ctx.build_cells(parts2)
    g = parts2.numpy()
    p = ctx.permutation()
    # divv and n_ngb travel with their particles (bit-exact)
    inv0 = np.empty(n, np.int64)
    inv0[p0] = np.arange(n)
    src = inv0[p]
    assert np.array_equal(g["divv"], g0["divv"][src])
    assert np.array_equal(g["n_ngb"], g0["n_ngb"][src])
    dt = 3e-4
    feats = ctx.hp_features(parts2, dt).cpu().numpy().astype(np.float64)
    nc = ctx.stats()["nc"]
    cells = oracle.cell_keys(g["x"], g["y"], g["z"], 1.0, nc)
    count = np.bincount(cells, minlength=nc ** 3)[cells]
    ref = hp.features(g["h"], g["divv"], g["n_ngb"], g["vsig"], count, 1.0 / nc, dt)
    assert np.allclose(feats, ref, rtol=1e-5, atol=1e-5)


def _state_close(g1, g2, p1, p2, rtol):
    i1, i2 = np.argsort(p1), np.argsort(p2)
    for k in ("x", "y", "z"):
        dx = g1[k][i1] - g2[k][i2]
        dx -= np.rint(dx)
        assert np.abs(dx).max() < 1e-9, k
    for k in ("vx", "vy", "vz"):
        assert np.abs(g1[k][i1] - g2[k][i2]).max() <= rtol * (np.abs(g1[k]).max() + 1e-30), k
    assert (np.abs(g1["h"][i1] - g2["h"][i2]) / g1["h"][i1]).max() <= rtol


@pytest.mark.parametrize("graph", [False, True])
def test_hp_steps_reach_the_same_root(graph):
    """Steps whose iterations start at a (random-weight) predictor's guess end at the
    same smoothing lengths, positions and velocities as plain steps."""
    from paper_1508_00115_gb300 import binding
    d = _uniform_moving(6000, 28)
    out = []
    # random weights; guesses within a few per cent of h_prev (target scale 0.02),
    # so that the six passes of a captured step converge too
    norm = _norm()
    norm[12], norm[13] = 0.0, 0.02
    w, f = hp.to_library(hp.glorot(29), norm)
    for flags in (0, binding.SPH_FLAG_HPREDICT):
        ctx = binding.Context(d["x"].size, h_tol=1e-6, flags=flags)
        if flags:
            ctx.hp_load(w, f)
        parts = binding.Particles(d)
        if graph:
            ctx.steps(parts, 3, 4e-4)
        else:
            for _ in range(3):
                ctx.step(parts, 4e-4)
        out.append((parts.numpy(), ctx.permutation()))
    (g1, p1), (g2, p2) = out
    _state_close(g1, g2, p1, p2, 1e-5)


def test_hp_batched_adaptive_graph_steps_reach_the_same_root():
    """Learned guess + batched boxes on adaptive cells, steps replayed from a CUDA
    graph (the headline form): same smoothing lengths, positions and velocities as
    the same steps without the guess."""
    from paper_1508_00115_gb300 import binding
    boxes = []
    for b, nb in enumerate((4000, 900, 2500 + 3)):
        d = inputs.plummer_mix(nb, seed=60 + b, n_halos=max(1, nb // 1000))
        boxes.append(inputs.random_velocities(d, 0.05, 70 + b))
    offs = [0]
    for b in boxes:
        offs.append(offs[-1] + b["x"].size)
    d = {k: np.concatenate([b[k] for b in boxes]) for k in inputs.FIELDS}
    norm = _norm()
    norm[12], norm[13] = 0.0, 0.02
    w, f = hp.to_library(hp.glorot(31), norm)
    out = []
    for flags in (binding.SPH_FLAG_ADAPTIVE, binding.SPH_FLAG_ADAPTIVE | binding.SPH_FLAG_HPREDICT):
        ctx = binding.Context(d["x"].size, h_tol=1e-6, flags=flags | binding.SPH_FLAG_TREE_H_GUESS,
                              box_offsets=offs)
        if flags & binding.SPH_FLAG_HPREDICT:
            ctx.hp_load(w, f)
        parts = binding.Particles(d)
        ctx.steps(parts, 3, 2e-4)
        assert ctx.stats()["graph_steps"] == 3
        out.append((parts.numpy(), ctx.permutation()))
        ctx.close()
    (g1, p1), (g2, p2) = out
    _state_close(g1, g2, p1, p2, 1e-5)


def test_hp_collect_samples_during_steps():
    from paper_1508_00115_gb300 import binding
    n = 5000
    d = _uniform_moving(n, 30)
    ctx = binding.Context(n, h_tol=1e-6)
    parts = binding.Particles(d)
    cap = 3 * n + 10
    F = torch.zeros((cap, 6), dtype=torch.float32, device="cuda")
    T = torch.zeros(cap, dtype=torch.float32, device="cuda")
    ctx.hp_collect(F, T, cap)
    for _ in range(4):  # the fourth step does not fit
        ctx.step(parts, 3e-4)
    assert ctx.stats()["hp_samples"] == 3 * n
    t = T[: 3 * n].cpu().numpy()
    f = F[: 3 * n].cpu().numpy()
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(t))
    assert np.all(T[3 * n:].cpu().numpy() == 0)
    # a step changes h by a small amount in a smooth flow
    assert np.abs(t).max() < 0.2
    # the targets are the log-ratios of consecutive converged h: the last step's
    # target plus its h_prev gives the final h
    g = parts.numpy()
    assert np.all(np.abs(t[2 * n:]) < 0.2)
    assert np.all(g["h"] > 0)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 311373])
def test_hp_inference_ragged_tiles(n):
    """Tensor-core inference takes 128 particles per tile and loops over tiles in a
    persistent grid: a single particle, one short of a tile, a whole tile, one over,
    and more than two waves of the grid's CTAs (8 per SM), against the oracle."""
    ctx = _ctx()
    w, f = hp.to_library(hp.glorot(31), _norm())
    ctx.hp_load(w, f)
    P, norm = hp.from_library(w, f)
    X, _ = _data(n, 32)
    out = ctx.hp_eval(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = hp.forward(P, norm, X, bf16=True)
    err = np.abs(out - ref)
    assert out.shape == (n,)
    assert err.max() <= 1e-4, err.max()
    if n >= 1000:
        assert np.quantile(err, 0.999) <= 1e-6
