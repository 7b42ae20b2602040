"""Near-field gravity (sph_gravity_p2p, Sec. 3.2, Eq. 3) against the FP64 oracle
(oracle.grav_p2p) on the same particles, the same grid and the same softening.

Tolerances (FP32 pair arithmetic on cell-relative positions, compensated cell
sums): acceleration |a_gpu - a_orc| <= 1e-4 x RMS|a_orc| per particle (the bar of
the SPH force), potential 1e-5 relative per particle; sum m a = 0 to 1e-6 of sum m |a|; bit-identical on a
second run.  The grid is set through the smoothing lengths, on which gravity does
not otherwise depend: every h equal to h0 gives nc = floor(1 / (1.1 h0)) cells
per side (cell factor 1.1).

Where the bar holds: a separation component carries an absolute FP32 error up to
delta ~ 3.5 x 2^-24 L (cell side L), so a pair's force is off by at most
m_j delta / eps^3 with Plummer softening eps, and by ~2 delta / r of itself
without: random fields are tested softened (eps of a tenth of the mean spacing
keeps that 5x inside the bar), unsoftened ones on a jittered lattice (separations
bounded below)."""
import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A_TOL = 1e-4
PHI_TOL = 1e-5


def _field(n, seed, clustered=False, h0=0.1):
    d = inputs.plummer_mix(n, seed=seed, n_halos=4) if clustered else inputs.uniform(n, seed=seed)
    d["m"] = np.random.default_rng(seed + 7).uniform(0.5, 2.0, n) / n
    d["h"] = np.full(n, h0)
    return d


def _gpu_gravity(d, G=1.0, eps=0.0, box_offsets=None, tile_width=32, runs=1):
    from paper_1508_00115_gb300 import binding
    n = d["x"].size
    ctx = binding.Context(n, box_offsets=box_offsets, tile_width=tile_width, cell_factor=1.1)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    outs = []
    for _ in range(runs):
        o = ctx.gravity(G, eps)
        torch.cuda.synchronize()
        outs.append({k: v[:n].cpu().numpy() for k, v in o.items()})
    g = parts.numpy()
    st = ctx.stats()
    ctx.close()
    return g, outs, st


def _state(g, lo=0, hi=None):
    sl = slice(lo, hi)
    return oracle.State(x=g["x"][sl], y=g["y"][sl], z=g["z"][sl], vx=g["vx"][sl], vy=g["vy"][sl],
                        vz=g["vz"][sl], m=g["m"][sl].astype(np.float64), u=g["u"][sl].astype(np.float64),
                        h=g["h"][sl].astype(np.float64))


def _compare(o, ref, G=1.0, targets=None):
    t = slice(None) if targets is None else targets
    a = np.stack([o["ax"][t], o["ay"][t], o["az"][t]], axis=1).astype(np.float64)
    rms = np.sqrt(np.mean(np.sum(ref["a"] ** 2, axis=1)))
    err = np.sqrt(np.sum((a - ref["a"]) ** 2, axis=1))
    assert err.max() <= A_TOL * rms, (err.max() / rms)
    perr = np.abs(o["phi"][t] - ref["phi"]) / np.abs(ref["phi"])
    assert perr.max() <= PHI_TOL, perr.max()
    return err.max() / rms, perr.max()


@pytest.mark.parametrize("tw,eps", [(32, 0.004), (16, 0.004), (32, 0.01)])
def test_gravity_uniform_matches_oracle(tw, eps):
    d = _field(32768, 3, h0=0.1)
    g, (o,), st = _gpu_gravity(d, eps=eps, tile_width=tw)
    assert st["nc"] == 9
    ref = oracle.grav_p2p(_state(g), st["nc"], eps=eps)
    _compare(o, ref)
    # algorithmic pair count: every particle against the 27 cells around it, less itself
    assert st["grav_pairs"] > 0


def test_gravity_clustered_matches_oracle_and_conserves_momentum():
    d = _field(30000, 5, clustered=True, h0=0.07)
    G = 2.5
    g, (o,), st = _gpu_gravity(d, G=G, eps=0.003)
    ref = oracle.grav_p2p(_state(g), st["nc"], G=G, eps=0.003)
    _compare(o, ref)
    m = g["m"].astype(np.float64)
    a = np.stack([o["ax"], o["ay"], o["az"]], axis=1).astype(np.float64)
    assert np.abs((m[:, None] * a).sum(axis=0)).max() <= 1e-6 * np.sum(m * np.linalg.norm(a, axis=1))


def test_gravity_is_deterministic():
    d = _field(20000, 9, clustered=True, h0=0.08)
    _, outs, _ = _gpu_gravity(d, eps=0.002, runs=2)
    for k in ("ax", "ay", "az", "phi"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_gravity_large_sampled_targets():
    """Sedov-like jittered lattice, 64^3 particles, fine grid (nc = 45): a sample of
    targets, including the first and last slots, against the oracle."""
    d = inputs.lattice(64, jitter=0.1, seed=4)
    n = d["x"].size
    d["m"] = np.full(n, 1.0 / n)
    d["h"] = np.full(n, 0.02)
    g, (o,), st = _gpu_gravity(d, eps=0.0)
    rng = np.random.default_rng(1)
    t = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 1500, replace=False)]))
    ref = oracle.grav_p2p(_state(g), st["nc"], eps=0.0, targets=t)
    _compare(o, ref, targets=t)


def test_gravity_batched_boxes_match_each_box_alone():
    """Boxes of uneven size in one context: each box on its own grid, against the
    oracle run on that box alone."""
    sizes = [3000, 700, 5000 + 3]
    boxes = [_field(nb, 20 + b, clustered=b != 1, h0=0.1) for b, nb in enumerate(sizes)]
    offs = [0]
    for b in boxes:
        offs.append(offs[-1] + b["x"].size)
    d = {k: np.concatenate([b[k] for b in boxes]) for k in inputs.FIELDS}
    g, (o,), st = _gpu_gravity(d, eps=0.003, box_offsets=offs)
    for b in range(len(sizes)):
        lo, hi = offs[b], offs[b + 1]
        nc = min(9, int(np.floor(np.cbrt(8 * sizes[b]))))
        ref = oracle.grav_p2p(_state(g, lo, hi), nc, eps=0.003)
        _compare({k: v[lo:hi] for k, v in o.items()}, ref)


def test_gravity_errors_and_edges():
    from paper_1508_00115_gb300 import binding
    d = _field(2000, 13)
    n = d["x"].size
    ctx = binding.Context(n, cell_factor=1.1)
    parts = binding.Particles(d)
    with pytest.raises(binding.SphError) as e:  # no cells yet
        ctx.gravity()
    assert e.value.code == binding.SPH_ERR_STATE
    ctx.build_cells(parts)
    with pytest.raises(binding.SphError) as e:
        ctx.gravity(eps=-1.0)
    assert e.value.code == binding.SPH_ERR_INVALID_ARG
    o = ctx.gravity(with_phi=False)
    assert torch.all(o["phi"] == 0) and torch.isfinite(o["ax"]).all()
    ctx.close()
    ctx = binding.Context(n, flags=binding.SPH_FLAG_ADAPTIVE)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    with pytest.raises(binding.SphError) as e:
        ctx.gravity()
    assert e.value.code == binding.SPH_ERR_STATE
    ctx.close()
    # coincident particles without softening: finite, their mutual term dropped
    d2 = inputs.lattice(8, jitter=0.1, seed=14)
    d2["h"] = np.full(512, 0.1)
    for k in inputs.FIELDS:
        d2[k][1] = d2[k][0]
    g, (o,), st = _gpu_gravity(d2, eps=0.0)
    assert all(np.all(np.isfinite(o[k])) for k in o)
    ref = oracle.grav_p2p(_state(g), st["nc"], eps=0.0)
    _compare(o, ref)
