"""Individual time-steps on the GPU (sph_step_bins) against the oracle's scheme.

Where the scheme makes no choice it must be the global step bit for bit (one
level; every particle in one shared bin).  With a hierarchy of bins (a hot region
inside cooler gas) it must match oracle.step_bins: the same bins for every
particle, the same substeps and particle updates, and the state within the
tolerances of the global-step parity test (FP32 pair sums, FP64 kicks and drifts).
Bin decisions are integers taken from floating point; the test picks dt_max so that
no decision of the oracle's run lies within 5e-5 (in log2) of a bin boundary, far
outside the FP32 differences of the two paths.
"""
import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ARRAYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "dudt", "vsig", "rho")


def _hydro_ctx(d, **params):
    from paper_1508_00115_gb300 import binding
    n = int(d["x"].size)
    ctx = binding.Context(n, **params)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    return ctx, parts


def _equal(a, b):
    for k in ARRAYS:
        assert np.array_equal(a[k], b[k]), k


def test_single_level_is_sph_step_bit_for_bit():
    d = inputs.random_velocities(inputs.uniform(3000, seed=21), 0.3, 22)
    d["u"] = np.random.default_rng(23).uniform(0.5, 2.0, 3000)
    c1, p1 = _hydro_ctx(d)
    c2, p2 = _hydro_ctx(d)
    g = p1.numpy()
    dt = 0.5 * 0.1 * float(np.min(g["h"] / g["vsig"]))
    c1.step(p1, dt)
    cons, st = c2.step_bins(p2, dt, 0)
    assert st["substeps"] == 1 and st["updates"] == 3000 and st["bin_count"][0] == 3000
    _equal(p1.numpy(), p2.numpy())
    assert np.array_equal(c1.permutation(), c2.permutation())


def test_one_shared_bin_is_repeated_steps_bit_for_bit():
    d = inputs.random_velocities(inputs.lattice(16, 1.0, jitter=0.1, seed=8, u0=1.0), 0.02, 9)
    n = d["x"].size
    c1, p1 = _hydro_ctx(d)
    c2, p2 = _hydro_ctx(d)
    g = p1.numpy()
    dtc = 0.1 * g["h"].astype(np.float64) / g["vsig"].astype(np.float64)
    assert dtc.max() < 1.3 * dtc.min()
    dt_max = 2.9 * dtc.min()  # every CFL step in [dt_max/2.9, dt_max/2.2]: bin 2
    for _ in range(4):
        c1.step(p1, dt_max / 4)
    cons, st = c2.step_bins(p2, dt_max, 4)
    assert st["substeps"] == 4 and st["updates"] == 4 * n and st["bin_count"][2] == n
    assert np.all(c2.bins() == 2)
    _equal(p1.numpy(), p2.numpy())


def _hot_spot(n, seed, factor):
    d = inputs.random_velocities(inputs.uniform(n, seed=seed), 0.3, seed + 1)
    d["u"] = np.random.default_rng(seed + 2).uniform(0.5, 2.0, n)
    r2 = (d["x"] - 0.5) ** 2 + (d["y"] - 0.5) ** 2 + (d["z"] - 0.5) ** 2
    d["u"][r2 < 0.2 ** 2] *= factor
    return d


def test_hierarchical_bins_match_oracle():
    from paper_1508_00115_gb300 import binding
    n, levels = 2500, 3
    d = _hot_spot(n, 31, 30.0)
    s = oracle.State(**{k: np.asarray(d[k], np.float64) for k in inputs.FIELDS})
    acc = oracle.hydro(s)
    dtc = 0.1 * acc["h"] / acc["vsig"]
    dt_max = 5.0 * dtc.min()
    for _ in range(40):  # a dt_max whose bin decisions all keep clear of a boundary
        ref, racc, rst = oracle.step_bins(s, acc, dt_max, levels)
        if rst["margin"] > 5e-5:
            break
        dt_max *= 1.0173
    else:
        pytest.fail("no dt_max with clear bin decisions")
    assert len(np.unique(rst["bins"])) >= 3  # a real hierarchy
    ctx = binding.Context(n, h_tol=1e-6)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    cons, st = ctx.step_bins(parts, dt_max, levels)
    g = parts.numpy()
    idx = ctx.permutation()  # slot k holds the input particle idx[k]
    assert np.array_equal(ctx.bins(), rst["bins"][idx])
    assert st["substeps"] == rst["substeps"] and st["updates"] == rst["active"]
    assert st["cfl_over"] == rst["over"]
    for k in ("x", "y", "z"):
        dx = g[k] - getattr(ref, k)[idx]
        dx -= np.rint(dx)
        assert np.abs(dx).max() < 1e-7, k
    vscale = np.sqrt(np.mean(ref.vx ** 2 + ref.vy ** 2 + ref.vz ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - getattr(ref, k)[idx]).max() < 1e-4 * vscale, k
    assert (np.abs(g["u"] - ref.u[idx]) / ref.u[idx]).max() < 1e-4
    assert (np.abs(g["h"] - ref.h[idx]) / ref.h[idx]).max() < 1e-4
    ascale = np.sqrt(np.mean(np.sum(racc["a"] ** 2, axis=1)))
    for j, k in enumerate(("ax", "ay", "az")):
        assert np.abs(g[k] - racc["a"][idx, j]).max() < 1e-3 * ascale, k
    # momentum is not conserved exactly by individual steps; energy stays close
    e0 = float(np.sum(s.m * (0.5 * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2) + s.u)))
    assert abs(cons["e_tot"] - e0) < 1e-2 * e0


def test_bins_edge_cases():
    from paper_1508_00115_gb300 import binding
    d = inputs.uniform(500, seed=4)
    ctx, parts = _hydro_ctx(d)
    with pytest.raises(binding.SphError) as e:  # no binned step yet
        ctx.bins()
    assert e.value.code == binding.SPH_ERR_STATE
    for dt, levels in ((0.0, 2), (-1.0, 2), (float("nan"), 2), (1e-3, -1), (1e-3, binding.SPH_MAX_BINS + 1)):
        with pytest.raises(binding.SphError) as e:
            ctx.step_bins(parts, dt, levels)
        assert e.value.code == binding.SPH_ERR_INVALID_ARG
    # empty set: one step end, nothing to update
    ctx0 = binding.Context(0)
    p0 = binding.Particles({k: np.zeros(0) for k in inputs.FIELDS})
    cons, st = ctx0.step_bins(p0, 1e-3, 3)
    assert st["substeps"] == 1 and st["updates"] == 0 and cons["e_tot"] == 0.0
    assert ctx0.bins().size == 0


def _blast(n, seed, lattice=False):
    """A hot sphere (u = 10) in cold gas at rest (u = 1e-4): CFL steps ~350x apart.
    lattice: n^3 particles on a jittered lattice (nearly equal h), else n random."""
    if lattice:
        d = inputs.lattice(n, 1.0, jitter=0.3, seed=seed, u0=1e-4)
        n = d["x"].size
    else:
        d = inputs.uniform(n, seed=seed)
    for k in ("vx", "vy", "vz"):
        d[k] = np.zeros(n)
    d["u"] = np.full(n, 1e-4)
    r2 = (d["x"] - 0.5) ** 2 + (d["y"] - 0.5) ** 2 + (d["z"] - 0.5) ** 2
    d["u"][r2 < (0.15 if lattice else 0.12) ** 2] = 10.0
    return d


@pytest.mark.parametrize("grid", ["uniform", "adaptive", "uniform-wide"])
def test_limiter_matches_oracle(grid):
    """The time-step limiter with wake-up against oracle.step_bins(limiter=2) on a blast
    into cold gas: the same bins, substeps, particle updates, raised bins and
    wake-ups (all integers), and the state within the tolerances above.  The limiter's
    neighbour decisions are FP64 on both sides; the pairs that decide a raise sit
    next to a jump of several bins, far from the h boundary in this setup.
    uniform-wide: a 12^3 jittered lattice, the grid planned from h guesses 1.8x below
    the converged h (between 1.4 and 1.6 cell sides, within the 1.8 up to which the
    plan is kept): every cutoff exceeds the cell side, and the limiter searches the
    125 cells around each particle."""
    from paper_1508_00115_gb300 import binding
    levels = 8
    d = _blast(12, 41, lattice=True) if grid == "uniform-wide" else _blast(1200, 41)
    n = int(d["x"].size)
    s = oracle.State(**{k: np.asarray(d[k], np.float64) for k in inputs.FIELDS})
    acc = oracle.hydro(s)
    dtc = 0.1 * acc["h"] / acc["vsig"]
    dt_max = 16.0 * dtc.min()
    for _ in range(40):
        ref, racc, rst = oracle.step_bins(s, acc, dt_max, levels, limiter=binding.SPH_BIN_LIMIT_LEVELS)
        if rst["margin"] > 5e-5:
            break
        dt_max *= 1.0173
    else:
        pytest.fail("no dt_max with clear bin decisions")
    assert rst["limited"] > 0 and rst["woken"] > 0
    flags = binding.SPH_FLAG_BIN_LIMITER | (binding.SPH_FLAG_ADAPTIVE if grid == "adaptive" else 0)
    ctx = binding.Context(n, h_tol=1e-6, flags=flags)
    if grid == "uniform-wide":
        d = dict(d, h=acc["h"] / 1.8)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    if grid == "uniform-wide":
        L = ctx.stats()["cell_size"]
        assert acc["h"].min() > 1.05 * L and acc["h"].max() < 1.8 * L
    ctx.density(parts)
    ctx.force(parts)
    cons, st = ctx.step_bins(parts, dt_max, levels)
    g = parts.numpy()
    idx = ctx.permutation()
    assert np.array_equal(ctx.bins(), rst["bins"][idx])
    assert st["substeps"] == rst["substeps"] and st["updates"] == rst["active"]
    assert st["limited"] == rst["limited"] and st["woken"] == rst["woken"]
    assert st["cfl_over"] == rst["over"] and st["limit_sweeps"] >= st["substeps"]
    for k in ("x", "y", "z"):
        dx = g[k] - getattr(ref, k)[idx]
        dx -= np.rint(dx)
        assert np.abs(dx).max() < 1e-7, k
    vscale = np.sqrt(np.mean(ref.vx ** 2 + ref.vy ** 2 + ref.vz ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - getattr(ref, k)[idx]).max() < 1e-4 * vscale, k
    assert (np.abs(g["u"] - ref.u[idx]) / ref.u[idx]).max() < 1e-4
    assert (np.abs(g["h"] - ref.h[idx]) / ref.h[idx]).max() < 1e-4


def test_limiter_off_is_unchanged_and_on_is_a_no_op_in_one_bin():
    """Every particle in one bin: the limiter finds nothing to raise or wake, and the
    run is bit for bit the one without it (and both the repeated global step)."""
    from paper_1508_00115_gb300 import binding
    d = inputs.random_velocities(inputs.lattice(16, 1.0, jitter=0.1, seed=8, u0=1.0), 0.02, 9)
    c1, p1 = _hydro_ctx(d)
    c2, p2 = _hydro_ctx(d, flags=binding.SPH_FLAG_BIN_LIMITER)
    g = p1.numpy()
    dt_max = 2.9 * float(np.min(0.1 * g["h"].astype(np.float64) / g["vsig"].astype(np.float64)))
    _, s1 = c1.step_bins(p1, dt_max, 4)
    _, s2 = c2.step_bins(p2, dt_max, 4)
    assert s2["limited"] == 0 and s2["woken"] == 0 and s2["limit_sweeps"] == s2["substeps"]
    assert s1["limit_sweeps"] == 0
    _equal(p1.numpy(), p2.numpy())


def test_limiter_batched_boxes_match_each_box_alone():
    """Two blasts in two periodic boxes of one context (one limiter pass over all
    boxes) against each box in a context of its own: the same bins, updates, raised
    bins and wake-ups, and the same state up to rounding -- a batched run also
    drifts each box at the other box's step ends, which splits its drifts and
    moves its FP32 sums by an ulp."""
    from paper_1508_00115_gb300 import binding
    levels = 7
    ds = [_blast(900, 51), _blast(1400, 52)]
    runs = []
    for d in ds:
        ctx, parts = _hydro_ctx(d, flags=binding.SPH_FLAG_BIN_LIMITER)
        runs.append((ctx, parts))
    g0 = runs[0][1].numpy()
    dt_max = 16.0 * float(np.min(0.1 * g0["h"].astype(np.float64) / g0["vsig"].astype(np.float64)))
    alone = []
    for ctx, parts in runs:
        _, st = ctx.step_bins(parts, dt_max, levels)
        alone.append((st, parts.numpy(), ctx.bins(), ctx.permutation()))
        assert st["limited"] > 0 and st["woken"] > 0
    sizes = [d["x"].size for d in ds]
    offs = np.array([0, sizes[0], sizes[0] + sizes[1]], dtype=np.int64)
    db = {k: np.concatenate([d[k] for d in ds]) for k in inputs.FIELDS}
    ctx = binding.Context(int(offs[-1]), box_offsets=offs, flags=binding.SPH_FLAG_BIN_LIMITER)
    parts = binding.Particles(db)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    _, stb = ctx.step_bins(parts, dt_max, levels)
    gb, bb, pb = parts.numpy(), ctx.bins(), ctx.permutation()
    # step ends: those of either box (their union)
    assert max(a[0]["substeps"] for a in alone) <= stb["substeps"] <= sum(a[0]["substeps"] for a in alone)
    assert stb["updates"] == sum(a[0]["updates"] for a in alone)
    assert stb["limited"] == sum(a[0]["limited"] for a in alone)
    assert stb["woken"] == sum(a[0]["woken"] for a in alone)
    for b, (st, g, bins, perm) in enumerate(alone):
        sl = slice(int(offs[b]), int(offs[b + 1]))
        ib = np.argsort(pb[sl] - offs[b])
        ia = np.argsort(perm)
        assert np.array_equal(bb[sl][ib], bins[ia])
        for k in ("x", "y", "z"):
            dx = gb[k][sl][ib] - g[k][ia]
            dx -= np.rint(dx)
            assert np.abs(dx).max() < 1e-8, k
        for k in ("vx", "vy", "vz", "u", "h"):
            x, y = gb[k][sl][ib], g[k][ia]
            assert np.abs(x - y).max() <= 1e-5 * np.abs(y).max(), k
