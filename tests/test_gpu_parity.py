"""Parity of the CUDA path (called through the C-ABI) with the FP64 oracle.

Tolerances (from the precision design: FP32 pair arithmetic on cell-relative
positions with compensated sums, FP64 decisions at the cutoff):
  density       |rho_gpu - rho_orc| / rho_orc <= 1e-5 at the GPU's h
  h criterion   |N_w(h_gpu)/N_ngb - 1| <= h_tol (+ FP32 rounding of h), in FP64
  neighbours    counts and set fingerprints bit-exact
  cell keys     bit-exact
  acceleration  |a_gpu - a_orc| <= 1e-4 * RMS|a_orc|   (same for du/dt)
"""
import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import inputs

from _gpu_util import check_density, check_force, check_ghost, gpu_hydro, oracle_state, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _uniform_moving(n, seed):
    d = inputs.uniform(n, seed=seed)
    d = inputs.random_velocities(d, 0.3, seed + 100)
    rng = np.random.default_rng(seed + 200)
    d["u"] = rng.uniform(0.5, 2.0, n)
    return d


@pytest.mark.parametrize("n,seed", [(1000, 3), (4096 + 17, 4), (12345, 5)])
def test_density_force_small_ragged(n, seed):
    d = _uniform_moving(n, seed)
    ctx, parts, g = gpu_hydro(d)
    s = oracle_state(g)
    t = np.arange(n)
    dd = check_density(g, s)
    check_ghost(g, s, dd, t)
    check_force(g, s)
    # the GPU's composite permutation maps every slot to a distinct input particle
    assert np.array_equal(np.sort(g["perm"]), np.arange(n))
    assert np.allclose(g["x"], np.mod(d["x"][g["perm"]], 1.0), rtol=0, atol=0)


def test_config1_uniform_32k_full():
    """32^3 = 32768 uniform equal-mass particles, rho0 = 1, u = 1, v = 0: one
    density + h iteration + force, every particle compared."""
    d = inputs.uniform(32768, seed=1)
    ctx, parts, g = gpu_hydro(d)
    s = oracle_state(g)
    dd = check_density(g, s)
    check_ghost(g, s, dd, np.arange(s.n))
    check_force(g, s)
    assert g["iters"] >= 2


def test_cell_keys_bit_exact():
    d = _uniform_moving(20000, 8)
    ctx, parts, g = gpu_hydro(d)
    nc = g["stats"]["nc"]
    keys = ctx.cell_keys()
    ok = oracle.cell_keys(g["x"], g["y"], g["z"], 1.0, nc)
    assert np.array_equal(keys.astype(np.int64), ok)
    assert np.all(np.diff(keys) >= 0)


def test_lattice_symmetry():
    d = inputs.lattice(20)
    ctx, parts, g = gpu_hydro(d)
    assert (g["h"].max() - g["h"].min()) <= 2e-6 * g["h"].mean()
    assert np.all(g["n_ngb"] == g["n_ngb"][0])
    s = oracle_state(g)
    check_density(g, s)
    a = np.sqrt(g["ax"] ** 2 + g["ay"] ** 2 + g["az"] ** 2)
    term = g["m"][0] * g["P"][0] / g["rho"][0] ** 2 / g["h"][0] ** 4
    assert a.max() < 1e-4 * term


def test_momentum_antisymmetry_gpu():
    d = _uniform_moving(30000, 9)
    ctx, parts, g = gpu_hydro(d)
    a = np.stack([g["ax"], g["ay"], g["az"]], axis=1).astype(np.float64)
    m = g["m"].astype(np.float64)[:, None]
    tot = np.abs((m * a).sum(axis=0))
    assert np.all(tot <= 1e-6 * (m * np.abs(a)).sum())


def test_deterministic():
    d = _uniform_moving(20000, 10)
    _, _, g1 = gpu_hydro(d)
    _, _, g2 = gpu_hydro(d)
    for k in ("rho", "h", "ax", "ay", "az", "dudt", "vsig", "n_ngb", "perm"):
        assert np.array_equal(g1[k], g2[k]), k


@pytest.mark.slow
def test_sedov_128_sampled():
    """Sedov-Taylor blast, 128^3 jittered lattice, full size in the launch
    configuration the bench times; sampled targets against the brute force."""
    d = inputs.sedov(128, seed=2)
    ctx, parts, g = gpu_hydro(d)
    s = oracle_state(g)
    rng = np.random.default_rng(7)
    hot = int(np.argmax(g["u"]))
    td = np.unique(np.concatenate([rng.choice(s.n, 2048, replace=False), [hot]]))
    dd = check_density(g, s, targets=td)
    check_ghost(g, s, dd, td)
    tf = np.unique(np.concatenate([rng.choice(s.n, 256, replace=False), [hot]]))
    check_force(g, s, targets=tf)


def test_step_matches_oracle():
    """Two KDK steps (fixed dt) on the GPU vs the oracle's integrator."""
    from paper_1508_00115_gb300 import binding
    n = 4000
    d = _uniform_moving(n, 12)
    ctx = binding.Context(n, h_tol=1e-6)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    g0 = parts.numpy()
    perm0 = ctx.permutation()
    s = oracle.State(x=g0["x"], y=g0["y"], z=g0["z"], vx=g0["vx"], vy=g0["vy"], vz=g0["vz"],
                     m=g0["m"].astype(np.float64), u=g0["u"].astype(np.float64),
                     h=g0["h"].astype(np.float64))
    acc = oracle.hydro(s)
    dt = 0.5 * oracle.cfl_dt(acc["h"], acc["vsig"])
    for _ in range(2):
        s, acc, _ = oracle.step(s, acc, dt)
        ctx.step(parts, dt)
    g = parts.numpy()
    perm = ctx.permutation()
    # map GPU slots back to the oracle's order (the oracle kept the first build's order)
    inv = np.empty(n, np.int64)
    inv[perm0] = np.arange(n)
    idx = inv[perm]
    for k in ("x", "y", "z"):
        dx = g[k] - getattr(s, k)[idx]
        dx -= np.rint(dx)
        assert np.abs(dx).max() < 1e-8
    vscale = np.sqrt(np.mean(s.vx ** 2 + s.vy ** 2 + s.vz ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - getattr(s, k)[idx]).max() < 1e-5 * vscale
    assert rel(g["u"], s.u[idx]).max() < 1e-5
    assert rel(g["h"], s.h[idx]).max() < 1e-5


def test_edge_cases():
    from paper_1508_00115_gb300 import binding
    # h beyond a third of the box cannot be held by a periodic grid
    d = inputs.uniform(200, seed=1)
    d["h"][:] = 0.4
    ctx = binding.Context(200)
    parts = binding.Particles(d)
    with pytest.raises(binding.SphError) as e:
        ctx.build_cells(parts)
    assert e.value.code == binding.SPH_ERR_H_EXCEEDS_CELL
    # non-converged: one pass from a poor guess
    d = inputs.uniform(5000, seed=2)
    d["h"] *= 0.5
    ctx = binding.Context(5000, max_h_iter=1)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    with pytest.raises(binding.SphError) as e:
        ctx.density(parts)
    assert e.value.code == binding.SPH_ERR_NOT_CONVERGED
    # force before density on the current positions
    ctx.build_cells(parts)
    with pytest.raises(binding.SphError) as e:
        ctx.force(parts)
    assert e.value.code == binding.SPH_ERR_STATE
    # empty set
    ctx0 = binding.Context(0)
    p0 = binding.Particles({k: np.zeros(0) for k in inputs.FIELDS})
    ctx0.build_cells(p0)
    assert ctx0.density(p0) == 0
    ctx0.force(p0)
    # NaN smoothing length
    d = inputs.uniform(300, seed=3)
    d["h"][5] = np.nan
    ctx = binding.Context(300)
    parts = binding.Particles(d)
    with pytest.raises(binding.SphError) as e:
        ctx.build_cells(parts)
    assert e.value.code == binding.SPH_ERR_NAN


def test_autotuned_schedule_parity():
    """The autotuner rebuilds cells with other tile widths / cell factors; results
    must still match the oracle."""
    from paper_1508_00115_gb300 import binding
    d = _uniform_moving(9000, 14)
    ctx, parts, g = gpu_hydro(d, flags=binding.SPH_FLAG_NGB_HASH | binding.SPH_FLAG_AUTOTUNE)
    assert g["stats"]["tile_width"] in (16, 32)
    s = oracle_state(g)
    dd = check_density(g, s)
    check_ghost(g, s, dd, np.arange(s.n))
    check_force(g, s)


@pytest.mark.parametrize("tw", [16, 32])
def test_tile_widths_parity(tw):
    d = _uniform_moving(7000, 15)
    ctx, parts, g = gpu_hydro(d, tile_width=tw, cell_factor=1.3)
    s = oracle_state(g)
    check_density(g, s)
    check_force(g, s)


def test_h_growth_forces_rebuild():
    """A guess far below the converged h forces cells to be rebuilt mid-iteration;
    the result still matches the oracle."""
    d = inputs.uniform(6000, seed=13)
    d["h"] *= 0.3
    ctx, parts, g = gpu_hydro(d)
    s = oracle_state(g)
    check_density(g, s)
    check_force(g, s)
