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
    # a step over the pass budget completes (force and closing kick included) and
    # reports the status at its end: the state stays consistent for the next call
    ctx.force(parts)
    before = parts.numpy()
    perm0 = ctx.permutation()
    dt = 1e-4
    ctx.step(parts, dt, allow=(binding.SPH_ERR_NOT_CONVERGED,))
    after = parts.numpy()
    assert all(np.all(np.isfinite(after[k])) for k in ("x", "vx", "ax", "rho", "h"))
    i0, i1 = np.argsort(perm0), np.argsort(ctx.permutation())
    dx = after["x"][i1] - before["x"][i0] - (before["vx"][i0] + before["ax"][i0].astype(np.float64) * dt / 2) * dt
    assert np.abs(dx - np.rint(dx)).max() < 1e-12  # drifted by (v + a dt/2) dt
    with pytest.raises(binding.SphError) as e:
        ctx.step(parts, dt)
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


def test_radius_two_stencil():
    """Cells planned for a guess at 0.7x the converged h (jittered lattice, nearly
    uniform h): the converged h reach past one cell but stay within two, so the
    passes use the radius-2 stencil instead of re-binning."""
    d = inputs.lattice(20, jitter=0.3, seed=16)
    d["h"] *= 0.7
    ctx, parts, g = gpu_hydro(d, cell_factor=1.0)
    assert g["stats"]["rebuilds"] == 0
    assert g["h"].max() > g["stats"]["cell_size"]
    s = oracle_state(g)
    check_density(g, s)
    check_force(g, s)


def _boxes(sizes, seed):
    """Independent periodic unit boxes of uneven occupancy, concatenated; equal
    masses 1/N_box; random velocities."""
    parts, offs = [], [0]
    for k, nb in enumerate(sizes):
        b = inputs.random_velocities(inputs.uniform(nb, seed=seed + k), 0.2, seed + 50 + k)
        parts.append(b)
        offs.append(offs[-1] + nb)
    d = {k: np.concatenate([b[k] for b in parts]) for k in inputs.FIELDS}
    return d, offs


def test_batched_boxes_match_each_box_alone():
    """Several uneven periodic boxes in one context (one launch per pass): every
    box must match the oracle run on that box alone."""
    sizes = [1200, 5000, 300 + 17, 9000]
    d, offs = _boxes(sizes, 60)
    ctx, parts, g = gpu_hydro(d, box_offsets=offs)
    perm = g["perm"]
    for b in range(len(sizes)):
        sl = np.arange(offs[b], offs[b + 1])
        assert np.all((perm[sl] >= offs[b]) & (perm[sl] < offs[b + 1]))  # boxes stay contiguous
        sub = {k: g[k][sl] for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "rho", "P", "c", "f",
                                     "divv", "curl", "n_ngb", "ax", "ay", "az", "dudt", "vsig")}
        sub["perm"] = perm[sl]
        sub["ngb_hash"] = g["ngb_hash"][sl]
        s = oracle_state(sub)
        dd = check_density(sub, s)
        check_force(sub, s)


def _state_equal(g1, g2, perm1, perm2, rtol):
    i1 = np.argsort(perm1)
    i2 = np.argsort(perm2)
    for k in ("x", "y", "z"):
        dx = g1[k][i1] - g2[k][i2]
        dx -= np.rint(dx)
        assert np.abs(dx).max() < 1e-9, k
    for k in ("vx", "vy", "vz"):
        scale = np.abs(g1[k]).max() + 1e-30
        assert np.abs(g1[k][i1] - g2[k][i2]).max() <= rtol * scale, k
    assert rel(g1["u"][i1], g2["u"][i2]).max() <= rtol
    assert rel(g1["h"][i1], g2["h"][i2]).max() <= rtol


@pytest.mark.parametrize("dt", [0.0, 4e-4])
def test_graph_steps_match_host_steps(dt):
    """sph_steps (one captured step replayed) against sph_step called in a loop."""
    from paper_1508_00115_gb300 import binding
    d = _uniform_moving(6000, 17)
    out = []
    for mode in ("host", "graph"):
        ctx = binding.Context(d["x"].size, h_tol=1e-6)
        parts = binding.Particles(d)
        if mode == "host":
            for _ in range(3):
                ctx.step(parts, dt)
        else:
            ctx.steps(parts, 3, dt)
            assert ctx.stats()["graph_steps"] == 3
        out.append((parts.numpy(), ctx.permutation()))
    (g1, p1), (g2, p2) = out
    _state_equal(g1, g2, p1, p2, 1e-5)


def test_graph_steps_batched_boxes_match_oracle():
    """Batched boxes stepped by the captured graph, each box against the oracle's
    integrator (common dt)."""
    from paper_1508_00115_gb300 import binding
    sizes = [3000, 1500, 4500]
    d, offs = _boxes(sizes, 80)
    ctx = binding.Context(d["x"].size, box_offsets=offs, h_tol=1e-6)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    ctx.density(parts)
    ctx.force(parts)
    g0 = parts.numpy()
    perm0 = ctx.permutation()
    dt = 0.5 * min(float(np.min(g0["h"][g0["vsig"] > 0] / g0["vsig"][g0["vsig"] > 0])) * 0.1, 1e9)
    ctx.steps(parts, 2, dt)
    g = parts.numpy()
    perm = ctx.permutation()
    for b in range(len(sizes)):
        sl0 = np.arange(offs[b], offs[b + 1])
        s = oracle.State(**{k: g0[k][sl0].astype(np.float64) for k in inputs.FIELDS})
        acc = oracle.hydro(s)
        for _ in range(2):
            s, acc, _ = oracle.step(s, acc, dt)
        # GPU slots of box b, mapped to the first build's order inside the box
        sl = np.arange(offs[b], offs[b + 1])
        inv = np.empty(d["x"].size, np.int64)
        inv[perm0] = np.arange(d["x"].size)
        idx = inv[perm[sl]] - offs[b]
        for k in ("x", "y", "z"):
            dx = g[k][sl] - getattr(s, k)[idx]
            dx -= np.rint(dx)
            assert np.abs(dx).max() < 1e-8
        vscale = np.sqrt(np.mean(s.vx ** 2 + s.vy ** 2 + s.vz ** 2))
        for k in ("vx", "vy", "vz"):
            assert np.abs(g[k][sl] - getattr(s, k)[idx]).max() < 1e-5 * vscale
        assert rel(g["u"][sl], s.u[idx]).max() < 1e-5


@pytest.mark.parametrize("tw", [16, 32])
def test_axis_sweep_parity(tw):
    """SPH_FLAG_AXIS_SWEEP: neighbour cells read along the axis joining the two cells,
    up to the projected cutoff; results must match the oracle like the default."""
    from paper_1508_00115_gb300 import binding
    d = _uniform_moving(15000, 33)
    ctx, parts, g = gpu_hydro(d, flags=binding.SPH_FLAG_NGB_HASH | binding.SPH_FLAG_AXIS_SWEEP, tile_width=tw)
    s = oracle_state(g)
    dd = check_density(g, s)
    check_ghost(g, s, dd, np.arange(s.n))
    check_force(g, s)
    # a few steps with the sweep on (cells rebuilt and re-sorted every step)
    for _ in range(2):
        ctx.step(parts, 2e-4)


@pytest.mark.parametrize("pin,adaptive", [(True, False), (False, False), (True, True)])
def test_step_host_matches_device_step(pin, adaptive):
    """sph_step_host (host arrays, copies inside the call -- the results go back on a
    second stream as soon as the step is done with them) gives exactly what sph_step
    gives on device arrays: the same kernels in the same order."""
    from paper_1508_00115_gb300 import binding
    if adaptive:
        d = inputs.random_velocities(inputs.plummer_mix(8000, seed=93, n_halos=4), 0.2, 94)
    else:
        d = _uniform_moving(5000, 91)
    n = d["x"].size
    dt = 3e-4
    fl = binding.SPH_FLAG_ADAPTIVE if adaptive else 0
    ctx_d = binding.Context(n, h_tol=1e-6, flags=fl)
    pd = binding.Particles(d)
    ctx_h = binding.Context(n, h_tol=1e-6, flags=fl)
    ph = binding.Particles(d, device="cpu", pin=pin)
    for k in range(3):
        used_d, cons_d = ctx_d.step(pd, dt if k else 0.0)
        used_h, cons_h = ctx_h.step_host(ph, dt if k else 0.0)
        assert used_d == used_h
        assert cons_d["e_tot"] == cons_h["e_tot"]
    gd, gh = pd.numpy(), ph.numpy()
    for key in gd:
        assert np.array_equal(gd[key], gh[key]), key
    assert np.array_equal(ctx_d.permutation(), ctx_h.permutation())
