"""Pins of the oracle's individual time-steps (oracle.time_bins, oracle.step_bins).

The scheme must reduce to the pinned global leapfrog where it has no choice to
make: with one level it is one global step of dt_max; when every particle sits in
the same bin b it is 2^b global steps of dt_max / 2^b.  Groups of particles that do
not interact evolve as if simulated alone, whatever bins the other group takes.
The bin rule itself is checked on hand cases.
"""
import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import inputs


def _state(d):
    return oracle.State(**{k: np.asarray(d[k], np.float64) for k in inputs.FIELDS})


def _moving(n, seed, sigma=0.3):
    d = inputs.uniform(n, seed=seed)
    d = inputs.random_velocities(d, sigma, seed + 100)
    d["u"] = np.random.default_rng(seed + 200).uniform(0.5, 2.0, n)
    return d


def test_time_bins_rule():
    """Bin b = largest dt_max/2^b not above cfl h/vsig; the smallest bin if none is;
    bin 0 without a signal velocity; then smaller until s is a multiple of 2^(L-b)."""
    cfl = 0.1
    h = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    dtc = np.array([1.0, 0.5, 0.49, 0.126, 0.01, np.inf])  # cfl h / vsig
    vsig = np.where(np.isfinite(dtc), cfl * h / np.where(np.isfinite(dtc), dtc, 1.0), 0.0)
    b, over, margin = oracle.time_bins(h, vsig, 1.0, 3, 0, cfl)
    assert list(b) == [0, 1, 2, 3, 3, 0]
    assert over == 1  # 0.01 < 1/8
    # alignment: at s = 4 (L = 3) steps of 8 units cannot start, steps of 4 can;
    # at s = 6 only steps of 2 or 1
    b4, _, _ = oracle.time_bins(h, vsig, 1.0, 3, 4, cfl)
    assert list(b4) == [1, 1, 2, 3, 3, 1]
    b6, _, _ = oracle.time_bins(h, vsig, 1.0, 3, 6, cfl)
    assert list(b6) == [2, 2, 2, 3, 3, 2]
    b7, _, _ = oracle.time_bins(h, vsig, 1.0, 3, 7, cfl)
    assert list(b7) == [3] * 6
    # 0.5 sits on a boundary
    assert margin == pytest.approx(0.0, abs=1e-12)


@pytest.fixture(scope="module")
def moving_hydro():
    s = _state(_moving(400, 11))
    acc = oracle.hydro(s)
    return s, acc


def _same(a: oracle.State, b: oracle.State, tol):
    for k in ("x", "y", "z"):
        d = getattr(a, k) - getattr(b, k)
        d -= np.rint(d)
        assert np.abs(d).max() <= tol
    for k in ("vx", "vy", "vz", "u", "h"):
        x, y = getattr(a, k), getattr(b, k)
        assert np.abs(x - y).max() <= tol * max(1.0, np.abs(y).max())


def test_single_level_is_the_global_step(moving_hydro):
    s, acc = moving_hydro
    dt = 0.5 * oracle.cfl_dt(acc["h"], acc["vsig"])
    g, gacc, _ = oracle.step(s, acc, dt)
    b, bacc, st = oracle.step_bins(s, acc, dt, 0)
    assert st["substeps"] == 1 and st["active"] == s.n
    _same(b, g, 1e-13)
    assert np.abs(bacc["a"] - gacc["a"]).max() <= 1e-12 * np.abs(gacc["a"]).max()


def test_one_shared_bin_is_repeated_global_steps():
    """All CFL steps between dt_max/4 and dt_max/2: every particle stays in bin 2,
    and the run is four global steps of dt_max/4."""
    d = inputs.random_velocities(inputs.lattice(8, 1.0, jitter=0.3, seed=8, u0=1.0), 0.05, 9)
    s = _state(d)
    acc = oracle.hydro(s)
    dtc = 0.1 * acc["h"] / acc["vsig"]
    assert dtc.max() < 1.6 * dtc.min()  # one octave holds them
    dt_max = 3.0 * dtc.min()
    b, bacc, st = oracle.step_bins(s, acc, dt_max, 4)
    assert np.all(st["bins"] == 2) and st["substeps"] == 4 and st["active"] == 4 * s.n
    g, gacc = s, acc
    for _ in range(4):
        g, gacc, _ = oracle.step(g, gacc, dt_max / 4)
    _same(b, g, 1e-12)


def test_groups_that_do_not_interact_evolve_alone():
    """A hot clump and a cold clump, far apart in the periodic box: the hot one takes
    small steps, the cold one large ones, and each evolves exactly as when it is
    alone (up to the rounding of drifts taken in pieces)."""
    hot = inputs.lattice(6, 0.12, jitter=0.1, seed=3, u0=1.0)
    cold = inputs.lattice(6, 0.12, jitter=0.1, seed=4, u0=0.02)
    for d, off in ((hot, 0.19), (cold, 0.69)):
        for k in ("x", "y", "z"):
            d[k] = d[k] + off
        d["m"] = np.full(d["x"].size, 1.0 / 432)
    hot = inputs.random_velocities(hot, 0.2, 5)
    cold = inputs.random_velocities(cold, 0.02, 6)
    both = {k: np.concatenate([hot[k], cold[k]]) for k in inputs.FIELDS}
    sb = _state(both)
    ab = oracle.hydro(sb)
    # clumps 0.5 apart with sides 0.12: no particle's support reaches the other clump
    assert ab["h"].max() < 0.15
    na = hot["x"].size
    dt_max = 6.0 * oracle.cfl_dt(ab["h"], ab["vsig"])
    rb, _, stb = oracle.step_bins(sb, ab, dt_max, 4)
    assert stb["bins"][:na].min() > stb["bins"][na:].max()  # the hot clump steps finer
    for sl, d in ((slice(0, na), hot), (slice(na, None), cold)):
        s1 = _state(d)
        a1 = oracle.hydro(s1)
        r1, _, _ = oracle.step_bins(s1, a1, dt_max, 4)
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
            x = getattr(rb, k)[sl]
            y = getattr(r1, k)
            assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max()), k


def test_all_in_the_top_bin_is_one_global_step(moving_hydro):
    """Every CFL step above dt_max: every particle takes bin 0 whatever the depth of
    the grid, and the call is one global step of dt_max."""
    s, acc = moving_hydro
    dt = 0.5 * oracle.cfl_dt(acc["h"], acc["vsig"])
    g, _, _ = oracle.step(s, acc, dt)
    b, _, st = oracle.step_bins(s, acc, dt, 5)
    assert np.all(st["bins"] == 0) and st["substeps"] == 1 and st["active"] == s.n
    _same(b, g, 1e-13)


def test_individual_steps_converge_at_second_order():
    """Against a fine global-step reference over the same interval, halving every
    particle's step (C_CFL / 2, the same hierarchy one level deeper) cuts the error
    about 4x: the per-particle leapfrog with neighbours predicted from the middle of
    their own steps stays second order (predicting them to their step ends instead
    falls to first order: ~2x)."""
    d = inputs.random_velocities(inputs.uniform(600, seed=41), 0.3, 42)
    d["u"] = np.random.default_rng(43).uniform(0.5, 2.0, 600)
    r2 = (d["x"] - 0.5) ** 2 + (d["y"] - 0.5) ** 2 + (d["z"] - 0.5) ** 2
    d["u"][r2 < 0.25 ** 2] *= 30.0  # a hot region: bins spread over three levels
    s = _state(d)
    acc = oracle.hydro(s)
    T = 4.0 * float(np.max(0.1 * acc["h"] / acc["vsig"]))
    g, ga = s, acc
    for _ in range(256):
        g, ga, _ = oracle.step(g, ga, T / 256)
    ev, eu = [], []
    for cfl in (0.2, 0.1, 0.05):
        b, _, st = oracle.step_bins(s, acc, T, 8, oracle.Params(cfl=cfl))
        assert len(np.unique(st["bins"])) >= 3 and st["over"] == 0
        ev.append(np.sqrt(np.mean((b.vx - g.vx) ** 2 + (b.vy - g.vy) ** 2 + (b.vz - g.vz) ** 2)))
        eu.append(np.abs(b.u - g.u).max())
    for k in range(2):
        assert eu[k] / eu[k + 1] > 3.2, eu
        assert ev[k] / ev[k + 1] > 2.8, ev
