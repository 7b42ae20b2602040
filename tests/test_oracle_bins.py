"""Pins of the oracle's individual time-steps (oracle.time_bins, oracle.step_bins).

The scheme must reduce to the pinned global leapfrog where it has no choice to
make: with one level it is one global step of dt_max; when every particle sits in
the same bin b it is 2^b global steps of dt_max / 2^b.  Groups of particles that do
not interact evolve as if simulated alone, whatever bins the other group takes.
The bin rule itself is checked on hand cases.

The time-step limiter with wake-up (Saitoh & Makino 2009) is pinned on a hand case
whose fixed point is worked out below, by the properties that define it on random
inputs (neighbour sets brute-forced here in another form of the minimal image),
by changing nothing where it has nothing to limit, and by what it is for: a blast
running into cold gas whose particles sleep on long steps.
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


@pytest.mark.parametrize("limiter", [None, 2])
def test_individual_steps_converge_at_second_order(limiter):
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
        b, _, st = oracle.step_bins(s, acc, T, 8, oracle.Params(cfl=cfl), limiter=limiter)
        assert len(np.unique(st["bins"])) >= 3 and st["over"] == 0
        ev.append(np.sqrt(np.mean((b.vx - g.vx) ** 2 + (b.vy - g.vy) ** 2 + (b.vz - g.vz) ** 2)))
        eu.append(np.abs(b.u - g.u).max())
    for k in range(2):
        assert eu[k] / eu[k + 1] > 3.2, eu
        assert ev[k] / ev[k + 1] > 2.8, ev


def _pairs_brute(s, h):
    """Neighbour matrix r_ij < max(h_i, h_j), j != i: separations per axis as
    min(|d|, box - |d|) (another form of the minimal image)."""
    r2 = np.zeros((s.n, s.n))
    for c in ("x", "y", "z"):
        v = getattr(s, c)
        d = np.abs(v[:, None] - v[None, :])
        d = np.minimum(d, s.box - d)
        r2 += d * d
    hm = np.maximum(h[:, None], h[None, :])
    m = r2 < hm * hm
    np.fill_diagonal(m, False)
    return m


def test_limit_bins_hand_case():
    """Four particles on a line, h = 0.1, spacing 0.08 (each one's neighbours are the
    next ones; A and C are 0.16 apart: not neighbours), 2^6 units per dt_max, now s =
    16 and levels = 2.  A is active with CFL bin 5; B, asleep in bin 0 (its step ends
    at 64), must rise to 5 - 2 = 3 and is woken: a bin-3 step is 8 units, so its step
    now ends at 24.  C is active with CFL bin 0 (at s = 16 only bins >= 2 start a
    step, so the caller gives it at least 2): B's new bin 3 pulls it to 1 -- no, to
    max(2, 3 - 2) = 2, unchanged.  D asleep in bin 4 (step ending at 20) is C's
    neighbour: 4 - 2 = 2 <= C's 2, and C, active, raises nobody above its own
    level minus 2.  A second pass with C at bin 4 (CFL) pulls D nowhere (4 - 2 = 2 <
    4) and B to max(3, 2) = 3."""
    x = np.array([0.30, 0.38, 0.46, 0.54])
    d = {"x": x, "y": np.full(4, 0.5), "z": np.full(4, 0.5)}
    for k in ("vx", "vy", "vz"):
        d[k] = np.zeros(4)
    d.update(m=np.ones(4), u=np.ones(4), h=np.full(4, 0.1))
    s = _state(d)
    h = d["h"]
    act = np.array([True, False, True, False])
    T = np.array([0, 64, 0, 20])
    bins, Tn, lim, wk = oracle.limit_bins(s, h, [5, 0, 2, 4], act, T, 16, 6, 2)
    assert list(bins) == [5, 3, 2, 4] and list(Tn) == [0, 24, 0, 20]
    assert lim == 0 and list(wk) == [False, True, False, False]
    # C at bin 4: D (bin 4) needs nothing, B is held at 3 by A
    bins, Tn, lim, wk = oracle.limit_bins(s, h, [5, 0, 4, 4], act, T, 16, 6, 2)
    assert list(bins) == [5, 3, 4, 4] and list(Tn) == [0, 24, 0, 20] and lim == 0
    # A coarse (bin 2) and D very fine (bin 6, asleep): C (active) rises to 6 - 2 = 4;
    # then C wakes B: 4 - 2 = 2 > 0, a bin-2 step is 16 units: its step ends at 32
    bins, Tn, lim, wk = oracle.limit_bins(s, h, [2, 0, 2, 6], act, np.array([0, 64, 0, 17]), 16, 6, 2)
    assert list(bins) == [2, 2, 4, 6] and list(Tn) == [0, 32, 0, 17]
    assert lim == 1 and list(wk) == [False, True, False, False]
    # one level: the chain D(6) -> C(5) -> B(4) -> A(3), B woken to a 4-unit step
    bins, Tn, lim, wk = oracle.limit_bins(s, h, [2, 0, 2, 6], act, np.array([0, 64, 0, 17]), 16, 6, 1)
    assert list(bins) == [3, 4, 5, 6] and list(Tn) == [0, 20, 0, 17] and lim == 2


def test_limit_bins_is_the_least_fixed_point():
    """Random positions, h, bins and activity: afterwards no pair with an active
    member is more than `levels` bins apart, no bin went down, every raised bin is
    exactly some neighbour's bin minus `levels` (nothing is raised further than a
    constraint asks: the least fixed point), and exactly the inactive particles whose
    raised step ends before their old one were cut, to the first end after now."""
    rng = np.random.default_rng(5)
    n, B, now = 300, 10, 3 * 64
    d = inputs.uniform(n, seed=77)
    d["h"] = rng.uniform(0.05, 0.15, n)
    s = _state(d)
    act = rng.random(n) < 0.4
    b0 = rng.integers(0, 5, n)
    b0[rng.random(n) < 0.05] = 9  # a few very fine particles
    b0[act] = np.maximum(b0[act], 4)  # active bins divide now = 3 * 2^6: bins >= 4
    D0 = np.left_shift(1, B - b0)
    T0 = np.where(act, 0, (now // D0 + 1) * D0)
    for L in (1, 2, 3):
        bins, T, lim, wk = oracle.limit_bins(s, d["h"], b0, act, T0, now, B, L)
        m = _pairs_brute(s, d["h"])
        assert np.all(bins >= b0)
        i, j = np.nonzero(m)
        sel = act[i]
        assert np.all(bins[i[sel]] >= bins[j[sel]] - L)
        assert np.all(bins[j[sel]] >= bins[i[sel]] - L)
        for k in np.nonzero(bins != b0)[0]:
            g = np.nonzero(m[k])[0]
            if not act[k]:
                g = g[act[g]]
            assert bins[k] == bins[g].max() - L
        assert lim == int(np.sum(act & (bins != b0)))
        D = np.left_shift(1, B - bins)
        cut = ~act & ((now // D + 1) * D < T0)
        assert np.array_equal(wk, cut)
        assert np.all(T[cut] > now) and np.all(T[cut] % D[cut] == 0) and np.all(T[cut] - now <= D[cut])
        assert np.array_equal(T[~cut], T0[~cut])
        assert cut.any() and lim > 0


def test_limiter_changes_nothing_in_one_bin():
    d = inputs.random_velocities(inputs.lattice(8, 1.0, jitter=0.3, seed=8, u0=1.0), 0.05, 9)
    s = _state(d)
    acc = oracle.hydro(s)
    dt_max = 3.0 * float(np.min(0.1 * acc["h"] / acc["vsig"]))
    a, _, sa = oracle.step_bins(s, acc, dt_max, 4)
    b, _, sb = oracle.step_bins(s, acc, dt_max, 4, limiter=2)
    assert sb["limited"] == 0 and sb["woken"] == 0 and sb["active"] == sa["active"]
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def test_limiter_keeps_groups_that_do_not_interact_apart():
    """The clumps of the test above, the cold one much colder: their bins end up
    further apart than the limiter lets neighbours be, and each clump still evolves
    exactly as when it is alone."""
    hot = inputs.lattice(6, 0.12, jitter=0.1, seed=3, u0=1.0)
    cold = inputs.lattice(6, 0.12, jitter=0.1, seed=4, u0=0.0005)
    for d, off in ((hot, 0.19), (cold, 0.69)):
        for k in ("x", "y", "z"):
            d[k] = d[k] + off
        d["m"] = np.full(d["x"].size, 1.0 / 432)
    hot = inputs.random_velocities(hot, 0.2, 5)
    cold = inputs.random_velocities(cold, 0.001, 6)
    both = {k: np.concatenate([hot[k], cold[k]]) for k in inputs.FIELDS}
    sb = _state(both)
    ab = oracle.hydro(sb)
    na = hot["x"].size
    dt_max = 40.0 * oracle.cfl_dt(ab["h"], ab["vsig"])
    rb, _, stb = oracle.step_bins(sb, ab, dt_max, 7, limiter=2)
    assert np.all(stb["kicked"] == 2 << 7)
    assert stb["bins"][:na].min() > stb["bins"][na:].max() + 2  # further apart than the limiter allows
    for sl, d in ((slice(0, na), hot), (slice(na, None), cold)):
        s1 = _state(d)
        a1 = oracle.hydro(s1)
        r1, _, _ = oracle.step_bins(s1, a1, dt_max, 7, limiter=2)
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
            x, y = getattr(rb, k)[sl], getattr(r1, k)
            assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max()), k


def test_limiter_lets_a_blast_wake_cold_gas():
    """A hot sphere (u = 10) in cold gas at rest (u = 1e-4): the cold particles'
    CFL steps are ~350 times the hot ones', so without the limiter the blast reaches
    particles that sleep through it.  Against 256 global steps over the same
    interval, the limiter cuts the velocity error by more than an order of
    magnitude; it raises bins and wakes sleepers to do so."""
    n = 600
    d = inputs.uniform(n, seed=41)
    for k in ("vx", "vy", "vz"):
        d[k] = np.zeros(n)
    d["u"] = np.full(n, 1e-4)
    r2 = (d["x"] - 0.5) ** 2 + (d["y"] - 0.5) ** 2 + (d["z"] - 0.5) ** 2
    d["u"][r2 < 0.12 ** 2] = 10.0
    s = _state(d)
    acc = oracle.hydro(s)
    dtc = 0.1 * acc["h"] / acc["vsig"]
    assert dtc.max() > 300 * dtc.min()
    T = 32 * dtc.min()
    g, ga = s, acc
    for _ in range(256):
        g, ga, _ = oracle.step(g, ga, T / 256)
    err = {}
    for lim in (None, 2):
        b, _, st = oracle.step_bins(s, acc, T, 8, limiter=lim)
        # each particle's steps, cut ones included, tile [0, T]: its opening and
        # closing half kicks add up to twice the interval
        assert np.all(st["kicked"] == 2 << 8)
        err[lim] = np.sqrt(np.mean((b.vx - g.vx) ** 2 + (b.vy - g.vy) ** 2 + (b.vz - g.vz) ** 2))
        if lim:
            assert st["limited"] > 0 and st["woken"] > 0
    vrms = np.sqrt(np.mean(g.vx ** 2 + g.vy ** 2 + g.vz ** 2))
    assert err[None] > 0.02 * vrms  # sleeping through the blast
    assert err[2] < 0.05 * err[None] and err[2] < 1e-3 * vrms
