"""FP64 brute-force CPU oracle for the SPH neighbour sums -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never imports the CUDA package and
the CUDA package never imports it; the two share only the seeded input
generators (``paper_1508_00115_gb300/inputs.py``, which holds none of the
method's arithmetic).

What each function follows (Theuns et al. 2015, "Swift: task-based
hydrodynamics and gravity for cosmological simulations"):

* :func:`density_at_h`, :func:`solve_h` -- Sec. 2, Eq. 1 (density), the
  smoothing-length criterion in the sentence after Eq. 2, and the velocity
  divergence / curl estimates the viscosity switch needs.
* :func:`ghost` -- Sec. 2: equation of state and "density before pressure
  gradient"; the grad-h factor of the Gadget-2 formulation the paper adopts.
* :func:`force` -- Sec. 2, Eq. 2 in the Gadget-2 form, with artificial
  viscosity.
* :func:`step` -- Sec. 2, the time integration of the particles: a
  kick-drift-kick leapfrog (the integrator is not named in the paper).
* :func:`time_bins`, :func:`step_bins` -- the same leapfrog with individual,
  power-of-two time-steps (the Gadget-2 scheme the paper's force law comes from;
  the paper itself is silent on time-stepping).
* :func:`grav_p2p` -- Sec. 3.2, Eq. 3: the near-field gravity tasks in which all
  particles of a cell interact with all particles of the adjacent cells
  (softened, minimal image).

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, OpenMP over targets,
``-ffp-contract=off``); this file only marshals arrays and composes the step.
Parity pins: ``tests/test_oracle_pins.py``, for the individual time-steps
``tests/test_oracle_bins.py``, for the gravity near field
``tests/test_oracle_gravity.py`` (no function here is unpinned).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FOUR_PI_3 = 4.0 * np.pi / 3.0


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        lib.orc_w.restype = d
        lib.orc_w.argtypes = [d]
        lib.orc_dw.restype = d
        lib.orc_dw.argtypes = [d]
        lib.orc_wrap.restype = None
        lib.orc_wrap.argtypes = [i64, d, P]
        lib.orc_cell_key.restype = i64
        lib.orc_cell_key.argtypes = [d, d, d, d, i64]
        lib.orc_hash_id.restype = ctypes.c_uint64
        lib.orc_hash_id.argtypes = [ctypes.c_uint64]
        lib.orc_density_at_h.restype = ctypes.c_int
        lib.orc_density_at_h.argtypes = [i64, d] + [P] * 8 + [i64, P, P, P, P, P]
        lib.orc_solve_h.restype = ctypes.c_int
        lib.orc_solve_h.argtypes = ([i64, d] + [P] * 7 + [P, d, d, d, i64, P, P]
                                    + [P, P, P, P, P])
        lib.orc_ghost.restype = None
        lib.orc_ghost.argtypes = [i64] + [P] * 6 + [d, ctypes.c_int] + [P] * 4
        lib.orc_force.restype = ctypes.c_int
        lib.orc_force.argtypes = ([i64, d] + [P] * 7 + [P] * 6 + [d, i64, P]
                                  + [P] * 6)
        lib.orc_grav_p2p.restype = ctypes.c_int
        lib.orc_grav_p2p.argtypes = [i64, d, P, P, P, P, i64, d, d, i64, P, P, P, P, P]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def w(q: float) -> float:
    """Cubic-spline shape w(q), support q <= 1 (normalised: int 4 pi q^2 w = 1)."""
    return float(_load().orc_w(float(q)))


def dw(q: float) -> float:
    """dw/dq of the cubic-spline shape."""
    return float(_load().orc_dw(float(q)))


def hash_id(i: int) -> int:
    """splitmix64 finaliser of a particle id (neighbour-set fingerprint term)."""
    return int(_load().orc_hash_id(ctypes.c_uint64(int(i))))


def wrap(x: np.ndarray, box: float) -> np.ndarray:
    """Periodic wrap into [0, box) (FP64)."""
    out = _f64(x).copy()
    _load().orc_wrap(out.size, float(box), _p(out))
    return out


def cell_keys(x, y, z, box: float, nc: int) -> np.ndarray:
    """Linear cell key (iz*nc+iy)*nc+ix of each wrapped position."""
    lib = _load()
    return np.array([lib.orc_cell_key(float(a), float(b), float(c), float(box), int(nc))
                     for a, b, c in zip(x, y, z)], dtype=np.int64)


@dataclass
class State:
    """Particle state, FP64 SoA.  ``box`` is the periodic box side."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    u: np.ndarray
    h: np.ndarray
    box: float = 1.0
    ids: np.ndarray | None = field(default=None)

    @property
    def n(self) -> int:
        return int(self.x.size)

    def copy(self) -> "State":
        return State(*(np.array(getattr(self, k), dtype=np.float64) for k in
                       ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")),
                     box=self.box,
                     ids=None if self.ids is None else self.ids.copy())

    def _arrs(self):
        return [_f64(getattr(self, k)) for k in ("x", "y", "z", "vx", "vy", "vz", "m")]


def _targets(n, targets):
    if targets is None:
        return None, n
    t = np.ascontiguousarray(targets, dtype=np.int64)
    return t, int(t.size)


def _ids(s: State):
    if s.ids is None:
        return None
    return np.ascontiguousarray(s.ids, dtype=np.uint64)


def density_at_h(s: State, h=None, targets=None) -> dict:
    """Eq. 1 and companions at the given smoothing lengths (default s.h).

    Returns dict of arrays over targets: rho, nw, dnw_dh, drho_dh, divv, curl (n,3),
    curl_abs, n_ngb, ngb_hash.
    """
    lib = _load()
    h = _f64(s.h if h is None else h)
    t, nt = _targets(s.n, targets)
    out = np.zeros((nt, 8))
    nngb = np.zeros(nt, dtype=np.int64)
    hh = np.zeros(nt, dtype=np.uint64)
    arrs = s._arrs()
    ids = _ids(s)
    lib.orc_density_at_h(s.n, float(s.box), *[_p(a) for a in arrs], _p(h), nt, _p(t),
                         _p(ids), _p(out), _p(nngb), _p(hh))
    return _density_dict(out, nngb, hh)


def _density_dict(out, nngb, hh):
    curl = out[:, 5:8].copy()
    return dict(rho=out[:, 0].copy(), nw=out[:, 1].copy(), dnw_dh=out[:, 2].copy(),
                drho_dh=out[:, 3].copy(), divv=out[:, 4].copy(), curl=curl,
                curl_abs=np.sqrt((curl * curl).sum(axis=1)), n_ngb=nngb, ngb_hash=hh)


def solve_h(s: State, h_guess=None, n_ngb: float = 48.0, tol: float = 1e-12,
            h_max: float | None = None, targets=None) -> dict:
    """Smoothing lengths with N_w(h) = n_ngb (Newton + bisection), plus the density
    sums at the solved h.  Returns the density_at_h dict plus 'h' and 'iters'."""
    lib = _load()
    hg = _f64(s.h if h_guess is None else h_guess)
    t, nt = _targets(s.n, targets)
    if h_max is None:
        h_max = s.box / 2.0
    hout = np.zeros(nt)
    iters = np.zeros(nt, dtype=np.int32)
    out = np.zeros((nt, 8))
    nngb = np.zeros(nt, dtype=np.int64)
    hh = np.zeros(nt, dtype=np.uint64)
    arrs = s._arrs()
    ids = _ids(s)
    bad = lib.orc_solve_h(s.n, float(s.box), *[_p(a) for a in arrs], _p(hg), float(n_ngb),
                          float(tol), float(h_max), nt, _p(t), _p(ids), _p(hout), _p(iters),
                          _p(out), _p(nngb), _p(hh))
    if bad:
        raise RuntimeError(f"oracle: {bad} smoothing lengths exceed h_max={h_max}")
    d = _density_dict(out, nngb, hh)
    d["h"] = hout
    d["iters"] = iters
    return d


def ghost(rho, drho_dh, divv, curl_abs, u, h, gamma: float = 5.0 / 3.0,
          use_balsara: bool = True) -> dict:
    """P, c, f (grad-h) and Balsara B per particle."""
    lib = _load()
    arrs = [_f64(a) for a in (rho, drho_dh, divv, curl_abs, u, h)]
    n = arrs[0].size
    P, c, f, B = (np.zeros(n) for _ in range(4))
    lib.orc_ghost(n, *[_p(a) for a in arrs], float(gamma), int(bool(use_balsara)),
                  _p(P), _p(c), _p(f), _p(B))
    return dict(P=P, c=c, f=f, B=B)


def force(s: State, h, rho, P, c, f, B, alpha: float = 0.8, targets=None) -> dict:
    """Pressure-gradient + viscosity sums (Gadget-2 form of Eq. 2).  Per-particle
    inputs are full-length arrays; outputs are over targets."""
    lib = _load()
    t, nt = _targets(s.n, targets)
    ins = [_f64(a) for a in (h, rho, P, c, f, B)]
    ax, ay, az, dudt, vsig = (np.zeros(nt) for _ in range(5))
    npairs = np.zeros(nt, dtype=np.int64)
    arrs = s._arrs()
    lib.orc_force(s.n, float(s.box), *[_p(a) for a in arrs], *[_p(a) for a in ins],
                  float(alpha), nt, _p(t), _p(ax), _p(ay), _p(az), _p(dudt), _p(vsig),
                  _p(npairs))
    return dict(a=np.stack([ax, ay, az], axis=1), dudt=dudt, vsig=vsig, n_pairs=npairs)


@dataclass
class Params:
    gamma: float = 5.0 / 3.0
    n_ngb: float = 48.0
    alpha: float = 0.8
    cfl: float = 0.1
    use_balsara: bool = True
    h_tol: float = 1e-12


def hydro(s: State, p: Params = Params(), h_guess=None) -> dict:
    """Density (with h solve), ghost and force for every particle."""
    d = solve_h(s, h_guess=h_guess, n_ngb=p.n_ngb, tol=p.h_tol)
    g = ghost(d["rho"], d["drho_dh"], d["divv"], d["curl_abs"], s.u, d["h"], p.gamma,
              p.use_balsara)
    fr = force(s, d["h"], d["rho"], g["P"], g["c"], g["f"], g["B"], p.alpha)
    out = dict(d)
    out.update(g)
    out.update(fr)
    return out


def cfl_dt(h, vsig, cfl: float = 0.1) -> float:
    """dt = C_CFL min_i h_i / vsig_i over particles with vsig_i > 0."""
    h = _f64(h)
    v = _f64(vsig)
    ok = v > 0
    return float(cfl * np.min(h[ok] / v[ok])) if ok.any() else float("inf")


def conserved(s: State) -> dict:
    """Total momentum, kinetic and thermal energy (FP64)."""
    mv = np.array([np.sum(s.m * s.vx), np.sum(s.m * s.vy), np.sum(s.m * s.vz)])
    ek = float(np.sum(0.5 * s.m * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2)))
    eu = float(np.sum(s.m * s.u))
    return dict(momentum=mv, e_kin=ek, e_th=eu, e_tot=ek + eu)


def step(s: State, acc: dict, dt: float, p: Params = Params()) -> tuple[State, dict, int]:
    """One kick-drift-kick step.  ``acc`` holds the hydro result at the start of the
    step (keys a, dudt, h).  The hydro pass at the end of the drift sees velocities
    and internal energies predicted to the synchronised time,
    v_pred = v_half + a_old dt/2 and u_pred = u_half + (du/dt)_old dt/2 (the
    Gadget-2 prediction; the paper names no integrator).  Internal energy is floored
    at 0 after each kick and prediction; the number of floored values is returned.
    Returns (new state, new hydro, floors)."""
    n2 = s.copy()
    a = acc["a"]
    floors = 0
    half = 0.5 * dt
    n2.vx = n2.vx + a[:, 0] * half
    n2.vy = n2.vy + a[:, 1] * half
    n2.vz = n2.vz + a[:, 2] * half
    n2.u = n2.u + acc["dudt"] * half
    floors += int(np.sum(n2.u < 0))
    n2.u = np.maximum(n2.u, 0.0)
    n2.x = wrap(n2.x + n2.vx * dt, s.box)
    n2.y = wrap(n2.y + n2.vy * dt, s.box)
    n2.z = wrap(n2.z + n2.vz * dt, s.box)
    pred = n2.copy()
    pred.vx = n2.vx + a[:, 0] * half
    pred.vy = n2.vy + a[:, 1] * half
    pred.vz = n2.vz + a[:, 2] * half
    pred.u = np.maximum(n2.u + acc["dudt"] * half, 0.0)
    res = hydro(pred, p, h_guess=acc["h"])
    n2.h = res["h"].copy()
    a2 = res["a"]
    n2.vx = n2.vx + a2[:, 0] * half
    n2.vy = n2.vy + a2[:, 1] * half
    n2.vz = n2.vz + a2[:, 2] * half
    n2.u = n2.u + res["dudt"] * half
    floors += int(np.sum(n2.u < 0))
    n2.u = np.maximum(n2.u, 0.0)
    return n2, res, floors


def time_bins(h, vsig, dt_max: float, n_bins: int, s_now: int, cfl: float = 0.1):
    """Time bins of particles that start a step at integer time s_now (unit
    dt_max / 2^n_bins).  Bin b means a step of dt_max / 2^b: the largest such step not
    above the particle's CFL step cfl h / vsig (bin n_bins if even that one is
    above it; those are counted), then made smaller until s_now is a multiple of
    the step's length, so that every step starts and ends on its own grid.
    Returns (bins, number of particles whose CFL step is below the smallest bin,
    margin): margin is the smallest distance, in log2, of a CFL step from a bin
    boundary dt_max / 2^k inside the range of bins (inf if none), i.e. how far the
    decisions are from flipping."""
    h = _f64(h)
    v = _f64(vsig)
    dtc = np.full(h.size, np.inf)
    ok = v > 0
    dtc[ok] = cfl * h[ok] / v[ok]
    b = np.full(h.size, n_bins, dtype=np.int64)
    for k in range(n_bins, -1, -1):  # ends at the smallest k that fits
        b = np.where(dt_max * 2.0 ** (-k) <= dtc, k, b)
    over = int(np.sum(dt_max * 2.0 ** (-n_bins) > dtc))
    lg = np.log2(dt_max / dtc[ok]) if ok.any() else np.zeros(0)
    lg = lg[(lg > -1.0) & (lg < n_bins + 1.0)]
    margin = float(np.min(np.abs(lg - np.rint(lg)))) if lg.size else float("inf")
    for i in range(h.size):
        while b[i] < n_bins and s_now % (1 << (n_bins - b[i])) != 0:
            b[i] += 1
    return b, over, margin


def _neighbours(s: State, h, idx):
    """For each particle i of idx, every j != i with r_ij < max(h_i, h_j) (the pairs
    of the force sum, Eq. 8), r_ij^2 in the operation order of the plain definition:
    dx = x_i - x_j, minimal image dx - box rint(dx / box), r^2 = (dx^2 + dy^2) + dz^2."""
    out = []
    for i in idx:
        d = []
        for c in ("x", "y", "z"):
            v = getattr(s, c)
            dd = v[i] - v
            dd = dd - s.box * np.rint(dd / s.box)
            d.append(dd)
        r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        hh = np.maximum(h[i] * h[i], h * h)
        nb = np.nonzero(r2 < hh)[0]
        out.append(nb[nb != i])
    return out


def limit_bins(s: State, h, bins, active, T, s_now: int, n_bins: int, levels: int = 2):
    """Time-step limiter with wake-up (Saitoh & Makino 2009; the paper is silent on
    time-stepping) at integer time s_now, after the particles whose step ends there
    (``active``) took their CFL bins.

    Neighbours are the pairs of the force sum, r_ij < max(h_i, h_j).  The bins are
    raised to the least fixed point, reached by Jacobi sweeps from the given ones, of
      active i:    b_i = max(b_i, max over all neighbours j of b_j - levels)
      inactive j:  b_j = max(b_j, max over active neighbours i of b_i - levels),
    so that afterwards no pair with an active member has bins more than ``levels``
    apart.  (An active particle's bin already divides s_now, and a larger bin still
    does.)  An inactive particle whose raised bin's step D' = 2^(n_bins - b) ends
    before its current step, at T' = (s_now // D' + 1) D' < T, is woken: its step is
    cut to end at T'.

    Returns (bins, T, limited: active particles whose bin was raised, woken: mask of
    the particles whose step was cut).  The caller corrects the cut particles'
    opening half kick by (T' - T) / 2."""
    bins = np.array(bins, dtype=np.int64)
    T = np.array(T, dtype=np.int64)
    act = np.asarray(active, dtype=bool)
    everyone = np.arange(s.n)
    ngb = _neighbours(s, h, everyone)
    start = bins.copy()
    while True:
        prev = bins.copy()
        for i in everyone:
            g = ngb[i] if act[i] else ngb[i][act[ngb[i]]]
            if g.size:
                bins[i] = max(prev[i], int(prev[g].max()) - levels)
        if np.array_equal(bins, prev):
            break
    limited = int(np.sum(act & (bins != start)))
    D = np.left_shift(1, n_bins - bins)
    Tn = (s_now // D + 1) * D
    woken = ~act & (Tn < T)
    T[woken] = Tn[woken]
    return bins, T, limited, woken


def step_bins(s: State, acc: dict, dt_max: float, n_bins: int,
              p: Params = Params(), limiter: int | None = None) -> tuple[State, dict, dict]:
    """Advance by dt_max with individual time-steps: the kick-drift-kick leapfrog of
    :func:`step` per particle, each on its own power-of-two step (:func:`time_bins`).

    ``acc`` is the hydro result of a synchronised state (keys a, dudt, vsig, h, rho,
    P, c, f, B).  Time runs on an integer grid of dt_max / 2^n_bins; every particle
    carries the start s0 and end T of its current step.  At the start every particle
    takes its opening half kick.  Then, from one step end to the next: all particles
    drift to the smallest T; the particles whose step ends there are active; the
    density (with the h solve) and the force are evaluated for the active ones only,
    against every particle at its drifted position, with velocities and internal
    energies predicted to the current time (v_half + a (t - t_mid), t_mid = (s0 + T)
    / 2 the middle of the particle's own step), while the inactive particles keep h,
    rho, P, c, f and B from their last evaluation; the active ones take their closing
    half kick (T - s0) / 2, a new bin, and (before dt_max is reached) the opening half
    kick of their next step.  At dt_max every particle is synchronised again.

    ``limiter`` (levels, e.g. 2: no step more than 4 times a neighbour's): after the
    active particles (all of them at the start) take their CFL bins, the bins are
    raised by :func:`limit_bins` (Saitoh & Makino 2009), and every inactive particle
    whose step it cut takes the difference of its opening half kick, v += a (T' - T)
    dt-unit / 2 and u likewise (floored at 0, counted).
    ``limiter=None`` is the scheme without them.

    Returns (state, hydro dict of the final synchronised state, stats with
    floors, substeps, active (particle updates), over (CFL steps below the
    smallest bin), margin (the closest any bin decision came to a boundary, in
    log2), bins (the bins of the last steps), kicked (each particle's half-kick
    lengths summed, in units: 2^(n_bins + 1) when its steps tile the interval), and
    with a limiter limited (bins raised by it) and woken (wake-ups))."""
    B = int(n_bins)
    unit = dt_max / 2.0 ** B
    end = 1 << B
    n2 = s.copy()
    st = {k: np.array(acc[k], dtype=np.float64) for k in ("h", "rho", "P", "c", "f", "B", "dudt", "vsig")}
    st["a"] = np.array(acc["a"], dtype=np.float64)
    n2.h = st["h"].copy()
    floors = 0
    limited = 0
    woken = 0
    kicked = np.zeros(s.n, dtype=np.int64)  # each particle's half-kick lengths, summed

    def kick(idx, length):
        """v += a L/2 dt-unit, u likewise (floored), for the particles idx."""
        nonlocal floors
        kicked[idx] += np.asarray(length, dtype=np.int64)
        half = 0.5 * (np.asarray(length, dtype=np.int64).astype(np.float64) * unit)
        n2.vx[idx] = n2.vx[idx] + st["a"][idx, 0] * half
        n2.vy[idx] = n2.vy[idx] + st["a"][idx, 1] * half
        n2.vz[idx] = n2.vz[idx] + st["a"][idx, 2] * half
        u = n2.u[idx] + st["dudt"][idx] * half
        floors += int(np.sum(u < 0))
        n2.u[idx] = np.maximum(u, 0.0)

    def limit(act, bins, S):
        """The limiter and wake-up at S (:func:`limit_bins`); the cut steps' opening
        half kicks corrected to their new length."""
        nonlocal limited, woken, T
        if limiter is None:
            return bins
        bins, Tn, nl, wk = limit_bins(n2, st["h"], bins, act, T, S, B, limiter)
        idx = np.nonzero(wk)[0]
        kick(idx, Tn[idx] - T[idx])
        T = Tn
        limited += nl
        woken += int(idx.size)
        return bins

    everyone = np.arange(s.n)
    bins, over, margin = time_bins(st["h"], st["vsig"], dt_max, B, 0, p.cfl)
    s0 = np.zeros(s.n, dtype=np.int64)
    T = np.zeros(s.n, dtype=np.int64)
    bins = limit(np.ones(s.n, dtype=bool), bins, 0)
    T[:] = np.left_shift(1, B - bins)
    kick(everyone, T - s0)
    S = 0
    substeps = 0
    updates = 0
    while S < end:
        S_next = int(T.min())
        dt = (S_next - S) * unit
        n2.x = wrap(n2.x + n2.vx * dt, s.box)
        n2.y = wrap(n2.y + n2.vy * dt, s.box)
        n2.z = wrap(n2.z + n2.vz * dt, s.box)
        S = S_next
        substeps += 1
        act = T == S
        idx = np.nonzero(act)[0]
        updates += int(idx.size)
        tau = 0.5 * ((2 * S - s0 - T).astype(np.float64) * unit)
        pred = n2.copy()
        pred.vx = n2.vx + st["a"][:, 0] * tau
        pred.vy = n2.vy + st["a"][:, 1] * tau
        pred.vz = n2.vz + st["a"][:, 2] * tau
        pred.u = np.maximum(n2.u + st["dudt"] * tau, 0.0)
        d = solve_h(pred, h_guess=st["h"], n_ngb=p.n_ngb, tol=p.h_tol, targets=idx)
        g = ghost(d["rho"], d["drho_dh"], d["divv"], d["curl_abs"], pred.u[idx], d["h"], p.gamma,
                  p.use_balsara)
        st["h"][idx] = d["h"]
        st["rho"][idx] = d["rho"]
        for k in ("P", "c", "f", "B"):
            st[k][idx] = g[k]
        fr = force(pred, st["h"], st["rho"], st["P"], st["c"], st["f"], st["B"], p.alpha, targets=idx)
        st["a"][idx] = fr["a"]
        st["dudt"][idx] = fr["dudt"]
        st["vsig"][idx] = fr["vsig"]
        n2.h[idx] = d["h"]
        kick(idx, T[idx] - s0[idx])  # closing half kick on the step that ends now
        nb, o, mg = time_bins(st["h"][idx], st["vsig"][idx], dt_max, B, S, p.cfl)
        over += o
        margin = min(margin, mg)
        bins[idx] = nb
        if S < end:
            bins = limit(act, bins, S)
            s0[idx] = S
            T[idx] = S + np.left_shift(1, B - bins[idx])
            kick(idx, T[idx] - s0[idx])  # opening half kick of the next step
    stats = dict(floors=floors, substeps=substeps, active=updates, over=over, margin=margin, bins=bins,
                 kicked=kicked)
    if limiter is not None:
        stats.update(limited=limited, woken=woken)
    return n2, st, stats


def grav_p2p(s: State, nc: int, G: float = 1.0, eps: float = 0.0, targets=None) -> dict:
    """Near-field gravity of Sec. 3.2 (Eq. 3, Plummer-softened, minimal image): for
    each target, the sum over every other particle in its own cell and the 26
    adjacent cells of the periodic nc^3 grid.  Returns a (nt, 3) and phi (nt)."""
    lib = _load()
    t, nt = _targets(s.n, targets)
    a = np.zeros((3, nt))
    phi = np.zeros(nt)
    rc = lib.orc_grav_p2p(s.n, float(s.box), _p(_f64(s.x)), _p(_f64(s.y)), _p(_f64(s.z)), _p(_f64(s.m)),
                          int(nc), float(G), float(eps), nt, _p(t), _p(a[0]), _p(a[1]), _p(a[2]), _p(phi))
    if rc:
        raise RuntimeError(f"orc_grav_p2p failed ({rc})")
    return {"a": np.ascontiguousarray(a.T), "phi": phi}
