"""Pins of the gravity near-field oracle (Sec. 3.2, Eq. 3: the node-node tasks in
which all particles of a cell interact with all particles of the adjacent cells).

Each pin is chosen so that a plausible slip fails at least one of them: the
hand-derived two-body values (softened and not), Newton's third law (sum m a = 0),
a = -grad of the pair potential energy by central differences (catches a wrong
power of r or of the softening, a sign, m_i for m_j), the symmetry of an odd
periodic lattice (catches a wrong minimal image), dimensional scaling, and a
cell-by-cell enumeration of the near field on tiny inputs (catches a wrong
adjacency test)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state(x, y, z, m, box=1.0):
    n = len(x)
    z0 = np.zeros(n)
    return oracle.State(x=np.asarray(x, float), y=np.asarray(y, float), z=np.asarray(z, float), vx=z0, vy=z0,
                        vz=z0, m=np.asarray(m, float), u=np.ones(n), h=np.ones(n), box=box)


def _value(expr: str) -> float:
    return float(eval(expr, {"sqrt": math.sqrt}))


def test_two_body_golden():
    g = json.load(open(os.path.join(GOLDEN, "gravity_two_body.json")))["values"]
    s = _state([0.45, 0.55], [0.5, 0.5], [0.5, 0.5], [0.5, 0.25])
    for key, eps in (("eps0", 0.0), ("eps1_20", 0.05)):
        r = oracle.grav_p2p(s, 3, eps=eps)
        v = g[key]
        assert r["a"][0, 0] == pytest.approx(_value(v["a1x"]), rel=1e-14)
        assert r["a"][1, 0] == pytest.approx(_value(v["a2x"]), rel=1e-14)
        assert np.all(r["a"][:, 1:] == 0.0)
        assert r["phi"][0] == pytest.approx(_value(v["phi1"]), rel=1e-14)
        assert r["phi"][1] == pytest.approx(_value(v["phi2"]), rel=1e-14)
    s2 = _state([0.05, 0.55], [0.5, 0.5], [0.5, 0.5], [0.5, 0.25])
    r = oracle.grav_p2p(s2, 5)
    assert np.all(r["a"] == 0.0) and np.all(r["phi"] == 0.0)


def _random(n, seed, clustered=False):
    if clustered:
        d = inputs.plummer_mix(n, seed=seed, n_halos=3)
    else:
        d = inputs.uniform(n, seed=seed)
    m = np.random.default_rng(seed + 1).uniform(0.5, 2.0, n) / n
    return _state(d["x"], d["y"], d["z"], m)


@pytest.mark.parametrize("nc,eps", [(3, 0.0), (4, 0.01), (7, 0.002)])
def test_newtons_third_law(nc, eps):
    """The near-field pair set is symmetric (adjacency is), so sum_i m_i a_i = 0."""
    s = _random(1500, 11 + nc, clustered=nc == 7)
    r = oracle.grav_p2p(s, nc, eps=eps)
    p = (s.m[:, None] * r["a"]).sum(axis=0)
    assert np.abs(p).max() <= 1e-12 * np.sum(s.m * np.linalg.norm(r["a"], axis=1))


@pytest.mark.parametrize("nc,eps", [(3, 0.02), (5, 0.005)])
def test_force_is_minus_gradient_of_pair_energy(nc, eps):
    """W = 1/2 sum_i m_i phi_i; every pair appears once from each side, so moving
    particle k changes W by m_k times the change of its own phi_k.  Central
    differences of phi_k in each axis (no particle changes cell) give -a_k."""
    s = _random(600, 21 + nc)
    r = oracle.grav_p2p(s, nc, eps=eps)
    rng = np.random.default_rng(5)
    L = 1.0 / nc
    checked = 0
    for k in rng.choice(s.n, 40, replace=False):
        pos = np.array([s.x[k], s.y[k], s.z[k]])
        frac = pos / L - np.floor(pos / L)
        if np.any(np.minimum(frac, 1 - frac) < 1e-3):
            continue  # too close to a cell face
        sep = np.stack([s.x[k] - s.x, s.y[k] - s.y, s.z[k] - s.z])
        if np.min(np.abs(np.abs(sep - np.rint(sep)) - 0.5)) < 1e-5:
            continue  # a partner near half a box away: the minimal image has a kink there
        d = 1e-6
        for ax, arr in enumerate(("x", "y", "z")):
            sp, sm = s.copy(), s.copy()
            getattr(sp, arr)[k] += d
            getattr(sm, arr)[k] -= d
            g = (oracle.grav_p2p(sp, nc, eps=eps, targets=[k])["phi"][0]
                 - oracle.grav_p2p(sm, nc, eps=eps, targets=[k])["phi"][0]) / (2 * d)
            assert g == pytest.approx(-r["a"][k, ax], rel=1e-5, abs=1e-6 * np.abs(r["a"][k]).max())
        checked += 1
    assert checked >= 20
    # and W itself: the sum over pairs of -G m_i m_j / r_ij, each pair once
    W = 0.5 * np.sum(s.m * r["phi"])
    i, j = np.triu_indices(s.n, 1)
    cell = np.minimum(np.floor(np.stack([s.x, s.y, s.z]) / L).astype(int), nc - 1)
    dc = np.abs(cell[:, i] - cell[:, j])
    near = np.all((dc <= 1) | (dc == nc - 1), axis=0)
    d = np.stack([s.x[i] - s.x[j], s.y[i] - s.y[j], s.z[i] - s.z[j]])
    d -= np.rint(d)
    pair = -s.m[i] * s.m[j] / np.sqrt((d ** 2).sum(axis=0) + eps * eps)
    assert W == pytest.approx(pair[near].sum(), rel=1e-12)


def test_odd_periodic_lattice_has_no_net_force():
    """5^3 lattice, nc = 3 (every particle sees all others at their minimal images,
    offsets -2..2 spacings in each axis): zero acceleration by symmetry; every phi
    equal."""
    k = (np.arange(5) + 0.5) / 5
    X, Y, Z = np.meshgrid(k, k, k, indexing="ij")
    s = _state(X.ravel(), Y.ravel(), Z.ravel(), np.full(125, 1 / 125))
    r = oracle.grav_p2p(s, 3, eps=0.0)
    scale = 1 / 125 / 0.2 ** 2
    assert np.abs(r["a"]).max() <= 1e-12 * scale
    assert np.ptp(r["phi"]) <= 1e-13 * np.abs(r["phi"]).max()


def test_dimensional_scaling():
    """Positions, box and softening scaled by lam, masses by mu, G by g:
    a scales by g mu / lam^2, phi by g mu / lam."""
    s = _random(800, 31)
    r = oracle.grav_p2p(s, 4, G=1.0, eps=0.01)
    lam, mu, gg = 3.0, 0.5, 2.5
    t = _state(s.x * lam, s.y * lam, s.z * lam, s.m * mu, box=lam)
    q = oracle.grav_p2p(t, 4, G=gg, eps=0.01 * lam)
    np.testing.assert_allclose(q["a"], r["a"] * gg * mu / lam ** 2, rtol=1e-12, atol=1e-12 * np.abs(q["a"]).max())
    np.testing.assert_allclose(q["phi"], r["phi"] * gg * mu / lam, rtol=1e-12)


@pytest.mark.parametrize("nc", [3, 4, 6])
def test_near_field_enumerated_cell_by_cell(nc):
    """Tiny inputs: the near field gathered cell by cell (the set of the 27 cells
    around each particle's cell, then every particle in them) in plain Python gives
    the oracle's sums."""
    s = _random(150, 41 + nc, clustered=True)
    eps = 0.003
    L = 1.0 / nc
    cell = [tuple(min(int(math.floor(c / L)), nc - 1) for c in (s.x[i], s.y[i], s.z[i])) for i in range(s.n)]
    members = {}
    for i, c in enumerate(cell):
        members.setdefault(c, []).append(i)
    r = oracle.grav_p2p(s, nc, eps=eps)
    for i in range(s.n):
        near = {((cell[i][0] + a) % nc, (cell[i][1] + b) % nc, (cell[i][2] + c) % nc)
                for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
        acc = [0.0, 0.0, 0.0]
        phi = 0.0
        for c in near:
            for j in members.get(c, []):
                if j == i:
                    continue
                d = [s.x[i] - s.x[j], s.y[i] - s.y[j], s.z[i] - s.z[j]]
                d = [v - round(v) for v in d]
                r2 = sum(v * v for v in d) + eps * eps
                inv = 1 / math.sqrt(r2)
                for k in range(3):
                    acc[k] -= s.m[j] * d[k] * inv ** 3
                phi -= s.m[j] * inv
        np.testing.assert_allclose(r["a"][i], acc, rtol=1e-11, atol=1e-11 * max(abs(v) for v in acc))
        assert r["phi"][i] == pytest.approx(phi, rel=1e-12)


def test_unsoftened_coincident_pair_contributes_nothing():
    s = _state([0.3, 0.3, 0.6], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [1.0, 1.0, 1.0])
    r = oracle.grav_p2p(s, 3, eps=0.0)
    assert np.all(np.isfinite(r["a"])) and np.all(np.isfinite(r["phi"]))
    # particles 0 and 1 see only particle 2, at 0.3
    assert r["a"][0, 0] == pytest.approx(1 / 0.09, rel=1e-12)
    assert r["phi"][0] == pytest.approx(-1 / 0.3, rel=1e-12)
