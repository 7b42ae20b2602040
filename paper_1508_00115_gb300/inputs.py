"""Seeded synthetic particle sets shaped like the paper's workloads.

This module serves BOTH the CUDA path (bench, tests) and the FP64 oracle; it
holds none of the SPH arithmetic -- only random numbers and geometry of the
initial conditions.  Every generator uses numpy's PCG64 (``default_rng``) with
an explicit seed and returns FP64 SoA arrays:

    x, y, z, vx, vy, vz, m, u, h   (h = initial smoothing-length guess)

The paper measures on an EAGLE cosmological snapshot (Sec. 3.1, Fig. 4) that is
not available here; these seeded distributions stand in for it (uniform gas, a
jittered lattice with a point explosion, and a clustered halo field whose
smoothing lengths span about three decades).
"""
from __future__ import annotations

import math

import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")


def h_guess(n: int, box: float = 1.0, n_ngb: float = 48.0) -> float:
    """Radius of the sphere that holds n_ngb particles at the mean density."""
    return (3.0 * n_ngb / (4.0 * math.pi * n)) ** (1.0 / 3.0) * box


def _pack(x, y, z, vx, vy, vz, m, u, h):
    return dict(x=np.ascontiguousarray(x, np.float64), y=np.ascontiguousarray(y, np.float64),
                z=np.ascontiguousarray(z, np.float64), vx=np.ascontiguousarray(vx, np.float64),
                vy=np.ascontiguousarray(vy, np.float64), vz=np.ascontiguousarray(vz, np.float64),
                m=np.ascontiguousarray(m, np.float64), u=np.ascontiguousarray(u, np.float64),
                h=np.ascontiguousarray(h, np.float64))


def uniform(n: int, seed: int = 1, box: float = 1.0, u0: float = 1.0,
            vel_sigma: float = 0.0, n_ngb: float = 48.0) -> dict:
    """n equal-mass (1/n) particles, uniform-random in a periodic box, u = u0.
    Optional Gaussian velocities of dispersion vel_sigma (0 = at rest)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n)) * box
    if vel_sigma > 0:
        vel = rng.normal(0.0, vel_sigma, (3, n))
    else:
        vel = np.zeros((3, n))
    m = np.full(n, 1.0 / n)
    u = np.full(n, u0)
    h = np.full(n, h_guess(n, box, n_ngb))
    return _pack(pos[0], pos[1], pos[2], vel[0], vel[1], vel[2], m, u, h)


def lattice(n_side: int, box: float = 1.0, jitter: float = 0.0, seed: int = 0,
            u0: float = 1.0, n_ngb: float = 48.0) -> dict:
    """Cubic lattice of n_side^3 points at ((i + 1/2) + jitter*U(-1/2,1/2)) * box/n_side."""
    a = box / n_side
    g = (np.arange(n_side) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    if jitter > 0:
        rng = np.random.default_rng(seed)
        pos = pos + (rng.random(pos.shape) - 0.5) * jitter * a
        pos = np.mod(pos, box)
    n = pos.shape[1]
    z0 = np.zeros(n)
    return _pack(pos[0], pos[1], pos[2], z0, z0.copy(), z0.copy(), np.full(n, 1.0 / n),
                 np.full(n, u0), np.full(n, h_guess(n, box, n_ngb)))


def sedov(n_side: int = 128, seed: int = 2, u_bg: float = 1e-5, u_hot: float = 1.0) -> dict:
    """Sedov-Taylor point explosion: n_side^3 jittered lattice (spacing 1/n_side plus
    a uniform jitter of total width 0.1 spacing), rho = 1, v = 0, u = u_bg except the
    particle nearest the box centre, which gets u_hot."""
    d = lattice(n_side, 1.0, jitter=0.1, seed=seed, u0=u_bg)
    r2 = (d["x"] - 0.5) ** 2 + (d["y"] - 0.5) ** 2 + (d["z"] - 0.5) ** 2
    d["u"][int(np.argmin(r2))] = u_hot
    return d


def plummer_mix(n: int, seed: int = 3, box: float = 1.0, n_halos: int = 200,
                f_halo: float = 0.7, a_min: float = 1e-3, a_max: float = 1e-2,
                mass_slope: float = -1.9, m_lo: float = 1.0, m_hi: float = 100.0,
                r_trunc: float = 10.0, u0: float = 1.0, n_ngb: float = 48.0) -> dict:
    """Clustered halo field: a fraction f_halo of n particles in n_halos Plummer
    spheres (centres uniform, scale radii log-uniform in [a_min, a_max], halo masses
    from dN/dM ~ M^mass_slope on [m_lo, m_hi], particle counts proportional to mass,
    radii from the Plummer inverse CDF truncated at r_trunc * a, isotropic
    directions), the rest uniform; periodic wrap; equal masses 1/n; v = 0."""
    rng = np.random.default_rng(seed)
    n_halo_tot = int(round(f_halo * n))
    centres = rng.random((n_halos, 3)) * box
    scale = np.exp(rng.uniform(math.log(a_min), math.log(a_max), n_halos)) * box
    # inverse CDF of a power law p(M) ~ M^s on [m_lo, m_hi] (s != -1)
    s1 = mass_slope + 1.0
    uu = rng.random(n_halos)
    masses = (m_lo ** s1 + uu * (m_hi ** s1 - m_lo ** s1)) ** (1.0 / s1)
    counts = np.floor(masses / masses.sum() * n_halo_tot).astype(np.int64)
    counts[: n_halo_tot - counts.sum()] += 1
    parts = []
    for c, a, k in zip(centres, scale, counts):
        if k == 0:
            continue
        # Plummer enclosed-mass fraction X = r^3/(r^2+a^2)^(3/2), truncated at r_trunc*a
        x_max = r_trunc ** 3 / (r_trunc ** 2 + 1.0) ** 1.5
        X = rng.random(k) * x_max
        r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        v = rng.normal(size=(k, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        parts.append(c + v * r[:, None])
    halo = np.concatenate(parts, axis=0) if parts else np.zeros((0, 3))
    bg = rng.random((n - halo.shape[0], 3)) * box
    pos = np.mod(np.concatenate([halo, bg], axis=0), box).T
    perm = rng.permutation(n)
    pos = pos[:, perm]
    z0 = np.zeros(n)
    return _pack(pos[0], pos[1], pos[2], z0, z0.copy(), z0.copy(), np.full(n, 1.0 / n),
                 np.full(n, u0), np.full(n, h_guess(n, box, n_ngb)))


def random_velocities(d: dict, sigma: float, seed: int) -> dict:
    """Copy of d with Gaussian velocities of dispersion sigma."""
    rng = np.random.default_rng(seed)
    out = {k: v.copy() for k, v in d.items()}
    v = rng.normal(0.0, sigma, (3, out["x"].size))
    out["vx"], out["vy"], out["vz"] = v[0], v[1], v[2]
    return out
