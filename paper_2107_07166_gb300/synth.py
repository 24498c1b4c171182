"""Seeded synthetic particle sets (inputs only: no FMM arithmetic lives here).

Both the CUDA path and the CPU oracle are fed from these generators so that they see
identical bytes.  Units: G = 1, total mass 1 per system unless stated.  Every set is
shifted so that its centre of mass is at the origin.

* Plummer sphere (scale radius a): radii by inverting the cumulative mass
  M(<r) = r^3 / (r^2 + a^2)^(3/2), i.e. r = a (u^(-2/3) - 1)^(-1/2), with u drawn
  uniformly in (0, u_max] (u_max = 0.999 cuts the extended halo); isotropic directions;
  speeds q * v_esc with q drawn from q^2 (1 - q^2)^(7/2) by rejection.
* Hernquist sphere (scale a): M(<r) = r^2 / (r + a)^2, r = a sqrt(u) / (1 - sqrt(u)).
* Exponential disk + Hernquist bulge (the rotating galaxy workload).
* Binary of two Plummer spheres.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cz = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * np.pi * rng.random(n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def _centre(x: np.ndarray, m: np.ndarray) -> np.ndarray:
    c = (m[:, None] * x).sum(axis=0) / m.sum()
    return x - c


def plummer(n: int, seed: int, a: float = 1.0, mass: float = 1.0, u_max: float = 0.999,
            velocities: bool = False):
    """Plummer sphere of n equal-mass particles.  Returns (x[n,3], m[n]) or (x, m, v)."""
    rng = _rng(seed)
    u = u_max * (1.0 - rng.random(n))          # (0, u_max]
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    m = np.full(n, mass / n)
    x = _centre(x, m)
    if not velocities:
        return x, m
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        q1 = rng.random(todo.size)
        q2 = 0.1 * rng.random(todo.size)
        ok = q2 < q1 * q1 * (1.0 - q1 * q1) ** 3.5
        q[todo[ok]] = q1[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0 * mass / a) * (1.0 + (r / a) ** 2) ** -0.25
    v = (q * vesc)[:, None] * _isotropic(rng, n)
    v -= v.mean(axis=0)
    return x, m, v


def hernquist(n: int, seed: int, a: float = 1.0, mass: float = 1.0, u_max: float = 0.999):
    """Hernquist sphere of n equal-mass particles.  Returns (x[n,3], m[n])."""
    rng = _rng(seed)
    u = u_max * (1.0 - rng.random(n))
    su = np.sqrt(u)
    r = a * su / (1.0 - su)
    x = r[:, None] * _isotropic(rng, n)
    m = np.full(n, mass / n)
    return _centre(x, m), m


def disk_bulge(n: int, seed: int, rd: float = 1.0, z0: float = 0.1, f_disk: float = 0.8,
               a_bulge: float = 0.2, velocities: bool = False):
    """Exponential disk (surface density ~ exp(-R/rd), cut at 10 rd; vertical
    sech^2(z/z0)) holding f_disk of the mass, plus a Hernquist bulge.  Total mass 1.
    With velocities, disk particles rotate on circular orbits about z at the speed
    sqrt(M(<r) / r) of the spherically averaged enclosed mass and bulge particles get an
    isotropic direction at half that speed: a rotating galaxy with net angular momentum."""
    rng = _rng(seed)
    nd = int(round(f_disk * n))
    nb = n - nd
    # cylindrical radius from the Gamma(2) cumulative 1 - (1 + s) e^-s, by bisection
    u = rng.random(nd) * (1.0 - 11.0 * np.exp(-10.0))
    lo, hi = np.zeros(nd), np.full(nd, 10.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        f = 1.0 - (1.0 + mid) * np.exp(-mid)
        lo = np.where(f < u, mid, lo)
        hi = np.where(f < u, hi, mid)
    R = rd * 0.5 * (lo + hi)
    ph = 2.0 * np.pi * rng.random(nd)
    w = rng.random(nd)
    z = z0 * np.arctanh(2.0 * w - 1.0 + 1e-16 * (0.5 - w))   # sech^2 vertical profile
    xd = np.stack([R * np.cos(ph), R * np.sin(ph), z], axis=1)
    ub = 0.999 * (1.0 - rng.random(nb))
    sb = np.sqrt(ub)
    rb = a_bulge * sb / (1.0 - sb)
    xb = rb[:, None] * _isotropic(rng, nb)
    x = np.concatenate([xd, xb], axis=0)
    m = np.concatenate([np.full(nd, f_disk / max(nd, 1)), np.full(nb, (1.0 - f_disk) / max(nb, 1))])
    x = _centre(x, m)
    if not velocities:
        return x, m
    r = np.linalg.norm(x, axis=1)
    order = np.argsort(r, kind="stable")
    menc = np.empty(n)
    menc[order] = np.cumsum(m[order])
    vc = np.sqrt(menc / np.maximum(r, 1e-12))
    v = np.zeros_like(x)
    v[:nd, 0] = -vc[:nd] * np.sin(ph)
    v[:nd, 1] = vc[:nd] * np.cos(ph)
    v[nd:] = (0.5 * vc[nd:])[:, None] * _isotropic(rng, nb)
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return x, m, v


def binary(n_each: int, seed_a: int, seed_b: int, separation: float = 10.0):
    """Two Plummer spheres (mass 1 each) at (+-separation/2, 0, 0)."""
    xa, ma = plummer(n_each, seed_a)
    xb, mb = plummer(n_each, seed_b)
    xa = xa + np.array([0.5 * separation, 0.0, 0.0])
    xb = xb - np.array([0.5 * separation, 0.0, 0.0])
    x = np.concatenate([xa, xb])
    m = np.concatenate([ma, mb])
    return _centre(x, m), m


def clusters_pair(n_each: int, seed: int, distance: float):
    """Two irregular clusters (unions of five Gaussian blobs, unit size), each shifted to its
    own mean, with centres `distance` apart along x: a stand-in for the two-shape test.
    Every particle has mass 1 / (2 n_each)."""
    rng = _rng(seed)
    out = []
    for s in (-0.5, 0.5):
        nb = 5
        centres = rng.normal(size=(nb, 3)) * 0.3
        scales = 0.1 + 0.2 * rng.random(nb)
        which = rng.integers(0, nb, n_each)
        x = centres[which] + rng.normal(size=(n_each, 3)) * scales[which, None]
        x -= x.mean(axis=0)
        out.append(x + np.array([s * distance, 0.0, 0.0]))
    x = np.concatenate(out)
    m = np.full(x.shape[0], 1.0 / x.shape[0])
    return x, m


def batch_sizes(n_sys: int, seed: int, n_min: int = 1024, n_max: int = 65536):
    """Particle counts and profiles (True: Plummer) of the systems of batch(n_sys, seed)."""
    rng = _rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_sys))).astype(np.int64)
    kinds = rng.random(n_sys) < 0.5
    return sizes, kinds


def batch_subset(n_sys: int, seed: int, idx, n_min: int = 1024, n_max: int = 65536):
    """The systems idx (increasing) of batch(n_sys, seed, n_min, n_max), concatenated:
    the same particles as the matching slices of the full batch.
    Returns (x[N, 3], m[N], offsets[len(idx) + 1])."""
    sizes, kinds = batch_sizes(n_sys, seed, n_min, n_max)
    idx = np.asarray(idx, dtype=np.int64)
    xs, ms = [], []
    for i in idx:
        gen = plummer if kinds[i] else hernquist
        x, m = gen(int(sizes[i]), seed + 1 + int(i))
        xs.append(x)
        ms.append(m)
    off = np.concatenate([[0], np.cumsum(sizes[idx])]).astype(np.int64)
    if not xs:
        return np.zeros((0, 3)), np.zeros(0), off
    return np.concatenate(xs), np.concatenate(ms), off


def batch(n_sys: int, seed: int, n_min: int = 1024, n_max: int = 65536):
    """Independent systems concatenated: system i has N_i = floor(exp U(ln n_min, ln n_max))
    particles, a Plummer or a Hernquist (a = 1) profile by a coin flip, seed seed + i.
    Returns (x[N, 3], m[N], offsets[n_sys + 1])."""
    return batch_subset(n_sys, seed, np.arange(n_sys), n_min, n_max)
