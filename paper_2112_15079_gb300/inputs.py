"""Seeded synthetic initial conditions shaped like the paper's Solar-System model.

The paper's model (Section 2) is the Sun, 30 major bodies heavier than 1e19 kg,
over a hundred minor moons around the planets, and main-belt asteroids with
masses uniform in [1e12, 3e17] kg, taken from JPL HORIZONS on 2019-12-22 in a
Sun-centred ecliptic frame.  Those data are not available here, so this module
draws seeded stand-ins with the same structure:

* ``major_bodies``  -- Sun (1 Msun, at rest at the origin) + 30 bodies, masses
  log-uniform in [1e19, 2e27] kg, semi-major axes log-uniform in [0.3, 40] AU,
  e ~ U[0, 0.25], i ~ U[0, 8] deg, node/periapsis/mean anomaly ~ U[0, 2pi).
* ``moons``         -- circular orbits of radius log-uniform in [1e-4, 5e-2] AU
  around hosts drawn (with replacement) from the major bodies heavier than
  1e23 kg, masses ~ U[1e15, 1e19] kg.
* ``asteroids``     -- a ~ U[2.1, 3.3] AU, e ~ U[0, 0.3], i ~ U[0, 20] deg,
  masses ~ U[1e12, 3e17] kg.

This module holds input construction only (Kepler-element to Cartesian
conversion); it contains none of the force or integrator arithmetic.  Units:
AU, day, solar mass, with ``G_AU_DAY`` below.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

#: Gaussian gravitational constant squared, AU^3 Msun^-1 day^-2.
G_AU_DAY = 2.9591220828e-4
#: IAU nominal solar mass in kg (only used to convert the mass ranges).
MSUN_KG = 1.98847e30
#: Step size of the paper's runs, in days.
DT_DAY = 0.1
#: Base seed of every workload (the paper's epoch, 2019-12-22).
BASE_SEED = 20191222


@dataclass
class System:
    """One N-body system in structure-of-arrays form (float64)."""

    r: np.ndarray  # [3, n] positions, AU
    v: np.ndarray  # [3, n] velocities, AU/day
    m: np.ndarray  # [n] masses, Msun
    G: float = G_AU_DAY
    dt: float = DT_DAY
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def kepler_to_cartesian(a, e, inc, node, peri, mean_anom, mu):
    """Position and velocity [3, k] of Keplerian orbits (elliptic, e < 1).

    Solves Kepler's equation E - e sin E = M by Newton's method, then rotates
    the perifocal state by R_z(node) R_x(inc) R_z(peri)."""
    a, e, inc, node, peri, M, mu = (np.asarray(t, dtype=np.float64)
                                    for t in (a, e, inc, node, peri, mean_anom, mu))
    E = M + e * np.sin(M)
    for _ in range(60):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.max(np.abs(dE), initial=0.0) < 1e-15:
            break
    cE, sE = np.cos(E), np.sin(E)
    q = np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = a * q * sE
    nmean = np.sqrt(mu / a**3)
    den = 1.0 - e * cE
    vxp = -a * nmean * sE / den
    vyp = a * nmean * q * cE / den
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    p1 = (cO * cw - sO * sw * ci, sO * cw + cO * sw * ci, sw * si)
    p2 = (-cO * sw - sO * cw * ci, -sO * sw + cO * cw * ci, cw * si)
    r = np.stack([p1[k] * xp + p2[k] * yp for k in range(3)])
    v = np.stack([p1[k] * vxp + p2[k] * vyp for k in range(3)])
    return r, v


def major_bodies(rng, G=G_AU_DAY, count=30):
    """Sun at the origin plus ``count`` major bodies on heliocentric orbits."""
    m_kg = _loguniform(rng, 1e19, 2e27, count)
    m = m_kg / MSUN_KG
    a = _loguniform(rng, 0.3, 40.0, count)
    e = rng.uniform(0.0, 0.25, count)
    inc = np.deg2rad(rng.uniform(0.0, 8.0, count))
    ang = rng.uniform(0.0, 2 * np.pi, (3, count))
    r, v = kepler_to_cartesian(a, e, inc, ang[0], ang[1], ang[2], G * (1.0 + m))
    r = np.concatenate([np.zeros((3, 1)), r], axis=1)
    v = np.concatenate([np.zeros((3, 1)), v], axis=1)
    m = np.concatenate([[1.0], m])
    return r, v, m, np.concatenate([[1.989e30], m_kg])


def _unit_vectors(rng, k):
    u = rng.normal(size=(3, k))
    return u / np.linalg.norm(u, axis=0)


def moons(rng, r_host, v_host, m_host, m_host_kg, G=G_AU_DAY, count=100, omega_dt_max=None):
    """``count`` moons on circular orbits around hosts heavier than 1e23 kg.

    Returns (r, v, m, stats) where stats counts moons whose period is shorter
    than 2 pi * 0.1 day (unresolved by the paper's step) and moons outside
    their host's Hill sphere (computed with the host's distance from the Sun).
    ``omega_dt_max``: if given, each drawn radius is raised, where needed, to
    the one at which the orbit's angular rate times the step (0.1 day) equals
    it, so every moon orbit is resolved by the step (the same draws
    otherwise)."""
    cand = np.nonzero(m_host_kg[1:] > 1e23)[0] + 1
    if cand.size == 0:
        raise ValueError("no major body heavier than 1e23 kg; draw another seed")
    host = rng.choice(cand, size=count, replace=True)
    R = _loguniform(rng, 1e-4, 5e-2, count)
    m = rng.uniform(1e15, 1e19, count) / MSUN_KG
    if omega_dt_max is not None:
        # omega = sqrt(G (M + m) / R^3) <= omega_dt_max / dt
        r_min = np.cbrt(G * (m_host[host] + m) * (DT_DAY / omega_dt_max) ** 2)
        R = np.maximum(R, r_min)
    u = _unit_vectors(rng, count)
    w = rng.normal(size=(3, count))
    w = w - u * np.sum(w * u, axis=0)
    w = w / np.linalg.norm(w, axis=0)
    speed = np.sqrt(G * (m_host[host] + m) / R)
    r = r_host[:, host] + R * u
    v = v_host[:, host] + speed * w
    omega_dt = speed / R * DT_DAY
    dist = np.linalg.norm(r_host[:, host], axis=0)
    hill = dist * np.cbrt(m_host[host] / 3.0)
    stats = {"moons_unresolved_omega_dt_gt_1": int(np.sum(omega_dt > 1.0)),
             "moons_outside_hill": int(np.sum(R > hill))}
    return r, v, m, stats


def asteroids(rng, G=G_AU_DAY, count=10294):
    """Main-belt asteroids on heliocentric Keplerian orbits."""
    a = rng.uniform(2.1, 3.3, count)
    e = rng.uniform(0.0, 0.3, count)
    inc = np.deg2rad(rng.uniform(0.0, 20.0, count))
    ang = rng.uniform(0.0, 2 * np.pi, (3, count))
    m = rng.uniform(1e12, 3e17, count) / MSUN_KG
    r, v = kepler_to_cartesian(a, e, inc, ang[0], ang[1], ang[2], G * (1.0 + m))
    return r, v, m


def solar_system(n: int = 10425, seed: int = BASE_SEED, n_moons: int = 100,
                 moon_omega_dt_max: float | None = None) -> System:
    """A Solar-System-shaped system of ``n`` bodies.

    n == 31: Sun + 30 major bodies.  Otherwise Sun + 30 major bodies +
    ``n_moons`` moons + (n - 31 - n_moons) asteroids, in that order.
    ``moon_omega_dt_max``: see ``moons`` (None: the radii as drawn)."""
    rng = np.random.default_rng(seed)
    r, v, m, m_kg = major_bodies(rng)
    info = {"seed": seed, "n_major": 31, "n_moons": 0, "n_asteroids": 0}
    if n < 31:
        raise ValueError("n must be >= 31")
    if n > 31:
        k_moons = min(n_moons, n - 31)
        rm, vm, mm, stats = moons(rng, r, v, m, m_kg, count=k_moons, omega_dt_max=moon_omega_dt_max)
        ra, va, ma = asteroids(rng, count=n - 31 - k_moons)
        r = np.concatenate([r, rm, ra], axis=1)
        v = np.concatenate([v, vm, va], axis=1)
        m = np.concatenate([m, mm, ma])
        info.update(n_moons=k_moons, n_asteroids=n - 31 - k_moons, **stats)
    return System(r=np.ascontiguousarray(r), v=np.ascontiguousarray(v),
                  m=np.ascontiguousarray(m), info=info)


def ensemble(n_systems: int = 256, seed: int = BASE_SEED, lo: int = 1000, hi: int = 20000,
             jitter_au: float = 1e-8) -> list[System]:
    """Independent systems: the 131-body major+moon set of ``solar_system`` plus
    a seeded asteroid count in {lo..hi}, positions jittered by N(0, jitter_au)."""
    base = solar_system(131, seed)
    out = []
    for s in range(n_systems):
        rng = np.random.default_rng(seed + 1 + s)
        k = int(rng.integers(lo, hi + 1))
        ra, va, ma = asteroids(rng, count=k)
        r = np.concatenate([base.r, ra], axis=1)
        v = np.concatenate([base.v, va], axis=1).copy()
        m = np.concatenate([base.m, ma])
        r = r + rng.normal(0.0, jitter_au, size=r.shape)
        out.append(System(r=np.ascontiguousarray(r), v=np.ascontiguousarray(v),
                          m=np.ascontiguousarray(m),
                          info={"seed": seed + 1 + s, "n_asteroids": k}))
    return out


def loss_targets(system: System, k: int = 64, seed: int = BASE_SEED + 7):
    """k seeded asteroid indices and target positions [3, k] for the trajectory
    loss L = sum_i |r_{idx_i}(T) - target_i|^2."""
    rng = np.random.default_rng(seed)
    n_ast = system.info.get("n_asteroids", 0)
    first = system.n - n_ast
    pool = np.arange(first, system.n) if n_ast >= k else np.arange(1, system.n)
    idx = np.sort(rng.choice(pool, size=k, replace=False))
    targets = system.r[:, idx] + rng.normal(0.0, 1e-2, size=(3, k))
    return idx, targets


def concat(systems: list[System]):
    """CSR layout of several systems: (offsets [S+1] int64, r [3, N], v [3, N], m [N])."""
    sizes = np.array([s.n for s in systems], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    r = np.ascontiguousarray(np.concatenate([s.r for s in systems], axis=1))
    v = np.ascontiguousarray(np.concatenate([s.v for s in systems], axis=1))
    m = np.ascontiguousarray(np.concatenate([s.m for s in systems]))
    return offsets, r, v, m
