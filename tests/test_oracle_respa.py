"""Pins of the oracle's close-encounter step (``oracle.respa``): impulse
multiple time stepping with close pairs sub-cycled, an extension beyond
Section 2's method (Tuckerman, Berne and Martyna, J. Chem. Phys. 97, 1990,
1992).  Each pin is something the method must reduce to or conserve:
- without close pairs it is velocity Verlet (Eqs. 3-4), to rounding;
- an isolated close pair has no far force, so it is velocity Verlet with
  the sub-step h = dt / k;
- total momentum is conserved (every force is a pair force, split by pairs);
- the scheme is time-reversible;
- a moon whose period is below the step (w dt > 2: Eqs. 3-4 unstable) keeps
  its orbit, and the sub-step error falls as h^2;
- the close-pair graph and the sub-step count follow their definitions.
"""
import math

import numpy as np
import pytest

import oracle

G = 2.9591220828e-4


def _kepler_circ(m_host, r_host, v_host, radius, m_sat, phase=0.3, incl=0.2):
    """A satellite on a circular orbit of `radius` around a host."""
    u = np.array([math.cos(phase), math.sin(phase) * math.cos(incl), math.sin(phase) * math.sin(incl)])
    w = np.array([-math.sin(phase), math.cos(phase) * math.cos(incl), math.cos(phase) * math.sin(incl)])
    speed = math.sqrt(G * (m_host + m_sat) / radius)
    return r_host + radius * u, v_host + speed * w


def _triple(moon_radius=2e-4, planet_mass=1e-3):
    """Sun, a planet at 5.2 AU, and a moon around the planet."""
    rs, vs = np.zeros(3), np.zeros(3)
    rp, vp = _kepler_circ(1.0, rs, vs, 5.2, planet_mass, phase=0.0, incl=0.02)
    rm, vm = _kepler_circ(planet_mass, rp, vp, moon_radius, 1e-9)
    r = np.stack([rs, rp, rm], axis=1)
    v = np.stack([vs, vp, vm], axis=1)
    m = np.array([1.0, planet_mass, 1e-9])
    return r, v, m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_without_close_pairs_it_is_velocity_verlet():
    rng = np.random.default_rng(5)
    n = 24
    r = rng.uniform(-3, 3, size=(3, n))
    v = rng.normal(0, 1e-3, size=(3, n))
    m = rng.uniform(1e-9, 1e-5, size=n)
    r1, v1, a1, npairs, kmax = oracle.respa(G, 0.1, 60, r, v, m, theta_c=1e9, theta_s=0.05)
    assert npairs == 0 and kmax == 0
    a0 = oracle.accel(G, r, m)
    r2, v2, a2 = oracle.verlet(G, 0.1, 60, r, v, m, a0)
    assert _rel(r1, r2) < 1e-13 and _rel(v1, v2) < 1e-12
    assert np.array_equal(a1, oracle.accel(G, r1, m))  # Eq. 1 at the final positions


def test_an_isolated_close_pair_is_verlet_at_the_sub_step():
    rh, vh = np.zeros(3), np.zeros(3)
    rm, vm = _kepler_circ(1e-3, rh, vh, 1e-3, 1e-9)
    r = np.stack([rh, rm], axis=1)
    v = np.stack([vh, vm], axis=1)
    m = np.array([1e-3, 1e-9])
    w = math.sqrt(G * (m[0] + m[1]) / 1e-3 ** 3)
    k = math.ceil(w * 0.1 / 0.05)
    r1, v1, _, npairs, kmax = oracle.respa(G, 0.1, 12, r, v, m, theta_c=0.5, theta_s=0.05)
    assert npairs == 1 and kmax == k == 35
    a0 = oracle.accel(G, r, m)
    r2, v2, _ = oracle.verlet(G, 0.1 / k, 12 * k, r, v, m, a0)
    assert _rel(r1, r2) < 1e-12 and _rel(v1, v2) < 1e-11


def test_momentum_is_conserved_and_the_scheme_is_reversible():
    r, v, m = _triple()
    rng = np.random.default_rng(9)
    extra_r = rng.uniform(-3, 3, size=(3, 6))
    extra_v = rng.normal(0, 5e-3, size=(3, 6))
    r = np.concatenate([r, extra_r], axis=1)
    v = np.concatenate([v, extra_v], axis=1)
    m = np.concatenate([m, rng.uniform(1e-10, 1e-8, size=6)])
    p0 = (m * v).sum(axis=1)
    r1, v1, _, npairs, kmax = oracle.respa(G, 0.1, 80, r, v, m, theta_c=0.5, theta_s=0.05)
    assert npairs == 1 and kmax > 1
    p1 = (m * v1).sum(axis=1)
    assert np.max(np.abs(p1 - p0)) <= 1e-14 * np.sum(np.abs(m * v))
    # back: reverse the velocities, the same number of steps, reverse again
    # (10 steps, ~4,000 sub-steps each way: rounding, not the scheme, sets the
    # bound; the sub-step count must come out the same both ways)
    r1, v1, _, _, k1 = oracle.respa(G, 0.1, 10, r, v, m, theta_c=0.5, theta_s=0.05)
    r2, v2, _, _, k2 = oracle.respa(G, 0.1, 10, r1, -v1, m, theta_c=0.5, theta_s=0.05)
    assert k1 == k2
    assert _rel(r2, r) < 1e-11 and _rel(-v2, v) < 1e-7


def _moon_state(r, v):
    return r[:, 2] - r[:, 1], v[:, 2] - v[:, 1]


def test_a_moon_faster_than_the_step_keeps_its_orbit():
    r, v, m = _triple(moon_radius=2e-4)
    w = math.sqrt(G * (m[1] + m[2]) / 2e-4 ** 3)
    assert w * 0.1 > 2.0  # Eqs. 3-4 are unstable for this moon
    steps = 3650
    r1, v1, _, npairs, kmax = oracle.respa(G, 0.1, steps, r, v, m, theta_c=0.5, theta_s=0.05)
    d, _ = _moon_state(r1, v1)
    assert npairs == 1 and abs(np.linalg.norm(d) / 2e-4 - 1.0) < 1e-3
    # plain Verlet loses the moon
    a0 = oracle.accel(G, r, m)
    r2, v2, _ = oracle.verlet(G, 0.1, steps, r, v, m, a0)
    d2, _ = _moon_state(r2, v2)
    assert abs(np.linalg.norm(d2) / 2e-4 - 1.0) > 0.1


def test_the_sub_step_error_is_second_order():
    r, v, m = _triple(moon_radius=4e-4)
    ref = oracle.respa(G, 0.1, 10, r, v, m, theta_c=0.5, theta_s=0.01 / 16)
    errs = []
    for ts in (0.04, 0.02, 0.01):
        out = oracle.respa(G, 0.1, 10, r, v, m, theta_c=0.5, theta_s=ts)
        errs.append(np.linalg.norm(_moon_state(out[0], out[1])[0] - _moon_state(ref[0], ref[1])[0]))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs


def test_close_pairs_and_clusters_follow_their_definitions():
    rs, vs = np.zeros(3), np.zeros(3)
    rp, vp = _kepler_circ(1.0, rs, vs, 5.2, 1e-3, phase=0.0)
    bodies_r, bodies_v, masses = [rs, rp], [vs, vp], [1.0, 1e-3]
    radii = (2e-4, 1e-3, 3e-2)  # w dt 10.7, 0.96, 0.006 around a 1e-3 host
    for i, R in enumerate(radii):
        rm, vm = _kepler_circ(1e-3, rp, vp, R, 1e-10, phase=1.0 + i)
        bodies_r.append(rm)
        bodies_v.append(vm)
        masses.append(1e-10)
    r = np.stack(bodies_r, axis=1)
    v = np.stack(bodies_v, axis=1)
    m = np.array(masses)
    # theta_c = 0.5: the two inner moons pair with the planet (one cluster of
    # three bodies); the outer moon and the Sun pair with nobody
    _, _, _, npairs, kmax = oracle.respa(G, 0.1, 1, r, v, m, theta_c=0.5, theta_s=0.05)
    period = 2 * math.pi * math.sqrt(2e-4 ** 3 / (G * (1e-3 + 1e-10)))
    assert npairs == 2
    assert kmax == math.ceil(2 * math.pi * 0.1 / period / 0.05)
    # theta_c above every pair's w dt: no pairs
    _, _, _, npairs, kmax = oracle.respa(G, 0.1, 1, r, v, m, theta_c=20.0, theta_s=0.05)
    assert npairs == 0 and kmax == 0
