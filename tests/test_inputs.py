"""The seeded input recipe (host logic, no GPU): the synthetic stand-ins for
the paper's Solar-System model (Section 2) have the stated structure and
distributions, and are reproducible from their seeds."""
import numpy as np
import pytest

from paper_2112_15079_gb300 import inputs

MSUN = inputs.MSUN_KG


def _elements(r, v, mu):
    """Semi-major axis, eccentricity and inclination (deg) of heliocentric
    two-body orbits from Cartesian states [3, k] (textbook relations)."""
    rn = np.linalg.norm(r, axis=0)
    v2 = np.sum(v * v, axis=0)
    a = 1.0 / (2.0 / rn - v2 / mu)
    h = np.cross(r.T, v.T).T
    evec = np.cross(v.T, h.T).T / mu - r / rn
    inc = np.degrees(np.arccos(h[2] / np.linalg.norm(h, axis=0)))
    return a, np.linalg.norm(evec, axis=0), inc


def test_kepler_to_cartesian_closed_forms():
    """Energy -mu/(2a) and |h| = sqrt(mu a (1 - e^2)) for random elements."""
    rng = np.random.default_rng(1)
    k = 200
    a = rng.uniform(0.3, 40, k)
    e = rng.uniform(0, 0.9, k)
    inc, node, peri, M = (rng.uniform(0, np.pi, k), *rng.uniform(0, 2 * np.pi, (3, k)))
    mu = inputs.G_AU_DAY * rng.uniform(1.0, 1.001, k)
    r, v = inputs.kepler_to_cartesian(a, e, inc, node, peri, M, mu)
    energy = 0.5 * np.sum(v * v, axis=0) - mu / np.linalg.norm(r, axis=0)
    np.testing.assert_allclose(energy, -mu / (2 * a), rtol=1e-12)
    h = np.linalg.norm(np.cross(r.T, v.T), axis=1)
    np.testing.assert_allclose(h, np.sqrt(mu * a * (1 - e * e)), rtol=1e-12)


def test_solar_system_structure_10425():
    s = inputs.solar_system(10425)
    assert s.n == 10425 and s.info["n_moons"] == 100 and s.info["n_asteroids"] == 10294
    assert s.m[0] == 1.0 and np.all(s.r[:, 0] == 0) and np.all(s.v[:, 0] == 0)  # Sun at rest at the origin
    major_kg = s.m[1:31] * MSUN
    assert major_kg.min() >= 1e19 * (1 - 1e-12) and major_kg.max() <= 2e27 * (1 + 1e-12)
    a, e, inc = _elements(s.r[:, 1:31], s.v[:, 1:31], s.G * (1 + s.m[1:31]))
    assert a.min() > 0.3 - 1e-9 and a.max() < 40 + 1e-9
    assert e.max() <= 0.25 + 1e-9 and inc.max() <= 8 + 1e-9
    ast = slice(131, None)
    ast_kg = s.m[ast] * MSUN
    assert ast_kg.min() >= 1e12 * (1 - 1e-12) and ast_kg.max() <= 3e17 * (1 + 1e-12)
    a, e, inc = _elements(s.r[:, ast], s.v[:, ast], s.G * (1 + s.m[ast]))
    assert a.min() > 2.1 - 1e-9 and a.max() < 3.3 + 1e-9
    assert e.max() <= 0.3 + 1e-9 and inc.max() <= 20 + 1e-9
    moon_kg = s.m[31:131] * MSUN
    assert moon_kg.min() >= 1e15 * (1 - 1e-12) and moon_kg.max() <= 1e19 * (1 + 1e-12)
    # every moon sits at 1e-4..5e-2 AU from a major body heavier than 1e23 kg
    d = np.linalg.norm(s.r[:, 31:131, None] - s.r[:, None, 1:31], axis=0)
    host = np.argmin(d, axis=1)
    assert np.all(d[np.arange(100), host] >= 1e-4 * (1 - 1e-9))
    assert np.all(d[np.arange(100), host] <= 5e-2 * (1 + 1e-9))
    assert np.all(s.m[1:31][host] * MSUN > 1e23)


def test_seeds_reproduce_and_differ():
    a, b, c = inputs.solar_system(500, seed=3), inputs.solar_system(500, seed=3), inputs.solar_system(500, seed=4)
    assert np.array_equal(a.r, b.r) and np.array_equal(a.v, b.v) and np.array_equal(a.m, b.m)
    assert not np.array_equal(a.r, c.r)


def test_small_and_moonless_variants():
    s31 = inputs.solar_system(31)
    assert s31.n == 31 and s31.info["n_moons"] == 0
    s = inputs.solar_system(500, n_moons=0)
    assert s.info["n_moons"] == 0 and s.info["n_asteroids"] == 469
    with pytest.raises(ValueError):
        inputs.solar_system(30)


def test_ensemble_and_concat():
    ens = inputs.ensemble(4)
    base = inputs.solar_system(131)
    for e in ens:
        k = e.info["n_asteroids"]
        assert 1000 <= k <= 20000 and e.n == 131 + k
        dev = np.abs(e.r[:, :131] - base.r)
        assert 0 < dev.max() < 1e-6  # N(0, 1e-8 AU) jitter
    off, r, v, m = inputs.concat(ens)
    assert off[0] == 0 and np.all(np.diff(off) == [e.n for e in ens]) and r.shape == (3, off[-1])


def test_loss_targets():
    s = inputs.solar_system(10425)
    idx, tgt = inputs.loss_targets(s)
    assert idx.shape == (64,) and np.all(np.diff(idx) > 0) and idx.min() >= 131
    assert tgt.shape == (3, 64) and np.abs(tgt - s.r[:, idx]).max() < 0.1


def test_resolved_moons_variant():
    """moon_omega_dt_max raises only the radii of moons whose orbit the step
    does not resolve; every other draw is the same."""
    base = inputs.solar_system(1031)
    res = inputs.solar_system(1031, moon_omega_dt_max=0.5)
    host_idx = slice(0, 31)
    assert np.array_equal(base.r[:, host_idx], res.r[:, host_idx])
    assert np.array_equal(base.r[:, 131:], res.r[:, 131:]) and np.array_equal(base.m, res.m)
    # moon radius and rate around the nearest major body (its host)
    def rates(s):
        d = s.r[:, 31:131, None] - s.r[:, None, 1:31]
        dist = np.linalg.norm(d, axis=0)
        k = dist.argmin(axis=1)
        R = dist[np.arange(100), k]
        M = s.m[1:31][k] + s.m[31:131]
        return R, np.sqrt(s.G * M / R**3) * inputs.DT_DAY
    R0, w0 = rates(base)
    R1, w1 = rates(res)
    assert w0.max() > 1.0  # the plain draw has unresolved moons
    assert w1.max() <= 0.5 * (1 + 1e-9)
    kept = w0 <= 0.5
    np.testing.assert_allclose(R1[kept], R0[kept], rtol=1e-12)
    assert np.all(R1[~kept] > R0[~kept])
