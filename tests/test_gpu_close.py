"""GPU parity of close-encounter handling (nbody_opts.close_omega_dt):
impulse multiple time stepping with the close pairs of each cluster
sub-cycled in FP64, against the oracle's close-encounter step
(``oracle.respa``, pinned in test_oracle_respa.py).

Gates (theta_c = 0.5, theta_s = 0.05 unless stated):
- the close pairs and the largest sub-step count equal the oracle's;
- an isolated close pair is velocity Verlet at the sub-step, to 1e-14 AU;
- trajectories of the 131-body model (Sun, 30 major bodies, 100 moons with
  the radii as drawn: 13 moons have w dt > 2) after 100 steps, and of the
  10,425-body model after 10 steps.  Cluster members within 1e-8 AU in
  both precisions: their far force and sub-cycle are FP64, and the fast
  moons' orbital phase picks up the last-bit differences of ~3e4
  sub-steps (observed 5e-10 AU).  Bodies in no cluster: FP64 median within
  1e-13 AU (observed 5e-15) and every one within 1e-10 AU (a slow moon of
  a cluster's host inherits the host's error, observed 1e-12); mixed every
  one within 5e-8 AU (its Eq. 1 error, 2e-6 of a moon's ~1e-2 AU/day^2
  host pull, over dt^2 n^2 / 2 = 50 day^2; observed 5e-9);
- over 3650 steps every moon with w dt > 2 keeps its distance to its host
  within 1 %, where plain Verlet (Eqs. 3-4) changes some by more than 10 %,
  and the total-energy drift is within 2x the oracle's;
- a run split over several calls, and one without CUDA graphs, is bitwise
  identical to one call;
- the entry points that do not cover close pairs refuse them (EINVAL).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2112_15079_gb300 import inputs

pytestmark = pytest.mark.gpu

TC, TS = 0.5, 0.05


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15079_gb300 import build
    build.build()
    from paper_2112_15079_gb300 import nbody
    return nbody


def _run(nb, s, precision, steps, tc=TC, ts=TS, **kw):
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, close_omega_dt=tc, substep_omega_dt=ts, **kw)
    info = b.close_info()
    if steps:
        b.step(steps)
    b.sync()
    st = b.state.cpu().numpy().copy()
    b.close()
    return st[:3], st[3:], info


def _close_pairs(s, tc=TC):
    """(p, j, w dt) of every close pair, from the definition (test-side)."""
    out = []
    for p in range(s.n):
        d = s.r[:, p + 1:] - s.r[:, p:p + 1]
        d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
        d3 = d2 * np.sqrt(d2)
        close = s.G * (s.m[p] + s.m[p + 1:]) * (s.dt * s.dt) > tc * tc * d3
        for jj in np.nonzero(close)[0]:
            j = p + 1 + int(jj)
            out.append((p, j, math.sqrt(s.G * (s.m[p] + s.m[j]) / d3[jj]) * s.dt))
    return out


class _Sys:
    def __init__(self, r, v, m, G=inputs.G_AU_DAY, dt=0.1):
        self.r, self.v, self.m, self.G, self.dt = r, v, m, G, dt
        self.n = m.shape[0]


@pytest.mark.parametrize("n", [131, 10425])
def test_close_set_matches_the_oracle(nb, n):
    s = inputs.solar_system(n)
    _, _, info = _run(nb, s, "fp64", 0)
    _, _, _, npairs, kmax = oracle.respa(s.G, s.dt, 0, s.r, s.v, s.m, TC, TS, openmp=True)
    assert info["pairs"] == npairs > 0 and info["k_max"] == kmax
    assert info["members"] >= 2 and 1 <= info["clusters"] <= info["pairs"]


def test_an_isolated_close_pair_is_verlet_at_the_sub_step(nb):
    G = inputs.G_AU_DAY
    rm = np.array([1e-3 * math.cos(0.3), 1e-3 * math.sin(0.3), 0.0])
    vm = math.sqrt(G * (1e-3 + 1e-9) / 1e-3) * np.array([-math.sin(0.3), math.cos(0.3), 0.0])
    s = _Sys(np.stack([np.zeros(3), rm], 1), np.stack([np.zeros(3), vm], 1), np.array([1e-3, 1e-9]))
    r, v, info = _run(nb, s, "fp64", 12)
    k = info["k_max"]
    assert info["pairs"] == 1 and k == math.ceil(math.sqrt(G * (1e-3 + 1e-9) / 1e-9) * 0.1 / TS)
    r2, v2, _ = oracle.verlet(G, 0.1 / k, 12 * k, s.r, s.v, s.m, oracle.accel(G, s.r, s.m))
    assert np.abs(r - r2).max() <= 1e-14 and np.abs(v - v2).max() <= 1e-12


def _members(s):
    return sorted({p for p, j, _ in _close_pairs(s)} | {j for p, j, _ in _close_pairs(s)})


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,steps", [(131, 100), (10425, 10)])
def test_trajectories_match_the_oracle(nb, precision, n, steps):
    s = inputs.solar_system(n)
    r, v, _ = _run(nb, s, precision, steps)
    ro, vo, _, _, _ = oracle.respa(s.G, s.dt, steps, s.r, s.v, s.m, TC, TS, openmp=True)
    err = np.linalg.norm(r - ro, axis=0)
    mem = np.zeros(s.n, bool)
    mem[_members(s)] = True
    assert err[mem].max() <= 1e-8, err[mem].max()
    if precision == "fp64":
        assert np.median(err[~mem]) <= 1e-13 and err[~mem].max() <= 1e-10, (np.median(err[~mem]), err[~mem].max())
    else:
        assert err[~mem].max() <= 5e-8, err[~mem].max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fast_moons_keep_their_orbits_and_energy_is_conserved(nb, precision):
    s = inputs.solar_system(131)
    fast = [(p, j) for p, j, wdt in _close_pairs(s) if wdt > 2.0]
    assert len(fast) >= 5
    d0 = np.array([np.linalg.norm(s.r[:, j] - s.r[:, p]) for p, j in fast])
    r, v, _ = _run(nb, s, precision, 3650)
    d1 = np.array([np.linalg.norm(r[:, j] - r[:, p]) for p, j in fast])
    assert np.abs(d1 / d0 - 1).max() <= 0.01
    rv, vv, _ = _run(nb, s, precision, 3650, tc=0.0)  # plain Verlet
    dv = np.array([np.linalg.norm(rv[:, j] - rv[:, p]) for p, j in fast])
    assert np.abs(dv / d0 - 1).max() > 0.1
    e0 = sum(oracle.energy(s.G, s.r, s.v, s.m))
    ro, vo, _, _, _ = oracle.respa(s.G, s.dt, 3650, s.r, s.v, s.m, TC, TS)
    drift_ref = abs(sum(oracle.energy(s.G, ro, vo, s.m)) - e0) / abs(e0)
    drift = abs(sum(oracle.energy(s.G, r, v, s.m)) - e0) / abs(e0)
    assert drift <= 2 * drift_ref, (drift, drift_ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_calls_and_graphs_are_bitwise(nb, precision):
    s = inputs.solar_system(2131)
    b1 = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, close_omega_dt=TC, substep_omega_dt=TS)
    b1.step(40)
    b2 = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, close_omega_dt=TC, substep_omega_dt=TS)
    b2.step(7)
    b2.step(33)
    b3 = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, close_omega_dt=TC, substep_omega_dt=TS,
                  graphs=False)
    b3.step(40)
    for b in (b1, b2, b3):
        b.sync()
    a1, a2, a3 = (b.state.cpu().numpy() for b in (b1, b2, b3))
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)
    for b in (b1, b2, b3):
        b.close()


def test_entry_points_without_close_pairs_refuse_them(nb):
    s = inputs.solar_system(131)
    with pytest.raises(nb.NBodyError):
        nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", integrator="rk4", close_omega_dt=TC)
    with pytest.raises(nb.NBodyError):
        nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", close_omega_dt=TC, substep_omega_dt=0.0)
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", close_omega_dt=TC, substep_omega_dt=TS)
    import torch
    g = torch.zeros((3, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NBodyError):
        b.grad(2, g)
    with pytest.raises(nb.NBodyError):
        b.kernel_times(2)
    b.close()


def test_batched_systems_are_handled_each_on_its_own(nb):
    """Two 131-body systems in one context: the close pairs never cross
    systems, and each system's trajectory equals the oracle's run alone."""
    s1 = inputs.solar_system(131)
    s2 = inputs.solar_system(131, seed=inputs.BASE_SEED + 7)
    off, r, v, m = inputs.concat([s1, s2])
    for precision in ("fp64", "mixed"):
        b = nb.NBody(r, v, m, off, G=s1.G, dt=s1.dt, precision=precision, close_omega_dt=TC, substep_omega_dt=TS)
        info = b.close_info()
        b.step(20)
        b.sync()
        st = b.state.cpu().numpy()
        b.close()
        pairs = 0
        for k, sy in enumerate((s1, s2)):
            ro, _, _, npairs, _ = oracle.respa(sy.G, sy.dt, 20, sy.r, sy.v, sy.m, TC, TS)
            pairs += npairs
            assert np.abs(st[:3, off[k]:off[k + 1]] - ro).max() <= 1e-8
        assert info["pairs"] == pairs


def test_reset_rebuilds_the_close_set(nb):
    """After nbody_reset to another state the context steps bitwise like a
    new one built on that state (the close pairs of the new positions)."""
    s1 = inputs.solar_system(131)
    s2 = inputs.solar_system(131, seed=inputs.BASE_SEED + 3)
    import torch
    b = nb.NBody(s1.r, s1.v, s1.m, G=s1.G, dt=s1.dt, precision="fp64", close_omega_dt=TC, substep_omega_dt=TS)
    b.step(5)
    b.state[0:3].copy_(torch.as_tensor(s2.r))
    b.state[3:6].copy_(torch.as_tensor(s2.v))
    b.m.copy_(torch.as_tensor(s2.m))
    b.reset()
    info = b.close_info()
    b.step(10)
    b.sync()
    c = nb.NBody(s2.r, s2.v, s2.m, G=s2.G, dt=s2.dt, precision="fp64", close_omega_dt=TC, substep_omega_dt=TS)
    assert c.close_info() == info
    c.step(10)
    c.sync()
    assert np.array_equal(b.state.cpu().numpy(), c.state.cpu().numpy())
    b.close()
    c.close()
