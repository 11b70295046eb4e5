"""GPU parity of the leapfrog integrator (drift-kick-drift, named in
Section 2 beside Verlet) against the oracle's leapfrog.

FP64: positions of the 31-body model within 1e-10 AU after 3650 steps;
several tiles with ragged tails within 1e-12 AU after 10 steps; the kept
acceleration is Eq. 1 at the last half-step positions (1e-13); the energy
drift matches the oracle's at dt = 0.4, 0.2.  Mixed: one step within the
force-error bound (dt^2 * 2e-6 * T_p for positions, dt * 2e-6 * T_p for
velocities, T_p = sum_j |term_pj| at the half-step positions, with a
factor 2)."""
import numpy as np
import pytest

import oracle
from paper_2112_15079_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15079_gb300 import build
    build.build()
    from paper_2112_15079_gb300 import nbody
    return nbody


def _lf(nb, s, precision, **kw):
    return nb.NBody(s.r, s.v, s.m, G=s.G, dt=kw.pop("dt", s.dt), precision=precision, integrator="leapfrog", **kw)


def test_leapfrog_fp64_31_bodies_3650_steps(nb):
    s = inputs.solar_system(31)
    b = _lf(nb, s, "fp64")
    b.step(3650)
    r_ref, v_ref, _ = oracle.leapfrog(s.G, s.dt, 3650, s.r, s.v, s.m)
    assert np.abs(b.r.cpu().numpy() - r_ref).max() <= 1e-10


@pytest.mark.parametrize("n", [2131, 5003])
def test_leapfrog_fp64_tiles_vs_oracle(nb, n):
    s = inputs.solar_system(n, seed=400 + n, n_moons=0)
    b = _lf(nb, s, "fp64")
    b.step(10)
    r_ref, v_ref, a_ref = oracle.leapfrog(s.G, s.dt, 10, s.r, s.v, s.m, openmp=True)
    assert np.abs(b.r.cpu().numpy() - r_ref).max() <= 1e-12
    assert np.abs(b.v.cpu().numpy() - v_ref).max() <= 1e-13
    a = b.accel().cpu().numpy()
    err = np.linalg.norm(a - a_ref, axis=0) / np.linalg.norm(a_ref, axis=0)
    assert err.max() <= 1e-12, err.max()  # same half-step positions to ~1e-15, Eq. 1 to 1e-13


@pytest.mark.parametrize("n", [2131, 5003])
def test_leapfrog_mixed_one_step_within_force_bound(nb, n):
    s = inputs.solar_system(n, seed=410 + n)
    b = _lf(nb, s, "mixed")
    b.step(1)
    r_ref, v_ref, _ = oracle.leapfrog(s.G, s.dt, 1, s.r, s.v, s.m, openmp=True)
    T = oracle.term_norm(s.G, s.r + 0.5 * s.dt * s.v, s.m, openmp=True)
    dr = np.linalg.norm(b.r.cpu().numpy() - r_ref, axis=0)
    dv = np.linalg.norm(b.v.cpu().numpy() - v_ref, axis=0)
    assert np.all(dr <= 2 * s.dt**2 * 2e-6 * T + 1e-15 * np.linalg.norm(r_ref, axis=0)), (dr / T).max()
    assert np.all(dv <= 2 * s.dt * 2e-6 * T + 1e-15 * np.linalg.norm(v_ref, axis=0)), (dv / T).max()


def test_leapfrog_energy_drift_matches_oracle(nb):
    s = inputs.solar_system(500, seed=31, n_moons=0)
    for dt in (0.4, 0.2):
        n = int(round(36.5 / dt))
        every = max(1, n // 20)
        b = _lf(nb, s, "fp64", dt=dt)
        e0 = b.energy()[0]
        st = {"r": s.r.copy(), "v": s.v.copy()}
        worst_g = worst_o = 0.0
        for _ in range(n // every):
            b.step(every)
            worst_g = max(worst_g, abs(b.energy()[0] - e0) / abs(e0))
            st["r"], st["v"], _ = oracle.leapfrog(s.G, dt, every, st["r"], st["v"], s.m, openmp=True)
            worst_o = max(worst_o, abs(sum(oracle.energy(s.G, st["r"], st["v"], s.m)) - e0) / abs(e0))
        assert abs(worst_g - worst_o) <= 1e-3 * worst_o + 1e-14, (dt, worst_g, worst_o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_leapfrog_graphs_split_calls_and_batches(nb, precision):
    """Graph replay, split calls and no-graph launches agree bitwise; a batch
    of uneven systems equals each system run alone (FP64: to 1e-12 AU)."""
    s = inputs.solar_system(2131, seed=35)
    outs = []
    for graphs, chunks in ((True, [70]), (True, [64, 6]), (False, [13, 57])):
        b = _lf(nb, s, precision, graphs=graphs)
        for c in chunks:
            b.step(c)
        outs.append(b.state.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    if precision == "fp64":
        systems = [inputs.solar_system(n, seed=sd, n_moons=0) for n, sd in ((31, 51), (700, 52), (1531, 53))]
        off, r, v, m = inputs.concat(systems)
        bb = nb.NBody(r, v, m, off, G=inputs.G_AU_DAY, dt=inputs.DT_DAY, precision="fp64", integrator="leapfrog")
        bb.step(10)
        rg = bb.r.cpu().numpy()
        for k, sysk in enumerate(systems):
            r_ref, _, _ = oracle.leapfrog(sysk.G, sysk.dt, 10, sysk.r, sysk.v, sysk.m)
            assert np.abs(rg[:, off[k]:off[k + 1]] - r_ref).max() <= 1e-12 * max(1.0, np.abs(r_ref).max())
