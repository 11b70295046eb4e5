"""Energy error against the step size (the accuracy criterion of Section 4,
the analogue of the paper's energy-error-vs-dt study): Verlet's error is of
order dt^2 (Section 2), so halving dt divides the maximum total-energy drift
by ~4.  The GPU's FP64 path reproduces the oracle's drift at every dt, and
the mixed path stays within 2x of it (the mixed-precision energy bound).

System: the Sun, 30 major bodies and 469 asteroids (no moons: their orbital
periods fall below dt and would dominate the error), 36.5 days at dt = 0.4,
0.2 and 0.1 day, energy sampled 20 times per run."""
import numpy as np
import pytest

import oracle
from paper_2112_15079_gb300 import inputs

pytestmark = pytest.mark.gpu

T_DAYS = 36.5
DTS = (0.4, 0.2, 0.1)


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15079_gb300 import build
    build.build()
    from paper_2112_15079_gb300 import nbody
    return nbody


def _oracle_drift(s, dt):
    n_steps = int(round(T_DAYS / dt))
    every = max(1, n_steps // 20)
    r, v, a = s.r.copy(), s.v.copy(), None
    e0 = sum(oracle.energy(s.G, r, v, s.m))
    worst = 0.0
    for _ in range(n_steps // every):
        r, v, a = oracle.verlet(s.G, dt, every, r, v, s.m, a, openmp=True)
        worst = max(worst, abs(sum(oracle.energy(s.G, r, v, s.m)) - e0) / abs(e0))
    return worst


def _gpu_drift(nb, s, dt, precision):
    n_steps = int(round(T_DAYS / dt))
    every = max(1, n_steps // 20)
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=dt, precision=precision)
    e0 = b.energy()[0]
    worst = 0.0
    for _ in range(n_steps // every):
        b.step(every)
        worst = max(worst, abs(b.energy()[0] - e0) / abs(e0))
    b.close()
    return worst


def test_energy_error_is_second_order_in_dt(nb):
    s = inputs.solar_system(500, seed=31, n_moons=0)
    ref = {dt: _oracle_drift(s, dt) for dt in DTS}
    for dt in DTS:
        g64 = _gpu_drift(nb, s, dt, "fp64")
        gmx = _gpu_drift(nb, s, dt, "mixed")
        assert abs(g64 - ref[dt]) <= 1e-3 * ref[dt] + 1e-13, (dt, g64, ref[dt])
        assert gmx <= 2.0 * ref[dt], (dt, gmx, ref[dt])
    for hi, lo in zip(DTS, DTS[1:]):
        ratio = ref[hi] / ref[lo]
        assert 3.0 <= ratio <= 5.0, (hi, lo, ratio)  # dt^2: 4 per halving
