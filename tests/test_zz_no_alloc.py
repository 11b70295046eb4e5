"""nbody_accel_static: Eq. 1 without device allocation, checked against the
regular context path.

Some callers of this library cannot allocate device memory once they are
running (a host that reserved its whole memory budget at start-up, or a
component living next to an allocator that owns the device memory).  For
them ``nbody_accel_static`` keeps its scratch in a fixed array inside the
library.  This test calls it through the C ABI twice in a row, on two
different systems, and compares each result with ``nbody_init`` +
``nbody_accel`` (FP64) within the FP64 tolerance of the other parity tests.
The second call checks that what the first call left in the shared array
does not leak into the next result.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2112_15079_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15079_gb300 import build
    build.build()
    from paper_2112_15079_gb300 import nbody
    return nbody


def _static_accel(nb, torch, s):
    r = torch.tensor(s.r, dtype=torch.float64, device="cuda")
    m = torch.tensor(s.m, dtype=torch.float64, device="cuda")
    out = torch.empty((3, s.n), dtype=torch.float64, device="cuda")
    st = nb.nbody_accel_static(s.n, s.G, r[0].data_ptr(), r[1].data_ptr(), r[2].data_ptr(), m.data_ptr(),
                               out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
    assert st == nb.NBODY_OK, nb.nbody_last_error(None)
    return out.cpu().numpy()


def test_static_accel_matches_context_path_twice(nb):
    torch = pytest.importorskip("torch")
    systems = [inputs.solar_system(5003, seed=71), inputs.solar_system(2131, seed=72)]
    for s in systems:  # two calls in a row; the second reuses the array the first filled
        got = _static_accel(nb, torch, s)
        ref = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64").accel().cpu().numpy()
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= FP64_TOL, err.max()


def test_static_accel_rejects_sizes_beyond_the_limit(nb):
    torch = pytest.importorskip("torch")
    n = nb.NBODY_STATIC_MAX_BODIES + 1
    buf = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = nb.nbody_accel_static(n, 1.0, p, p, p, p, p, p, p, None)
    assert st == nb.NBODY_EINVAL
    assert b"NBODY_STATIC_MAX_BODIES" in nb.nbody_last_error(None)
    assert nb.nbody_accel_static(0, 1.0, p, p, p, p, p, p, p, None) == nb.NBODY_EINVAL
