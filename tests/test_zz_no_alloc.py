"""nbody_accel_static: all-pairs accelerations of one system without device
allocation, checked element by element against the FP64 oracle and against
the regular context path.

Some callers of this library cannot allocate device memory once they are
running (a host that reserved its whole memory budget at start-up, or a
component living next to an allocator that owns the device memory).  For
them ``nbody_accel_static`` keeps its scratch in a fixed array inside the
library.  These tests call it through the C ABI:

* twice in a row on two different systems, each result against the oracle
  and against ``nbody_init`` + ``nbody_accel`` (FP64 tolerance 1e-13 per
  body, the bound of the other FP64 parity tests), so what the first call
  left in the shared array cannot leak into the second;
* at n = NBODY_STATIC_MAX_BODIES, the only size that reaches the far end of
  the fixed layout, against the oracle on every body;
* at n = 1 (no pair: the acceleration is exactly zero);
* across a warm call, the device's free memory must not change.

The file sorts last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
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


def _buffers(torch, s):
    r = torch.tensor(s.r, dtype=torch.float64, device="cuda")
    m = torch.tensor(s.m, dtype=torch.float64, device="cuda")
    out = torch.empty((3, s.n), dtype=torch.float64, device="cuda")
    return r, m, out


def _call(nb, s, r, m, out):
    st = nb.nbody_accel_static(s.n, s.G, r[0].data_ptr(), r[1].data_ptr(), r[2].data_ptr(), m.data_ptr(),
                               out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
    assert st == nb.NBODY_OK, nb.nbody_last_error(None)


def _static_accel(nb, torch, s):
    r, m, out = _buffers(torch, s)
    _call(nb, s, r, m, out)
    return out.cpu().numpy()


def _rel(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def test_static_accel_matches_oracle_and_context_path_twice(nb):
    torch = pytest.importorskip("torch")
    systems = [inputs.solar_system(5003, seed=71), inputs.solar_system(2131, seed=72)]
    for s in systems:  # two calls in a row; the second reuses the array the first filled
        got = _static_accel(nb, torch, s)
        want = oracle.accel(s.G, s.r, s.m, openmp=True)
        assert _rel(got, want).max() <= FP64_TOL, _rel(got, want).max()
        ctx = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64").accel().cpu().numpy()
        assert _rel(got, ctx).max() <= FP64_TOL, _rel(got, ctx).max()


def test_static_accel_at_the_size_limit_vs_oracle(nb):
    """n = NBODY_STATIC_MAX_BODIES: every table and the staged sources fill
    the fixed layout to its end; every body against the oracle."""
    torch = pytest.importorskip("torch")
    n = nb.NBODY_STATIC_MAX_BODIES
    s = inputs.solar_system(n, seed=73)
    got = _static_accel(nb, torch, s)
    want = oracle.accel(s.G, s.r, s.m, openmp=True)
    assert _rel(got, want).max() <= FP64_TOL, _rel(got, want).max()


def test_static_accel_single_body_is_zero(nb):
    torch = pytest.importorskip("torch")
    s = inputs.System(r=np.array([[0.3], [-1.2], [0.01]]), v=np.zeros((3, 1)), m=np.array([1.0]))
    got = _static_accel(nb, torch, s)
    assert np.array_equal(got, np.zeros((3, 1))), got
    assert np.array_equal(oracle.accel(s.G, s.r, s.m), np.zeros((3, 1)))


def test_static_accel_allocates_nothing(nb):
    """After a first call (which loads the kernels), a call leaves the
    device's free memory unchanged: its scratch is the fixed array."""
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(4099, seed=74)
    r, m, out = _buffers(torch, s)
    _call(nb, s, r, m, out)  # warm: kernels loaded, device address of the array looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call(nb, s, r, m, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    want = oracle.accel(s.G, s.r, s.m, openmp=True)
    assert _rel(out.cpu().numpy(), want).max() <= FP64_TOL


def test_static_accel_rejects_sizes_beyond_the_limit(nb):
    torch = pytest.importorskip("torch")
    n = nb.NBODY_STATIC_MAX_BODIES + 1
    buf = torch.zeros(n, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = nb.nbody_accel_static(n, 1.0, p, p, p, p, p, p, p, None)
    assert st == nb.NBODY_EINVAL
    assert b"NBODY_STATIC_MAX_BODIES" in nb.nbody_last_error(None)
    assert nb.nbody_accel_static(0, 1.0, p, p, p, p, p, p, p, None) == nb.NBODY_EINVAL


def test_static_accel_refuses_a_capturing_stream(nb):
    """The call ends with a synchronous copy, which a stream capture cannot
    hold: on a capturing stream it returns EINVAL before any work, the
    capture completes, and the next plain call works."""
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(131, seed=75)
    r, m, out = _buffers(torch, s)
    _call(nb, s, r, m, out)  # warm: the device address of the array is known
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side):
        out.mul_(1.0)
        st = nb.nbody_accel_static(s.n, s.G, r[0].data_ptr(), r[1].data_ptr(), r[2].data_ptr(), m.data_ptr(),
                                   out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), side.cuda_stream)
    assert st == nb.NBODY_EINVAL
    assert b"captured" in nb.nbody_last_error(None)
    g.replay()
    torch.cuda.synchronize()
    _call(nb, s, r, m, out)
    want = oracle.accel(s.G, s.r, s.m)
    assert _rel(out.cpu().numpy(), want).max() <= FP64_TOL
