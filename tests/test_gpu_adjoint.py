"""GPU adjoint (nbody_grad) against the oracle's adjoint, which is itself
pinned by central differences of its forward map (tests/test_oracle_pins.py).

Tolerance: relative error of the whole gradient vector (dL/dr0, dL/dv0,
dL/dm concatenated, each scaled so the blocks weigh alike) within 1e-6 in
FP64 and 1e-3 in mixed precision.
"""
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


def _loss_grads(s, T, idx, tgt, cv):
    """dL/dr_T, dL/dv_T of L = sum |r_idx(T) - tgt|^2 + cv sum |v_idx(T)|^2 at the
    oracle's final state."""
    rT, vT, _ = oracle.verlet(s.G, s.dt, T, s.r, s.v, s.m, openmp=True)
    gr = np.zeros((3, s.n))
    gv = np.zeros((3, s.n))
    gr[:, idx] = 2 * (rT[:, idx] - tgt)
    gv[:, idx] = 2 * cv * vT[:, idx]
    return gr, gv


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("mixed", 1e-3)])
@pytest.mark.parametrize("T,ckpt", [(1, 0), (25, 0), (230, 7)])
def test_grad_vs_oracle(nb, precision, tol, T, ckpt):
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(131, seed=61, n_moons=0)
    rng = np.random.default_rng(T)
    idx = np.sort(rng.choice(np.arange(31, s.n), 16, replace=False))
    tgt = s.r[:, idx] + rng.normal(0, 0.01, (3, idx.size))
    gr, gv = _loss_grads(s, T, idx, tgt, 3.0)
    ref = oracle.grad(s.G, s.dt, T, s.r, s.v, s.m, gr, gv, openmp=True)
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, ckpt_every=ckpt)
    got = [t.cpu().numpy() for t in b.grad(T, torch.tensor(gr), torch.tensor(gv))]
    for g, r in zip(got, ref):
        assert _rel(g, r) <= tol, (_rel(g, r), precision, T)


def test_grad_zero_steps_is_identity(nb):
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(31, seed=4)
    rng = np.random.default_rng(3)
    gr, gv = rng.normal(size=(3, s.n)), rng.normal(size=(3, s.n))
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64")
    dr, dv, dm = (t.cpu().numpy() for t in b.grad(0, torch.tensor(gr), torch.tensor(gv)))
    assert np.array_equal(dr, gr) and np.array_equal(dv, gv) and np.all(dm == 0)


def test_grad_leaves_state_untouched_and_is_repeatable(nb):
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(131, seed=5, n_moons=0)
    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", ckpt_every=10)
    b.step(7)
    before = b.state.clone()
    gr = torch.ones((3, s.n), dtype=torch.float64)
    g1 = b.grad(33, gr)
    g2 = b.grad(33, gr)
    assert torch.equal(b.state, before)
    for x, y in zip(g1, g2):
        assert torch.equal(x, y)
    b.step(1)  # the bound state still steps from where it was
    assert not torch.equal(b.state, before)


def test_autograd_function(nb):
    torch = pytest.importorskip("torch")
    from paper_2112_15079_gb300.autograd import trajectory
    s = inputs.solar_system(131, seed=9, n_moons=0)
    r0 = torch.tensor(s.r, device="cuda", requires_grad=True)
    v0 = torch.tensor(s.v, device="cuda", requires_grad=True)
    m = torch.tensor(s.m, device="cuda", requires_grad=True)
    rT, vT = trajectory(r0, v0, m, 40, s.G, s.dt)
    loss = (rT[:, 40:60] ** 2).sum() + 5.0 * (vT[:, 40:60] ** 2).sum()
    loss.backward()
    gr = np.zeros((3, s.n))
    gv = np.zeros((3, s.n))
    rr, vv, _ = oracle.verlet(s.G, s.dt, 40, s.r, s.v, s.m)
    gr[:, 40:60] = 2 * rr[:, 40:60]
    gv[:, 40:60] = 10.0 * vv[:, 40:60]
    ref = oracle.grad(s.G, s.dt, 40, s.r, s.v, s.m, gr, gv)
    for g, r in zip((r0.grad, v0.grad, m.grad), ref):
        assert _rel(g.cpu().numpy(), r) <= 1e-6


def test_grad_10425_bodies_64_asteroid_loss(nb):
    """The 10,425-body model, 100 steps, loss on 64 seeded asteroids."""
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(10425)
    idx, tgt = inputs.loss_targets(s)
    T = 100
    gr, gv = _loss_grads(s, T, idx, tgt, 0.0)
    ref = oracle.grad(s.G, s.dt, T, s.r, s.v, s.m, gr, None, openmp=True)
    for precision, tol in (("fp64", 1e-6), ("mixed", 1e-3)):
        b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, ckpt_every=30)
        got = [t.cpu().numpy() for t in b.grad(T, torch.tensor(gr))]
        for g, r in zip(got, ref):
            assert _rel(g, r) <= tol, (precision, _rel(g, r))


def test_grad_vs_gpu_central_difference(nb):
    """The adjoint against central differences of the GPU's own FP64 forward
    map (h = 1e-7 relative), along random directions in (r0, v0, m):
    u . grad L = (L(x + h u) - L(x - h u)) / 2h for L = sum_k |r_k(T) - t_k|^2
    over 64 seeded bodies.  Separated bodies (no moons), so the map is smooth
    on the scale of h."""
    torch = pytest.importorskip("torch")
    s = inputs.solar_system(300, seed=41, n_moons=0)
    T = 20
    idx, tgt = inputs.loss_targets(s)

    def loss(r, v, m):
        b = nb.NBody(r, v, m, G=s.G, dt=s.dt, precision="fp64")
        b.step(T)
        rT = b.r.cpu().numpy()
        b.close()
        return float(((rT[:, idx] - tgt) ** 2).sum())

    b = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64")
    b.step(T)
    rT = b.r.cpu().numpy()
    gr = np.zeros((3, s.n))
    gr[:, idx] = 2 * (rT[:, idx] - tgt)
    b2 = nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64")
    dr, dv, dm = (t.cpu().numpy() for t in b2.grad(T, torch.tensor(gr)))
    rng = np.random.default_rng(7)
    for _ in range(3):
        ur = rng.normal(size=(3, s.n)) * np.abs(s.r).max()
        uv = rng.normal(size=(3, s.n)) * np.abs(s.v).max()
        um = rng.normal(size=s.n) * s.m
        h = 1e-7
        fd = (loss(s.r + h * ur, s.v + h * uv, s.m + h * um) - loss(s.r - h * ur, s.v - h * uv, s.m - h * um)) / (2 * h)
        ad = float((dr * ur).sum() + (dv * uv).sum() + (dm * um).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-12, (fd, ad)
