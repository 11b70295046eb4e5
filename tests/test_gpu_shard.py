"""Row shards (nbody_shard / nbody_shard_step / nbody_shard_buffer): the
distributed form of the method, every rank stepping its own block of bodies
against all sources and the ranks exchanging their chunks of the source
buffer after every step.

One GPU here: world 1 runs through the C ABI as is, and worlds of 2 and 3
ranks run as that many contexts on the one GPU, the exchange being device
copies of each rank's chunk into the other ranks' buffers (what the
all-gather does across GPUs; no kernel waits for another).  The whole state,
assembled from every rank's own bodies, is compared with the oracle's
trajectory; bodies are moonless so trajectories stay comparable."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2112_15079_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15079_gb300 import build
    build.build()
    from paper_2112_15079_gb300 import nbody, shard
    return nbody, shard


def _local_group(shard, s, precision, world):
    """`world` shards on this GPU and an exchange that copies every rank's
    chunk into every other rank's buffer."""
    shards = [shard.ShardedNBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, rank=k, world=world,
                                 exchange=lambda sh: None) for k in range(world)]

    def step(n):
        for _ in range(n):
            for sh in shards:
                sh.step_local()
            bufs = [sh.stage_bytes() for sh in shards]
            cb = shards[0].chunk_bytes
            for k in range(world):
                for j in range(world):
                    if j != k:
                        bufs[j][k * cb:(k + 1) * cb].copy_(bufs[k][k * cb:(k + 1) * cb])

    def state():
        out = np.empty((6, s.n))
        for sh in shards:
            b, e = sh.own
            out[:, b:e] = sh.body.state[:, b:e].cpu().numpy()
        return out

    return shards, step, state


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("world,n", [(1, 1001), (2, 1001), (3, 1001), (3, 2048), (4, 5)])
def test_shards_follow_the_oracle(mods, precision, world, n):
    nbody, shard = mods
    s = inputs.solar_system(max(n, 31), seed=33, n_moons=0) if n >= 31 else inputs.System(
        r=np.array([[0.0, 1.0, -1.5, 2.0, 0.5], [0.0, 0.1, 0.3, -0.2, 2.5], [0.0, 0.0, 0.05, 0.0, -0.1]]),
        v=np.array([[0.0, 0.0, 0.001, -0.01, 0.002], [0.0, 0.017, -0.013, 0.011, 0.0], [0.0, 0.0, 0.0, 0.0, 0.001]]),
        m=np.array([1.0, 3e-6, 1e-5, 2e-7, 4e-6]))
    shards, step, state = _local_group(shard, s, precision, world)
    for sh in shards:  # the library's chunk layout is the one every rank derives
        assert sh.chunk_bytes == 32 * shard.chunk_layout(s.n, world)[0]
    T = 30
    step(T)
    for sh in shards:
        sh.sync()
    got = state()
    r_ref, v_ref, _ = oracle.verlet(s.G, s.dt, T, s.r, s.v, s.m, openmp=True)
    tol = 1e-12 if precision == "fp64" else 1e-7
    assert np.abs(got[:3] - r_ref).max() <= tol * max(1.0, np.abs(r_ref).max())
    assert np.abs(got[3:] - v_ref).max() <= tol * max(1e-2, np.abs(v_ref).max())
    for sh in shards:
        sh.close()


def test_shard_of_one_rank_matches_the_whole_context(mods):
    """World 1: the same sums as the unsharded context up to the order of the
    partial sums (FP64, 1e-14 relative after 30 steps)."""
    nbody, shard = mods
    s = inputs.solar_system(2131, seed=34, n_moons=0)
    sh = shard.ShardedNBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", rank=0, world=1,
                            exchange=lambda x: None)
    whole = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", small=False)
    sh.step(30)
    whole.step(30)
    a, b = sh.body.state.cpu().numpy(), whole.state.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_shard_errors(mods):
    nbody, shard = mods
    s = inputs.solar_system(131, seed=35, n_moons=0)
    b = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="mixed")
    ctx = b._ctx
    assert nbody.nbody_shard(ctx, 2, 2) == nbody.NBODY_EINVAL
    assert nbody.nbody_shard(ctx, -1, 2) == nbody.NBODY_EINVAL
    assert nbody.nbody_shard(ctx, 0, 0) == nbody.NBODY_EINVAL
    assert nbody.nbody_shard_step(ctx) == nbody.NBODY_EINVAL  # not a shard yet
    assert nbody.nbody_shard(ctx, 1, 2) == nbody.NBODY_OK
    assert nbody.nbody_shard(ctx, 0, 2) == nbody.NBODY_EINVAL  # already a shard
    for call in (lambda: nbody.nbody_step(ctx, 1), lambda: nbody.nbody_reset(ctx), lambda: nbody.nbody_reorder(ctx)):
        assert call() == nbody.NBODY_EINVAL
    assert b"nbody_shard_step" in nbody.nbody_last_error(ctx)
    p, cb = ctypes.c_void_p(), ctypes.c_int64()
    assert nbody.nbody_shard_buffer(ctx, ctypes.byref(p), ctypes.byref(cb)) == nbody.NBODY_OK
    assert p.value and cb.value == 32 * shard.chunk_layout(s.n, 2)[0]
    assert nbody.nbody_shard_step(ctx) == nbody.NBODY_OK
    b.sync()
    # several systems and other integrators are refused
    off, r, v, m = inputs.concat([inputs.solar_system(31, seed=1), inputs.solar_system(31, seed=2)])
    c = nbody.NBody(r, v, m, off, G=s.G, dt=s.dt, precision="fp64")
    assert nbody.nbody_shard(c._ctx, 0, 2) == nbody.NBODY_EINVAL
    d = nbody.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision="fp64", integrator="rk4")
    assert nbody.nbody_shard(d._ctx, 0, 2) == nbody.NBODY_EINVAL
