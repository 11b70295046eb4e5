"""The autotuner's result cache through the C ABI (nbody_opts.tune_cache):
nbody_autotune writes its winner; a later context with the same key starts
from the cached tiles and steps bitwise like a context given the same tiles
by hand; a damaged file or a stale entry leaves a context on the defaults."""
import json

import numpy as np
import pytest

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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_tune_cache_round_trip(nb, tmp_path, precision):
    s = inputs.solar_system(5003, seed=91)  # above the single-launch kernels' range: the tiles shape every step
    path = tmp_path / "tune.json"
    mk = lambda **kw: nb.NBody(s.r, s.v, s.m, G=s.G, dt=s.dt, precision=precision, **kw)
    default = mk().tiles
    a = mk(tune_cache=str(path))
    assert a.tiles == default  # no file yet
    best, _ = a.autotune(probe_steps=1)
    doc = json.loads(path.read_text())
    (entry,) = doc["entries"]
    assert {k: entry[k] for k in best} == best
    assert entry["precision"] == (1 if precision == "mixed" else 0) and entry["n_log2"] == 12
    # a cached entry with tiles other than the defaults and the winner
    other = ({"threads": 256, "ipt": 2, "tj": 256, "jsplit": 0, "ctas_per_sm": 2} if precision == "mixed"
             else {"threads": 256, "ipt": 1, "tj": 512, "jsplit": 0, "ctas_per_sm": 2})
    entry.update(other)
    path.write_text(json.dumps(doc))
    b = mk(tune_cache=str(path))
    assert b.tiles == other
    c = mk()
    c.tiles = other
    c.reset()
    for x in (b, c):
        x.step(20)
        x.sync()
    assert np.array_equal(b.state.cpu().numpy(), c.state.cpu().numpy())
    # a stale entry (other kernels) and a damaged file leave the defaults
    entry["kernels"] = "0" * 16
    path.write_text(json.dumps(doc))
    assert mk(tune_cache=str(path)).tiles == default
    path.write_text('{"format": "nbody-tune-cache", "version": 1, "entries": [')
    assert mk(tune_cache=str(path)).tiles == default
    # autotune over the damaged file writes a fresh one
    d = mk(tune_cache=str(path))
    best, _ = d.autotune(probe_steps=1)
    assert len(json.loads(path.read_text())["entries"]) == 1
