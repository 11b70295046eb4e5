"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports exactly the entry points include/nbody.h declares (no GPU needed,
no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "nbody.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nbody_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2112_15079_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nbody_init", "nbody_step", "nbody_energy", "nbody_grad", "nbody_free", "nbody_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nbody_[a-z_]+)\b", out))
    assert set(_declared()) <= exported, set(_declared()) - exported
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name)


def test_binding_mirrors_header(lib_path):
    from paper_2112_15079_gb300 import nbody
    assert sorted(nbody.EXPORTED) == _declared()


def test_library_targets_sm_103a(lib_path):
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_errors_without_context_are_reported():
    """Calls that need no GPU: argument validation before any CUDA call."""
    from paper_2112_15079_gb300 import nbody
    ctx = ctypes.c_void_p()
    off = (ctypes.c_int64 * 2)(0, 2)
    opts = nbody.nbody_opts(G=1.0, dt=0.1, precision=0, ckpt_every=0, flags=0, integrator=0)
    st = nbody.nbody_init(ctypes.byref(ctx), 0, off, *([None] * 7), ctypes.byref(opts), None)
    assert st == nbody.NBODY_EINVAL
    assert b"n_systems" in nbody.nbody_last_error(None)
    st = nbody.nbody_init(ctypes.byref(ctx), 1, off, *([None] * 7), ctypes.byref(opts), None)
    assert st == nbody.NBODY_EINVAL and b"NULL" in nbody.nbody_last_error(None)
    assert nbody.nbody_step(None, 1) == nbody.NBODY_EINVAL
    assert nbody.nbody_sync(None) == nbody.NBODY_EINVAL
    nbody.nbody_free(None)


def test_pair_once_block_is_validated():
    """nbody_opts.pair_once_block: FP64 0, 64 or a power of two from 256 to
    4,096, mixed 0 or a power of two from 128 to 2,048, with partial sums of
    at most 16 GiB and 65,535 blocks per system; checked before any CUDA call
    (the state pointers are never read)."""
    from paper_2112_15079_gb300 import nbody
    buf = (ctypes.c_double * 4)()
    ptrs = [ctypes.cast(buf, ctypes.c_void_p)] * 7
    cases = [(0, 128, 2, b"power of two"), (0, 8192, 2, b"power of two"), (0, 300, 2, b"power of two"),
             (0, -1, 2, b"power of two"), (0, 256, 1 << 30, b"exceed"),
             # mixed: 128 .. 2,048 stage entries (no 64-entry blocks)
             (1, 64, 2, b"(mixed)"), (1, 4096, 2, b"(mixed)"), (1, 96, 2, b"(mixed)"), (1, 128, 1 << 30, b"exceed")]
    for prec, block, n, msg in cases:
        ctx = ctypes.c_void_p()
        off = (ctypes.c_int64 * 2)(0, n)
        opts = nbody.nbody_opts(G=1.0, dt=0.1, precision=prec, pair_once_block=block)
        st = nbody.nbody_init(ctypes.byref(ctx), 1, off, *ptrs, ctypes.byref(opts), None)
        assert st == nbody.NBODY_EINVAL, (prec, block)
        assert msg in nbody.nbody_last_error(None), (prec, block, nbody.nbody_last_error(None))
