"""The block size of the pair-once force kernels (csrc/pair_once_plan.h),
built with g++ through tests/pair_once_shim.cpp and checked on the CPU.

The choice decides which kernel a context runs.  Checked, on a 152-SM GPU:
the FP64 64-body blocks from the size where the systems hold 1.5 block pairs
per SM (1,283 bodies; not 1,031) up to 65,536 bodies; above, the narrowest
wide block whose partial rows take at most 2 GiB (65,537: 256; 262,144:
1,024), 4,096 up to 16 GiB (1,048,576), none beyond (2,000,000); the mixed
kernel only from 65,536 bodies (512-entry blocks there, 2,048 at 262,144
and 1,048,576), not for the 256-system ensemble of at most 20,000 bodies
each; a requested size as asked.  These are the sizes the GPU tests and the
benchmark observe through nbody_pair_once.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15079_gb300", "csrc")
NSM = 152


@pytest.fixture(scope="module")
def po(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("po") / "libpo.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "pair_once_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.po_block.restype = ctypes.c_int
    lib.po_block.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
    lib.po_row_bytes.restype = ctypes.c_int64
    lib.po_row_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
    return lib


def _block(po, sizes, mixed, requested=0, nsm=NSM):
    a = np.ascontiguousarray(sizes, dtype=np.int64)
    return po.po_block(a.ctypes.data, a.size, int(mixed), nsm, requested)


@pytest.mark.parametrize("n,want", [(1031, 0), (1283, 64), (2131, 64), (10425, 64), (65536, 64), (65537, 256),
                                    (262144, 1024), (1048576, 4096), (2000000, 0)])
def test_fp64_single_system(po, n, want):
    assert _block(po, [n], mixed=False) == want


@pytest.mark.parametrize("n,want", [(10425, 0), (65535, 0), (65536, 512), (262144, 2048), (1048576, 2048)])
def test_mixed_single_system(po, n, want):
    assert _block(po, [n], mixed=True) == want


def test_wide_block_is_the_narrowest_within_the_budget(po):
    for n in (65537, 100003, 262144, 500000, 1048576, 1500000):
        b = _block(po, [n], mixed=False)
        budget = 2 << 30
        fits = [B for B in (256, 512, 1024, 2048, 4096) if po.po_row_bytes(np.array([n], np.int64).ctypes.data, 1, B)
                <= budget]
        assert b == (fits[0] if fits else 4096), (n, b, fits)
        assert po.po_row_bytes(np.array([n], np.int64).ctypes.data, 1, b) <= 16 << 30


def test_batches(po):
    rng = np.random.default_rng(3)
    small = rng.integers(100, 701, size=48)
    assert _block(po, small, mixed=False) == 64
    assert _block(po, small, mixed=True) == 0
    ensemble = 131 + rng.integers(1000, 20001, size=256)
    assert _block(po, ensemble, mixed=True) == 0  # largest system below 65,536 bodies
    assert _block(po, ensemble, mixed=False) == 64
    # one large system among small ones takes the wide FP64 blocks for all:
    # the narrowest whose rows ([rows of the largest system][3][all bodies])
    # take at most 2 GiB -- 2,048 here (1,024 would need 2.3 GB)
    mix = np.ascontiguousarray(np.concatenate([small, [300000]]), dtype=np.int64)
    assert _block(po, mix, mixed=False) == 2048
    assert po.po_row_bytes(mix.ctypes.data, mix.size, 1024) > 2 << 30 >= po.po_row_bytes(mix.ctypes.data, mix.size,
                                                                                         2048)


def test_requested_size_and_sm_count(po):
    assert _block(po, [10425], mixed=True, requested=128) == 128
    assert _block(po, [1031], mixed=False, requested=256) == 256
    # fewer SMs: 153 block pairs of 1,031 bodies are enough for 100 SMs
    assert _block(po, [1031], mixed=False, nsm=100) == 64
