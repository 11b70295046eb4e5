"""The autotuner's result cache (csrc/tune_cache.h), built with g++ through
tests/tune_cache_shim.cpp and checked on the CPU: entries written by one
context are found by the next one with the same key; a different key (other
kernels, size class, SM count, precision or integrator) finds nothing; a
damaged file never crashes and never yields an entry; writing keeps the
other entries and replaces a damaged file."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15079_gb300", "csrc")
KEY = dict(precision=1, integrator=0, n_log2=13, systems_log2=0, sms=152, kernels="0123456789abcdef")


@pytest.fixture(scope="module")
def tc(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("tc") / "libtc.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "tune_cache_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    I = ctypes.c_int
    lib.tc_store.argtypes = [ctypes.c_char_p, I, I, I, I, I, ctypes.c_char_p, ctypes.POINTER(I), ctypes.c_double]
    lib.tc_lookup.argtypes = [ctypes.c_char_p, I, I, I, I, I, ctypes.c_char_p, ctypes.POINTER(I),
                              ctypes.POINTER(ctypes.c_double)]
    lib.tc_floor_log2.argtypes = [ctypes.c_longlong]
    return lib


def store(tc, path, tiles, ms=0.5, **over):
    k = {**KEY, **over}
    t = (ctypes.c_int * 5)(*tiles)
    return tc.tc_store(str(path).encode(), k["precision"], k["integrator"], k["n_log2"], k["systems_log2"],
                       k["sms"], k["kernels"].encode(), t, ms)


def lookup(tc, path, **over):
    k = {**KEY, **over}
    t = (ctypes.c_int * 5)()
    ms = ctypes.c_double()
    ok = tc.tc_lookup(str(path).encode(), k["precision"], k["integrator"], k["n_log2"], k["systems_log2"],
                      k["sms"], k["kernels"].encode(), t, ctypes.byref(ms))
    return (list(t), ms.value) if ok else None


def test_round_trip_and_keys(tc, tmp_path):
    p = tmp_path / "tune.json"
    assert lookup(tc, p) is None  # no file
    assert store(tc, p, [512, 1, 1024, 0, 2], 0.0674) == 0
    assert lookup(tc, p) == ([512, 1, 1024, 0, 2], 0.0674)
    for field, value in (("kernels", "fedcba9876543210"), ("n_log2", 14), ("systems_log2", 1), ("sms", 148),
                         ("precision", 0), ("integrator", 1)):
        assert lookup(tc, p, **{field: value}) is None, field
    # a second key is added, the first kept; the same key again is replaced
    assert store(tc, p, [128, 1, 1024, 0, 3], 3.1, precision=0) == 0
    assert store(tc, p, [1024, 1, 512, 0, 1], 0.06) == 0
    assert lookup(tc, p) == ([1024, 1, 512, 0, 1], 0.06)
    assert lookup(tc, p, precision=0) == ([128, 1, 1024, 0, 3], 3.1)
    doc = json.loads(p.read_text())  # the file is plain JSON
    assert doc["format"] == "nbody-tune-cache" and doc["version"] == 1 and len(doc["entries"]) == 2
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]  # no temporary file left behind


@pytest.mark.parametrize("text", [
    "", "{", "not json", "[]", '{"format": "nbody-tune-cache", "version": 2, "entries": []}',
    '{"format": "other", "version": 1, "entries": []}',
    '{"format": "nbody-tune-cache", "version": 1, "entries": {}}',
    '{"format": "nbody-tune-cache", "version": 1, "entries": [{"precision": 1}]}',
    '{"format": "nbody-tune-cache", "version": 1, "entries": [{"precision": 1.5, "integrator": 0, "n_log2": 13, '
    '"systems_log2": 0, "sms": 152, "kernels": "0123456789abcdef", "threads": 512, "ipt": 1, "tj": 1024, '
    '"jsplit": 0, "ctas_per_sm": 2}]}',
    '{"format": "nbody-tune-cache", "version": 1, "entries": [{"precision": 1, "integrator": 0, "n_log2": 13, '
    '"systems_log2": 0, "sms": 152, "kernels": 7, "threads": 512, "ipt": 1, "tj": 1024, "jsplit": 0, '
    '"ctas_per_sm": 2}]}',
    "\x00\xff\xfe garbage",
])
def test_damaged_files_yield_nothing_and_are_replaced(tc, tmp_path, text):
    p = tmp_path / "tune.json"
    p.write_bytes(text.encode("latin-1"))
    assert lookup(tc, p) is None
    assert store(tc, p, [256, 2, 512, 0, 2]) == 0
    assert lookup(tc, p) == ([256, 2, 512, 0, 2], 0.5)
    assert len(json.loads(p.read_text())["entries"]) == 1


def test_truncated_file_and_good_entries_beside_bad_ones(tc, tmp_path):
    p = tmp_path / "tune.json"
    assert store(tc, p, [512, 1, 1024, 0, 2]) == 0
    assert store(tc, p, [128, 1, 1024, 0, 3], precision=0) == 0
    full = p.read_text()
    p.write_text(full[: len(full) // 2])  # cut in the middle: unreadable as a whole
    assert lookup(tc, p) is None and lookup(tc, p, precision=0) is None
    # one malformed entry does not hide the well-formed ones
    doc = json.loads(full)
    doc["entries"].insert(0, {"precision": "x"})
    p.write_text(json.dumps(doc))
    assert lookup(tc, p) == ([512, 1, 1024, 0, 2], 0.5)


def test_unwritable_location_is_reported(tc, tmp_path):
    assert store(tc, tmp_path / "no_such_dir" / "tune.json", [512, 1, 1024, 0, 2]) != 0


def test_size_classes(tc):
    assert [tc.tc_floor_log2(v) for v in (1, 2, 3, 31, 10425, 16384, 1 << 20)] == [0, 1, 1, 4, 13, 14, 20]
