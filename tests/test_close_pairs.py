"""The host close-pair finder of close-encounter handling
(csrc/close_pairs.h), built with g++ through tests/close_pairs_shim.cpp and
checked on the CPU against a brute-force search written here from the
definition: pair p < j of one system is close if
G (m_p + m_j) dt^2 > theta_c^2 |r_j - r_p|^3; clusters are the connected
components of the close pairs; a cluster takes
k = max over its pairs of ceil(w |dt| / theta_s), w = sqrt(G (m_p + m_j) / d^3).
Systems above 4,096 bodies exercise the heavy-body scan and the grid."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15079_gb300", "csrc")
G = 2.9591220828e-4


@pytest.fixture(scope="module")
def cp(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("cp") / "libcp.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "close_pairs_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.cp_find.restype = ctypes.c_int
    lib.cp_find.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_int64, P, P, P, P]
    return lib


def find(cp, r, m, offsets, dt, tc, ts, cap=100000):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    n = m.shape[0]
    pairs = np.zeros(2 * cap, np.int64)
    cluster = np.zeros(n, np.int32)
    kc = np.zeros(n, np.int32)
    meta = np.zeros(4, np.int64)
    rc = cp.cp_find(len(offsets) - 1, offsets.ctypes.data, r[0].ctypes.data, r[1].ctypes.data, r[2].ctypes.data,
                    m.ctypes.data, G, dt, tc, ts, cap, pairs.ctypes.data, cluster.ctypes.data, kc.ctypes.data,
                    meta.ctypes.data)
    return rc, pairs[:2 * int(meta[0])].reshape(-1, 2), cluster, kc, meta


def brute(r, m, offsets, dt, tc, ts):
    pairs, w = [], {}
    for s in range(len(offsets) - 1):
        b, e = offsets[s], offsets[s + 1]
        for p in range(b, e):
            d = r[:, p + 1:e] - r[:, p:p + 1]
            d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
            d3 = d2 * np.sqrt(d2)
            close = G * (m[p] + m[p + 1:e]) * (dt * dt) > tc * tc * d3
            for jj in np.nonzero(close)[0]:
                j = p + 1 + int(jj)
                pairs.append((p, j))
                w[(p, j)] = math.sqrt(G * (m[p] + m[j]) / d3[jj])
    # connected components
    parent = list(range(len(m)))

    def root(i):
        while parent[i] != i:
            i = parent[i]
        return i
    for p, j in pairs:
        parent[root(p)] = root(j)
    k = {}
    for (p, j), wv in w.items():
        kk = max(1, math.ceil(wv * abs(dt) / ts))
        k[root(p)] = max(k.get(root(p), 0), kk)
    return sorted(pairs), root, k


def _system(rng, n, n_heavy=5, moons=20):
    """Sun, a few planets with moons, and a cloud of light bodies."""
    r = [np.zeros(3)]
    m = [1.0]
    hosts = []
    for i in range(n_heavy):
        a = 1.0 + 2.0 * i
        ph = rng.uniform(0, 2 * np.pi)
        r.append(np.array([a * np.cos(ph), a * np.sin(ph), 0.01 * rng.normal()]))
        m.append(10 ** rng.uniform(-6, -3))
        hosts.append(len(m) - 1)
    for i in range(moons):
        h = hosts[rng.integers(len(hosts))]
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        r.append(r[h] + 10 ** rng.uniform(-4, -1.5) * u)
        m.append(10 ** rng.uniform(-13, -9))
    rest = n - len(m)
    cloud = rng.uniform(-4, 4, size=(rest, 3))
    cloud[:, 2] *= 0.1
    # a few tight light pairs, so the grid has work
    for i in range(0, min(rest, 60), 2):
        cloud[i + 1] = cloud[i] + 1e-6 * rng.normal(size=3)
    r.extend(cloud)
    m.extend(10 ** rng.uniform(-14, -10, size=rest))
    return np.array(r).T.copy(), np.array(m)


@pytest.mark.parametrize("n,tc", [(300, 0.5), (300, 0.05), (5000, 0.5), (5000, 0.1), (9000, 0.02)])
def test_finder_matches_brute_force(cp, n, tc):
    rng = np.random.default_rng(n + int(1000 * tc))
    r, m = _system(rng, n)
    off = np.array([0, n], dtype=np.int64)
    rc, pairs, cluster, kc, meta = find(cp, r, m, off, 0.1, tc, 0.05)
    assert rc == 0
    bp, root, k = brute(r, m, off, 0.1, tc, 0.05)
    got = sorted(map(tuple, pairs.tolist()))
    assert got == bp
    assert meta[0] == len(bp) and meta[3] == (max(k.values()) if k else 0)
    # clusters: the same partition as the components, and each member's k
    members = sorted({p for pq in bp for p in pq})
    assert meta[2] == len(members)
    for p in range(n):
        if p not in members:
            assert cluster[p] == -1 and kc[p] == 0
    for p in members:
        for q in members:
            assert (cluster[p] == cluster[q]) == (root(p) == root(q))
        assert kc[p] == k[root(p)]


def test_systems_are_searched_separately_and_negative_dt(cp):
    rng = np.random.default_rng(3)
    r1, m1 = _system(rng, 200)
    r2, m2 = _system(rng, 4500)
    r = np.concatenate([r1, r2], axis=1)
    m = np.concatenate([m1, m2])
    off = np.array([0, 200, 4700], dtype=np.int64)
    # put a body of system 2 on top of a moon of system 1: no cross-system pair
    r[:, 250] = r[:, 10] + 1e-9
    for dt in (0.1, -0.1):
        rc, pairs, cluster, kc, meta = find(cp, r, m, off, dt, 0.5, 0.05)
        assert rc == 0
        bp, root, k = brute(r, m, off, dt, 0.5, 0.05)
        assert sorted(map(tuple, pairs.tolist())) == bp
        assert all((p < 200) == (j < 200) for p, j in bp)


def test_a_pair_too_fast_for_the_sub_step_limit_is_refused(cp):
    r = np.array([[0.0, 1e-9], [0.0, 0.0], [0.0, 0.0]])
    m = np.array([1.0, 1.0])
    rc, *_ = find(cp, r, m, np.array([0, 2]), 0.1, 0.5, 0.05)
    assert rc == 1
