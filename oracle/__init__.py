"""Oracle for the direct-sum N-body method with velocity Verlet (arXiv:2112.15079).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a thin ctypes
wrapper around ``nbody_oracle.c`` (plain FP64 C, built with gcc
``-O2 -ffp-contract=off``), plus a central finite-difference driver written
on top of the oracle's own forward map.  It shares no code with the CUDA
library in ``paper_2112_15079_gb300``.

Functions (all FP64 numpy arrays, structure-of-arrays):

* ``accel``      -- Eq. 1, the direct-sum acceleration.
* ``accel_rows`` -- Eq. 1 for a sample of target bodies.
* ``term_norm``  -- sum of the magnitudes of the terms of Eq. 1 (error scale).
* ``verlet``     -- Eqs. 3-4, velocity-Verlet steps (Eq. 1 for the force).
* ``rk4``        -- classical fourth-order Runge-Kutta steps on (r, v), the
                    higher-order method Section 2 names.
* ``leapfrog``   -- drift-kick-drift leapfrog steps (Section 2).
* ``respa``      -- close-encounter handling: impulse multiple time stepping
                    with close pairs sub-cycled (an extension beyond Section 2).
* ``energy``     -- total energy (kinetic, potential), the accuracy criterion
                    of Sections 2 and 4.
* ``vjp``        -- vector-Jacobian product of Eq. 1 w.r.t. positions and masses.
* ``grad``       -- dL/d(r0, v0, m) of a loss on the final state by the
                    discrete adjoint of Eqs. 1, 3, 4 (optionally with the
                    magnitude sums that scale each element's rounding error).
* ``fd_grad_dir``-- central finite difference of the same loss along a direction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[bool, ctypes.CDLL] = {}

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def _so_path(openmp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if openmp else "liboracle.so")


def build(openmp: bool | None = None) -> None:
    """Compile the oracle (single-threaded and OpenMP variants) with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    variants = [False, True] if openmp is None else [openmp]
    for omp in variants:
        out = _so_path(omp)
        if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def _lib(openmp: bool = False) -> ctypes.CDLL:
    with _LOCK:
        if openmp not in _LIBS:
            build(openmp)
            lib = ctypes.CDLL(_so_path(openmp))
            lib.oracle_accel.argtypes = [_I64, ctypes.c_double] + [_D] * 7
            lib.oracle_accel.restype = None
            lib.oracle_accel_rows.argtypes = ([_I64, ctypes.c_double] + [_D] * 4
                                              + [_I64, ctypes.POINTER(_I64)] + [_D] * 3)
            lib.oracle_accel_rows.restype = None
            lib.oracle_term_norm_rows.argtypes = ([_I64, ctypes.c_double] + [_D] * 4
                                                  + [_I64, ctypes.POINTER(_I64), _D])
            lib.oracle_term_norm_rows.restype = None
            lib.oracle_verlet.argtypes = ([_I64, ctypes.c_double, ctypes.c_double, _I64]
                                          + [_D] * 10)
            lib.oracle_verlet.restype = ctypes.c_int
            lib.oracle_rk4.argtypes = lib.oracle_verlet.argtypes
            lib.oracle_rk4.restype = ctypes.c_int
            lib.oracle_leapfrog.argtypes = lib.oracle_verlet.argtypes
            lib.oracle_leapfrog.restype = ctypes.c_int
            lib.oracle_energy.argtypes = [_I64, ctypes.c_double] + [_D] * 9
            lib.oracle_energy.restype = None
            lib.oracle_vjp.argtypes = [_I64, ctypes.c_double] + [_D] * 11
            lib.oracle_vjp.restype = None
            lib.oracle_grad.argtypes = ([_I64, ctypes.c_double, ctypes.c_double, _I64]
                                        + [_D] * 15)
            lib.oracle_grad.restype = ctypes.c_int
            lib.oracle_respa.argtypes = ([_I64, ctypes.c_double, ctypes.c_double, _I64, ctypes.c_double,
                                          ctypes.c_double] + [_D] * 10 + [ctypes.POINTER(_I64)] * 2)
            lib.oracle_respa.restype = ctypes.c_int
            lib.oracle_openmp_threads.argtypes = []
            lib.oracle_openmp_threads.restype = ctypes.c_int
            _LIBS[openmp] = lib
        return _LIBS[openmp]


def _c(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads(openmp: bool = True) -> int:
    """Threads the OpenMP build uses (1 for the single-threaded build)."""
    return max(1, _lib(openmp).oracle_openmp_threads())


def accel(G: float, r: np.ndarray, m: np.ndarray, openmp: bool = False) -> np.ndarray:
    """Eq. 1 at positions r [3, n] (x, y, z rows) and masses m [n]; returns [3, n]."""
    r = _f64(r)
    m = _f64(m)
    n = m.shape[0]
    a = np.zeros((3, n))
    _lib(openmp).oracle_accel(n, G, _c(r[0]), _c(r[1]), _c(r[2]), _c(m),
                              _c(a[0]), _c(a[1]), _c(a[2]))
    return a


def accel_rows(G: float, r: np.ndarray, m: np.ndarray, rows, openmp: bool = False) -> np.ndarray:
    """Eq. 1 for the target bodies ``rows`` only; returns [3, len(rows)]."""
    r = _f64(r)
    m = _f64(m)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    a = np.zeros((3, rows.shape[0]))
    _lib(openmp).oracle_accel_rows(m.shape[0], G, _c(r[0]), _c(r[1]), _c(r[2]), _c(m),
                                   rows.shape[0], rows.ctypes.data_as(ctypes.POINTER(_I64)),
                                   _c(a[0]), _c(a[1]), _c(a[2]))
    return a


def term_norm(G: float, r: np.ndarray, m: np.ndarray, rows=None, openmp: bool = False) -> np.ndarray:
    """T_p = sum_{j != p} G m_j / |r_j - r_p|^2 (magnitudes of the terms of
    Eq. 1) for ``rows`` (all bodies when None)."""
    r = _f64(r)
    m = _f64(m)
    n = m.shape[0]
    if rows is None:
        rows_p, k = None, n
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        rows_p, k = rows.ctypes.data_as(ctypes.POINTER(_I64)), rows.shape[0]
    t = np.zeros(k)
    _lib(openmp).oracle_term_norm_rows(n, G, _c(r[0]), _c(r[1]), _c(r[2]), _c(m), k, rows_p, _c(t))
    return t


def verlet(G: float, dt: float, n_steps: int, r: np.ndarray, v: np.ndarray, m: np.ndarray,
           a: np.ndarray | None = None, openmp: bool = False):
    """Eqs. 3-4 for n_steps from (r, v) [3, n]; returns (r, v, a) after the steps.

    ``a`` is the acceleration at the entry positions (computed by Eq. 1 when None).
    """
    r = _f64(r).copy()
    v = _f64(v).copy()
    m = _f64(m)
    a = accel(G, r, m, openmp) if a is None else _f64(a).copy()
    rc = _lib(openmp).oracle_verlet(m.shape[0], G, dt, int(n_steps),
                                    _c(r[0]), _c(r[1]), _c(r[2]), _c(v[0]), _c(v[1]), _c(v[2]),
                                    _c(m), _c(a[0]), _c(a[1]), _c(a[2]))
    if rc != 0:
        raise MemoryError("oracle_verlet: allocation failed")
    return r, v, a


def leapfrog(G: float, dt: float, n_steps: int, r: np.ndarray, v: np.ndarray, m: np.ndarray,
             openmp: bool = False):
    """Drift-kick-drift leapfrog (Section 2 names leapfrog beside Verlet) for
    n_steps from (r, v) [3, n]; returns (r, v, a) after the steps, a = Eq. 1
    at the last half-step positions."""
    r = _f64(r).copy()
    v = _f64(v).copy()
    m = _f64(m)
    a = np.zeros_like(r)
    rc = _lib(openmp).oracle_leapfrog(m.shape[0], G, dt, int(n_steps),
                                      _c(r[0]), _c(r[1]), _c(r[2]), _c(v[0]), _c(v[1]), _c(v[2]),
                                      _c(m), _c(a[0]), _c(a[1]), _c(a[2]))
    if rc != 0:
        raise MemoryError("oracle_leapfrog: allocation failed")
    return r, v, a


def rk4(G: float, dt: float, n_steps: int, r: np.ndarray, v: np.ndarray, m: np.ndarray,
        openmp: bool = False):
    """Classical fourth-order Runge-Kutta (the higher-order method Section 2
    names) on y = (r, v), y' = (v, A(r)), for n_steps from (r, v) [3, n];
    returns (r, v, a) after the steps, a = Eq. 1 at the final positions."""
    r = _f64(r).copy()
    v = _f64(v).copy()
    m = _f64(m)
    a = np.zeros_like(r)
    rc = _lib(openmp).oracle_rk4(m.shape[0], G, dt, int(n_steps),
                                 _c(r[0]), _c(r[1]), _c(r[2]), _c(v[0]), _c(v[1]), _c(v[2]),
                                 _c(m), _c(a[0]), _c(a[1]), _c(a[2]))
    if rc != 0:
        raise MemoryError("oracle_rk4: allocation failed")
    return r, v, a


def respa(G: float, dt: float, n_steps: int, r: np.ndarray, v: np.ndarray, m: np.ndarray,
          theta_c: float, theta_s: float, openmp: bool = False):
    """Close-encounter handling: n_steps impulse multiple-time-step steps
    (close pairs, w dt > theta_c, sub-cycled per cluster with
    k = ceil(w_max dt / theta_s) velocity-Verlet sub-steps on their own
    forces; the rest of Eq. 1 as half kicks of dt).  Returns (r, v, a,
    n_close_pairs, k_max); a = Eq. 1 at the final positions."""
    r = _f64(r).copy()
    v = _f64(v).copy()
    m = _f64(m)
    n = m.shape[0]
    a = np.zeros((3, n))
    npairs = _I64(0)
    kmax = _I64(0)
    rc = _lib(openmp).oracle_respa(n, G, dt, int(n_steps), float(theta_c), float(theta_s),
                                   _c(r[0]), _c(r[1]), _c(r[2]), _c(v[0]), _c(v[1]), _c(v[2]), _c(m),
                                   _c(a[0]), _c(a[1]), _c(a[2]), ctypes.byref(npairs), ctypes.byref(kmax))
    if rc == -2:
        raise ValueError("a close pair would need more than 1e6 sub-steps per step")
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return r, v, a, int(npairs.value), int(kmax.value)


def energy(G: float, r: np.ndarray, v: np.ndarray, m: np.ndarray):
    """(E_kin, E_pot) with Neumaier summation; the total is their sum."""
    r = _f64(r)
    v = _f64(v)
    m = _f64(m)
    ek = ctypes.c_double()
    ep = ctypes.c_double()
    _lib(False).oracle_energy(m.shape[0], G, _c(r[0]), _c(r[1]), _c(r[2]),
                              _c(v[0]), _c(v[1]), _c(v[2]), _c(m),
                              ctypes.byref(ek), ctypes.byref(ep))
    return ek.value, ep.value


def vjp(G: float, r: np.ndarray, m: np.ndarray, w: np.ndarray, openmp: bool = False):
    """(J^T w [3, n], (dA/dm)^T w [n]) of Eq. 1 at (r, m)."""
    r = _f64(r)
    m = _f64(m)
    w = _f64(w)
    n = m.shape[0]
    rho = np.zeros((3, n))
    gm = np.zeros(n)
    _lib(openmp).oracle_vjp(n, G, _c(r[0]), _c(r[1]), _c(r[2]), _c(m),
                            _c(w[0]), _c(w[1]), _c(w[2]),
                            _c(rho[0]), _c(rho[1]), _c(rho[2]), _c(gm))
    return rho, gm


def grad(G: float, dt: float, T: int, r0, v0, m, dL_dr_T, dL_dv_T=None, openmp: bool = False,
         magnitudes: bool = False):
    """(dL/dr0 [3, n], dL/dv0 [3, n], dL/dm [n]) through T Verlet steps.

    magnitudes=True also returns, in the same sweep, the sums of the
    magnitudes of the elementary terms of each element (same shapes): the
    condition-free scale of each gradient element (see oracle_grad)."""
    r0 = _f64(r0)
    v0 = _f64(v0)
    m = _f64(m)
    n = m.shape[0]
    gr = _f64(dL_dr_T).reshape(3, n)
    gv = None if dL_dv_T is None else _f64(dL_dv_T).reshape(3, n)
    out_r = np.zeros((3, n))
    out_v = np.zeros((3, n))
    out_m = np.zeros(n)
    mags = [np.zeros((3, n)), np.zeros((3, n)), np.zeros(n)] if magnitudes else None
    rc = _lib(openmp).oracle_grad(n, G, dt, int(T), _c(r0[0]), _c(r0[1]), _c(r0[2]),
                                  _c(v0[0]), _c(v0[1]), _c(v0[2]), _c(m), _c(gr),
                                  _c(gv) if gv is not None else None,
                                  _c(out_r), _c(out_v), _c(out_m),
                                  *([_c(a) for a in mags] if mags else [None, None, None]))
    if rc != 0:
        raise MemoryError("oracle_grad: allocation failed")
    if magnitudes:
        return out_r, out_v, out_m, mags[0], mags[1], mags[2]
    return out_r, out_v, out_m


def fd_grad_dir(loss, G: float, dt: float, T: int, r0, v0, m, dr, dv, dm, h: float,
                openmp: bool = False) -> float:
    """Central difference (L(x + h u) - L(x - h u)) / (2h) of ``loss(r_T, v_T)``
    along the direction u = (dr, dv, dm), using the oracle's forward map."""
    vals = []
    for s in (+1.0, -1.0):
        r, v, _ = verlet(G, dt, T, r0 + s * h * dr, v0 + s * h * dv, m + s * h * dm,
                         openmp=openmp)
        vals.append(loss(r, v))
    return (vals[0] - vals[1]) / (2.0 * h)
