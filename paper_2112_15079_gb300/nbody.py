"""ctypes binding of ``libnbody.so`` (C ABI in ``include/nbody.h``).

The functions ``nbody_*`` mirror the C entry points one to one and only
marshal arguments; every step of the computation runs in the library's CUDA
kernels.  ``NBody`` is a convenience wrapper that owns the state as torch
CUDA tensors (device memory and the current stream come from torch).

Importing this module loads the library and raises ``ImportError`` when it
has not been built (``python -m paper_2112_15079_gb300.build``): there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbody.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2112_15079_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)

NBODY_OK, NBODY_EINVAL, NBODY_ENOMEM, NBODY_ECUDA, NBODY_ENONFINITE, NBODY_ETIMEOUT = range(6)
NBODY_FP64, NBODY_MIXED = 0, 1
NBODY_FLAG_NO_GRAPH = 1
NBODY_FLAG_NO_SMALL = 2
NBODY_FLAG_NO_SYM = 4
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ETIMEOUT"}
PRECISIONS = {"fp64": NBODY_FP64, "mixed": NBODY_MIXED}
NBODY_VERLET, NBODY_RK4, NBODY_LEAPFROG = 0, 1, 2
INTEGRATORS = {"verlet": NBODY_VERLET, "rk4": NBODY_RK4, "leapfrog": NBODY_LEAPFROG}


class nbody_opts(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32), ("flags", ctypes.c_int32), ("integrator", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p), ("close_omega_dt", ctypes.c_double),
                ("substep_omega_dt", ctypes.c_double), ("pair_once_block", ctypes.c_int32)]


class nbody_tiles(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ipt", ctypes.c_int32), ("tj", ctypes.c_int32),
                ("jsplit", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_P = ctypes.c_void_p
_S = ctypes.c_int  # nbody_status
_SIGS = {
    "nbody_init": (_S, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)] + [_P] * 7
                   + [ctypes.POINTER(nbody_opts), _P]),
    "nbody_step": (_S, [_P, ctypes.c_int64]),
    "nbody_accel": (_S, [_P, _P, _P, _P]),
    "nbody_reset": (_S, [_P]),
    "nbody_reorder": (_S, [_P]),
    "nbody_pair_once": (_S, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "nbody_close_info": (_S, [_P, ctypes.POINTER(ctypes.c_int64)] + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "nbody_energy": (_S, [_P, ctypes.POINTER(ctypes.c_double)]),
    "nbody_grad": (_S, [_P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "nbody_sync": (_S, [_P]),
    "nbody_get_tiles": (_S, [_P, ctypes.POINTER(nbody_tiles)]),
    "nbody_set_tiles": (_S, [_P, ctypes.POINTER(nbody_tiles)]),
    "nbody_autotune": (_S, [_P, ctypes.c_int32, ctypes.POINTER(nbody_tiles), ctypes.POINTER(ctypes.c_double)]),
    "nbody_kernel_times": (_S, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "nbody_free": (None, [_P]),
    "nbody_last_error": (ctypes.c_char_p, [_P]),
    "nbody_peaks": (_S, [ctypes.POINTER(ctypes.c_double)]),
    "nbody_accel_static": (_S, [ctypes.c_int64, ctypes.c_double] + [_P] * 8),
    "nbody_shard": (_S, [_P, ctypes.c_int32, ctypes.c_int32]),
    "nbody_shard_step": (_S, [_P]),
    "nbody_shard_buffer": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class NBodyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != NBODY_OK:
        msg = nbody_last_error(ctx)
        raise NBodyError(status, msg.decode() if msg else "")


def peaks() -> dict:
    """Measured instruction throughputs (1e9 lane-ops/s) and the SM clock."""
    out = (ctypes.c_double * 8)()
    check(nbody_peaks(out))
    keys = ["ffma", "dfma", "rsqrt_f32", "rsqrt_f64", "cvt_f32_f64", "ffma2_lanes", "sm_mhz", "sms"]
    return dict(zip(keys, list(out)))


NBODY_STATIC_MAX_BODIES = 65536


def accel_static(r, m, G: float, stream=None):
    """Eq. 1 accelerations [3, n] (FP64) of one system through
    ``nbody_accel_static``, which allocates no device memory itself (its
    scratch is a fixed array inside the library).  r: [3, n] and m: [n] CUDA
    float64 tensors; the result tensor is allocated here, by torch."""
    torch = _torch()
    n = int(m.shape[0])
    r = r.contiguous()
    out = torch.empty((3, n), dtype=torch.float64, device=r.device)
    s = stream if stream is not None else torch.cuda.current_stream(r.device)
    check(nbody_accel_static(n, float(G), r[0].data_ptr(), r[1].data_ptr(), r[2].data_ptr(), m.data_ptr(),
                             out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), _P(s.cuda_stream or None)))
    return out


def _torch():
    import torch
    return torch


class NBody:
    """State of one or more independent systems, bound to the library.

    r, v: [3, N] (numpy or torch), m: [N]; offsets: [n_systems + 1] CSR
    boundaries (default: one system).  The state lives in ``self.state``, a
    [6, N] float64 CUDA tensor (rows x, y, z, vx, vy, vz), updated in place."""

    def __init__(self, r, v, m, offsets=None, *, G: float, dt: float, precision: str = "fp64",
                 ckpt_every: int = 0, graphs: bool = True, small: bool = True, device=None, stream=None,
                 integrator: str = "verlet", tune_cache: str | None = None, close_omega_dt: float = 0.0,
                 substep_omega_dt: float = 0.05, pair_once: bool = True, pair_once_block: int = 0):
        torch = _torch()
        device = torch.device(device if device is not None else "cuda")
        self.device = device
        r = torch.as_tensor(np.asarray(r) if not torch.is_tensor(r) else r, dtype=torch.float64)
        v = torch.as_tensor(np.asarray(v) if not torch.is_tensor(v) else v, dtype=torch.float64)
        m = torch.as_tensor(np.asarray(m) if not torch.is_tensor(m) else m, dtype=torch.float64)
        n = int(m.shape[0])
        self.n = n
        self.state = torch.empty((6, n), dtype=torch.float64, device=device)
        self.state[0:3].copy_(r.reshape(3, n))
        self.state[3:6].copy_(v.reshape(3, n))
        self.m = m.reshape(n).to(device).contiguous()
        off = np.array([0, n] if offsets is None else offsets, dtype=np.int64)
        self.offsets = off
        self.n_systems = len(off) - 1
        self.G, self.dt, self.precision, self.integrator = float(G), float(dt), precision, integrator
        self._stream = stream if stream is not None else torch.cuda.current_stream(device)
        opts = nbody_opts(G=self.G, dt=self.dt, precision=PRECISIONS[precision], ckpt_every=int(ckpt_every),
                          flags=(0 if graphs else NBODY_FLAG_NO_GRAPH) | (0 if small else NBODY_FLAG_NO_SMALL)
                          | (0 if pair_once else NBODY_FLAG_NO_SYM),
                          integrator=INTEGRATORS[integrator],
                          tune_cache=None if tune_cache is None else os.fsencode(tune_cache),
                          close_omega_dt=float(close_omega_dt), substep_omega_dt=float(substep_omega_dt),
                          pair_once_block=int(pair_once_block))
        self._ctx = _P()
        s = self.state
        ptrs = [s[k].data_ptr() for k in range(6)] + [self.m.data_ptr()]
        off_c = (ctypes.c_int64 * len(off))(*off.tolist())
        with torch.cuda.device(device):
            check(nbody_init(ctypes.byref(self._ctx), self.n_systems, off_c, *ptrs, ctypes.byref(opts),
                             _P(self._stream.cuda_stream or None)))

    # -- views -----------------------------------------------------------
    @property
    def r(self):
        return self.state[0:3]

    @property
    def v(self):
        return self.state[3:6]

    # -- calls -----------------------------------------------------------
    def step(self, n_steps: int = 1) -> None:
        check(nbody_step(self._ctx, int(n_steps)), self._ctx)

    def accel(self):
        a = _torch().empty((3, self.n), dtype=_torch().float64, device=self.device)
        check(nbody_accel(self._ctx, a[0].data_ptr(), a[1].data_ptr(), a[2].data_ptr()), self._ctx)
        return a

    def reset(self) -> None:
        check(nbody_reset(self._ctx), self._ctx)

    @property
    def pair_once(self) -> bool:
        """Whether the force launches evaluate each pair once (FP64 from ~1,200
        bodies, mixed from 65,536; see ``pair_once_block``)."""
        return self.pair_once_block > 0

    @property
    def pair_once_block(self) -> int:
        """Block size of the pair-once force kernel (FP64 bodies, 64 ..
        4,096; mixed stage entries, 128 .. 2,048), or 0 when the force
        launches evaluate every ordered pair."""
        on = ctypes.c_int32()
        check(nbody_pair_once(self._ctx, ctypes.byref(on)), self._ctx)
        return int(on.value)

    def close_info(self) -> dict:
        """Close-encounter handling: close pairs, clusters, cluster members
        and the largest sub-step count per step (all 0 when off)."""
        npairs = ctypes.c_int64()
        ncl, nmem, kmax = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(nbody_close_info(self._ctx, ctypes.byref(npairs), ctypes.byref(ncl), ctypes.byref(nmem),
                               ctypes.byref(kmax)), self._ctx)
        return {"pairs": npairs.value, "clusters": ncl.value, "members": nmem.value, "k_max": kmax.value}

    def reorder(self) -> None:
        """Mixed precision: re-sort the sources spatially at the current
        positions (a performance hint for long runs; no-op in FP64)."""
        check(nbody_reorder(self._ctx), self._ctx)

    def energy(self) -> np.ndarray:
        out = (ctypes.c_double * self.n_systems)()
        check(nbody_energy(self._ctx, out), self._ctx)
        return np.array(list(out))

    def grad(self, n_steps: int, dL_dr_T, dL_dv_T=None):
        """(dL/dr0 [3, N], dL/dv0 [3, N], dL/dm [N]) through n_steps steps
        from the snapshot taken at construction / reset()."""
        torch = _torch()
        gr = torch.as_tensor(dL_dr_T, dtype=torch.float64, device=self.device).reshape(3, self.n).contiguous()
        gv = None if dL_dv_T is None else torch.as_tensor(dL_dv_T, dtype=torch.float64,
                                                          device=self.device).reshape(3, self.n).contiguous()
        dr = torch.empty((3, self.n), dtype=torch.float64, device=self.device)
        dv = torch.empty_like(dr)
        dm = torch.empty((self.n,), dtype=torch.float64, device=self.device)
        check(nbody_grad(self._ctx, int(n_steps), gr.data_ptr(), None if gv is None else gv.data_ptr(),
                         dr.data_ptr(), dv.data_ptr(), dm.data_ptr()), self._ctx)
        return dr, dv, dm

    def sync(self) -> None:
        check(nbody_sync(self._ctx), self._ctx)

    @property
    def tiles(self) -> dict:
        t = nbody_tiles()
        check(nbody_get_tiles(self._ctx, ctypes.byref(t)), self._ctx)
        return t.as_dict()

    @tiles.setter
    def tiles(self, d: dict) -> None:
        t = nbody_tiles(**{k: int(d[k]) for k, _ in nbody_tiles._fields_})
        check(nbody_set_tiles(self._ctx, ctypes.byref(t)), self._ctx)

    def autotune(self, probe_steps: int = 4):
        t = nbody_tiles()
        ms = ctypes.c_double()
        check(nbody_autotune(self._ctx, int(probe_steps), ctypes.byref(t), ctypes.byref(ms)), self._ctx)
        return t.as_dict(), ms.value

    def kernel_times(self, n_steps: int) -> dict:
        """Advance n_steps Verlet steps with each kernel timed alone (CUDA
        events on this context's stream): mean force-kernel, Verlet-kernel and
        per-step milliseconds."""
        out = (ctypes.c_double * 4)()
        check(nbody_kernel_times(self._ctx, int(n_steps), out), self._ctx)
        return {"force_ms": out[0], "verlet_ms": out[1], "step_ms": out[2], "steps": int(out[3])}

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            nbody_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
