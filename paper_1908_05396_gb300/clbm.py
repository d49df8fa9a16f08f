"""Thin ctypes binding of the C ABI in ``include/clbm.h``.

Argument marshalling only: every step of the method runs inside
``libclbm.so``.  There is no CPU fallback; if the library has not been built
(``paper_1908_05396_gb300.build.build()``), importing the library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
F64, F32, F16S, F16R = 0, 1, 2, 3
PERIODIC, WALL, LID = 0, 1, 2
ROUND_NEAREST, ROUND_STOCHASTIC = 0, 1
DTYPES = {"f64": F64, "f32": F32, "f16s": F16S, "f16r": F16R}

_LOCK = threading.Lock()
_LIB = None


class CLBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"clbm error {code}: {msg}")
        self.code = code


class Domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("face", ctypes.c_int * 6), ("rho0", ctypes.c_double),
                ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("check_interval", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("in_place", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p
# clbm_alloc_fn / clbm_free_fn
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p)
_ALLOCATOR = None   # the registered callbacks, kept alive while registered


def library_path() -> str:
    return _build.LIB


def lib():
    """Load ``libclbm.so`` (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError(f"libclbm.so not built at {path}; run "
                                  "paper_1908_05396_gb300.build.build() first")
            L = ctypes.CDLL(path)
            L.clbm_create.argtypes = [ctypes.POINTER(Domain), ctypes.c_double, ctypes.c_double,
                                      _D, _D, ctypes.c_int, ctypes.POINTER(_H)]
            L.clbm_step.argtypes = [_H, ctypes.c_int64]
            L.clbm_fields.argtypes = [_H, _D, _D, _D]
            L.clbm_fields_device.argtypes = [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.clbm_residual.argtypes = [_H, _D]
            L.clbm_mass.argtypes = [_H, _D]
            L.clbm_get_state.argtypes = [_H, _D]
            L.clbm_set_state.argtypes = [_H, _D]
            L.clbm_steps_done.argtypes = [_H, ctypes.POINTER(ctypes.c_int64)]
            L.clbm_sync.argtypes = [_H]
            L.clbm_destroy.argtypes = [_H]
            L.clbm_last_error.argtypes = [_H]
            L.clbm_last_error.restype = ctypes.c_char_p
            L.clbm_collide_nodes.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             _D, _D, _D, _D, _D, ctypes.c_int64]
            L.clbm_autotune.argtypes = [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        _D]
            L.clbm_set_launch.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.clbm_set_rates.argtypes = [_H, _D]
            L.clbm_set_rounding.argtypes = [_H, ctypes.c_int]
            L.clbm_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
            L.clbm_probe_fma_rate.argtypes = [ctypes.c_int, _D]
            L.clbm_omega_nodes.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _D, _D, _D, _D,
                                           ctypes.c_int64]
            for name in ("clbm_probe_fma_rate", "clbm_omega_nodes", "clbm_autotune", "clbm_set_launch", "clbm_set_rates", "clbm_set_rounding", "clbm_set_allocator",
                         "clbm_create", "clbm_step", "clbm_fields", "clbm_fields_device",
                         "clbm_residual", "clbm_mass", "clbm_get_state", "clbm_set_state",
                         "clbm_steps_done", "clbm_sync", "clbm_destroy", "clbm_collide_nodes"):
                getattr(L, name).restype = ctypes.c_int
            _LIB = L
    return _LIB


def set_allocator(alloc=None, free=None) -> None:
    """Take the device buffers of lattices created from now on from
    ``alloc(nbytes, device, stream) -> int`` (a 256-byte aligned device
    pointer, 0 when out of memory) and return them through
    ``free(ptr, nbytes, device, stream)`` (``clbm_set_allocator``); ``stream``
    is the lattice's CUDA stream as an int.  No arguments: back to cudaMalloc.
    Lattices keep the allocator they were created with."""
    global _ALLOCATOR
    L = lib()
    if alloc is None and free is None:
        _check(L.clbm_set_allocator(_ALLOC_FN(), _FREE_FN(), None))   # NULL, NULL
        _RETIRED.append(_ALLOCATOR)
        _ALLOCATOR = None
        return
    if alloc is None or free is None:
        raise ValueError("give both alloc and free, or neither")

    def _alloc(nbytes, device, stream, user):
        return int(alloc(int(nbytes), int(device), int(stream or 0)) or 0)

    def _free(ptr, nbytes, device, stream, user):
        free(int(ptr or 0), int(nbytes), int(device), int(stream or 0))

    cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(L.clbm_set_allocator(cbs[0], cbs[1], None))
    # lattices created under an earlier allocator still free through it
    _RETIRED.append(_ALLOCATOR)
    _ALLOCATOR = cbs


_RETIRED = []


def use_torch_allocator() -> None:
    """Route lattice device memory through PyTorch's caching allocator, so
    that lattices and tensors share one pool (``torch.cuda.memory_allocated``
    counts the lattices)."""
    import torch

    def alloc(nbytes, device, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

    def free(ptr, nbytes, device, stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec3(v):
    if v is None:
        return None
    return (ctypes.c_double * 3)(*[float(x) for x in v])


def _check(rc: int, h=None):
    if rc != OK:
        msg = lib().clbm_last_error(h)
        raise CLBMError(rc, msg.decode() if msg else "")


class Lattice:
    """One lattice on the current CUDA device (a ``clbm_handle``)."""

    def __init__(self, nx, ny, nz, face=(PERIODIC,) * 6, K=0.1, n=1.0, U_lid=None,
                 body_force=None, dtype="f64", rho0=1.0, nu_min=0.0, nu_max=0.0,
                 check_interval=100, stream=None, in_place=False):
        L = lib()
        d = Domain()
        d.in_place = 1 if in_place else 0
        d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
        for i, f in enumerate(face):
            d.face[i] = int(f)
        d.rho0, d.nu_min, d.nu_max = float(rho0), float(nu_min), float(nu_max)
        d.check_interval = int(check_interval)
        d.stream = stream
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        self.dtype = dtype
        self.check_interval = int(check_interval)
        h = _H()
        code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        _check(L.clbm_create(ctypes.byref(d), float(K), float(n), _vec3(U_lid),
                             _vec3(body_force), code, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def step(self, nsteps: int) -> int:
        rc = lib().clbm_step(self._h, int(nsteps))
        if rc not in (OK, ERR_DIVERGED):
            _check(rc, self._h)
        return rc

    def fields(self, out=None):
        """(rho (nz,ny,nx), u (3,nz,ny,nx), gamma_dot (nz,ny,nx)) as FP64 numpy arrays;
        `out` may give the three host arrays to fill (e.g. views of pinned memory)."""
        if out is None:
            rho, u, gd = np.empty(self.shape), np.empty((3,) + self.shape), np.empty(self.shape)
        else:
            rho, u, gd = out
            for a, shp in ((rho, self.shape), (u, (3,) + self.shape), (gd, self.shape)):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == shp
        _check(lib().clbm_fields(self._h, _dp(rho), _dp(u), _dp(gd)), self._h)
        return rho, u, gd

    def fields_device(self, rho=None, u=None, gamma_dot=None):
        """Write the fields into caller-owned CUDA tensors (float64, contiguous)."""
        def ptr(t, n):
            if t is None:
                return None
            assert t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == n
            return ctypes.c_void_p(t.data_ptr())
        _check(lib().clbm_fields_device(self._h, ptr(rho, self.N), ptr(u, 3 * self.N),
                                        ptr(gamma_dot, self.N)), self._h)

    def residual(self) -> tuple[float, int]:
        out = ctypes.c_double(0.0)
        rc = lib().clbm_residual(self._h, ctypes.byref(out))
        if rc not in (OK, ERR_DIVERGED):
            _check(rc, self._h)
        return out.value, rc

    def mass(self) -> float:
        out = ctypes.c_double(0.0)
        _check(lib().clbm_mass(self._h, ctypes.byref(out)), self._h)
        return out.value

    def get_state(self) -> np.ndarray:
        f = np.empty((19,) + self.shape)
        _check(lib().clbm_get_state(self._h, _dp(f)), self._h)
        return f

    def set_state(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (19,) + self.shape
        _check(lib().clbm_set_state(self._h, _dp(f)), self._h)

    def autotune(self, steps: int = 10) -> dict:
        """Time the launch-shape candidates and keep the fastest (state restored)."""
        bx, by, npt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        us = ctypes.c_double()
        _check(lib().clbm_autotune(self._h, int(steps), ctypes.byref(bx), ctypes.byref(by),
                                   ctypes.byref(npt), ctypes.byref(us)), self._h)
        return dict(block=(bx.value, by.value), npt=npt.value, us_per_step=us.value)

    def set_rates(self, omega) -> None:
        """Relaxation rates omega_9..omega_18: a sequence of 10, or a dict
        {j: omega_j} (missing rates stay 1)."""
        if isinstance(omega, dict):
            omega = [float(omega.get(j, 1.0)) for j in range(9, 19)]
        w = np.ascontiguousarray(omega, dtype=np.float64)
        assert w.shape == (10,)
        _check(lib().clbm_set_rates(self._h, _dp(w)), self._h)

    def set_rounding(self, mode) -> None:
        """FP16 store rounding of an F16S lattice: ROUND_NEAREST (default) or
        ROUND_STOCHASTIC (also accepted as "nearest" / "stochastic")."""
        if isinstance(mode, str):
            mode = {"nearest": ROUND_NEAREST, "stochastic": ROUND_STOCHASTIC}[mode]
        _check(lib().clbm_set_rounding(self._h, int(mode)), self._h)

    def set_launch(self, block_x: int, block_y: int, npt: int) -> None:
        _check(lib().clbm_set_launch(self._h, int(block_x), int(block_y), int(npt)), self._h)

    def steps_done(self) -> int:
        out = ctypes.c_int64(0)
        _check(lib().clbm_steps_done(self._h, ctypes.byref(out)), self._h)
        return out.value

    def sync(self) -> None:
        _check(lib().clbm_sync(self._h), self._h)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().clbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def collide_nodes(f: np.ndarray, K: float, n: float, dtype="f64", body_force=None, rho0=1.0,
                  nu_min=0.0, nu_max=0.0):
    """Collide M independent nodes on the GPU: f is (19, M) plain FP64."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    M = f.shape[1]
    out = np.empty_like(f)
    rho = np.empty(M)
    u = np.empty((3, M))
    gd = np.empty(M)
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().clbm_collide_nodes(code, float(K), float(n), _vec3(body_force), float(rho0),
                                    float(nu_min), float(nu_max), _dp(f), _dp(out), _dp(rho),
                                    _dp(u), _dp(gd), M))
    return dict(ft=out, rho=rho, u=u, gamma_dot=gd)


def step_noalloc(nx, ny, nz, face, K, n, U_lid, body_force, dtype, src, dst, u_prev, stats,
                 rho0=1.0, nu_min=0.0, nu_max=0.0, stream=None) -> int:
    """One check step between caller-owned device buffers (``clbm_step_noalloc``).

    ``src``, ``dst``, ``u_prev`` and ``stats`` are device addresses (ints) of
    buffers the caller owns, in the dense layouts the header documents.
    Returns the status code; the message of a failure is in
    ``last_error()``."""
    L = lib()
    if not hasattr(L, "_noalloc_ready"):
        L.clbm_step_noalloc.argtypes = [ctypes.POINTER(Domain), ctypes.c_double, ctypes.c_double,
                                        _D, _D, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
        L.clbm_step_noalloc.restype = ctypes.c_int
        L._noalloc_ready = True
    d = Domain()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    for i, f in enumerate(face):
        d.face[i] = int(f)
    d.rho0, d.nu_min, d.nu_max = float(rho0), float(nu_min), float(nu_max)
    d.stream = stream
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return L.clbm_step_noalloc(ctypes.byref(d), float(K), float(n), _vec3(U_lid), _vec3(body_force),
                               code, ctypes.c_void_p(src), ctypes.c_void_p(dst),
                               ctypes.c_void_p(u_prev), ctypes.c_void_p(stats))


def omega_nodes(rho: np.ndarray, m: np.ndarray, K: float, n: float, dtype="f64", nu_min=0.0,
                nu_max=0.0):
    """omega_nu and |gamma_dot| of M nodes from rho (M,) and the non-equilibrium
    moments m^(1)_4..9 given as an array (6, M) (``clbm_omega_nodes``)."""
    L = lib()
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    M = rho.shape[0]
    assert m.shape == (6, M)
    omega = np.empty(M)
    gd = np.empty(M)
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(L.clbm_omega_nodes(code, float(K), float(n), float(nu_min), float(nu_max), _dp(rho),
                              _dp(m), _dp(omega), _dp(gd), M))
    return omega, gd


def probe_fma_rate(dtype="f64") -> float:
    """FMA throughput of the current device in FLOP/s (``clbm_probe_fma_rate``)."""
    L = lib()
    out = ctypes.c_double(0.0)
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(L.clbm_probe_fma_rate(code, ctypes.byref(out)))
    return out.value


def last_error() -> str:
    msg = lib().clbm_last_error(None)
    return msg.decode() if msg else ""


class Batch:
    """Many lattices of one storage form stepped together (``clbm_batch``)."""

    def __init__(self, dtype="f32", capacity=64, check_interval=100, stream=None):
        L = lib()
        if not hasattr(L, "_batch_ready"):
            B = ctypes.c_void_p
            L.clbm_batch_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.POINTER(B)]
            L.clbm_batch_add.argtypes = [B, _H, ctypes.POINTER(ctypes.c_int)]
            L.clbm_batch_remove.argtypes = [B, ctypes.c_int]
            L.clbm_batch_detach.argtypes = [B, _H]
            L.clbm_batch_step.argtypes = [B, ctypes.c_int64]
            L.clbm_batch_stats.argtypes = [B, ctypes.c_int, _D, _D, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int64)]
            L.clbm_batch_set_launch.argtypes = [B, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int]
            L.clbm_batch_set_lattice_launch.argtypes = [B, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_int]
            L.clbm_batch_stats_all.argtypes = [B, _D, _D, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int64)]
            L.clbm_batch_autotune.argtypes = [B, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4 + [_D]
            L.clbm_batch_sync.argtypes = [B]
            L.clbm_batch_destroy.argtypes = [B]
            L.clbm_batch_last_error.argtypes = [B]
            L.clbm_batch_last_error.restype = ctypes.c_char_p
            for n in ("clbm_batch_create", "clbm_batch_add", "clbm_batch_remove", "clbm_batch_detach",
                      "clbm_batch_step", "clbm_batch_stats", "clbm_batch_set_launch",
                      "clbm_batch_set_lattice_launch", "clbm_batch_stats_all",
                      "clbm_batch_autotune", "clbm_batch_sync", "clbm_batch_destroy"):
                getattr(L, n).restype = ctypes.c_int
            L._batch_ready = True
        self._b = ctypes.c_void_p()
        code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.check_interval = int(check_interval)
        self.capacity = int(capacity)
        self._bcheck(L.clbm_batch_create(code, int(capacity), int(check_interval), stream,
                                         ctypes.byref(self._b)), create=True)
        self.members = {}

    def _bcheck(self, rc, create=False):
        if rc != OK:
            L = lib()
            msg = L.clbm_last_error(None) if create else L.clbm_batch_last_error(self._b)
            raise CLBMError(rc, msg.decode() if msg else "")

    def add(self, lat: "Lattice") -> int:
        slot = ctypes.c_int()
        self._bcheck(lib().clbm_batch_add(self._b, lat.handle, ctypes.byref(slot)))
        self.members[slot.value] = lat
        return slot.value

    def remove(self, slot: int) -> "Lattice":
        self._bcheck(lib().clbm_batch_remove(self._b, int(slot)))
        return self.members.pop(slot)

    def step(self, nsteps: int) -> None:
        self._bcheck(lib().clbm_batch_step(self._b, int(nsteps)))

    def stats(self, slot: int) -> dict:
        R, m = ctypes.c_double(), ctypes.c_double()
        dv, st = ctypes.c_int(), ctypes.c_int64()
        self._bcheck(lib().clbm_batch_stats(self._b, int(slot), ctypes.byref(R), ctypes.byref(m),
                                            ctypes.byref(dv), ctypes.byref(st)))
        return dict(residual=R.value, mass=m.value, diverged=bool(dv.value), steps=st.value)

    def stats_all(self) -> dict:
        """``stats`` of every slot as arrays of ``capacity`` entries (empty
        slots: residual and mass NaN, diverged False, steps -1); one sync."""
        n = self.capacity
        R = np.empty(n, dtype=np.float64)
        m = np.empty(n, dtype=np.float64)
        dv = (ctypes.c_int * n)()
        st = (ctypes.c_int64 * n)()
        self._bcheck(lib().clbm_batch_stats_all(self._b, _dp(R), _dp(m), dv, st))
        return dict(residual=R, mass=m, diverged=np.array(dv[:], dtype=bool),
                    steps=np.array(st[:], dtype=np.int64))

    def set_launch(self, block_x, block_y, zc, blocks_per_sm) -> None:
        """The persistent kernel with this launch shape."""
        self._bcheck(lib().clbm_batch_set_launch(self._b, int(block_x), int(block_y), int(zc),
                                                 int(blocks_per_sm)))

    def set_lattice_launch(self, block_x, block_y, npt, streams) -> None:
        """One launch of each lattice's own step kernel per step, on `streams` streams."""
        self._bcheck(lib().clbm_batch_set_lattice_launch(self._b, int(block_x), int(block_y),
                                                         int(npt), int(streams)))

    def autotune(self, steps: int = 6) -> dict:
        """Time the launch choices and keep the fastest; the returned dict
        can be given back to ``apply_launch``."""
        v = [ctypes.c_int() for _ in range(4)]
        us = ctypes.c_double()
        self._bcheck(lib().clbm_batch_autotune(self._b, int(steps), *[ctypes.byref(x) for x in v],
                                               ctypes.byref(us)))
        if v[2].value == 0:
            return dict(mode="per_lattice", block=(v[0].value, v[1].value),
                        npt=5 if v[3].value < 0 else 1, streams=abs(v[3].value),
                        us_per_step=us.value)
        return dict(mode="persistent", block=(v[0].value, v[1].value), zc=v[2].value,
                    blocks_per_sm=v[3].value, us_per_step=us.value)

    def apply_launch(self, info: dict) -> None:
        """Set the launch an ``autotune`` result describes."""
        if info["mode"] == "per_lattice":
            self.set_lattice_launch(*info["block"], info["npt"], info["streams"])
        else:
            self.set_launch(*info["block"], info["zc"], info["blocks_per_sm"])

    def sync(self) -> None:
        self._bcheck(lib().clbm_batch_sync(self._b))

    def close(self) -> None:
        if getattr(self, "_b", None):
            lib().clbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Request(ctypes.Structure):
    _fields_ = [("dom", Domain), ("K", ctypes.c_double), ("n", ctypes.c_double),
                ("U_lid", ctypes.c_double * 3), ("body_force", ctypes.c_double * 3),
                ("tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("plateau_checks", ctypes.c_int), ("keep_fields", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("steps", ctypes.c_int64),
                ("residual", ctypes.c_double), ("mass", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("N", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("active", ctypes.c_int64), ("done", ctypes.c_int64),
                ("used_bytes", ctypes.c_double), ("lattice_updates", ctypes.c_double),
                ("busy_seconds", ctypes.c_double), ("clock", ctypes.c_double)]


SOLVE_STATUS = {0: "converged", 1: "max_steps", 2: "plateau", 3: "diverged", 4: "rejected",
                5: "cancelled", 6: "error"}


class Server:
    """Continuous-batching solve server (``clbm_server``)."""

    def __init__(self, dtype="f16s", hbm_budget_bytes=150e9, max_active=64, check_interval=100):
        L = lib()
        if not hasattr(L, "_server_ready"):
            S = ctypes.c_void_p
            L.clbm_server_create.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(S)]
            L.clbm_server_submit.argtypes = [S, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]
            L.clbm_server_wait.argtypes = [S, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(Result)]
            L.clbm_server_results.argtypes = [S, ctypes.POINTER(Result), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]
            L.clbm_server_fields.argtypes = [S, ctypes.c_int64, _D, _D, _D]
            L.clbm_server_release.argtypes = [S, ctypes.c_int64]
            L.clbm_server_info.argtypes = [S, ctypes.POINTER(ServerStats)]
            L.clbm_server_set_rounding.argtypes = [S, ctypes.c_int]
            L.clbm_server_destroy.argtypes = [S]
            L.clbm_server_last_error.argtypes = [S]
            L.clbm_server_last_error.restype = ctypes.c_char_p
            for n in ("clbm_server_create", "clbm_server_submit", "clbm_server_wait",
                      "clbm_server_results", "clbm_server_fields", "clbm_server_release",
                      "clbm_server_info", "clbm_server_set_rounding", "clbm_server_destroy"):
                getattr(L, n).restype = ctypes.c_int
            L._server_ready = True
        self._s = ctypes.c_void_p()
        code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        rc = L.clbm_server_create(code, float(hbm_budget_bytes), int(max_active),
                                  int(check_interval), ctypes.byref(self._s))
        if rc != OK:
            msg = L.clbm_last_error(None)
            raise CLBMError(rc, msg.decode() if msg else "")
        self.shapes = {}

    def _scheck(self, rc):
        if rc != OK:
            msg = lib().clbm_server_last_error(self._s)
            raise CLBMError(rc, msg.decode() if msg else "")

    def set_rounding(self, mode) -> None:
        """Store rounding of the lattices admitted from now on (F16S servers):
        ROUND_NEAREST or ROUND_STOCHASTIC, or "nearest" / "stochastic"."""
        if isinstance(mode, str):
            mode = {"nearest": ROUND_NEAREST, "stochastic": ROUND_STOCHASTIC}[mode]
        self._scheck(lib().clbm_server_set_rounding(self._s, int(mode)))

    def submit(self, nx, ny, nz, face, K, n, U_lid=None, body_force=None, tol=1e-7,
               max_steps=0, plateau_checks=0, keep_fields=False, rho0=1.0, nu_min=0.0,
               nu_max=0.0) -> int:
        r = Request()
        r.dom.nx, r.dom.ny, r.dom.nz = int(nx), int(ny), int(nz)
        for i, f in enumerate(face):
            r.dom.face[i] = int(f)
        r.dom.rho0, r.dom.nu_min, r.dom.nu_max = float(rho0), float(nu_min), float(nu_max)
        r.K, r.n = float(K), float(n)
        for i in range(3):
            r.U_lid[i] = float(U_lid[i]) if U_lid is not None else 0.0
            r.body_force[i] = float(body_force[i]) if body_force is not None else 0.0
        r.tol, r.max_steps = float(tol), int(max_steps)
        r.plateau_checks, r.keep_fields = int(plateau_checks), int(bool(keep_fields))
        rid = ctypes.c_int64()
        self._scheck(lib().clbm_server_submit(self._s, ctypes.byref(r), ctypes.byref(rid)))
        self.shapes[rid.value] = (int(nz), int(ny), int(nx))
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        res = Result()
        self._scheck(lib().clbm_server_wait(self._s, int(rid), float(timeout), ctypes.byref(res)))
        return res.as_dict()

    def results(self, max_n: int = 4096) -> list:
        arr = (Result * max_n)()
        n = ctypes.c_int()
        self._scheck(lib().clbm_server_results(self._s, arr, max_n, ctypes.byref(n)))
        return [arr[i].as_dict() for i in range(n.value)]

    def fields(self, rid: int):
        shape = self.shapes[rid]
        rho, u, gd = np.empty(shape), np.empty((3,) + shape), np.empty(shape)
        self._scheck(lib().clbm_server_fields(self._s, int(rid), _dp(rho), _dp(u), _dp(gd)))
        return rho, u, gd

    def release(self, rid: int) -> None:
        self._scheck(lib().clbm_server_release(self._s, int(rid)))

    def info(self) -> dict:
        st = ServerStats()
        self._scheck(lib().clbm_server_info(self._s, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self) -> None:
        if getattr(self, "_s", None):
            lib().clbm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
