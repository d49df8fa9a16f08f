"""FP64 CPU oracle of the D3Q19 cascaded central-moment LBM for power-law fluids.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product library never loads it, and it shares no code with the CUDA path.

The arithmetic lives in ``clbm_oracle.c`` (plain C, FP64, ``-ffp-contract=off``,
one OpenMP loop over z-planes that does not change any result).  This module
compiles it with gcc and exposes it through ctypes.

Each function follows the paper (Adam, Hajabdollahi & Premnath, Sec. 3):
  * ``collide``      -- Eqs. hydrodynamicfields1/2, rawmomentdistributionfunction1,
                        collisionkernelg4..g18, strainratetensor,
                        localvarationsrelaxationtimes, cascadedcollision1.
  * ``run``          -- Eq. cascadedstreaming1 with the boundaries of Sec. 4.
  * ``fields``       -- Eqs. hydrodynamicfields1/2 and shearrateexpression.
  * ``omega_solve``  -- Eq. localvarationsrelaxationtimes with Eq. 6.
Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

PERIODIC, WALL, LID = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [_SRC, os.path.join(_HERE, "clbm_oracle.h")]
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(d) for d in deps)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("face", ctypes.c_int * 6),
        ("K", ctypes.c_double), ("n", ctypes.c_double),
        ("U", ctypes.c_double * 3), ("F", ctypes.c_double * 3),
        ("rho0", ctypes.c_double),
        ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
        ("omega", ctypes.c_double * 19),
        ("attractor_over_rho", ctypes.c_int),
    ]


class _NodeInfo(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double), ("u", ctypes.c_double * 3),
        ("gamma_dot", ctypes.c_double), ("omega_nu", ctypes.c_double),
        ("g", ctypes.c_double * 19),
    ]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_default_params.argtypes = [P]
            lib.orc_omega_solve.argtypes = [P, ctypes.c_double, D, D]
            lib.orc_omega_solve.restype = ctypes.c_double
            lib.orc_collide.argtypes = [P, D, D, ctypes.POINTER(_NodeInfo)]
            lib.orc_rest_state.argtypes = [P, D]
            lib.orc_run.argtypes = [P, D, D, ctypes.c_int64]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_pull.argtypes = [P, D, D]
            lib.orc_fields.argtypes = [P, D, D, D, D]
            lib.orc_residual.argtypes = [D, D, ctypes.c_int64, ctypes.c_int64]
            lib.orc_residual.restype = ctypes.c_double
            lib.orc_mass.argtypes = [P, D]
            lib.orc_mass.restype = ctypes.c_double
            lib.orc_velocities.argtypes = [ctypes.POINTER(ctypes.c_int * 57)]
            lib.orc_weights.argtypes = [D]
            lib.orc_kmatrix.argtypes = [D]
            _LIB = lib
    return _LIB


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Problem statement of one lattice (mirrors ``orc_params``)."""
    nx: int = 1
    ny: int = 1
    nz: int = 1
    face: tuple = (PERIODIC,) * 6        # (-x, +x, -y, +y, -z, +z)
    K: float = 0.1                        # consistency coefficient mu_p
    n: float = 1.0                        # power-law index
    U: tuple = (0.0, 0.0, 0.0)            # lid velocity
    F: tuple = (0.0, 0.0, 0.0)            # body force
    rho0: float = 1.0
    nu_min: float = 5e-4
    nu_max: float = 10.0
    omega_high: dict = field(default_factory=dict)  # {j: omega_j}, j = 9..18
    attractor_over_rho: bool = True

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def c(self) -> _Params:
        p = _Params()
        _lib().orc_default_params(ctypes.byref(p))
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        for i, v in enumerate(self.face):
            p.face[i] = int(v)
        p.K, p.n = float(self.K), float(self.n)
        for i in range(3):
            p.U[i] = float(self.U[i])
            p.F[i] = float(self.F[i])
        p.rho0 = float(self.rho0)
        p.nu_min, p.nu_max = float(self.nu_min), float(self.nu_max)
        for j, w in self.omega_high.items():
            p.omega[int(j)] = float(w)
        p.attractor_over_rho = 1 if self.attractor_over_rho else 0
        return p


def velocities() -> np.ndarray:
    buf = (ctypes.c_int * 57)()
    _lib().orc_velocities(ctypes.byref(buf))
    return np.array(buf[:], dtype=np.int64).reshape(19, 3)


def weights() -> np.ndarray:
    w = np.zeros(19)
    _lib().orc_weights(_dp(w))
    return w


def kmatrix() -> np.ndarray:
    K = np.zeros((19, 19))
    _lib().orc_kmatrix(_dp(K))
    return K


def omega_solve(p: Params, rho: float, m: np.ndarray) -> tuple[float, float]:
    """omega_nu and |gamma_dot| from m^(1)_4..9 (array of 10, entries 4..9 used)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    assert m.shape == (10,)
    gd = ctypes.c_double(0.0)
    pc = p.c()
    w = _lib().orc_omega_solve(ctypes.byref(pc), float(rho), _dp(m), ctypes.byref(gd))
    return w, gd.value


def collide(p: Params, f: np.ndarray) -> dict:
    """One node: pre-collision f (19,) -> dict(ft, rho, u, gamma_dot, omega_nu, g)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (19,)
    ft = np.zeros(19)
    info = _NodeInfo()
    pc = p.c()
    _lib().orc_collide(ctypes.byref(pc), _dp(f), _dp(ft), ctypes.byref(info))
    return dict(ft=ft, rho=info.rho, u=np.array(info.u[:]),
                gamma_dot=info.gamma_dot, omega_nu=info.omega_nu,
                g=np.array(info.g[:]))


def rest_state(p: Params) -> np.ndarray:
    f = np.zeros((19, p.nz, p.ny, p.nx))
    pc = p.c()
    _lib().orc_rest_state(ctypes.byref(pc), _dp(f))
    return f


def run(p: Params, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Return the state after ``nsteps`` steps from ``f`` (19, nz, ny, nx)."""
    A = np.array(f, dtype=np.float64, order="C", copy=True)
    assert A.shape == (19, p.nz, p.ny, p.nx)
    B = np.empty_like(A)
    pc = p.c()
    rc = _lib().orc_run(ctypes.byref(pc), _dp(A), _dp(B), int(nsteps))
    assert rc == 0
    return A


def pull(p: Params, f: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(A)
    pc = p.c()
    _lib().orc_pull(ctypes.byref(pc), _dp(A), _dp(out))
    return out


def fields(p: Params, f: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(rho (nz,ny,nx), u (3,nz,ny,nx), gamma_dot (nz,ny,nx)) of the state."""
    A = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.empty((p.nz, p.ny, p.nx))
    u = np.empty((3, p.nz, p.ny, p.nx))
    gd = np.empty((p.nz, p.ny, p.nx))
    pc = p.c()
    _lib().orc_fields(ctypes.byref(pc), _dp(A), _dp(rho), _dp(u), _dp(gd))
    return rho, u, gd


def residual(u: np.ndarray, u_prev: np.ndarray, delta: int) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(u_prev, dtype=np.float64)
    assert u.shape == v.shape and u.shape[0] == 3
    return _lib().orc_residual(_dp(u), _dp(v), u.size // 3, int(delta))


def mass(p: Params, f: np.ndarray) -> float:
    A = np.ascontiguousarray(f, dtype=np.float64)
    pc = p.c()
    return _lib().orc_mass(ctypes.byref(pc), _dp(A))
