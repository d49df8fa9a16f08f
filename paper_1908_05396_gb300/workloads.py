"""Seeded synthetic workloads: problem statements and random inputs.

This module holds no arithmetic of the method.  It turns the benchmark
problems of the paper (Sec. 4) into lattice parameters through their defining
dimensionless groups, and draws seeded random numbers.  Both the tests and the
benchmark take their inputs from here; the CPU oracle and the CUDA library are
then fed the same values.

Problems:
  * lid-driven cubic cavity, Re = rho H^n U^(2-n) / K (Sec. 4.3), lid on +y
    moving in +x, every other face a no-slip wall;
  * power-law channel, Re = rho (H/2)^n u_max^(2-n) / K and the body force
    from the printed u_max (Sec. 4.1), walls at -y/+y, periodic x and z;
  * the batched set of cavities and the serving request trace are seeded
    draws of these two problems.
"""
from __future__ import annotations

import dataclasses

import numpy as np

PERIODIC, WALL, LID = 0, 1, 2
CAVITY_FACES = (WALL, WALL, WALL, LID, WALL, WALL)
CHANNEL_FACES = (PERIODIC, PERIODIC, WALL, WALL, PERIODIC, PERIODIC)


@dataclasses.dataclass
class Problem:
    kind: str
    nx: int
    ny: int
    nz: int
    face: tuple
    K: float
    n: float
    U_lid: tuple = (0.0, 0.0, 0.0)
    body_force: tuple = (0.0, 0.0, 0.0)
    Re: float = 0.0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def kwargs(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, face=self.face, K=self.K, n=self.n,
                    U_lid=self.U_lid, body_force=self.body_force)


def cavity(L: int, Re: float, n: float, U: float = 0.05, rho0: float = 1.0,
           dims: tuple | None = None) -> Problem:
    K = rho0 * L ** n * U ** (2.0 - n) / Re
    nx, ny, nz = dims if dims else (L, L, L)
    return Problem("cavity", nx, ny, nz, CAVITY_FACES, K, n, U_lid=(U, 0.0, 0.0), Re=Re)


def channel(H: int, n: float, u_max: float = 0.02, G: float | None = None,
            Re: float | None = None, nx: int = 4, nz: int = 4, rho0: float = 1.0) -> Problem:
    """Either the force G (then K from u_max) or Re (then K and G) is given."""
    h = H / 2.0
    if G is not None:
        K = G * (n / (n + 1.0) * h ** ((n + 1.0) / n) / u_max) ** n
    else:
        K = rho0 * h ** n * u_max ** (2.0 - n) / Re
        G = K * (u_max * (n + 1.0) / n) ** n / h ** (n + 1.0)
    Re_ = rho0 * h ** n * u_max ** (2.0 - n) / K
    return Problem("channel", nx, H, nz, CHANNEL_FACES, K, n, body_force=(G, 0.0, 0.0), Re=Re_)


def channel_profile(p: Problem) -> tuple[np.ndarray, np.ndarray]:
    """Analytic power-law channel velocity at the node centres (Sec. 4.1)."""
    H, n, G, K = p.ny, p.n, p.body_force[0], p.K
    y = np.arange(H) + 0.5 - H / 2.0
    u = n / (n + 1.0) * (G / K) ** (1.0 / n) * ((H / 2.0) ** ((n + 1.0) / n) - np.abs(y) ** ((n + 1.0) / n))
    return y, u


def noise(shape, seed: int, amp: float = 1.0) -> np.ndarray:
    """Seeded uniform noise in [-amp, amp]."""
    return np.random.default_rng(seed).uniform(-amp, amp, size=shape)


def batch_cavities(count: int = 64, seed: int = 0, L_range=(32, 96), Re_range=(50.0, 500.0),
                   n_range=(0.4, 1.6), U: float = 0.05) -> list[Problem]:
    """The batched workload: cavities of uneven size, Re and n (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        Re = float(rng.uniform(*Re_range))
        n = float(rng.uniform(*n_range))
        out.append(cavity(L, Re, n, U=U))
    return out


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the trace
    problem: Problem


def serving_trace(count: int = 256, seed: int = 0, rate: float = 20.0,
                  cavity_L=(32, 192), channel_H=(32, 256), Re_range=(50.0, 1000.0),
                  n_range=(0.4, 1.6), U: float = 0.05, u_c: float = 0.02) -> list[Request]:
    """Poisson arrivals (mean ``rate`` per second) of cavity and channel solves,
    half each, with random size, Re and n (seeded)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        Re = float(rng.uniform(*Re_range))
        n = float(rng.uniform(*n_range))
        if rng.uniform() < 0.5:
            L = int(rng.integers(cavity_L[0], cavity_L[1] + 1))
            prob = cavity(L, Re, n, U=U)
        else:
            H = int(rng.integers(channel_H[0], channel_H[1] + 1))
            prob = channel(H, n, u_max=u_c, Re=Re, nx=8, nz=8)
        out.append(Request(i, t, prob))
    return out
