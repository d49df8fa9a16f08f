"""Stability limit of the cascaded scheme in the lid-driven cubic cavity.

Sec. 5 (second study) finds, on a 64^3 cavity, the largest lid velocity U_p
for which a run stays stable for 50,000 steps, for a consistency coefficient
set through mu_p = c_s^2 (tau_p - 1/2) and power-law indices n = 0.8, 1, 1.5.
Sec. 3.1 sets the rates omega_9..omega_18 to 1 and notes that tuning them
(the bulk rate omega_9 and the rates of the third and fourth orders) can raise
stability further; here every case carries its own set of rates.

The limit of each case is found by bisection over U_p.  Every bisection round
runs all open cases at once, each as a lattice of one batch, so one round costs
about as much as one long run.  A run counts as unstable once a divergence
check of the library trips: a non-finite value, or a density outside
[0.5, 2].  The cavity is the one of Sec. 4.3: the lid on +y moving in +x,
every other face a no-slip wall, rho0 = 1.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Sequence

CS2 = 1.0 / 3.0
CAVITY_FACES = (1, 1, 1, 2, 1, 1)      # walls; the lid on +y


@dataclasses.dataclass(frozen=True)
class Case:
    """One stability case: power-law index n, tau_p (mu_p = c_s^2 (tau_p - 1/2))
    and the rates omega_9..omega_18 (None: all 1, the choice of Sec. 3.1)."""
    n: float
    tau_p: float
    rates: tuple | None = None
    label: str = "unit"

    @property
    def K(self) -> float:
        return CS2 * (self.tau_p - 0.5)


Runner = Callable[[Sequence[Case], Sequence[float]], list]


def batch_runner(L: int = 64, steps: int = 50_000, dtype: str = "f32",
                 check_interval: int = 1000, chunk: int = 5000, autotune: bool = True) -> Runner:
    """A runner that steps every (case, U_p) pair as an L^3 cavity of one batch
    for `steps` steps and returns, per pair, whether it stayed stable.  Runs
    that diverge leave the batch at the next chunk boundary."""
    from . import clbm

    if steps % check_interval or chunk % check_interval:
        raise ValueError("steps and chunk must be multiples of check_interval")
    launch = {}

    def run(cases: Sequence[Case], U: Sequence[float]) -> list:
        stable = [True] * len(cases)
        if not cases:
            return stable
        with clbm.Batch(dtype, capacity=len(cases), check_interval=check_interval) as b:
            slots = {}
            try:
                for i, (c, u) in enumerate(zip(cases, U)):
                    lat = clbm.Lattice(L, L, L, face=CAVITY_FACES, K=c.K, n=c.n,
                                       U_lid=(float(u), 0.0, 0.0), dtype=dtype,
                                       check_interval=check_interval)
                    if c.rates is not None:
                        lat.set_rates(list(c.rates))
                    slots[b.add(lat)] = i
                if autotune and not launch:
                    launch.update(b.autotune())
                elif launch:
                    b.apply_launch(launch)
                done = 0
                while done < steps and slots:
                    k = min(chunk, steps - done)
                    b.step(k)
                    done += k
                    diverged = b.stats_all()["diverged"]
                    for s, i in list(slots.items()):
                        if diverged[s]:
                            stable[i] = False
                            b.remove(s).close()
                            del slots[s]
            finally:
                for s in list(slots):
                    b.remove(s).close()
        return stable

    return run


def max_lid_velocity(cases: Sequence[Case], run: Runner, u_hi: float = 0.25,
                     rounds: int = 8) -> list:
    """For each case, (u_stable, u_unstable): the largest lid velocity found
    stable and the smallest found unstable, u_unstable - u_stable =
    u_hi / 2^rounds.  A case already stable at u_hi gives (u_hi, None); u = 0
    (a fluid at rest) counts as stable without a run."""
    lo = [0.0] * len(cases)
    hi: list = [u_hi] * len(cases)
    ok = run(cases, hi)
    open_ = []
    for i, s in enumerate(ok):
        if s:
            lo[i], hi[i] = u_hi, None
        else:
            open_.append(i)
    for _ in range(rounds):
        if not open_:
            break
        mids = [(lo[i] + hi[i]) / 2 for i in open_]
        ok = run([cases[i] for i in open_], mids)
        for i, m, s in zip(open_, mids, ok):
            if s:
                lo[i] = m
            else:
                hi[i] = m
    return list(zip(lo, hi))
