"""The paper's flow validations run on the GPU path at the paper's sizes
(Sec. 4.1, 4.2): the power-law channel against its analytic profile, second-
order grid convergence under diffusive scaling over H = 16..128, and the square
duct at n = 1 against its series solution.  The CPU oracle pins the same
closed forms at smaller sizes (test_oracle_flows)."""
import numpy as np
import pytest

from paper_1908_05396_gb300 import workloads as wl
from test_oracle_flows import _analytic_channel

pytestmark = pytest.mark.gpu

P, W_ = wl.PERIODIC, wl.WALL


@pytest.fixture(scope="module")
def clbm():
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import clbm as c
    c.lib()
    return c


def _steady(lat, tol, chunk, max_steps):
    """Step until the residual (Eq. of reading c11, over the lattice's check
    interval) is at most tol; returns the steps taken."""
    steps = 0
    while steps < max_steps:
        lat.step(chunk)
        steps += chunk
        R, rc = lat.residual()
        assert rc == 0, "diverged"
        if R <= tol:
            return steps
    raise AssertionError(f"not steady after {steps} steps (R = {R})")


def _channel(H, n, umax, Re, nx=1, nz=1):
    # Re = rho (H/2)^n u_max^(2-n) / K (Sec. 4.1); G from the printed u_max
    K = (H / 2) ** n * umax ** (2 - n) / Re
    G = K * (umax * (n + 1) / n) ** n / (H / 2) ** (n + 1)
    prob = wl.Problem("channel", nx, H, nz, (P, P, W_, W_, P, P), K=K, n=n, body_force=(G, 0.0, 0.0))
    return prob, G, K


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_channel_configuration_matches_power_law_profile(clbm, dtype):
    # The channel configuration: 4 x 64 x 4, n = 0.5, G = 1e-6, K for u_c = 0.02,
    # run to steady state; the analytic profile of Sec. 4.1 within 1e-2.
    H, n, G = 64, 0.5, 1e-6
    K = G * (n / (n + 1) * (H / 2) ** ((n + 1) / n) / 0.02) ** n
    prob = wl.Problem("channel", 4, H, 4, (P, P, W_, W_, P, P), K=K, n=n, body_force=(G, 0.0, 0.0))
    with clbm.Lattice(**prob.kwargs(), dtype=dtype, check_interval=100) as lat:
        _steady(lat, 1e-10 if dtype == "f64" else 1e-8, 20000, 2_000_000)
        _, u, gd = lat.fields()
    _, ua = _analytic_channel(H, n, G, K)
    un = u[0].mean(axis=(0, 2))
    assert abs(ua.max() - 0.02) < 1e-6      # centreline between the two middle nodes
    assert np.linalg.norm(un - ua) / np.linalg.norm(ua) < 1e-2
    # the shear-rate output (Eq. strainratetensor, from the non-equilibrium
    # moments) against the analytic |du/dy| = (G |y| / K)^(1/n), away from
    # the centreline, where it vanishes, and from the wall nodes
    y = np.arange(H) + 0.5 - H / 2
    gd_a = (G * np.abs(y) / K) ** (1.0 / n)
    sel = (np.abs(y) > H / 8) & (np.abs(y) < H / 2 - 2)
    gdn = gd.mean(axis=(0, 2))
    err = np.abs(gdn[sel] - gd_a[sel]) / gd_a[sel]
    assert err.max() <= (1e-5 if dtype == "f64" else 1e-3)   # measured 2.5e-6 / 2.1e-4
    # the profile is the same in every x column and z plane
    assert np.abs(u[0] - un[None, :, None]).max() <= (1e-9 if dtype == "f64" else 1e-5) * ua.max()


@pytest.mark.parametrize("n", [0.8, 1.0, 1.5])
def test_channel_grid_convergence_h16_to_h128(clbm, n):
    # Diffusive scaling at fixed Re: u_max ~ 1/H; the error against the
    # analytic profile falls as H^-2 (slope of the two finest grids).
    errs, Hs = [], [16, 32, 64, 128]
    for H in Hs:
        prob, G, K = _channel(H, n, umax=0.04 * 16 / H, Re=4.0)
        with clbm.Lattice(**prob.kwargs(), dtype="f64", check_interval=100) as lat:
            _steady(lat, 1e-12, 20000, 4_000_000)
            _, u, _ = lat.fields()
        _, ua = _analytic_channel(H, n, G, K)
        errs.append(np.linalg.norm(u[0, 0, :, 0] - ua) / np.linalg.norm(ua))
    slope = np.log(errs[3] / errs[2]) / np.log(Hs[3] / Hs[2])
    assert -2.3 <= slope <= -1.7, (errs, slope)
    assert errs[2] < 1e-2


def _duct_series(a, Y, Z, terms=80):
    # Newtonian flow in a square duct of half-width a under unit pressure
    # gradient over viscosity (Sec. 4.2): the classical Fourier series.
    s = np.zeros_like(Y)
    for k in range(1, terms):
        m = 2 * k - 1
        s += (-1) ** (k - 1) * (1 - np.cosh(m * np.pi * Z / (2 * a)) / np.cosh(m * np.pi / 2)) \
            * np.cos(m * np.pi * Y / (2 * a)) / m ** 3
    return 16 * a ** 2 / np.pi ** 3 * s


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_square_duct_newtonian_matches_series(clbm, dtype):
    # 4 x 44 x 44, periodic in x, walls in y and z, n = 1, force for u_max 0.02.
    N, K = 44, 0.1
    a = N / 2
    y = np.arange(N) + 0.5 - a
    Y, Z = np.meshgrid(y, y, indexing="ij")             # [y][z]
    F = 0.02 * K / _duct_series(a, np.zeros(1), np.zeros(1))[0]
    prob = wl.Problem("duct", 4, N, N, (P, P, W_, W_, W_, W_), K=K, n=1.0, body_force=(F, 0.0, 0.0))
    with clbm.Lattice(**prob.kwargs(), dtype=dtype, check_interval=100) as lat:
        _steady(lat, 1e-10 if dtype == "f64" else 1e-8, 5000, 1_000_000)
        _, u, _ = lat.fields()
    un = u[0].mean(axis=2).T                             # [z][y] -> [y][z]
    ua = F / K * _duct_series(a, Y, Z)
    err = np.linalg.norm(un - ua) / np.linalg.norm(ua)
    assert err < 1e-2, err
    # symmetric under y <-> z and under reflections
    assert np.abs(un - un.T).max() <= 1e-6 * ua.max()
    assert np.abs(un - un[::-1, :]).max() <= 1e-6 * ua.max()
