"""Flow-level pins of the oracle against closed forms and invariants.

P8   power-law channel (Sec. 4.1, analytic u(y)) and second-order grid
     convergence under diffusive scaling (Sec. 4.1, Fig. 4 claim);
P9   |gamma_dot| output against the analytic shear rate of the channel and
     against spectral velocity gradients of a 3D periodic flow;
P10  square duct at n = 1 against the series of Sec. 4.2;
     lid: plane Couette flow between a wall and the moving lid (exactly
     linear for every n, since the shear stress is uniform);
P11  cavity mirror symmetry about the mid z-plane and exact mass conservation;
P12  one step on tiny lattices against a dense restatement (f~ = f + K g^ with
     g^ from the linear solve of Eq. centralmomentrelaxation, then streaming
     by an explicit index map with halfway bounce-back and the lid term).
"""
import numpy as np
import pytest

from test_oracle_collision import _solve_g

P, W_, L_ = 0, 1, 2


def _run_to_steady(oracle, p, f, chunk, tol, max_steps):
    prev = None
    steps = 0
    while steps < max_steps:
        f = oracle.run(p, f, chunk)
        steps += chunk
        _, u, _ = oracle.fields(p, f)
        if prev is not None and oracle.residual(u.reshape(3, -1), prev.reshape(3, -1), chunk) < tol:
            return f, steps
        prev = u.copy()
    raise AssertionError(f"not steady after {steps} steps")


def _channel(oracle, H, n, umax, Re, nx=1):
    # Re = rho (H/2)^n u_max^(2-n) / K  (Sec. 4.1); G from the printed u_max.
    K = (H / 2) ** n * umax ** (2 - n) / Re
    G = K * (umax * (n + 1) / n) ** n / (H / 2) ** (n + 1)
    p = oracle.Params(nx=nx, ny=H, nz=1, face=(P, P, W_, W_, P, P), K=K, n=n, F=(G, 0, 0))
    return p, G, K


def _analytic_channel(H, n, G, K):
    y = np.arange(H) + 0.5 - H / 2
    u = n / (n + 1) * (G / K) ** (1 / n) * ((H / 2) ** ((n + 1) / n) - np.abs(y) ** ((n + 1) / n))
    return y, u


@pytest.mark.parametrize("n", [0.5, 1.0, 1.5])
def test_channel_matches_power_law_profile(oracle, n):
    H = 32
    p, G, K = _channel(oracle, H, n, umax=0.02, Re=4.0)
    f, _ = _run_to_steady(oracle, p, oracle.rest_state(p), 1000, 1e-11, 400000)
    rho, u, gd = oracle.fields(p, f)
    y, ua = _analytic_channel(H, n, G, K)
    un = u[0, 0, :, 0]
    assert np.linalg.norm(un - ua) / np.linalg.norm(ua) < 1e-2
    assert np.abs(u[1:]).max() < 1e-12 * np.abs(un).max() + 1e-18
    # P9: |gamma_dot| = |du/dy| = (G |y| / K)^(1/n), away from the centreline
    gda = (G * np.abs(y) / K) ** (1 / n)
    sel = np.abs(y) > 3
    assert np.abs(gd[0, :, 0][sel] - gda[sel]).max() < 2e-2 * gda.max()


@pytest.mark.parametrize("n", [0.8, 1.0, 1.5])
def test_channel_second_order_grid_convergence(oracle, n):
    errs, Hs = [], [8, 16, 32]
    for H in Hs:
        # diffusive scaling: u_max ~ 1/H at fixed Re
        p, G, K = _channel(oracle, H, n, umax=0.08 * 8 / H, Re=4.0)
        f, _ = _run_to_steady(oracle, p, oracle.rest_state(p), 500, 1e-12, 400000)
        _, u, _ = oracle.fields(p, f)
        _, ua = _analytic_channel(H, n, G, K)
        errs.append(np.linalg.norm(u[0, 0, :, 0] - ua) / np.linalg.norm(ua))
    # Slope of the two finest grids: for n > 1 the exact profile has an
    # unbounded second derivative at the centreline (|y|^(1/n - 1)), and the
    # coarsest grid is not yet asymptotic there.
    slope = np.log(errs[2] / errs[1]) / np.log(Hs[2] / Hs[1])
    assert -2.3 <= slope <= -1.7, (errs, slope)


def test_duct_newtonian_matches_series(oracle):
    N = 24
    a = N / 2
    K = 0.1                     # n = 1: mu = K
    umax_target = 0.02
    # centre value of the series with unit prefactor, to set F for u_max
    y = np.arange(N) + 0.5 - a
    Y, Z = np.meshgrid(y, y, indexing="ij")      # [y][z]

    def series(Yv, Zv):
        s = np.zeros_like(Yv)
        for k in range(1, 60):
            m = 2 * k - 1
            s += (-1) ** (k - 1) * (1 - np.cosh(m * np.pi * Zv / (2 * a)) / np.cosh(m * np.pi / 2)) \
                * np.cos(m * np.pi * Yv / (2 * a)) / m ** 3
        return 16 * a ** 2 / (np.pi ** 3) * s

    F = umax_target * K / series(np.zeros(1), np.zeros(1))[0]
    p = oracle.Params(nx=1, ny=N, nz=N, face=(P, P, W_, W_, W_, W_), K=K, n=1.0, F=(F, 0, 0))
    f, _ = _run_to_steady(oracle, p, oracle.rest_state(p), 1000, 1e-10, 200000)
    _, u, _ = oracle.fields(p, f)
    un = u[0, :, :, 0].T                  # [z][y] -> [y][z]
    ua = F / K * series(Y, Z)
    assert np.linalg.norm(un - ua) / np.linalg.norm(ua) < 1e-2


@pytest.mark.parametrize("n", [0.6, 1.0, 1.4])
@pytest.mark.parametrize("axis", [0, 2])
def test_lid_couette_is_linear(oracle, n, axis):
    H, U = 16, 0.02
    Uv = [0.0, 0.0, 0.0]
    Uv[axis] = U
    # K such that nu = 0.05 at the uniform shear rate U/H
    K = 0.05 * (U / H) ** (1 - n)
    p = oracle.Params(nx=1, ny=H, nz=1, face=(P, P, W_, L_, P, P), K=K, n=n, U=tuple(Uv))
    f, _ = _run_to_steady(oracle, p, oracle.rest_state(p), 1000, 1e-12, 400000)
    _, u, _ = oracle.fields(p, f)
    y = np.arange(H) + 0.5                 # wall at y = 0, lid at y = H
    np.testing.assert_allclose(u[axis, 0, :, 0], U * y / H, rtol=0, atol=2e-4 * U)
    assert abs(oracle.mass(p, f) - H) < 1e-12 * H


def test_cavity_mirror_symmetry_and_mass(oracle):
    L = 10
    p = oracle.Params(nx=L, ny=L, nz=L, face=(W_, W_, W_, L_, W_, W_), K=0.05 * L ** 0.8 / 100,
                      n=0.8, U=(0.05, 0, 0))
    f0 = oracle.rest_state(p)
    f = oracle.run(p, f0, 300)
    _, u, _ = oracle.fields(p, f)
    # mirror z -> L-1-z: u_x, u_y even, u_z odd
    np.testing.assert_allclose(u[0], u[0][::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[1], u[1][::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[2], -u[2][::-1], rtol=0, atol=1e-14)
    # lid drags the fluid under it in +x
    assert u[0, :, L - 1, :].mean() > 0.01
    m0 = oracle.mass(p, f0)
    assert abs(oracle.mass(p, f) - m0) < 1e-12 * m0


def _dense_step(oracle, p, A):
    """One step restated densely: stream by an index map, collide by the
    linear solve of the central-moment relaxation (n = 1, no force)."""
    e = oracle.velocities()
    w = oracle.weights()
    K = oracle.kmatrix()
    opp = [int(np.flatnonzero((e == -e[a]).all(1))[0]) for a in range(19)]
    nz, ny, nx = A.shape[1:]
    dims = (nx, ny, nz)
    f = np.empty_like(A)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for a in range(19):
                    s = [x - e[a, 0], y - e[a, 1], z - e[a, 2]]
                    out = lid = False
                    for d in range(3):
                        if not 0 <= s[d] < dims[d]:
                            face = p.face[2 * d + (0 if s[d] < 0 else 1)]
                            if face == P:
                                s[d] %= dims[d]
                            else:
                                out = True
                                lid = lid or face == L_
                    if out:
                        v = A[opp[a], z, y, x]
                        if lid:
                            v += 6 * w[a] * p.rho0 * float(e[a] @ np.array(p.U))
                    else:
                        v = A[a, s[2], s[1], s[0]]
                    f[a, z, y, x] = v
    B = np.empty_like(A)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                fn = f[:, z, y, x]
                rho = fn.sum()
                om = np.ones(19)
                om[4:9] = 1.0 / (3.0 * p.K / rho + 0.5)
                B[:, z, y, x] = fn + K @ _solve_g(e.astype(float), K, fn, om)
    return B


@pytest.mark.parametrize("shape,faces", [
    ((2, 3, 4), (P, P, P, P, P, P)),
    ((3, 4, 2), (P, P, W_, L_, P, P)),
    ((3, 3, 3), (W_, W_, W_, L_, W_, W_)),
])
def test_tiny_lattice_step_matches_dense_restatement(oracle, shape, faces):
    nx, ny, nz = shape
    rng = np.random.default_rng(7)
    p = oracle.Params(nx=nx, ny=ny, nz=nz, face=faces, K=0.03, n=1.0, U=(0.04, 0, 0.01))
    w = oracle.weights()
    A = w[:, None, None, None] * (1 + 0.2 * rng.uniform(-1, 1, (19, nz, ny, nx)))
    B1 = oracle.run(p, A, 1)
    B2 = _dense_step(oracle, p, A)
    np.testing.assert_allclose(B1, B2, rtol=0, atol=1e-14)


def test_shear_rate_matches_spectral_velocity_gradient(oracle):
    # Smooth 3D periodic flow: all six strain components are nonzero.
    L = 24
    k = 2 * np.pi / L
    x = np.arange(L)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    a = 0.01
    ux = a * (np.sin(k * Z) + np.sin(k * X) * np.cos(k * Y) + 0.5 * np.sin(k * X) * np.cos(k * Z))
    uy = a * (np.sin(k * X) - np.cos(k * X) * np.sin(k * Y) + 0.7 * np.cos(k * Z))
    uz = a * (np.sin(k * Y) - 0.5 * np.cos(k * X) * np.sin(k * Z))
    e = oracle.velocities().astype(float)
    w = oracle.weights()
    # second-order equilibrium as the initial state; the non-equilibrium part
    # builds up within a few relaxation times
    eu = np.einsum("ad,dzyx->azyx", e, np.stack([ux, uy, uz]))
    usq = ux ** 2 + uy ** 2 + uz ** 2
    f = w[:, None, None, None] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * usq)
    p = oracle.Params(nx=L, ny=L, nz=L, K=0.05, n=1.0)
    f = oracle.run(p, f, 30)
    _, u, gd = oracle.fields(p, f)
    kk = np.fft.fftfreq(L) * 2 * np.pi
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")

    def d(fld, K_):
        return np.real(np.fft.ifftn(1j * K_ * np.fft.fftn(fld)))
    grads = [[d(u[i], Kd) for Kd in (KX, KY, KZ)] for i in range(3)]
    S = [[0.5 * (grads[i][j] + grads[j][i]) for j in range(3)] for i in range(3)]
    gd_spec = np.sqrt(2 * sum(S[i][j] ** 2 for i in range(3) for j in range(3)))
    err = np.abs(gd - gd_spec).max() / gd_spec.max()
    assert err < 0.03, err


def test_residual_definition(oracle):
    rng = np.random.default_rng(9)
    u = rng.normal(size=(3, 50))
    assert oracle.residual(u, u, 100) == 0.0
    assert abs(oracle.residual(u, np.zeros_like(u), 100) - 1e-2) < 1e-15
    assert abs(oracle.residual(2 * u, u, 10) - 0.05) < 1e-15


def test_uniform_force_accelerates_periodic_box(oracle):
    # Uniform force on a periodic box at rest: every step adds F to the
    # momentum (F/2 before and F/2 after the collision [c7]), the state stays
    # uniform, and the output velocity u* = (j + F/2)/rho after t steps is
    # (t + 1/2) F / rho0, the time-centred value of the exact u = F t / rho.
    F = (1e-4, 2e-5, -3e-5)
    for n in (0.7, 1.0, 1.3):
        p = oracle.Params(nx=2, ny=3, nz=2, K=0.05, n=n, F=F)
        f = oracle.rest_state(p)
        for t in (1, 7, 40):
            ft = oracle.run(p, f, t)
            rho, u, _ = oracle.fields(p, ft)
            np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
            for d in range(3):
                np.testing.assert_allclose(u[d], (t + 0.5) * F[d], rtol=1e-12, atol=1e-18)
