"""Pins of the oracle's collision against what the paper fixes.

P2  g^_4..18 re-derived by solving the central-moment relaxation equation
    (Eq. centralmomentrelaxation) order by order as small dense linear systems,
    for random states and random distinct relaxation rates.  This is a second
    route to the printed closed forms (Eqs. collisionkernelg4..g18) and catches
    any dropped term, sign, index or bracket in them.
P3  Mass and momentum are collision invariants (Sec. 3.1: g^_0..3 = 0); with a
    body force the momentum changes by exactly F.
P4  Equilibrium at rest is a fixed point for any density (reading [c4]); the
    literal attractor without 1/rho is not.
P5  With every rate 1 the post-collision central moments equal the factorised
    attractors (Eq. discretecentralmomentattractors).
P6  n = 1: omega_nu = [K/(rho c_s^2) + 1/2]^-1 bitwise (Eq. localvarationsrelaxationtimes).
P7  The omega_nu solve returns the root of its defining equation, or a clamp
    with the sign that makes the clamp the root [c6].
"""
import numpy as np
import pytest

SEEDS = range(6)


def _random_state(oracle, rng, amp=0.3):
    w = oracle.weights()
    return w * (1.0 + amp * rng.uniform(-1, 1, 19)) * rng.uniform(0.8, 1.25)


def _central_combos(c):
    ex, ey, ez = c[:, 0], c[:, 1], c[:, 2]
    # The relaxed combinations that pair with g^_4..g^_18, in order.
    return np.array([
        ex * ey, ex * ez, ey * ez,
        ex ** 2 - ey ** 2, ex ** 2 + ey ** 2 - 2 * ez ** 2, ex ** 2 + ey ** 2 + ez ** 2,
        ex * ey ** 2 + ex * ez ** 2, ex ** 2 * ey + ey * ez ** 2, ex ** 2 * ez + ey ** 2 * ez,
        ex * ey ** 2 - ex * ez ** 2, ey * ez ** 2 - ex ** 2 * ey, ex ** 2 * ez - ey ** 2 * ez,
        ex ** 2 * ey ** 2 + ex ** 2 * ez ** 2 + ey ** 2 * ez ** 2,
        ex ** 2 * ey ** 2 + ex ** 2 * ez ** 2 - 2 * ey ** 2 * ez ** 2,
        ex ** 2 * ey ** 2 - ex ** 2 * ez ** 2])


def _solve_g(e, K, fs, omega, over_rho=True):
    """g^ from Eq. centralmomentrelaxation, one order at a time.

    For each relaxed combination c_j of central moments:
        <c_j(e - u) | K g^> = omega_j (c_j(kappa^at) - c_j(kappa)),
    second order first, then third, then fourth, whose attractor uses the
    post-collision diagonal second moments.
    """
    rho = fs.sum()
    u = fs @ e / rho
    c = e - u
    C = _central_combos(c)
    M = C @ K[:, 4:]
    kap = C @ fs
    g = np.zeros(19)
    at2 = np.array([0, 0, 0, 0, 0, rho])          # 3 c_s^2 rho for the trace
    g[4:10] = np.linalg.solve(M[0:6, 0:6], omega[4:10] * (at2 - kap[0:6]))
    post = fs + K @ g
    kt = [(c[:, i] ** 2) @ post for i in range(3)]
    b3 = omega[10:16] * (0.0 - kap[6:12]) - M[6:12, 0:6] @ g[4:10]
    g[10:16] = np.linalg.solve(M[6:12, 6:12], b3)
    s = 1.0 / rho if over_rho else 1.0
    at4 = s * np.array([kt[0] * kt[1] + kt[0] * kt[2] + kt[1] * kt[2],
                        kt[0] * kt[1] + kt[0] * kt[2] - 2 * kt[1] * kt[2],
                        kt[0] * kt[1] - kt[0] * kt[2]])
    b4 = omega[16:19] * (at4 - kap[12:15]) - M[12:15, 0:12] @ g[4:16]
    g[16:19] = np.linalg.solve(M[12:15, 12:15], b4)
    return g


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("n", [1.0, 0.6, 1.4])
def test_g_rederived_from_central_moment_relaxation(oracle, seed, n):
    rng = np.random.default_rng(100 + seed)
    e = oracle.velocities().astype(float)
    K = oracle.kmatrix()
    for _ in range(40):
        f = _random_state(oracle, rng)
        om = {j: rng.uniform(0.3, 1.9) for j in range(9, 19)}
        p = oracle.Params(K=rng.uniform(0.005, 0.2), n=n, omega_high=om)
        r = oracle.collide(p, f)
        omega = np.zeros(19)
        omega[4:9] = r["omega_nu"]
        for j in range(9, 19):
            omega[j] = om[j]
        g = _solve_g(e, K, f, omega)
        scale = np.abs(r["g"]).max()
        np.testing.assert_allclose(r["g"], g, rtol=0, atol=1e-12 * scale)
        # and the post-collision populations are f + K g^ (no force here)
        np.testing.assert_allclose(r["ft"], f + K @ g, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", SEEDS)
def test_mass_momentum_conserved(oracle, seed):
    rng = np.random.default_rng(200 + seed)
    e = oracle.velocities().astype(float)
    for n in (0.5, 1.0, 1.5):
        for F in ((0, 0, 0), tuple(rng.uniform(-1e-3, 1e-3, 3))):
            p = oracle.Params(K=0.02, n=n, F=F)
            f = _random_state(oracle, rng)
            r = oracle.collide(p, f)
            assert abs(r["ft"].sum() - f.sum()) <= 1e-15 * f.sum()
            np.testing.assert_allclose(r["ft"] @ e - f @ e, F, rtol=0, atol=1e-16)


@pytest.mark.parametrize("rho", [0.9, 1.0, 1.05, 1.3])
def test_rest_equilibrium_is_fixed_point(oracle, rho):
    w = oracle.weights()
    for n in (0.5, 1.0, 1.5):
        p = oracle.Params(K=0.01, n=n)
        r = oracle.collide(p, w * rho)
        np.testing.assert_allclose(r["ft"], w * rho, rtol=0, atol=1e-15)
        assert r["gamma_dot"] < 1e-15


def test_literal_attractor_breaks_rest_fixed_point(oracle):
    # Reading [c4]: without 1/rho the 4th-order attractor differs from the
    # Maxwellian c_s^4 rho away from rho = 1, and the rest state moves.
    w = oracle.weights()
    p = oracle.Params(K=0.01, n=1.0, attractor_over_rho=False)
    np.testing.assert_allclose(oracle.collide(p, w)["ft"], w, atol=1e-16)
    r = oracle.collide(p, w * 1.05)
    assert np.abs(r["ft"] - w * 1.05).max() > 1e-3


def test_unit_rates_reach_attractors(oracle):
    rng = np.random.default_rng(300)
    e = oracle.velocities().astype(float)
    for _ in range(30):
        f = _random_state(oracle, rng)
        rho = f.sum()
        # omega_nu = 1 exactly needs nu = 1/6: Newtonian with K = rho/6.
        p = oracle.Params(K=rho / 6.0, n=1.0)
        r = oracle.collide(p, f)
        assert abs(r["omega_nu"] - 1.0) < 1e-15
        ft = r["ft"]
        u = ft @ e / rho
        c = e - u
        cm = _central_combos(c) @ ft
        kxx, kyy, kzz = ((c[:, i] ** 2) @ ft for i in range(3))
        # Second order: diagonal c_s^2 rho, off-diagonal 0.
        np.testing.assert_allclose([kxx, kyy, kzz], [rho / 3] * 3, atol=1e-15)
        np.testing.assert_allclose(cm[0:3], 0, atol=1e-15)
        # Third order: 0.
        np.testing.assert_allclose(cm[6:12], 0, atol=1e-15)
        # Fourth order: k~ii k~jj / rho.
        at4 = [(kxx * kyy + kxx * kzz + kyy * kzz) / rho,
               (kxx * kyy + kxx * kzz - 2 * kyy * kzz) / rho,
               (kxx * kyy - kxx * kzz) / rho]
        np.testing.assert_allclose(cm[12:15], at4, atol=1e-15)
        # A second collision with the same rates leaves the state unchanged.
        r2 = oracle.collide(oracle.Params(K=ft.sum() / 6.0, n=1.0), ft)
        np.testing.assert_allclose(r2["ft"], ft, atol=2e-16)


@pytest.mark.parametrize("seed", SEEDS)
def test_forced_unit_rates_source_moments(oracle, seed):
    # Reading [c7]: half of the source S_a is added before and half after the
    # collision, and the moments of S are 0, F and u*F + Fu* (u* the
    # half-force velocity).  With every rate 1 the collision takes the second
    # central moments about u* to c_s^2 rho delta_ij (Eq.
    # discretecentralmomentattractors), so after the second half of the
    # source the raw second moments are fixed in closed form:
    #   sum_a ft_a e_ai e_aj = rho (delta_ij / 3 + u*_i u*_j)
    #                          + (u*_i F_j + F_i u*_j) / 2.
    # A wrong sign or a dropped term in the second-order part of S, or S
    # evaluated at j/rho instead of u*, moves the right-hand side by at least
    # |u||F|/2 or |F|^2/4 (>= 1e-6 here), far above round-off.
    rng = np.random.default_rng(700 + seed)
    e = oracle.velocities().astype(float)
    for _ in range(20):
        f = _random_state(oracle, rng)
        F = rng.uniform(-1e-2, 1e-2, 3)
        rho = f.sum()
        j = f @ e
        us = (j + 0.5 * F) / rho
        p = oracle.Params(K=rho / 6.0, n=1.0, F=tuple(F))
        r = oracle.collide(p, f)
        assert abs(r["omega_nu"] - 1.0) < 1e-15
        np.testing.assert_allclose(r["u"], us, rtol=0, atol=1e-16)
        ft = r["ft"]
        assert abs(ft.sum() - rho) <= 1e-15 * rho
        np.testing.assert_allclose(ft @ e, j + F, rtol=0, atol=1e-16)
        second = np.einsum("a,ai,aj->ij", ft, e, e)
        expect = rho * (np.eye(3) / 3 + np.outer(us, us)) + 0.5 * (np.outer(us, F)
                                                                  + np.outer(F, us))
        np.testing.assert_allclose(second, expect, rtol=0, atol=2e-15)


def test_newtonian_rate_closed_form(oracle):
    rng = np.random.default_rng(400)
    for _ in range(50):
        f = _random_state(oracle, rng)
        K = rng.uniform(1e-3, 0.5)
        r = oracle.collide(oracle.Params(K=K, n=1.0), f)
        rho = r["rho"]     # the oracle's own sum, so the comparison is bitwise
        assert abs(rho - f.sum()) <= 1e-15 * rho
        assert r["omega_nu"] == 1.0 / (3.0 * (K / rho) + 0.5)


def _h(oracle, p, rho, m, omega):
    """Eq. localvarationsrelaxationtimes residual, with gamma_dot from the
    invariant of Eq. shearrateexpression written as omega^2 A + B: the
    omega-part of S_ij (Eq. strainratetensor) is traceless."""
    P = np.array([[-(m[7] + m[8]), -3 * m[4], -3 * m[5]],
                  [-3 * m[4], -(-2 * m[7] + m[8]), -3 * m[6]],
                  [-3 * m[5], -3 * m[6], -(m[7] - 2 * m[8])]]) / (2 * rho)
    Q = -p.omega_high.get(9, 1.0) * m[9] / (2 * rho) * np.eye(3)
    S = omega * P + Q
    gd = np.sqrt(2 * np.sum(S * S))
    nu = p.K / rho * gd ** (p.n - 1.0) if gd > 0 else (np.inf if p.n < 1 else 0.0)
    nu_c = min(max(nu, p.nu_min), p.nu_max)
    return 1.0 / omega - 0.5 - 3.0 * nu_c, 1.0 / omega - 0.5 - 3.0 * nu, gd


def test_omega_solve_root_or_clamp(oracle):
    rng = np.random.default_rng(500)
    for _ in range(300):
        n = rng.uniform(0.3, 1.8)
        p = oracle.Params(K=10 ** rng.uniform(-4, 0), n=n)
        rho = rng.uniform(0.9, 1.1)
        m = np.zeros(10)
        m[4:10] = rng.normal(size=6) * 10 ** rng.uniform(-9, -1)
        w, gd = oracle.omega_solve(p, rho, m)
        lo = 1 / (3 * p.nu_max + 0.5)
        hi = 1 / (3 * p.nu_min + 0.5)
        assert lo <= w <= hi
        hc, hu, gd2 = _h(oracle, p, rho, m, w)
        assert abs(gd - gd2) <= 1e-12 * gd2 + 1e-300
        at_hi = abs(w - hi) <= 1e-15 * hi
        at_lo = abs(w - lo) <= 1e-15 * lo
        if not (at_hi or at_lo):
            # interior root of the clamped equation: also the unclamped root
            assert abs(hc) < 1e-10 * (1 / w) and abs(hu) < 1e-10 * (1 / w)
        elif at_hi:
            assert hu >= -1e-12          # nu(gamma_dot) <= nu_min
        else:
            assert hu <= 1e-12           # nu(gamma_dot) >= nu_max


def test_omega_solve_zero_shear(oracle):
    m = np.zeros(10)
    lo = 1 / (3 * 10.0 + 0.5)
    hi = 1 / (3 * 5e-4 + 0.5)
    # n < 1: nu -> infinity, clamped to nu_max; n > 1: nu -> 0, clamped to
    # nu_min (the root sits on the clamp up to the rounding of h there).
    assert oracle.omega_solve(oracle.Params(K=0.01, n=0.5), 1.0, m) == (lo, 0.0)
    w, gd = oracle.omega_solve(oracle.Params(K=0.01, n=1.5), 1.0, m)
    assert abs(w - hi) <= 4e-16 * hi and gd == 0.0
    w, gd = oracle.omega_solve(oracle.Params(K=0.01, n=1.0), 1.0, m)
    assert w == 1 / (3 * 0.01 + 0.5) and gd == 0.0
