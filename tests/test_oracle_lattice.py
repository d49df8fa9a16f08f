"""Pins of the oracle's lattice constants against what the paper prints.

* velocity set: the component vectors |1>, |e_x>, |e_y>, |e_z> of Sec. 3;
* weights: not printed; fixed by c_s^2 = 1/3 and the fourth-order Maxwellian
  central moment c_s^4 rho (Sec. 3, Maxwellian central moments);
* K: the printed element listing (Eq. collisionmatrix1), the printed moment
  table (Eq. momentscascadedcollisionterm) and the printed post-collision list
  (Sec. 3.3).  The oracle builds K from the basis definitions; the printed
  matrix and the printed list each differ from it in exactly one entry, and
  in each case the other printed source sides with the definitions.
"""
import os

import numpy as np

from conftest import GOLDEN

# Sec. 3: |1>, |e_x>, |e_y>, |e_z> as printed after the raw basis.
PRINTED_EX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
PRINTED_EY = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1]
PRINTED_EZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_velocity_set_matches_printed_components(oracle):
    e = oracle.velocities()
    assert e[:, 0].tolist() == PRINTED_EX
    assert e[:, 1].tolist() == PRINTED_EY
    assert e[:, 2].tolist() == PRINTED_EZ


def test_weights_fixed_by_isotropy(oracle):
    # Three symmetry classes (rest, |e|^2 = 1, |e|^2 = 2).  Mass 1, second
    # moment c_s^2 = 1/3, mixed fourth moment c_s^4 = 1/9 fix them uniquely.
    e = oracle.velocities().astype(float)
    s = (e ** 2).sum(1)
    cls = [(s == 0), (s == 1), (s == 2)]
    Amat = np.array([[c.sum() for c in cls],
                     [(e[c, 0] ** 2).sum() for c in cls],
                     [(e[c, 0] ** 2 * e[c, 1] ** 2).sum() for c in cls]])
    wc = np.linalg.solve(Amat, [1.0, 1.0 / 3.0, 1.0 / 9.0])
    w = oracle.weights()
    for c, v in zip(cls, wc):
        np.testing.assert_allclose(w[c], v, rtol=0, atol=1e-15)
    # Maxwellian moments up to fourth order (Sec. 3): odd moments vanish,
    # <e_x^4> = 3 c_s^4.
    assert abs(w @ e[:, 0]) < 1e-16 and abs(w @ (e[:, 0] * e[:, 1])) < 1e-16
    assert abs(w @ e[:, 0] ** 4 - 1.0 / 3.0) < 1e-16


def test_kmatrix_orthogonal_with_expected_norms(oracle):
    K = oracle.kmatrix()
    G = K.T @ K
    assert np.array_equal(G, np.diag(np.diag(G)))
    # Norms of the Gram-Schmidt basis, sum_alpha K_alpha,j^2.
    expect = [19, 10, 10, 10, 4, 4, 4, 12, 36, 2394, 40, 40, 40, 8, 8, 8, 252, 72, 24]
    assert np.diag(G).tolist() == expect


def test_kmatrix_vs_printed_matrix_single_typo(oracle):
    K = oracle.kmatrix()
    P = _load("K_printed.txt")
    diff = np.argwhere(K != P)
    # Reading [c1]: the printed (alpha=15, j=14) entry is -1; the definition
    # K_14 = e_z^2 e_y - e_y e_x^2 at e = (0, 1, 1) gives +1.
    assert diff.tolist() == [[15, 14]]
    assert P[15, 14] == -1 and K[15, 14] == 1
    # With the printed entry the matrix is not orthogonal and column 14 has
    # nonzero mass, so g^_14 would create mass.
    assert P[:, 14].sum() == -2 and K[:, 14].sum() == 0


def test_kmatrix_vs_printed_post_collision_list_single_typo(oracle):
    K = oracle.kmatrix()
    L = _load("post_collision_printed.txt")
    diff = np.argwhere(K != L)
    # Reading [c2]: f~_15 is printed with -g^_6; K_6 = e_y e_z = +1 there.
    assert diff.tolist() == [[15, 6]]
    P = _load("K_printed.txt")
    # The printed list sides with the definition at (15, 14), the printed
    # matrix at (15, 6): the two printed sources agree everywhere else.
    assert np.argwhere(P != L).tolist() == [[15, 6], [15, 14]]


def test_moment_table_matches_printed(oracle):
    K = oracle.kmatrix()
    e = oracle.velocities()
    T = _load("moment_table_printed.txt")
    for row in T:
        m, n, p = (int(v) for v in row[:3])
        mono = e[:, 0] ** m * e[:, 1] ** n * e[:, 2] ** p
        # The table lists g^_4..18 only: g^_0..3 vanish (collision invariants).
        assert np.array_equal((mono @ K)[4:], row[3 + 4:]), (m, n, p)
        assert not row[3:3 + 4].any()
    # Zeroth and first moments of K g^ vanish unless g^_0..3 are nonzero.
    for mono in (np.ones(19), e[:, 0], e[:, 1], e[:, 2]):
        assert np.count_nonzero(mono @ K) == 1
