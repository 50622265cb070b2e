"""Pins of the oracle's wall-corrected mobility and wall forces (oracle/wall.py).

Blake's Green's function must satisfy no slip on the wall and incompressibility; the
regularised mobility must be reciprocal (M_ij(x, y) = M_ji(y, x)^T, which the asymmetric
construction does not give for free), reproduce the published self-mobility of a sphere
above a wall, tend to the unbounded RPY tensor far from the wall and stay positive definite
above it; the wall force is minus the derivative of the Sec. 6.2 potential.
"""
import numpy as np
import pytest

from oracle import rpy, wall


@pytest.fixture(scope="module", autouse=True)
def _symbolic():
    wall._symbolic()


def test_blake_no_slip_on_the_wall():
    rng = np.random.default_rng(1)
    for _ in range(10):
        y = np.array([*rng.uniform(-2, 2, 2), rng.uniform(0.5, 4.0)])
        x = np.array([*rng.uniform(-5, 5, 2), 0.0])
        G = wall.blake(x, y)
        scale = np.abs(wall.blake(x + np.array([0, 0, 1.0]), y)).max()
        assert np.abs(G).max() < 1e-14 * scale


def test_blake_is_divergence_free():
    rng = np.random.default_rng(2)
    eps = 1e-5
    for _ in range(5):
        y = np.array([*rng.uniform(-1, 1, 2), rng.uniform(1.0, 3.0)])
        x = np.array([*rng.uniform(-3, 3, 2), rng.uniform(0.5, 4.0)])
        div = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            div += (wall.blake(x + e, y)[k] - wall.blake(x - e, y)[k]) / (2 * eps)
        assert np.abs(div).max() < 1e-7 * np.abs(wall.blake(x, y)).max()


def test_wall_mobility_is_reciprocal():
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = np.array([*rng.uniform(-3, 3, 2), rng.uniform(1.05, 5.0)])
        y = np.array([*rng.uniform(-3, 3, 2), rng.uniform(1.05, 5.0)])
        np.testing.assert_allclose(wall.wall_correction(x, y, 1.0, 1.0), wall.wall_correction(y, x, 1.0, 1.0).T,
                                   rtol=0, atol=1e-14)


@pytest.mark.parametrize("h", [1.1, 1.5, 2.5, 6.0])
def test_self_mobility_above_a_wall(h):
    a, eta = 1.0, 1.0
    mu0 = 1.0 / (6 * np.pi * eta * a)
    x = np.array([0.4, -0.7, h * a])
    M = mu0 * np.eye(3) + wall.wall_correction(x, x, a, eta)
    s = a / h
    par = 1 - 9 * s / 16 + s ** 3 / 8 - s ** 5 / 16
    perp = 1 - 9 * s / 8 + s ** 3 / 2 - s ** 5 / 8
    np.testing.assert_allclose(M, mu0 * np.diag([par, par, perp]), rtol=0, atol=1e-14)


def test_far_from_the_wall_it_is_unbounded_rpy():
    rng = np.random.default_rng(4)
    r = rng.uniform(0, 6, size=(20, 3))
    M0 = rpy.rpy_matrix(r, 1.0, 1.0)
    # the correction decays like a/h (9a/8h of the self term normal to the wall)
    for h in (1e4, 1e6):
        diff = np.abs(wall.wall_matrix(r + np.array([0.0, 0.0, h]), 1.0, 1.0) - M0).max()
        assert diff < 1.2 * (9.0 / 8.0 / h) * np.abs(M0).max()


def test_wall_mobility_is_positive_definite_above_the_wall():
    rng = np.random.default_rng(5)
    for trial in range(5):
        r = rng.uniform(0, 5, size=(40, 3))
        r[:, 2] = rng.uniform(1.02, 3.0, 40)      # every blob just above the wall, many overlapping
        M = wall.wall_matrix(r, 1.0, 1.0)
        np.testing.assert_allclose(M, M.T, atol=1e-15)
        assert np.linalg.eigvalsh(M).min() > 0
    with pytest.raises(ValueError):
        wall.wall_matrix(np.array([[0.0, 0.0, 0.9]]), 1.0, 1.0)


def test_wall_force_is_minus_the_potential_gradient():
    h = np.linspace(1.05, 4.0, 30)
    eps = 1e-6
    fd = -(wall.wall_potential(h + eps, 23.0, 0.5, 1.0) - wall.wall_potential(h - eps, 23.0, 0.5, 1.0)) / (2 * eps)
    np.testing.assert_allclose(wall.wall_force(h, 23.0, 0.5, 1.0), fd, rtol=1e-7)
    f = wall.blob_wall_forces(np.array([[0, 0, 2.0], [0, 0, 3.0], [5, 0, 2.0]]), np.array([0, 0, 1]), 2, 0.0, 0.5,
                              1.0, 0.18)
    np.testing.assert_allclose(f[:, 2], [-0.09, -0.09, -0.18])
