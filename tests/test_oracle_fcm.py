"""Pins of the oracle's fluctuating FCM (Sec. 4.2) in a periodic cube.

* The grid operators (truncated envelopes, FFT Stokes solve, trapezoidal averaging) equal
  the reciprocal-lattice sum of the continuous operators, evaluated without any grid.
* The lattice sum has Hasimoto's periodic self-mobility, mu0 (1 - 2.837297 a/L + O(a/L)^3),
  with mu0 = 1/(6 pi eta a) when sigma = a/sqrt(pi) (Sec. 4.2).
* J = S*: the grid mobility is symmetric and positive semi-definite; spreading keeps the
  total force.
* Fluctuation-dissipation (Eq. fluctu_dissip): the covariance of J L^-1 D W with the stress
  variances of Sec. 6.1 is exactly (2 kT/dt) J L^-1 S, checked with the dense operators on a
  small grid.
"""
import numpy as np
import pytest

from oracle import fcm

A = 1.0
SIGMA = A / np.sqrt(np.pi)


def _grid_matrix(g, r):
    n = r.shape[0]
    M = np.zeros((3 * n, 3 * n))
    for c in range(3 * n):
        e = np.zeros(3 * n)
        e[c] = 1.0
        M[:, c] = fcm.mobility_apply(g, r, e).reshape(-1)
    return M


def _particles(n, L, seed):
    return np.random.default_rng(seed).uniform(0.0, L, size=(n, 3))


def test_grid_operators_equal_the_lattice_sum():
    L, N = 10.0, 32                       # sigma / h = 1.80, as in Sec. 6.1 (1.86)
    r = _particles(5, L, 1)
    lat = fcm.lattice_mobility(L, SIGMA, r)
    wide = _grid_matrix(fcm.Grid(N, L, SIGMA, R_t=4.5), r)      # envelope tails below 1e-13
    assert np.abs(wide - lat).max() < 1e-11 * np.abs(lat).max()
    # Sec. 6.1's truncation at 3a changes the operator at the 1e-5 level
    paper = _grid_matrix(fcm.Grid(N, L, SIGMA, R_t=3.0), r)
    err = np.abs(paper - lat).max() / np.abs(lat).max()
    assert 1e-9 < err < 2e-5, err


def test_lattice_self_mobility_is_hasimoto():
    mu0 = 1.0 / (6.0 * np.pi * A)
    e = {}
    for L in (10.0, 20.0, 30.0):
        Ms = fcm.lattice_mobility(L, SIGMA, np.zeros((1, 3)))
        np.testing.assert_allclose(Ms, Ms[0, 0] * np.eye(3), atol=1e-14)   # cubic symmetry
        e[L] = Ms[0, 0] / mu0 - (1.0 - 2.837297 * A / L)
        assert abs(e[L]) < 6.0 * (A / L) ** 3, (L, e[L])
    assert 4.0 < e[10.0] / e[20.0] < 12.0      # the remainder falls like (a/L)^3


def test_grid_mobility_symmetric_positive_and_force_conserving():
    L, N = 10.0, 32
    g = fcm.Grid(N, L, SIGMA, R_t=3.0)
    r = _particles(6, L, 2)
    M = _grid_matrix(g, r)
    np.testing.assert_allclose(M, M.T, atol=1e-15 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > -1e-14 * np.abs(M).max()
    lam = np.random.default_rng(3).standard_normal((6, 3))
    f = fcm.spread(fcm.Grid(N, L, SIGMA, R_t=4.5), r, lam)
    np.testing.assert_allclose(f.reshape(3, -1).sum(axis=1) * g.h ** 3, lam.sum(axis=0), atol=1e-11)


def test_fluctuation_dissipation_is_exact_on_the_grid():
    g = fcm.Grid(8, 8.0, 0.9, R_t=3.5)
    r = _particles(3, g.L, 4)
    kT, dt = 1.3, 0.02
    M = _grid_matrix(g, r)
    env = fcm.envelopes(g, r)
    n6 = 6 * g.N ** 3
    B = np.zeros((9, n6))
    for c in range(n6):
        e = np.zeros(n6)
        e[c] = 1.0
        u = fcm.fluctuating_field(g, fcm.stress(g, e, kT, dt))
        B[:, c] = fcm.average(g, r, u, env).reshape(-1)
    cov = B @ B.T                                  # the normals are independent N(0, 1)
    np.testing.assert_allclose(cov, 2.0 * kT / dt * M, rtol=0, atol=1e-10 * np.abs(M).max() * 2.0 * kT / dt)


def test_brownian_velocity_is_reproducible_and_zero_mean_field():
    g = fcm.Grid(16, 8.0, 0.9, R_t=3.5)
    r = _particles(4, g.L, 5)
    v1, u1 = fcm.brownian_velocity(g, r, seed=11, susp=0, step=3, kT=1.0, dt=0.01)
    v2, u2 = fcm.brownian_velocity(g, r, seed=11, susp=0, step=3, kT=1.0, dt=0.01)
    v3, _ = fcm.brownian_velocity(g, r, seed=11, susp=0, step=4, kT=1.0, dt=0.01)
    np.testing.assert_array_equal(v1, v2)
    assert np.abs(v1 - v3).max() > 0.1 * np.abs(v1).max()
    # the solve removes the mean flow and the field is divergence free
    np.testing.assert_allclose(u1.reshape(3, -1).mean(axis=1), 0.0, atol=1e-12)
    kz, ky, kx, keep = fcm.wavenumbers(g)
    uh = np.fft.fftn(u1, axes=(1, 2, 3))
    assert np.abs(kx * uh[0] + ky * uh[1] + kz * uh[2]).max() < 1e-9 * np.abs(uh).max()


def test_envelopes_equal_a_search_of_every_grid_point():
    g = fcm.Grid(32, 10.0, SIGMA, R_t=3.0)
    r = np.concatenate([_particles(6, g.L, 6), [[0.0, 9.99, 5.0], [-0.2, 10.3, 20.1]]])   # edges and outside
    c = np.arange(g.N) * g.h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    X = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    for (idx, w), ri in zip(fcm.envelopes(g, r), r):
        d = X - ri
        d -= g.L * np.round(d / g.L)
        d2 = (d * d).sum(axis=1)
        want = np.flatnonzero(d2 <= g.R_t ** 2)
        order = np.argsort(idx)
        np.testing.assert_array_equal(idx[order], want)
        ref = (2 * np.pi * g.sigma ** 2) ** -1.5 * np.exp(-d2[want] / (2 * g.sigma ** 2))
        np.testing.assert_allclose(w[order], ref, rtol=1e-13, atol=0)


def test_fcm_step_divergence_rfd_is_unbiased_for_fd():
    """Step 3 with FCM re-averages one fluctuating field at perturbed states (Sec. 5): the
    random finite difference (Eq. rfd_div) at the unit vectors sums to the finite difference
    over every body coordinate (Eq. FD) of the same field, and over random W-tilde it is
    unbiased for it."""
    from oracle import geometry as G, rigid
    from oracle.gdc import Params, fd_divergence, rfd_divergence
    from synthetic import shapes
    grid = fcm.Grid(32, 10.0, SIGMA, R_t=3.0)
    lay = G.Layout([shapes.icosahedron()], np.array([0]))
    rng = np.random.default_rng(7)
    Y = np.array([[4.0, 5.0, 5.0]])
    g = rng.standard_normal((1, 4))
    q = g / np.linalg.norm(g, axis=1, keepdims=True)
    p = Params(dt=0.01, kT=1.0, rfd_delta=1e-4)
    _, ufield = fcm.brownian_velocity(grid, G.blob_positions(lay, Y, q), seed=5, susp=0, step=0, kT=1.0, dt=0.01)

    def project(Ys, qs):
        rs = G.blob_positions(lay, Ys, qs)
        Ks = rigid.k_matrix(rs, Ys, lay.blob_body)
        return rigid.lsq_velocity(Ks, rigid.rigid_basis(Ks, lay.n_bodies),
                                  fcm.average(grid, rs, ufield).reshape(-1)).reshape(-1, 6)

    calV = project(Y, q)
    fd = fd_divergence(lay, Y, q, None, calV, p, project)
    unit = sum(rfd_divergence(lay, Y, q, None, np.eye(6)[i], calV, p, project) for i in range(6))
    assert abs(unit - fd) < 1e-10 * abs(fd), (unit, fd)
    samples = np.array([rfd_divergence(lay, Y, q, None, rng.standard_normal(6), calV, p, project) for _ in range(2000)])
    se = samples.std() / np.sqrt(samples.size)
    assert abs(fd) > 5 * se, "the divergence must be resolvable for the test to have power"
    assert abs(samples.mean() - fd) < 4 * se, (samples.mean(), fd, se)
