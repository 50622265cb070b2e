"""Pins of the oracle's RPY matrix, K maps, saddle solve, body mobility and square roots."""
import numpy as np
import pytest

from oracle import geometry as G
from oracle import matfree, rigid, rpy
from synthetic import shapes

A, ETA = 1.0, 1.0
MU0 = 1.0 / (6 * np.pi * ETA * A)


def _oseen(rvec):
    r = np.linalg.norm(rvec)
    return (np.eye(3) + np.outer(rvec, rvec) / r ** 2) / (8 * np.pi * ETA * r)


def test_self_term():
    # Single-blob translational mobility 1/(6 pi eta a).
    np.testing.assert_allclose(rpy.rpy_pair(np.zeros(3), A, ETA), MU0 * np.eye(3))
    M = rpy.rpy_matrix(np.zeros((1, 3)), 2.5, 3.0)
    np.testing.assert_allclose(M, np.eye(3) / (6 * np.pi * 3.0 * 2.5))


def test_far_field_is_oseen_plus_laplacian():
    # For separated blobs RPY = (1 + a^2/3 Laplacian) Oseen.  The Laplacian is taken here by a
    # 7-point finite difference of the Oseen tensor, independently of the printed coefficients.
    rng = np.random.default_rng(0)
    h = 1e-3
    for rad in (2.0, 2.7, 4.0, 9.0):
        rv = rng.standard_normal(3)
        rv *= rad / np.linalg.norm(rv)
        lap = -6 * _oseen(rv)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap = lap + _oseen(rv + e) + _oseen(rv - e)
        lap /= h * h
        ref = _oseen(rv) + A * A / 3.0 * lap
        np.testing.assert_allclose(rpy.rpy_pair(rv, A, ETA), ref, rtol=2e-6, atol=1e-9)
    # and tends to Oseen far away
    rv = np.array([1e4, 3e3, -2e3])
    np.testing.assert_allclose(rpy.rpy_pair(rv, A, ETA), _oseen(rv), rtol=1e-7)


def test_overlap_branch_continuity():
    # The overlap branch is linear in r; it must meet the far branch at r = 2a and the self term at r = 0.
    e = np.array([0.3, -0.4, np.sqrt(0.75)])
    below = rpy.rpy_pair(e * (2 * A - 1e-12), A, ETA)
    above = rpy.rpy_pair(e * (2 * A + 1e-12), A, ETA)
    np.testing.assert_allclose(below, above, atol=1e-12)
    np.testing.assert_allclose(rpy.rpy_pair(e * 1e-12, A, ETA), MU0 * np.eye(3), atol=1e-12)
    # midway value is the average of the end points for a linear branch
    mid = rpy.rpy_pair(e * A, A, ETA)
    np.testing.assert_allclose(mid, 0.5 * (MU0 * np.eye(3) + below), atol=1e-14)


def test_symmetric_positive_definite_with_overlaps():
    rng = np.random.default_rng(1)
    for n in (5, 30, 80):
        r = rng.uniform(0, 0.9 * n ** (1 / 3), size=(n, 3))  # dense: many overlapping pairs
        M = rpy.rpy_matrix(r, A, ETA)
        np.testing.assert_allclose(M, M.T, atol=1e-15)
        assert np.linalg.eigvalsh(M).min() > 0
    # blob-spacing-a boomerang: heavily overlapping
    M = rpy.rpy_matrix(G.centred_template(shapes.boomerang()), A, ETA)
    assert np.linalg.eigvalsh(M).min() > 0


def test_dense_matches_blockwise_and_rows():
    rng = np.random.default_rng(2)
    r = rng.uniform(0, 6, size=(25, 3))
    r[3] = r[4]  # coincident blobs take the self term
    M = rpy.rpy_matrix(r, A, ETA)
    np.testing.assert_allclose(M, rpy.rpy_matrix_loops(r, A, ETA), atol=1e-15)
    lam = rng.standard_normal((25, 3))
    rows = [0, 3, 4, 24]
    u = (M @ lam.reshape(-1)).reshape(-1, 3)
    np.testing.assert_allclose(matfree.rpy_rows(r, lam, rows, A, ETA), u[rows], atol=1e-14)


def _layout_state(templates, body_tmpl, seed=0, spread=12.0):
    rng = np.random.default_rng(seed)
    lay = G.Layout(templates, body_tmpl)
    Y = rng.uniform(0, spread, size=(lay.n_bodies, 3))
    g = rng.standard_normal((lay.n_bodies, 4))
    q = g / np.linalg.norm(g, axis=1, keepdims=True)
    return lay, Y, q


def test_k_is_rigid_motion_of_blobs():
    # K V must be the blob velocity of the rigid motion that moves (Y, q) by (Ydot, Omega)
    # with the quaternion update of App. A; checked by differentiating the positions.
    lay, Y, q = _layout_state([shapes.boomerang(), shapes.icosahedron()], [0, 1, 1])
    rng = np.random.default_rng(3)
    V = rng.standard_normal((lay.n_bodies, 6))
    r = G.blob_positions(lay, Y, q)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    h = 1e-6
    rp = G.blob_positions(lay, *G.advance(Y, q, V, h))
    rm = G.blob_positions(lay, *G.advance(Y, q, V, -h))
    np.testing.assert_allclose(K @ V.reshape(-1), ((rp - rm) / (2 * h)).reshape(-1), atol=1e-8)
    # K^T lambda = [sum lambda; sum (r - Y) x lambda]
    lam = rng.standard_normal((lay.n_blobs, 3))
    ft = (K.T @ lam.reshape(-1)).reshape(-1, 6)
    for p in range(lay.n_bodies):
        sel = lay.blob_body == p
        np.testing.assert_allclose(ft[p, :3], lam[sel].sum(0), atol=1e-13)
        np.testing.assert_allclose(ft[p, 3:], np.cross(r[sel] - Y[p], lam[sel]).sum(0), atol=1e-12)


def test_ktk_closed_form():
    # Sec. 5 prints (K^T K)^(p) in closed form.
    lay, Y, q = _layout_state([shapes.boomerang(), shapes.rod(7)], [0, 1])
    r = G.blob_positions(lay, Y, q)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    KtK = K.T @ K
    for p in range(2):
        np.testing.assert_allclose(KtK[6 * p:6 * p + 6, 6 * p:6 * p + 6],
                                   rigid.ktk_closed_form(r, Y, lay.blob_body, p), atol=1e-11)


def _dumbbell_N(d):
    lay = G.Layout([shapes.dumbbell(d)], [0])
    Y = np.zeros((1, 3))
    q = np.array([[1.0, 0, 0, 0]])
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, A, ETA)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    B = rigid.rigid_basis(K, 1)
    return rigid.body_mobility(M, K, B), B


@pytest.mark.parametrize("d", [1.0, 2.0, 3.5, 8.0])
def test_dumbbell_closed_form(d):
    # Two blobs on the x axis: with M_12 = mu_par xx + mu_perp (I - xx),
    # N_par = (mu0 + mu_par)/2, N_perp = (mu0 + mu_perp)/2, rotation perp = 2 (mu0 - mu_perp)/d^2,
    # axial spin absent.
    M12 = rpy.rpy_pair(np.array([d, 0, 0]), A, ETA)
    mu_par, mu_perp = M12[0, 0], M12[1, 1]
    N, B = _dumbbell_N(d)
    assert B.shape[1] == 5
    np.testing.assert_allclose(N[0, 0], (MU0 + mu_par) / 2, rtol=1e-12)
    np.testing.assert_allclose(N[1, 1], (MU0 + mu_perp) / 2, rtol=1e-12)
    np.testing.assert_allclose(N[2, 2], (MU0 + mu_perp) / 2, rtol=1e-12)
    np.testing.assert_allclose(N[4, 4], 2 * (MU0 - mu_perp) / d ** 2, rtol=1e-12)
    np.testing.assert_allclose(N[5, 5], 2 * (MU0 - mu_perp) / d ** 2, rtol=1e-12)
    assert abs(N[3, 3]) < 1e-14 and np.abs(N[3]).max() < 1e-14
    np.testing.assert_allclose(N[:3, 3:], 0, atol=1e-14)


def test_icosahedron_is_isotropic():
    lay = G.Layout([shapes.icosahedron()], [0])
    rng = np.random.default_rng(4)
    g = rng.standard_normal(4)
    q = (g / np.linalg.norm(g))[None, :]
    Y = rng.standard_normal((1, 3))
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, A, ETA)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    N = rigid.body_mobility(M, K, rigid.rigid_basis(K, 1))
    np.testing.assert_allclose(N[:3, :3], N[0, 0] * np.eye(3), atol=1e-14)
    np.testing.assert_allclose(N[3:, 3:], N[3, 3] * np.eye(3), atol=1e-14)
    np.testing.assert_allclose(N[:3, 3:], 0, atol=1e-14)
    # shell of radius 2a is less mobile than a single blob
    assert N[0, 0] < MU0


def test_mobility_invariance_and_spd():
    templates = [shapes.boomerang(), shapes.icosahedron(), shapes.rod(5)]
    lay, Y, q = _layout_state(templates, [0, 1, 2], seed=5, spread=9.0)
    from oracle.gdc import Params, body_mobility_at
    p = Params()
    N = body_mobility_at(lay, Y, q, p)
    np.testing.assert_allclose(N, N.T, atol=1e-13)
    w = np.linalg.eigvalsh(N)
    assert (w > -1e-14).all() and (w > 1e-8).sum() == 6 * 3 - 1  # rod axial spin is the only null
    # translation invariance
    np.testing.assert_allclose(body_mobility_at(lay, Y + np.array([3.0, -7.0, 1.5]), q, p), N, atol=1e-13)
    # rotation covariance: rotating the whole suspension by Q gives Rt N Rt^T
    Q = G.quat_exp(np.array([0.3, -1.1, 0.7]))
    R = G.rotation_matrix(Q)
    Y2 = Y @ R.T
    q2 = np.array([G.quat_mul(Q, qq) for qq in q])
    N2 = body_mobility_at(lay, Y2, q2, p)
    Rt = np.kron(np.eye(6), R)
    np.testing.assert_allclose(N2, Rt @ N @ Rt.T, atol=1e-12)


def test_saddle_solve_equals_mobility_and_brute_force():
    templates = [shapes.boomerang(), shapes.triangle(), shapes.rod(4)]
    lay, Y, q = _layout_state(templates, [0, 1, 2], seed=6, spread=8.0)
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, A, ETA)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    B = rigid.rigid_basis(K, lay.n_bodies)
    rng = np.random.default_rng(7)
    F = rng.standard_normal(6 * lay.n_bodies)
    F = B @ (B.T @ F)  # a rod carries no axial torque
    lam, V = rigid.saddle_solve(M, K, B, np.zeros(3 * lay.n_blobs), F)
    N = rigid.body_mobility(M, K, B)
    np.testing.assert_allclose(V, N @ F, rtol=1e-10, atol=1e-14)
    # residual of the original (unreduced) equations
    a1, a2 = rigid.saddle_apply(M, K, lam, V)
    np.testing.assert_allclose(a1, 0, atol=1e-12)
    np.testing.assert_allclose(a2, -F, atol=1e-12)
    # Brownian slip: V = N K^T M^-1 v (Eq. lin_sys_RMB and the text after it)
    vb = rng.standard_normal(3 * lay.n_blobs)
    lam2, V2 = rigid.saddle_solve(M, K, B, vb, np.zeros_like(F))
    np.testing.assert_allclose(V2, N @ K.T @ np.linalg.solve(M, vb), rtol=1e-9, atol=1e-13)


def test_lsq_and_square_roots():
    templates = [shapes.boomerang(), shapes.rod(6)]
    lay, Y, q = _layout_state(templates, [0, 1], seed=8, spread=6.0)
    r = G.blob_positions(lay, Y, q)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    B = rigid.rigid_basis(K, lay.n_bodies)
    rng = np.random.default_rng(9)
    vb = rng.standard_normal(3 * lay.n_blobs)
    V = rigid.lsq_velocity(K, B, vb)
    ref = np.linalg.lstsq(K, vb, rcond=None)[0]  # minimum-norm least squares
    np.testing.assert_allclose(V, ref, atol=1e-12)
    M = rpy.rpy_matrix(r, A, ETA)
    S = rigid.sqrtm_sym(M)
    np.testing.assert_allclose(S @ S, M, atol=1e-14)
    np.testing.assert_allclose(S, S.T, atol=1e-15)
    L = rigid.sqrtm_chol(M)
    np.testing.assert_allclose(L @ L.T, M, atol=1e-14)
