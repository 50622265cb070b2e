"""Pins of the oracle's square roots of M (Sec. 4.1 Lanczos, Eq. v_brown_RMB).

The block-preconditioned root S = L (L^-1 M L^-T)^(1/2) is pinned by what fixes it
independently of its own formula: S S^T = M; L L^T equals the body blocks of the dense
RPY matrix; a lone body makes L^-1 M L^-T the identity, so S = L; the sample turns with a
rigid rotation of the whole suspension; and an independent Lanczos iteration on
L^-1 M L^-T started from W converges to L^-1 S W.
"""
import numpy as np

from oracle import geometry as G, rigid, rpy
from oracle.gdc import Params, brownian_slip
from synthetic import shapes


def _state(templates, body_tmpl, Y, seed=0):
    rng = np.random.default_rng(seed)
    lay = G.Layout(templates, body_tmpl)
    g = rng.standard_normal((lay.n_bodies, 4))
    return lay, np.asarray(Y, dtype=float), g / np.linalg.norm(g, axis=1, keepdims=True)


def _mixed():
    return _state([shapes.icosphere42(), shapes.rod(5), shapes.boomerang(6, 1.0)], [0, 1, 2, 1],
                  [[0, 0, 0], [9.0, 1.0, 0.0], [1.0, 10.0, 2.0], [-8.0, -3.0, 4.0]], seed=3)


def test_block_root_is_a_square_root_of_M():
    lay, Y, q = _mixed()
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, 1.0, 1.0)
    L = rigid.block_factor(lay, q, 1.0, 1.0)
    S = rigid.sqrtm_block(M, L)
    np.testing.assert_allclose(S @ S.T, M, atol=1e-13)
    # L L^T is M with every block between different bodies removed
    mask = lay.blob_body[:, None] == lay.blob_body[None, :]
    D = M * np.kron(mask, np.ones((3, 3)))
    np.testing.assert_allclose(L @ L.T, D, atol=1e-14)
    # and S differs from the symmetric root (it is a different sample of the same law)
    assert np.abs(S - rigid.sqrtm_sym(M)).max() > 1e-3


def test_lone_body_root_is_the_rotated_template_cholesky():
    lay, Y, q = _state([shapes.boomerang(11, 1.0)], [0], [[1.0, 2.0, 3.0]], seed=4)
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, 1.0, 1.0)
    L = rigid.block_factor(lay, q, 1.0, 1.0)
    np.testing.assert_allclose(rigid.sqrtm_block(M, L), L, atol=1e-13)
    Lt = np.linalg.cholesky(rpy.rpy_matrix(lay.templates[0], 1.0, 1.0))
    np.testing.assert_allclose(L, np.kron(np.eye(lay.n_blobs), G.rotation_matrix(q[0])) @ Lt, atol=1e-15)


def test_block_sample_turns_with_the_suspension():
    lay, Y, q = _mixed()
    W = np.random.default_rng(5).standard_normal(3 * lay.n_blobs)
    p = Params(sqrt_mode="block")
    _, _, _, _, vb = brownian_slip(lay, Y, q, W, p)
    u = np.array([0.3, -1.1, 0.7])
    Qq = G.quat_exp(u)
    Q = G.rotation_matrix(Qq)
    Y2 = Y @ Q.T + np.array([5.0, -2.0, 1.0])
    q2 = np.array([G.quat_mul(Qq, qq) for qq in q])
    _, _, _, _, vb2 = brownian_slip(lay, Y2, q2, W, p)
    np.testing.assert_allclose(vb2.reshape(-1, 3), vb.reshape(-1, 3) @ Q.T, atol=1e-11)


def test_lanczos_on_the_preconditioned_operator_converges_to_the_block_root():
    lay, Y, q = _mixed()
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, 1.0, 1.0)
    L = rigid.block_factor(lay, q, 1.0, 1.0)
    W = np.random.default_rng(6).standard_normal(3 * lay.n_blobs)
    Linv = np.linalg.inv(L)

    def op(x):
        return Linv @ (M @ (Linv.T @ x))

    # plain Lanczos with full reorthogonalisation, independent of the oracle's eigh root
    n = W.size
    V = np.zeros((n, 60))
    al, be = [], []
    V[:, 0] = W / np.linalg.norm(W)
    for k in range(59):
        w = op(V[:, k])
        for _ in range(2):
            w -= V[:, :k + 1] @ (V[:, :k + 1].T @ w)
        al.append(V[:, k] @ op(V[:, k]))
        b = np.linalg.norm(w)
        be.append(b)
        V[:, k + 1] = w / b
    k = len(al)
    T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
    th, Qt = np.linalg.eigh(T)
    y = np.linalg.norm(W) * V[:, :k] @ (Qt @ (np.sqrt(th) * Qt[0]))
    np.testing.assert_allclose(L @ y, rigid.sqrtm_block(M, L) @ W, rtol=0, atol=1e-8 * np.linalg.norm(W))


# ---- the oracle's Lanczos iterate (oracle/lanczos.py) ---------------------------------

from oracle import lanczos  # noqa: E402


def _preconditioned(lay, Y, q):
    r = G.blob_positions(lay, Y, q)
    M = rpy.rpy_matrix(r, 1.0, 1.0)
    L = rigid.block_factor(lay, q, 1.0, 1.0)
    Linv = np.linalg.inv(L)
    A = Linv @ M @ Linv.T
    return M, L, 0.5 * (A + A.T)


def test_lanczos_tends_to_the_dense_roots():
    lay, Y, q = _mixed()
    M, L, A = _preconditioned(lay, Y, q)
    W = np.random.default_rng(7).standard_normal(3 * lay.n_blobs)
    y, k, _ = lanczos.lanczos_sqrt(A, W, 1e-12)
    np.testing.assert_allclose(L @ y, rigid.sqrtm_block(M, L) @ W, rtol=0, atol=1e-9 * np.linalg.norm(W))
    y2, k2, _ = lanczos.lanczos_sqrt(M, W, 1e-12)
    np.testing.assert_allclose(y2, rigid.sqrtm_sym(M) @ W, rtol=0, atol=1e-9 * np.linalg.norm(W))
    assert k < k2   # the preconditioned operator needs fewer iterations


def test_lanczos_stops_at_the_first_small_change():
    lay, Y, q = _mixed()
    M, L, A = _preconditioned(lay, Y, q)
    W = np.random.default_rng(8).standard_normal(3 * lay.n_blobs)
    tol = 1e-4
    y, k, change = lanczos.lanczos_sqrt(A, W, tol)
    assert change < tol and k >= 3
    for j in range(2, k):
        assert lanczos.lanczos_sqrt(A, W, tol, fixed_k=j)[2] >= tol
    # a fixed count reproduces the iterate
    np.testing.assert_array_equal(lanczos.lanczos_sqrt(A, W, tol, fixed_k=k)[0], y)
    # the remaining error is of the order of the last change (geometric convergence)
    exact = rigid.sqrtm_sym(A) @ W
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 3 * tol


def test_lanczos_is_exact_on_an_operator_with_three_eigenvalues():
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.repeat([1.0, 4.0, 9.0], 10)
    A = (Q * lam) @ Q.T
    W = rng.standard_normal(30)
    y, k, _ = lanczos.lanczos_sqrt(A, W, 1e-14)
    assert k == 3   # the Krylov space of W has dimension 3
    np.testing.assert_allclose(y, (Q * np.sqrt(lam)) @ (Q.T @ W), atol=1e-12)


def test_lanczos_on_a_lone_body_stops_at_once():
    lay, Y, q = _state([shapes.icosphere42()], [0], [[0.0, 0.0, 0.0]], seed=10)
    M, L, A = _preconditioned(lay, Y, q)
    np.testing.assert_allclose(A, np.eye(A.shape[0]), atol=1e-12)
    W = np.random.default_rng(11).standard_normal(3 * lay.n_blobs)
    y, k, _ = lanczos.lanczos_sqrt(A, W, 1e-4)
    assert k == 1
    np.testing.assert_allclose(y, W, atol=1e-11)
