"""Pins of the oracle's quaternion, rotation and Philox code against independent facts."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import geometry as G
from oracle import philox


def _rand_q(rng, n):
    g = rng.standard_normal((n, 4))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_rotation_matrix_matches_scipy():
    # Eq. (quaternion_rotation_matrix) is the standard active rotation of a unit quaternion; scipy is an independent implementation.
    rng = np.random.default_rng(1)
    for q in _rand_q(rng, 20):
        R = G.rotation_matrix(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14


def test_hamilton_product_composes_rotations():
    # App. A: rotating by p * q is rotating by q and then by p.
    rng = np.random.default_rng(2)
    P, Q, S = _rand_q(rng, 3)
    np.testing.assert_allclose(G.rotation_matrix(G.quat_mul(P, Q)),
                               G.rotation_matrix(P) @ G.rotation_matrix(Q), atol=1e-14)
    np.testing.assert_allclose(G.quat_mul(G.quat_mul(P, Q), S), G.quat_mul(P, G.quat_mul(Q, S)),
                               atol=1e-15)
    np.testing.assert_allclose(G.quat_mul(np.array([1.0, 0, 0, 0]), Q), Q)
    # (q0, v) * (q0, -v) = identity
    np.testing.assert_allclose(G.quat_mul(Q, Q * np.array([1, -1, -1, -1])), [1, 0, 0, 0], atol=1e-15)


def test_quat_exp_is_rotation_vector():
    # exp(u) is the unit quaternion of the rotation by |u| about u/|u| (Sec. 2).
    rng = np.random.default_rng(3)
    for u in rng.standard_normal((10, 3)) * 2.0:
        e = G.quat_exp(u)
        assert abs(np.linalg.norm(e) - 1.0) < 1e-15
        ref = Rotation.from_rotvec(u).as_matrix()
        np.testing.assert_allclose(G.rotation_matrix(e), ref, atol=1e-14)
    np.testing.assert_allclose(G.quat_exp(np.zeros(3)), [1, 0, 0, 0])
    # tiny-u branch agrees with the closed form just above its threshold
    u = np.array([3e-9, -2e-9, 1e-9])
    np.testing.assert_allclose(G.quat_exp(u), [np.cos(np.linalg.norm(u) / 2), *(0.5 * u)], atol=1e-20)


def test_exp_derivative_is_psi():
    # App. A: d/dh [exp(h Omega) * q] at h = 0 equals Psi_q Omega = 1/2 (0, Omega) * q.
    rng = np.random.default_rng(4)
    q = _rand_q(rng, 1)[0]
    om = rng.standard_normal(3)
    h = 1e-6
    fd = (G.quat_mul(G.quat_exp(h * om), q) - G.quat_mul(G.quat_exp(-h * om), q)) / (2 * h)
    q0, qv = q[0], q[1:]
    psi = 0.5 * np.vstack([-qv[None, :], q0 * np.eye(3) - G.cross_matrix(qv)])
    np.testing.assert_allclose(fd, psi @ om, atol=1e-9)
    np.testing.assert_allclose(fd, 0.5 * G.quat_mul(np.concatenate([[0.0], om]), q), atol=1e-9)


def test_cross_matrix():
    rng = np.random.default_rng(5)
    v, w = rng.standard_normal((2, 3))
    np.testing.assert_allclose(G.cross_matrix(v) @ w, np.cross(v, w), atol=1e-15)
    np.testing.assert_allclose(G.cross_matrix(v).T, -G.cross_matrix(v))


def test_advance_preserves_norm():
    # App. A: the multiplicative update keeps |q| = 1 to rounding.
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((5, 3))
    q = _rand_q(rng, 5)
    V = rng.standard_normal((5, 6)) * 10
    for _ in range(50):
        Y, q = G.advance(Y, q, V, 0.37)
    assert np.abs(np.linalg.norm(q, axis=1) - 1.0).max() < 1e-13


def test_body_length_and_centroid():
    b = np.array([[0.0, 0, 0], [3.0, 0, 0], [0, 4.0, 0]])
    assert G.body_length(b) == 5.0
    np.testing.assert_allclose(G.centred_template(b).mean(axis=0), 0, atol=1e-15)
    assert G.body_length(b[:1]) == 0.0


# Known-answer vectors of Philox4x32-10 published with the Random123 library (Salmon et al. 2011).
_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", _KAT)
def test_philox_known_answers(ctr, key, expect):
    out = philox.philox4x32_10(np.array([ctr], dtype=np.uint64), key)[0]
    assert tuple(int(x) for x in out) == expect


def test_normals_statistics_and_determinism():
    z = philox.normals(1234, 3, 7, 0, 200001)
    assert z.shape == (200001,)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    # fourth moment of a normal is 3
    assert abs((z ** 4).mean() - 3.0) < 0.1
    np.testing.assert_array_equal(z, philox.normals(1234, 3, 7, 0, 200001))
    # a prefix of a longer draw is the shorter draw (counter-based)
    np.testing.assert_array_equal(z[:11], philox.normals(1234, 3, 7, 0, 11))
    assert not np.allclose(z[:100], philox.normals(1234, 3, 7, 1, 100))
    assert not np.allclose(z[:100], philox.normals(1234, 4, 7, 0, 100))
