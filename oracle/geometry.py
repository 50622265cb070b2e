"""Oracle geometry: quaternions, rotations and blob positions.  TEST INFRASTRUCTURE ONLY.

Conventions follow Sec. 2 and App. A: q = (q0, q1, q2, q3) with the scalar
part first; R(q) is Eq. (quaternion_rotation_matrix); exp(u) = (cos(|u|/2), sin(|u|/2) u/|u|); the
Hamilton product composes rotations so that exp(u) * q rotates by q first
and then by exp(u).
"""
from __future__ import annotations

import numpy as np


def rotation_matrix(q: np.ndarray) -> np.ndarray:
    """R(q) of Sec. 2, Eq. (quaternion_rotation_matrix), written entry by entry (q scalar first)."""
    q0, q1, q2, q3 = (float(x) for x in q)
    return np.array([
        [1.0 - 2.0 * q2 * q2 - 2.0 * q3 * q3, 2.0 * (q1 * q2 - q3 * q0), 2.0 * (q1 * q3 + q2 * q0)],
        [2.0 * (q1 * q2 + q3 * q0), 1.0 - 2.0 * q1 * q1 - 2.0 * q3 * q3, 2.0 * (q3 * q2 - q1 * q0)],
        [2.0 * (q1 * q3 - q2 * q0), 2.0 * (q3 * q2 + q1 * q0), 1.0 - 2.0 * q2 * q2 - 2.0 * q1 * q1],
    ])


def quat_mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Hamilton product (p0, p) * (q0, q) = (p0 q0 - p.q, p0 q + q0 p + p x q), App. A."""
    p0, pv = float(p[0]), np.asarray(p[1:], dtype=np.float64)
    q0, qv = float(q[0]), np.asarray(q[1:], dtype=np.float64)
    return np.concatenate([[p0 * q0 - pv @ qv], p0 * qv + q0 * pv + np.cross(pv, qv)])


def quat_exp(u: np.ndarray) -> np.ndarray:
    """Lie-algebra exponential of Sec. 2: exp(u) = (cos(|u|/2), sin(|u|/2) u/|u|).

    At u = 0 the limit sin(|u|/2)/|u| -> 1/2 is used (the map is smooth there).
    """
    u = np.asarray(u, dtype=np.float64)
    th = float(np.linalg.norm(u))
    if th < 1e-8:
        # sin(x/2)/x = 1/2 - x^2/48 + O(x^4)
        s = 0.5 - th * th / 48.0
    else:
        s = np.sin(0.5 * th) / th
    return np.concatenate([[np.cos(0.5 * th)], s * u])


def cross_matrix(v: np.ndarray) -> np.ndarray:
    """[v x] with entries [v x]_ij = eps_ikj v_k (Sec. 2.1), so that [v x] w = v x w."""
    v = np.asarray(v, dtype=np.float64)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    return np.einsum("ikj,k->ij", eps, v)


def centred_template(b: np.ndarray) -> np.ndarray:
    """Body-frame blobs relative to their centroid.

    The paper's Y_p is the body's centre of mass (Sec. 2); with equal blobs
    that is the blob centroid, so templates are centred on it.
    """
    b = np.asarray(b, dtype=np.float64)
    return b - b.mean(axis=0, keepdims=True)


def body_length(b: np.ndarray) -> float:
    """L_p: the largest distance between two blobs of the body (footnote to Sec. 3, step 3)."""
    b = np.asarray(b, dtype=np.float64)
    if b.shape[0] < 2:
        return 0.0
    d = np.linalg.norm(b[:, None, :] - b[None, :, :], axis=-1)
    return float(d.max())


class Layout:
    """Bodies, their templates and the blob ordering of one suspension.

    Blobs are ordered body by body, each body's blobs in template order;
    lambda = [lambda_1 .. lambda_M] and V = [V_1 .. V_N] with V_p = [Ydot_p, Omega_p]
    (Sec. 2.2).
    """

    def __init__(self, templates, body_tmpl):
        self.templates = [centred_template(t) for t in templates]
        self.body_tmpl = np.asarray(body_tmpl, dtype=np.int64)
        self.nb = np.array([self.templates[t].shape[0] for t in self.body_tmpl], dtype=np.int64)
        self.blob_off = np.concatenate([[0], np.cumsum(self.nb)]).astype(np.int64)
        self.n_bodies = int(self.body_tmpl.shape[0])
        self.n_blobs = int(self.blob_off[-1])
        self.blob_body = np.repeat(np.arange(self.n_bodies), self.nb)
        self.L = np.array([body_length(self.templates[t]) for t in self.body_tmpl])


def blob_positions(layout: Layout, Y: np.ndarray, q: np.ndarray) -> np.ndarray:
    """r_i = Y_p + R(q_p) b_i for every blob i of body p (Sec. 2)."""
    r = np.zeros((layout.n_blobs, 3))
    for p in range(layout.n_bodies):
        b = layout.templates[layout.body_tmpl[p]]
        r[layout.blob_off[p]:layout.blob_off[p + 1]] = Y[p][None, :] + b @ rotation_matrix(q[p]).T
    return r


def advance(Y: np.ndarray, q: np.ndarray, V: np.ndarray, h: float):
    """x -> x + h V with q -> exp(h Omega) * q (Sec. 3 steps 4 and 6, App. A).

    V is (N, 6) = [Ydot, Omega] per body; the Lie-algebra element starts from
    zero at every step, so u = h Omega.
    """
    Yn = Y + h * V[:, :3]
    qn = np.array([quat_mul(quat_exp(h * V[p, 3:]), q[p]) for p in range(Y.shape[0])])
    return Yn, qn
