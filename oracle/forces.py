"""Oracle soft repulsion between blobs of different bodies.  TEST INFRASTRUCTURE ONLY.

The force between two blobs a distance r apart is the (negative) derivative
of the soft-sphere potential of Sec. 6.3, Eq. (soft_sphere_potential):

  F(r) = A exp(-(r - 2a)/b)  for r >= 2a,
  F(r) = A                   for r <  2a  (the constant-force continuation
                                           that the linear branch of Eq. (soft_sphere_potential) gives),

directed along r_i - r_j (it pushes blob i away from blob j), with A = U0/b.
Blobs of the same body do not repel (their distances never change).  The
body force and torque are F_p = sum_i f_i and T_p = sum_i (r_i - Y_p) x f_i
(the K^T map of Eq. force_torque_balance_compact applied to the blob forces).
"""
from __future__ import annotations

import numpy as np


def blob_forces(r: np.ndarray, blob_body: np.ndarray, A: float, b: float, a: float) -> np.ndarray:
    m = r.shape[0]
    f = np.zeros((m, 3))
    if A == 0.0:
        return f
    for i in range(m):
        d = r[i][None, :] - r
        dist = np.linalg.norm(d, axis=1)
        other = blob_body != blob_body[i]
        mag = np.where(dist >= 2.0 * a, A * np.exp(-(dist - 2.0 * a) / b), A)
        with np.errstate(invalid="ignore", divide="ignore"):
            unit = d / dist[:, None]
        sel = other & (dist > 0.0)
        f[i] = (mag[sel, None] * unit[sel]).sum(axis=0)
    return f


def body_force_torque(r: np.ndarray, Y: np.ndarray, blob_body: np.ndarray, f: np.ndarray) -> np.ndarray:
    """[F_p; T_p] per body, flattened to 6N."""
    n = Y.shape[0]
    out = np.zeros((n, 6))
    for i in range(r.shape[0]):
        p = int(blob_body[i])
        out[p, :3] += f[i]
        out[p, 3:] += np.cross(r[i] - Y[p], f[i])
    return out.reshape(-1)
