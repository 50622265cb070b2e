"""Oracle RPY blob mobility M (Sec. 4.1).  TEST INFRASTRUCTURE ONLY.

The paper uses the Rotne-Prager-Yamakawa tensor for equal blobs of radius a
(Sec. 4.1) but does not print it; this is the textbook unbounded form
including the overlapping-blob branch, for i != j with r = r_i - r_j:

  r >= 2a : M_ij = 1/(8 pi eta r) [ (1 + 2a^2/(3 r^2)) I + (1 - 2a^2/r^2) rhat rhat^T ]
  r <  2a : M_ij = 1/(6 pi eta a) [ (1 - 9 r/(32 a)) I + (3 r/(32 a)) rhat rhat^T ]
  i == j  : M_ii = I / (6 pi eta a)

The two branches agree at r = 2a, and the overlap branch tends to the self
term as r -> 0, so the tie at r = 2a is immaterial.
"""
from __future__ import annotations

import numpy as np


def rpy_pair(rvec: np.ndarray, a: float, eta: float) -> np.ndarray:
    """3x3 block M_ij for the separation vector r_i - r_j (zero vector gives the self term)."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r = float(np.linalg.norm(rvec))
    if r == 0.0:
        return np.eye(3) / (6.0 * np.pi * eta * a)
    rr = np.outer(rvec, rvec) / (r * r)
    if r >= 2.0 * a:
        c = 1.0 / (8.0 * np.pi * eta * r)
        return c * ((1.0 + 2.0 * a * a / (3.0 * r * r)) * np.eye(3) + (1.0 - 2.0 * a * a / (r * r)) * rr)
    c = 1.0 / (6.0 * np.pi * eta * a)
    return c * ((1.0 - 9.0 * r / (32.0 * a)) * np.eye(3) + (3.0 * r / (32.0 * a)) * rr)


def rpy_matrix(r: np.ndarray, a: float, eta: float) -> np.ndarray:
    """Dense 3M x 3M blob mobility, block (i, j) = rpy_pair(r_i - r_j) (Eq. ddof_mob / Sec. 4.1)."""
    r = np.asarray(r, dtype=np.float64)
    m = r.shape[0]
    d = r[:, None, :] - r[None, :, :]
    dist = np.linalg.norm(d, axis=-1)
    eye = np.eye(3)
    safe = np.where(dist > 0.0, dist, 1.0)
    rr = d[..., :, None] * d[..., None, :] / (safe * safe)[..., None, None]
    far = dist >= 2.0 * a
    c_far = 1.0 / (8.0 * np.pi * eta * safe)
    f_far = c_far * (1.0 + 2.0 * a * a / (3.0 * safe * safe))
    g_far = c_far * (1.0 - 2.0 * a * a / (safe * safe))
    c0 = 1.0 / (6.0 * np.pi * eta * a)
    f_near = c0 * (1.0 - 9.0 * dist / (32.0 * a))
    g_near = c0 * (3.0 * dist / (32.0 * a))
    f = np.where(far, f_far, f_near)
    g = np.where(far, g_far, g_near)
    blocks = f[..., None, None] * eye + g[..., None, None] * rr
    # coincident blobs (including i == j) take the self term I/(6 pi eta a)
    blocks[dist == 0.0] = c0 * eye
    return blocks.transpose(0, 2, 1, 3).reshape(3 * m, 3 * m)


def rpy_matrix_loops(r: np.ndarray, a: float, eta: float) -> np.ndarray:
    """Same matrix built one block at a time from rpy_pair (brute-force cross-check)."""
    m = r.shape[0]
    M = np.zeros((3 * m, 3 * m))
    for i in range(m):
        for j in range(m):
            M[3 * i:3 * i + 3, 3 * j:3 * j + 3] = rpy_pair(r[i] - r[j], a, eta)
    return M
