"""Oracle matrix-free rows of the RPY product u = M lambda.  TEST INFRASTRUCTURE ONLY.

For suspensions too large to store M (65k blobs would need 309 GB), the
oracle evaluates selected rows u_i = sum_j M_ij lambda_j one target at a
time, straight from the pair formula of rpy.py (Sec. 4.1), in FP64.  Used
for sampled parity at full size and for the timed CPU baseline.
"""
from __future__ import annotations

import numpy as np

from . import forces


def rpy_rows(r: np.ndarray, lam: np.ndarray, rows, a: float, eta: float) -> np.ndarray:
    """u_i for every i in ``rows``; r is (M, 3), lam is (M, 3); returns (len(rows), 3)."""
    r = np.asarray(r, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(rows), 3))
    c_self = 1.0 / (6.0 * np.pi * eta * a)
    for k, i in enumerate(rows):
        d = r[i][None, :] - r
        dist = np.linalg.norm(d, axis=1)
        safe = np.where(dist > 0.0, dist, 1.0)
        dl = (d * lam).sum(axis=1) / (safe * safe)       # (rhat . lambda) / r
        far = dist >= 2.0 * a
        c_far = 1.0 / (8.0 * np.pi * eta * safe)
        f = np.where(far, c_far * (1.0 + 2.0 * a * a / (3.0 * safe * safe)),
                     c_self * (1.0 - 9.0 * dist / (32.0 * a)))
        g = np.where(far, c_far * (1.0 - 2.0 * a * a / (safe * safe)),
                     c_self * (3.0 * dist / (32.0 * a)))
        f = np.where(dist == 0.0, c_self, f)
        g = np.where(dist == 0.0, 0.0, g)
        out[k] = (f[:, None] * lam).sum(axis=0) + ((g * dl)[:, None] * d).sum(axis=0)
    return out


def repulsion_rows(r: np.ndarray, blob_body: np.ndarray, rows, A: float, b: float, a: float, potential: int = 0,
                   well_A: float = 0.0, well_lambda: float = 0.5) -> np.ndarray:
    """Blob pair forces f_i for the listed blobs (forces.py definition)."""
    out = np.zeros((len(rows), 3))
    for k, i in enumerate(rows):
        d = r[i][None, :] - r
        dist = np.linalg.norm(d, axis=1)
        sel = (blob_body != blob_body[i]) & (dist > 0.0)
        mag = forces.pair_force(dist[sel], a, A, b, potential, well_A, well_lambda)
        out[k] = (mag[:, None] * d[sel] / dist[sel, None]).sum(axis=0)
    return out
