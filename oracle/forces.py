"""Oracle pair forces between blobs of different bodies.  TEST INFRASTRUCTURE ONLY.

The force between two blobs a distance r apart is F(r) = -dU_k/dr for one of three pair
potentials, directed along r_i - r_j (F > 0 pushes blob i away from blob j):

  k = 0, soft sphere, Sec. 6.3, Eq. (soft_sphere_potential):
      U(r) = U0 exp((2a - r)/b) for r >= 2a, so F(r) = A exp(-(r - 2a)/b) with A = U0/b;
  k = 1, repel-attract, Sec. 6.4:       U_1 = U - phi_{3a};
  k = 2, repel-attract-repel, Sec. 6.4: U_2 = U - phi_{3a} + phi_{7a/2};

with the Gaussian wells phi_c(r) = A_w exp(-((r - c)/lambda)^2), whose force is
-dphi_c/dr = 2 A_w (r - c)/lambda^2 exp(-((r - c)/lambda)^2).  Below r = 2a every potential
continues linearly (Eq. soft_sphere_potential's first branch for U; the sentence after
U_2's definition for U_1 and U_2), so the force there is the force at 2a.

Blobs of the same body do not interact (their distances never change).  The body force
and torque are F_p = sum_i f_i and T_p = sum_i (r_i - Y_p) x f_i (the K^T map of
Eq. force_torque_balance_compact applied to the blob forces).
"""
from __future__ import annotations

import numpy as np


SOFT, REPEL_ATTRACT, REPEL_ATTRACT_REPEL = 0, 1, 2


def well_force(r: np.ndarray, c: float, well_A: float, well_lambda: float) -> np.ndarray:
    """-dphi_c/dr for phi_c(r) = well_A exp(-((r - c)/well_lambda)^2) (Sec. 6.4)."""
    x = (r - c) / well_lambda
    return 2.0 * well_A * x / well_lambda * np.exp(-x * x)


def pair_force(dist: np.ndarray, a: float, A: float, b: float, potential: int = SOFT, well_A: float = 0.0,
               well_lambda: float = 0.5) -> np.ndarray:
    """F_k(r) = -dU_k/dr, evaluated at max(r, 2a) (the linear continuation below 2a)."""
    rr = np.maximum(np.asarray(dist, dtype=float), 2.0 * a)
    F = A * np.exp(-(rr - 2.0 * a) / b) if A != 0.0 else np.zeros_like(rr)
    if potential in (REPEL_ATTRACT, REPEL_ATTRACT_REPEL):
        F = F - well_force(rr, 3.0 * a, well_A, well_lambda)
    if potential == REPEL_ATTRACT_REPEL:
        F = F + well_force(rr, 3.5 * a, well_A, well_lambda)
    return F


def blob_forces(r: np.ndarray, blob_body: np.ndarray, A: float, b: float, a: float, potential: int = SOFT,
                well_A: float = 0.0, well_lambda: float = 0.5, box: float | None = None) -> np.ndarray:
    """Blob forces f_i = sum over blobs j of other bodies of F_k(r_ij) (r_i - r_j)/r_ij.

    b and well_lambda are lengths (Sec. 6.4 uses A_w = 5 kT and lambda = 0.5 a).  In a
    periodic cube of side ``box`` (the FCM setting of Sec. 4.2) r_i - r_j is the minimum
    image: every other image of a blob is farther than box/2, where the forces have vanished
    for the cubes this is used with."""
    m = r.shape[0]
    f = np.zeros((m, 3))
    if A == 0.0 and (potential == SOFT or well_A == 0.0):
        return f
    for i in range(m):
        d = r[i][None, :] - r
        if box is not None:
            d -= box * np.round(d / box)
        dist = np.linalg.norm(d, axis=1)
        sel = (blob_body != blob_body[i]) & (dist > 0.0)
        mag = pair_force(dist[sel], a, A, b, potential, well_A, well_lambda)
        f[i] = (mag[:, None] * d[sel] / dist[sel, None]).sum(axis=0)
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
