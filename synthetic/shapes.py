"""Body-frame blob templates for the synthetic workloads.

These are *inputs*: rigid bodies made of blobs of radius ``a``.  Nothing here
computes any part of the gDC method; the templates are returned as given
(not re-centred), because centring on the blob centroid is part of the
method and is done by each consumer.

Shapes (all lengths in units of the blob radius ``a``):

* ``icosahedron(a)``      -- 12 blobs on the vertices of a regular
  icosahedron of circumradius 2a (edge 2.103a).
* ``icosphere42(a)``      -- 42 blobs: the icosahedron's 12 vertices plus its
  30 edge midpoints pushed out to the sphere, scaled so that the smallest
  blob-blob spacing is exactly 2a (circumradius 3.659a).
* ``rod(n, spacing, a)``  -- n collinear blobs along z.
* ``boomerang(n_arm, spacing, a)`` -- an L of two n_arm-blob arms that share
  the corner blob, at right angles, in the x-y plane (Sec. 6.2 uses blob
  spacing a for its boomerang).
"""
from __future__ import annotations

import itertools

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron_unit() -> np.ndarray:
    v = []
    for s1, s2 in itertools.product((-1.0, 1.0), repeat=2):
        v.append((0.0, s1, s2 * _PHI))
        v.append((s1, s2 * _PHI, 0.0))
        v.append((s2 * _PHI, 0.0, s1))
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v[0])


def icosahedron(a: float = 1.0) -> np.ndarray:
    return 2.0 * a * _icosahedron_unit()


def icosphere42(a: float = 1.0) -> np.ndarray:
    v = _icosahedron_unit()
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=-1)
    edge = d[d > 0].min()
    mids = []
    for i in range(12):
        for j in range(i + 1, 12):
            if abs(d[i, j] - edge) < 1e-9:
                m = 0.5 * (v[i] + v[j])
                mids.append(m / np.linalg.norm(m))
    pts = np.vstack([v, np.asarray(mids)])
    assert pts.shape == (42, 3)
    dd = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1)
    smin = dd[dd > 0].min()
    return pts * (2.0 * a / smin)


def rod(n: int, spacing: float = 2.0, a: float = 1.0) -> np.ndarray:
    z = np.arange(n, dtype=np.float64) * spacing * a
    return np.stack([np.zeros(n), np.zeros(n), z], axis=1)


def boomerang(n_arm: int = 11, spacing: float = 1.0, a: float = 1.0) -> np.ndarray:
    k = np.arange(1, n_arm, dtype=np.float64) * spacing * a
    corner = np.zeros((1, 3))
    arm_x = np.stack([k, np.zeros_like(k), np.zeros_like(k)], axis=1)
    arm_y = np.stack([np.zeros_like(k), k, np.zeros_like(k)], axis=1)
    return np.vstack([corner, arm_x, arm_y])


def triangle(side: float = 2.0, a: float = 1.0) -> np.ndarray:
    """Three blobs on an equilateral triangle (smallest non-collinear body)."""
    s = side * a
    return np.array([[0.0, 0.0, 0.0], [s, 0.0, 0.0], [0.5 * s, 0.5 * np.sqrt(3.0) * s, 0.0]])


def dumbbell(d: float, a: float = 1.0) -> np.ndarray:
    return np.array([[-0.5 * d * a, 0.0, 0.0], [0.5 * d * a, 0.0, 0.0]])
