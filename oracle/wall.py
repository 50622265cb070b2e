"""Oracle mobility of blobs above a no-slip wall, and the wall forces of Sec. 6.2.

TEST INFRASTRUCTURE ONLY.  The paper's RPY runs (Sec. 4.1, Sec. 6.2) use the RPY tensor
corrected for a planar no-slip wall (it cites Swan & Brady for it) without printing it.
Here it is built from its definition, the Rotne-Prager regularisation of the Green's
function of a point force above a wall:

* G(x, y): the velocity at x due to a unit point force at y = (y1, y2, h), h > 0, above the
  wall z = 0 (Blake's image system: the Stokeslet at y, minus the Stokeslet at the mirror
  point y* = (y1, y2, -h), plus the image source dipole and Stokes doublet at y*):
      8 pi eta G_ij = S_ij(x - y) - S_ij(R) + 2 h M_jk d/dR_k [ h R_i/|R|^3 - S_i3(R) ]
  with R = x - y*, S_ij(v) = delta_ij/|v| + v_i v_j/|v|^3 and M = diag(1, 1, -1);
* the wall-corrected mobility of two blobs of radius a at x (target) and y (source):
      M_ij(x, y) = RPY_ij(x - y) + (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) W_ij(x, y),
  RPY the unbounded tensor of rpy.py (its overlapping form included) and W the image part
  of G (G minus the free Stokeslet, smooth for blobs above the wall).  Each Laplacian is a
  Faxen operator: it averages over one sphere's surface (exact for these biharmonic terms).

The Laplacians are applied by symbolic differentiation (sympy), once per process, and the
result is evaluated numerically.  Pinned by: no slip of G on the wall, incompressibility,
the reciprocal symmetry M_ij(x, y) = M_ji(y, x), the self-mobility series of a sphere above
a wall (1 - 9a/16h + a^3/8h^3 - a^5/16h^5 parallel, 1 - 9a/8h + a^3/2h^3 - a^5/8h^5 normal,
in units of 1/(6 pi eta a)), positive definiteness above the wall, and the unbounded RPY
far from it.  Readings: a blob whose centre is at h <= a overlaps the wall, where the
correction is not a mobility; the oracle refuses such configurations.

Wall forces (Sec. 6.2): every blob at height h feels the repulsion of the potential
V(h) = V0 a exp(-(h - a)/b) / (h - a), i.e. the force -dV/dh along z; a body of weight mg
feels -mg along z, shared equally by its blobs (the blob centroid Y_p is its centre of
mass, so gravity exerts no torque about it).
"""
from __future__ import annotations

import functools

import numpy as np

from . import rpy


def _oseen(v, vn):
    import sympy as sp
    return [[sp.KroneckerDelta(i, j) / vn + v[i] * v[j] / vn ** 3 for j in range(3)] for i in range(3)]


@functools.lru_cache(maxsize=None)
def _symbolic():
    """The image part of Blake's Green's function and its Faxen-regularised form, as numpy
    functions of the mirror vector R = x - y*, the source height h and the radius a."""
    import sympy as sp
    R1, R2, R3 = sp.symbols("R1 R2 R3", real=True)
    h, a = sp.symbols("h a", positive=True)
    Rv = (R1, R2, R3)
    Rn = sp.sqrt(R1 ** 2 + R2 ** 2 + R3 ** 2)
    S = _oseen(Rv, Rn)
    mirror = (1, 1, -1)
    img = [[None] * 3 for _ in range(3)]
    reg = [[None] * 3 for _ in range(3)]
    lap = lambda f: sum(sp.diff(f, v, 2) for v in Rv)
    for i in range(3):
        dip = h * Rv[i] / Rn ** 3 - S[i][2]
        for j in range(3):
            f = -S[i][j] + 2 * h * mirror[j] * sp.diff(dip, Rv[j])
            img[i][j] = f
            # as a function of x and y: R = (x1 - y1, x2 - y2, x3 + y3), h = y3, so
            # Lap_x = Lap_R and Lap_y = Lap_R + 2 d2/dR3 dh + d2/dh2
            g = f + a ** 2 / 6 * (lap(f) + 2 * sp.diff(f, R3, h) + sp.diff(f, h, 2))
            reg[i][j] = g + a ** 2 / 6 * lap(g)
    args = (R1, R2, R3, h, a)
    return (sp.lambdify(args, sp.Matrix(img), "numpy", cse=True),
            sp.lambdify(args, sp.Matrix(reg), "numpy", cse=True))


def _mirror_vector(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return x[0] - y[0], x[1] - y[1], x[2] + y[2], y[2]


def blake(x, y, eta: float = 1.0) -> np.ndarray:
    """G(x, y) (3 x 3): velocity at x of a unit point force at y above the wall z = 0."""
    img, _ = _symbolic()
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    dn = np.linalg.norm(d)
    free = np.eye(3) / dn + np.outer(d, d) / dn ** 3
    R1, R2, R3, h = _mirror_vector(x, y)
    return (free + np.asarray(img(R1, R2, R3, h, 1.0), dtype=np.float64)) / (8.0 * np.pi * eta)


def wall_correction(x, y, a: float, eta: float) -> np.ndarray:
    """(1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) of the image part of G, for a target blob at x and a
    source blob at y (3 x 3)."""
    _, reg = _symbolic()
    R1, R2, R3, h = _mirror_vector(x, y)
    return np.asarray(reg(R1, R2, R3, h, a), dtype=np.float64) / (8.0 * np.pi * eta)


def wall_matrix(r: np.ndarray, a: float, eta: float) -> np.ndarray:
    """Dense 3M x 3M wall-corrected blob mobility: rpy.rpy_matrix plus the wall correction of
    every pair (self pairs included).  Every blob centre must be above z = a."""
    r = np.asarray(r, dtype=np.float64)
    if not (r[:, 2] > a).all():
        raise ValueError("a blob centre is at or below z = a: the blob overlaps the wall")
    m = r.shape[0]
    _, reg = _symbolic()
    X = np.repeat(r, m, axis=0)            # targets i (row-major over i, j)
    Ysrc = np.tile(r, (m, 1))              # sources j
    blocks = np.asarray(reg(X[:, 0] - Ysrc[:, 0], X[:, 1] - Ysrc[:, 1], X[:, 2] + Ysrc[:, 2], Ysrc[:, 2], a),
                        dtype=np.float64)   # (3, 3, m*m) after broadcasting
    blocks = np.broadcast_to(blocks, (3, 3, m * m)).reshape(3, 3, m, m).transpose(2, 0, 3, 1)
    return rpy.rpy_matrix(r, a, eta) + blocks.reshape(3 * m, 3 * m) / (8.0 * np.pi * eta)


def wall_force(h, V0: float, b: float, a: float):
    """-dV/dh for V(h) = V0 a exp(-(h - a)/b) / (h - a) (Sec. 6.2), for h > a."""
    h = np.asarray(h, dtype=np.float64)
    s = h - a
    return V0 * a * np.exp(-s / b) * (1.0 / (b * s) + 1.0 / (s * s))


def wall_potential(h, V0: float, b: float, a: float):
    h = np.asarray(h, dtype=np.float64)
    return V0 * a * np.exp(-(h - a) / b) / (h - a)


def blob_wall_forces(r: np.ndarray, blob_body: np.ndarray, n_bodies: int, V0: float, b: float, a: float,
                     weight: float) -> np.ndarray:
    """Per-blob forces (M, 3): the wall repulsion of every blob and the body weight shared
    equally by its blobs, both along z."""
    f = np.zeros_like(np.asarray(r, dtype=np.float64))
    if V0 != 0.0:
        f[:, 2] += wall_force(r[:, 2], V0, b, a)
    if weight != 0.0:
        counts = np.bincount(blob_body, minlength=n_bodies)
        f[:, 2] -= weight / counts[blob_body]
    return f
