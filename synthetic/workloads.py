"""Seeded synthetic suspensions with the shapes and sizes of the benchmark configs.

Every workload is generated from a seed, so nothing is read from disk.  The
generator places bodies by random sequential addition in a cube: each body
gets a uniform centre in [0, L)^3 and a uniform random unit quaternion
(a normalised 4-vector of N(0,1) draws, scalar part first), and is rejected
if any of its blobs comes closer than 2a to a blob of an already placed
body.  The domain is unbounded: bodies may stick out of the cube.

This module holds none of the method's arithmetic.  The rotation used for
the overlap test is scipy's, which shares no code with either the oracle
or the CUDA path.

Workloads (a = eta = kT = 1):

``c1``       4 icosahedra (12 blobs, circumradius 2a), 20a cube, seed 0, dt 0.01.
``c2``       256 rods of 10 blobs at spacing 2a in a 60a cube (~5% blob
             volume fraction), soft repulsion, dt 0.005, GMRES tol 1e-6.
``c3``       2,048 mixed bodies (42-blob icospheres, 15-blob rods, 21-blob
             boomerangs, a third each), 10% volume fraction, 53,253 blobs.
``c3_65k``   the same mix with 2,520 bodies (840 of each) = 65,520 blobs in a
             140a cube (10%): the 65k-blob throughput workload.
``c4``       512 independent suspensions, body counts uniform in 8..128,
             shapes uniform over {12-blob icosahedron, 10-blob rod,
             42-blob icosphere}, 5% volume fraction each, seeds per suspension.
``c5``       16,384 rods of 20 blobs (327,680 blobs) at 8% in a 257.9a cube,
             linear shear rate 1, dt 0.002.
``boomerang_wall``  15-blob boomerangs above a no-slip wall (the setting of Sec. 6.2),
             independent suspensions, with the wall repulsion and the weight of Sec. 6.2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence

import numpy as np
from scipy.spatial.transform import Rotation

from . import shapes


@dataclasses.dataclass
class Workload:
    name: str
    templates: List[np.ndarray]          # body-frame blob coordinates, n_t x 3
    body_tmpl: np.ndarray                # (N,) int32 template index of each body
    susp_body_off: np.ndarray            # (S+1,) int64 body offsets of suspensions
    Y: np.ndarray                        # (N, 3) body centres (blob centroids)
    q: np.ndarray                        # (N, 4) unit quaternions, scalar first
    params: Dict[str, float]
    box: np.ndarray                      # (S,) cube edge per suspension

    @property
    def n_bodies(self) -> int:
        return int(self.body_tmpl.shape[0])

    @property
    def n_susp(self) -> int:
        return int(self.susp_body_off.shape[0] - 1)

    @property
    def tmpl_nblobs(self) -> np.ndarray:
        return np.array([t.shape[0] for t in self.templates], dtype=np.int32)

    @property
    def n_blobs(self) -> int:
        return int(self.tmpl_nblobs[self.body_tmpl].sum())

    def susp_blob_counts(self) -> np.ndarray:
        nb = self.tmpl_nblobs[self.body_tmpl]
        off = self.susp_body_off
        return np.array([nb[off[s]:off[s + 1]].sum() for s in range(self.n_susp)], dtype=np.int64)

    def pair_evals_per_matvec(self) -> int:
        c = self.susp_blob_counts()
        return int((c.astype(np.float64) ** 2).sum())

    def subset(self, susp: Sequence[int]) -> "Workload":
        """The workload restricted to the listed suspensions (same order)."""
        off = self.susp_body_off
        idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in susp]).astype(np.int64)
        counts = [off[s + 1] - off[s] for s in susp]
        new_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return Workload(self.name + "_sub", self.templates, self.body_tmpl[idx].copy(), new_off,
                        self.Y[idx].copy(), self.q[idx].copy(), dict(self.params),
                        self.box[list(susp)].copy())

    def first_bodies(self, n: int) -> "Workload":
        """Single-suspension workload made of the first n bodies of suspension 0."""
        n = min(n, int(self.susp_body_off[1]))
        return Workload(f"{self.name}_first{n}", self.templates, self.body_tmpl[:n].copy(),
                        np.array([0, n], dtype=np.int64), self.Y[:n].copy(), self.q[:n].copy(),
                        dict(self.params), self.box[:1].copy())


def _centred(t: np.ndarray) -> np.ndarray:
    return t - t.mean(axis=0, keepdims=True)


def random_unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, 4))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


class _Grid:
    """Uniform hash grid of cell 2a for the overlap test of the placement."""

    def __init__(self, cell: float):
        self.cell = cell
        self.cells: Dict[tuple, List[tuple]] = {}

    def keys(self, pts: np.ndarray) -> np.ndarray:
        return np.floor(pts / self.cell).astype(np.int64)

    def conflict(self, pts: np.ndarray, dmin2: float) -> bool:
        """True when a stored point lies closer than sqrt(dmin2) to one of pts.

        With cell = sqrt(dmin2) such a point is in one of the 27 cells around the blob's
        cell; blobs are tested one at a time so that a rejected try usually stops early.
        """
        for (x, y, z), (i, j, k) in zip(pts.tolist(), self.keys(pts).tolist()):
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    for dk in (-1, 0, 1):
                        got = self.cells.get((i + di, j + dj, k + dk))
                        if got:
                            for (u, v, w) in got:
                                if (u - x) * (u - x) + (v - y) * (v - y) + (w - z) * (w - z) < dmin2:
                                    return True
        return False

    def add(self, pts: np.ndarray) -> None:
        for p, k in zip(pts.tolist(), map(tuple, self.keys(pts).tolist())):
            self.cells.setdefault(k, []).append(tuple(p))


def place_bodies(rng: np.random.Generator, templates: Sequence[np.ndarray], body_tmpl: np.ndarray,
                 box: float, a: float = 1.0, min_gap: float = 2.0, max_tries: int = 20000):
    """Random sequential addition of the bodies in ``body_tmpl`` into a cube of edge ``box``."""
    cen = [_centred(np.asarray(t, dtype=np.float64)) for t in templates]
    n = body_tmpl.shape[0]
    Y = np.zeros((n, 3))
    q = np.zeros((n, 4))
    dmin2 = (min_gap * a) ** 2
    # cell = 2a (min_gap * a): only blobs in the 27 cells around a cell can be closer than 2a.
    grid = _Grid(min_gap * a)
    for p in range(n):
        t = cen[int(body_tmpl[p])]
        for _ in range(max_tries):
            y = rng.uniform(0.0, box, size=3)
            qq = random_unit_quaternions(rng, 1)[0]
            rot = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]])  # scipy is scalar-last
            pts = y[None, :] + rot.apply(t)
            if not grid.conflict(pts, dmin2):
                break
        else:
            raise RuntimeError(f"could not place body {p} in a cube of edge {box}")
        Y[p] = y
        q[p] = qq
        grid.add(pts)
    return Y, q


def _box_for(templates, body_tmpl, phi: float, a: float = 1.0) -> float:
    nb = sum(templates[int(t)].shape[0] for t in body_tmpl)
    return (nb * 4.0 / 3.0 * math.pi * a ** 3 / phi) ** (1.0 / 3.0)


_BASE = dict(eta=1.0, kT=1.0, a=1.0, rep_A=0.0, rep_b=0.1, shear_rate=0.0,
             gmres_tol=1e-6, lanczos_tol=1e-4, rfd_delta=1e-6)


def c1(seed: int = 0) -> Workload:
    templates = [shapes.icosahedron()]
    bt = np.zeros(4, dtype=np.int32)
    rng = np.random.default_rng(seed)
    Y, q = place_bodies(rng, templates, bt, 20.0)
    params = dict(_BASE, dt=0.01, steps=100, seed=seed)
    return Workload("c1_4ico12", templates, bt, np.array([0, 4], dtype=np.int64), Y, q, params,
                    np.array([20.0]))


def c2(seed: int = 0, n_rods: int = 256, box: float = 60.0) -> Workload:
    templates = [shapes.rod(10, 2.0)]
    bt = np.zeros(n_rods, dtype=np.int32)
    rng = np.random.default_rng(seed)
    Y, q = place_bodies(rng, templates, bt, box)
    params = dict(_BASE, dt=0.005, steps=1000, seed=seed, rep_A=4.0, rep_b=0.1)
    return Workload(f"c2_{n_rods}rod10", templates, bt, np.array([0, n_rods], dtype=np.int64), Y, q,
                    params, np.array([box]))


def _mixed(n_bodies: int, seed: int, phi: float = 0.10, name: str = "c3") -> Workload:
    templates = [shapes.icosphere42(), shapes.rod(15, 2.0), shapes.boomerang(11, 1.0)]
    rng = np.random.default_rng(seed)
    bt = np.array([i % 3 for i in range(n_bodies)], dtype=np.int32)
    rng.shuffle(bt)
    box = _box_for(templates, bt, phi)
    Y, q = place_bodies(rng, templates, bt, box)
    params = dict(_BASE, dt=0.005, steps=200, seed=seed, rep_A=4.0, rep_b=0.1)
    return Workload(name, templates, bt, np.array([0, n_bodies], dtype=np.int64), Y, q, params,
                    np.array([box]))


def c3(seed: int = 0) -> Workload:
    return _mixed(2048, seed, name="c3_2048mixed")


def c3_65k(seed: int = 0) -> Workload:
    return _mixed(2520, seed, name="c3_65k_2520mixed")


def c4(seed: int = 0, n_susp: int = 512, nmin: int = 8, nmax: int = 128, phi: float = 0.05) -> Workload:
    templates = [shapes.icosahedron(), shapes.rod(10, 2.0), shapes.icosphere42()]
    rng = np.random.default_rng(seed)
    counts = rng.integers(nmin, nmax + 1, size=n_susp)
    bts, Ys, qs, boxes = [], [], [], []
    for s in range(n_susp):
        srng = np.random.default_rng([seed, s])
        bt = srng.integers(0, 3, size=int(counts[s])).astype(np.int32)
        box = _box_for(templates, bt, phi)
        Y, q = place_bodies(srng, templates, bt, box)
        bts.append(bt)
        Ys.append(Y)
        qs.append(q)
        boxes.append(box)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    params = dict(_BASE, dt=0.005, steps=100, seed=seed, rep_A=4.0, rep_b=0.1)
    return Workload(f"c4_{n_susp}susp", templates, np.concatenate(bts), off, np.vstack(Ys),
                    np.vstack(qs), params, np.asarray(boxes))


def c5(seed: int = 0, n_rods: int = 16384) -> Workload:
    templates = [shapes.rod(20, 2.0)]
    bt = np.zeros(n_rods, dtype=np.int32)
    rng = np.random.default_rng(seed)
    box = _box_for(templates, bt, 0.08)
    Y, q = place_bodies(rng, templates, bt, box)
    params = dict(_BASE, dt=0.002, steps=100, seed=seed, rep_A=4.0, rep_b=0.1, shear_rate=1.0,
                  lanczos_tol=1e-4)
    return Workload(f"c5_{n_rods}rod20", templates, bt, np.array([0, n_rods], dtype=np.int64), Y, q,
                    params, np.array([box]))


def boomerang_wall(n_susp: int = 36, bodies_per_susp: int = 1, seed: int = 0, spread: float = 12.0) -> Workload:
    """Boomerangs of 15 blobs at spacing a (two 8-blob arms sharing the corner, Sec. 6.2)
    above a no-slip wall at z = 0: n_susp independent suspensions (Sec. 6.2 runs 36) of
    bodies_per_susp boomerangs each, uniform random orientations, centres uniform in a
    spread x spread square at a height that keeps every blob at least 0.5a above z = a, no
    two bodies closer than 2a.  Wall repulsion V0 = 23 kT, b = 0.5a, weight mg = 0.18 kT/a,
    dt = 0.1 tau_D with tau_D = 6 pi eta a^3 / kT, GMRES and Lanczos tolerance 1e-4."""
    tmpl = shapes.boomerang(8, 1.0)
    cen = _centred(tmpl)
    reach = float(np.linalg.norm(cen, axis=1).max())
    rng = np.random.default_rng(seed)
    Ys, qs = [], []
    for s in range(n_susp):
        placed_Y, placed_pts = [], []
        for _ in range(bodies_per_susp):
            for _try in range(10000):
                y = np.array([*rng.uniform(0.0, spread, 2), 1.5 + reach + rng.uniform(0.0, 2.0)])
                qq = random_unit_quaternions(rng, 1)[0]
                pts = y[None, :] + Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).apply(cen)
                if all(np.min(np.linalg.norm(pts[:, None, :] - o[None, :, :], axis=-1)) >= 2.0 for o in placed_pts):
                    break
            else:
                raise RuntimeError("could not place a boomerang")
            placed_Y.append(y)
            placed_pts.append(pts)
            qs.append(qq)
        Ys.extend(placed_Y)
    n = n_susp * bodies_per_susp
    tau_d = 6.0 * math.pi
    params = dict(_BASE, dt=0.1 * tau_d, steps=100, seed=seed, gmres_tol=1e-4, lanczos_tol=1e-4, rfd_delta=1e-6,
                  wall=1, wall_V0=23.0, wall_b=0.5, body_weight=0.18)
    return Workload(f"boomerang_wall_{n_susp}x{bodies_per_susp}", [tmpl], np.zeros(n, dtype=np.int32),
                    (np.arange(n_susp + 1) * bodies_per_susp).astype(np.int64), np.array(Ys), np.array(qs), params,
                    np.full(n_susp, spread))


def mixed_small(n_bodies: int, seed: int = 0, phi: float = 0.10) -> Workload:
    """Small version of the c3 mix (same shapes and volume fraction) for parity tests."""
    return _mixed(n_bodies, seed, phi=phi, name=f"mixed{n_bodies}")


def batch_small(n_susp: int = 6, seed: int = 0, nmin: int = 2, nmax: int = 9) -> Workload:
    """Small version of the c4 batch for parity tests."""
    return c4(seed=seed, n_susp=n_susp, nmin=nmin, nmax=nmax)


BY_NAME = {"c1": c1, "c2": c2, "c3": c3, "c3_65k": c3_65k, "c4": c4, "c5": c5, "boomerang_wall": boomerang_wall,
           # half of c5's rods (163,840 blobs): a Lanczos basis of ~30 vectors already exceeds L2
           "c5_half": lambda seed=0: c5(seed=seed, n_rods=8192)}
