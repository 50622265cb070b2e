"""Pins of the oracle's pair forces for the potentials of Sec. 6.3 and Sec. 6.4.

The energies below are written from the paper's definitions: the soft sphere of
Eq. (soft_sphere_potential), the Gaussian wells phi_c(r) = A_w exp(-((r - c)/lambda)^2),
U_1 = U - phi_{3a} and U_2 = U - phi_{3a} + phi_{7a/2}, each continued below r = 2a by the
straight line that keeps it and its slope continuous.  The slope at 2a is taken here by a
central difference of the r >= 2a formula, so nothing of the oracle's force code is reused.
"""
import numpy as np
import pytest

from oracle import forces, geometry as G
from synthetic import shapes

# Sec. 6.3 and 6.4 (kT = a = 1): U0 = 20 kT, b = 0.5 a, A_w = 5 kT, lambda = 0.5 a
U0, B, AW, LAM = 20.0, 0.5, 5.0, 0.5


def _smooth_energy(r, potential, u0=U0, b=B, aw=AW, lam=LAM, a=1.0):
    """The r >= 2a branch of U_k, evaluated as written (also defined below 2a)."""
    e = u0 * np.exp((2 * a - r) / b)
    if potential >= 1:
        e = e - aw * np.exp(-((r - 3 * a) / (lam * a)) ** 2)
    if potential == 2:
        e = e + aw * np.exp(-((r - 3.5 * a) / (lam * a)) ** 2)
    return e


def _energy_pair(r, potential, **kw):
    a = kw.get("a", 1.0)
    h = 1e-5
    u2a = _smooth_energy(2 * a, potential, **kw)
    slope = (_smooth_energy(2 * a + h, potential, **kw) - _smooth_energy(2 * a - h, potential, **kw)) / (2 * h)
    return np.where(r >= 2 * a, _smooth_energy(r, potential, **kw), u2a + slope * (r - 2 * a))


def _energy(r, blob_body, potential, **kw):
    e = 0.0
    for i in range(r.shape[0]):
        d = np.linalg.norm(r[i + 1:] - r[i], axis=1)
        other = blob_body[i + 1:] != blob_body[i]
        e += _energy_pair(d[other], potential, **kw).sum()
    return e


def _oracle(r, blob_body, potential, u0=U0, b=B, aw=AW, lam=LAM, a=1.0):
    return forces.blob_forces(r, blob_body, u0 / b, b, a, potential, aw, lam * a)


def _three_bodies(seed):
    templates = [shapes.triangle(), shapes.rod(3), shapes.icosahedron()]
    rng = np.random.default_rng(seed)
    lay = G.Layout(templates, np.array([0, 1, 2]))
    # centres close enough that pairs fall below 2a, in the wells and beyond the barrier
    Y = np.array([[0.0, 0.0, 0.0], [2.6, 1.1, 0.4], [0.8, 4.4, -1.2]])
    g = rng.standard_normal((3, 4))
    q = g / np.linalg.norm(g, axis=1, keepdims=True)
    return lay, Y, q, G.blob_positions(lay, Y, q)


@pytest.mark.parametrize("potential,a", [(0, 1.0), (1, 1.0), (2, 1.0), (2, 0.8)])
def test_forces_are_minus_the_energy_gradient(potential, a):
    lay, Y, q, r = _three_bodies(seed=potential)
    r = r * a          # the same shapes with blob radius a (every length scales with a)
    d = np.linalg.norm(r[:, None] - r[None], axis=2)[lay.blob_body[:, None] != lay.blob_body[None]]
    assert d.min() < 2 * a and ((d > 2.6 * a) & (d < 4 * a)).any(), "pairs must span the continuation and the wells"
    f = _oracle(r, lay.blob_body, potential, b=B * a, a=a)
    h = 1e-6
    for i in range(r.shape[0]):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, c] += h
            rm[i, c] -= h
            g = (_energy(rp, lay.blob_body, potential, b=B * a, a=a) -
                 _energy(rm, lay.blob_body, potential, b=B * a, a=a)) / (2 * h)
            assert abs(f[i, c] + g) < 2e-6 * (1 + abs(g)), (i, c, f[i, c], -g)


def test_pair_forces_sum_to_zero_force_and_torque():
    lay, Y, q, r = _three_bodies(seed=5)
    f = _oracle(r, lay.blob_body, 2)
    assert np.abs(f).max() > 1.0
    np.testing.assert_allclose(f.sum(axis=0), 0.0, atol=1e-11)
    np.testing.assert_allclose(np.cross(r, f).sum(axis=0), 0.0, atol=1e-10)


def _extrema(r, F):
    """Minima (force + to -) and maxima (force - to +) of the energy, in order of r."""
    mins = [r[i + 1] for i in range(len(r) - 1) if F[i] > 0 and F[i + 1] <= 0]
    maxs = [r[i + 1] for i in range(len(r) - 1) if F[i] < 0 and F[i + 1] >= 0]
    return mins, maxs


def test_well_shapes():
    r = np.linspace(1.0, 7.0, 6001)
    F0, F1, F2 = (forces.pair_force(r, 1.0, U0 / B, B, k, AW, LAM) for k in (0, 1, 2))
    # constant force for overlapping blobs, continuous at 2a
    for F in (F0, F1, F2):
        assert np.all(F[r < 2.0] == F[np.searchsorted(r, 2.0)])
    assert np.all(F0 > 0)
    # repel-attract: repulsive at contact, then a well of negative energy near 3a; the soft
    # sphere outlasts the Gaussian, so a small bump (well below the well's depth) follows
    mins1, maxs1 = _extrema(r, F1)
    assert F1[0] > 0 and len(mins1) == 1 and 2.5 < mins1[0] < 3.5
    assert _energy_pair(mins1[0], 1) < -1.0
    assert all(m > mins1[0] and _energy_pair(m, 1) < 0.5 for m in maxs1)
    # repel-attract-repel: a well, then a barrier just beyond it, several kT high
    mins2, maxs2 = _extrema(r, F2)
    assert F2[0] > 0 and len(mins2) >= 1 and 2.5 < mins2[0] < 3.5
    assert len(maxs2) >= 1 and mins2[0] < maxs2[0] < 4.0
    assert _energy_pair(maxs2[0], 2) - _energy_pair(mins2[0], 2) > 2.0
    assert _energy_pair(maxs2[0], 2) > max([_energy_pair(m, 1) for m in maxs1] + [0.0]) + 2.0


def test_special_cases_reduce_to_the_soft_sphere():
    lay, Y, q, r = _three_bodies(seed=3)
    soft = _oracle(r, lay.blob_body, 0)
    np.testing.assert_array_equal(_oracle(r, lay.blob_body, 1, aw=0.0), soft)
    np.testing.assert_array_equal(_oracle(r, lay.blob_body, 2, aw=0.0), soft)
    # the wells alone, without the soft sphere, are minus the gradient of -phi_3a
    f = _oracle(r, lay.blob_body, 1, u0=0.0)
    g = _oracle(r, lay.blob_body, 1) - soft
    np.testing.assert_allclose(f, g, atol=1e-12)


def test_periodic_forces_are_the_sum_over_images():
    """In a periodic cube the minimum-image forces equal the sum over every image shift of
    -1, 0, 1 cube sides (all nearer images), computed by brute force."""
    lay, Y, q, r = _three_bodies(seed=4)
    box = 16.0                                     # force range ~6.5a < box / 2
    r = r + np.array([7.0, -9.0, 15.0])            # bodies straddle the cube's faces
    f = forces.blob_forces(r, lay.blob_body, U0 / B, B, 1.0, 2, AW, LAM, box=box)
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]) * box
    ref = np.zeros_like(r)
    for i in range(r.shape[0]):
        for j in range(r.shape[0]):
            if lay.blob_body[i] == lay.blob_body[j]:
                continue
            d = r[i] - r[j] - shifts
            dist = np.linalg.norm(d, axis=1)
            mag = forces.pair_force(dist, 1.0, U0 / B, B, 2, AW, LAM)
            mag[dist > 8.0] = 0.0                  # beyond the range: below 1e-15
            ref[i] += (mag[:, None] * d / dist[:, None]).sum(axis=0)
    np.testing.assert_allclose(f, ref, atol=1e-12 * np.abs(ref).max())
    # and translating one body by a cube side changes nothing
    r2 = r.copy()
    r2[lay.blob_body == 1] += np.array([box, -box, 0.0])
    np.testing.assert_allclose(forces.blob_forces(r2, lay.blob_body, U0 / B, B, 1.0, 2, AW, LAM, box=box), f,
                               atol=1e-12 * np.abs(f).max())


@pytest.mark.parametrize("potential", [0, 1, 2])
def test_matrix_free_rows_equal_the_dense_forces(potential):
    """oracle.matfree.repulsion_rows (the sampled-row oracle of the full-size tests) gives the
    rows of blob_forces, which the energy-gradient tests pin."""
    from oracle import matfree
    lay, Y, q, r = _three_bodies(seed=6 + potential)
    f = _oracle(r, lay.blob_body, potential)
    rows = np.array([0, 3, 5, r.shape[0] - 1])
    got = matfree.repulsion_rows(r, lay.blob_body, rows, U0 / B, B, 1.0, potential, AW, LAM)
    np.testing.assert_allclose(got, f[rows], atol=1e-13 * np.abs(f).max())
