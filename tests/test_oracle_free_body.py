"""Stochastic invariants of free bodies over many oracle gDC steps (pins of the oracle).

The same closed forms as the GPU test of free bodies, on a CPU-sized ensemble:

* a free 12-blob icosahedron: <|Y(t0 + t) - Y(t0)|^2> = 6 kT mu_t t, and each body axis
  decorrelates as <e(t0 + t) . e(t0)> = f^n with f = 1/3 + (2/3)(1 - s^2) exp(-s^2/2),
  s^2 = 2 kT mu_r dt (independent isotropic rotations by dt Omega);
* free rods started parallel reach uniformly distributed axes.

Windows of n steps that do not overlap are independent for a free body, so every
trajectory contributes several samples.  Tolerances are 4 standard errors of the samples.
"""
import numpy as np
import pytest

from oracle import geometry as G
from oracle.gdc import Params, body_mobility_at, gdc_step
from synthetic import shapes


def _run(lay, q0, p, n_rep, n_steps, seed):
    rng = np.random.default_rng(seed)
    nb = 3 * lay.n_blobs
    Ys, qs = [], []
    for r in range(n_rep):
        Y, q = np.zeros((1, 3)), q0[r:r + 1].copy()
        traj_Y, traj_q = [Y[0].copy()], [q[0].copy()]
        for _ in range(n_steps):
            o = gdc_step(lay, Y, q, rng.standard_normal(nb), rng.standard_normal(6), p)
            Y, q = o["Y1"], o["q1"]
            traj_Y.append(Y[0].copy())
            traj_q.append(q[0].copy())
        Ys.append(traj_Y)
        qs.append(traj_q)
    return np.array(Ys), np.array(qs)


@pytest.mark.slow
def test_oracle_free_icosahedron_msd_and_orientation_autocorrelation():
    lay = G.Layout([shapes.icosahedron()], [0])
    p = Params(dt=3.0, kT=1.0, rfd_delta=1e-6)
    N = body_mobility_at(lay, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), p)
    mu_t, mu_r = N[0, 0], N[3, 3]
    rng = np.random.default_rng(1)
    g = rng.standard_normal((100, 4))
    Ys, qs = _run(lay, g / np.linalg.norm(g, axis=1, keepdims=True), p, 100, 60, seed=2)
    lag = 20
    starts = np.arange(0, 60, lag)
    d2 = np.concatenate([((Ys[:, s + lag] - Ys[:, s]) ** 2).sum(axis=1) for s in starts])
    expect = 6 * p.kT * mu_t * lag * p.dt
    assert abs(d2.mean() - expect) < 4 * d2.std() / np.sqrt(d2.size), (d2.mean(), expect)
    R = np.array([[G.rotation_matrix(x) for x in row] for row in qs])
    corr = np.concatenate([np.einsum("nia,nia->n", R[:, s + lag], R[:, s]) / 3.0 for s in starts])
    s2 = 2 * p.kT * mu_r * p.dt
    f = 1.0 / 3.0 + 2.0 / 3.0 * (1 - s2) * np.exp(-s2 / 2)
    assert abs(corr.mean() - f ** lag) < 4 * corr.std() / np.sqrt(corr.size), (corr.mean(), f ** lag)
    assert f ** lag < 0.8


@pytest.mark.slow
def test_oracle_free_rods_reach_uniform_axes():
    lay = G.Layout([shapes.rod(10)], [0])
    N = body_mobility_at(lay, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), Params())
    dt = 0.2 / (2 * N[3, 3])                      # angular variance 0.2 per component per step
    p = Params(dt=dt, kT=1.0, rfd_delta=1e-6)
    n = 150
    Ys, qs = _run(lay, np.tile([1.0, 0, 0, 0], (n, 1)), p, n, 40, seed=3)
    cos_t = np.array([G.rotation_matrix(x)[2, 2] for x in qs[:, -1]])
    assert abs(cos_t.mean()) < 4 / np.sqrt(3 * n)
    assert abs((cos_t ** 2).mean() - 1.0 / 3.0) < 4 * np.sqrt(4.0 / 45.0 / n)
    # at the start every axis is along z: the test has power
    assert np.allclose([G.rotation_matrix(x)[2, 2] for x in qs[:, 0]], 1.0)
