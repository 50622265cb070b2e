"""Stochastic invariants of free bodies over many gDC steps, on the GPU.

Each suspension holds one body and nothing else, so a batched context advances many
independent replicas at once (the FP32-mixed path the benchmark times).  For a lone body
the gDC step's increment has the covariance 2 kT dt N (App. E) and, by symmetry, no drift,
so over many steps:

* a 12-blob icosahedron (N_tt = mu_t I, N_tr = 0, N_rr = mu_r I by its symmetry) has the
  translational mean-squared displacement <|Y(t) - Y(0)|^2> = 6 kT mu_t t = 2 tr(D_t) t;
* each body axis e of the icosahedron decorrelates as a product of independent isotropic
  random rotations: <e(t) . e(0)> = f^n after n steps, with f = 1/3 + (2/3) E[cos|theta|]
  for the rotation vector theta = dt Omega, isotropic Gaussian with per-component variance
  s^2 = 2 kT mu_r dt, whence E[cos|theta|] = (1 - s^2) exp(-s^2 / 2); as dt -> 0, f^n ->
  exp(-2 kT mu_r t), the orientation autocorrelation of an isotropic rotor;
* rods of collinear blobs started parallel end up with uniformly distributed axes:
  cos(theta) to the start direction is uniform on [-1, 1].

mu_t and mu_r come from the oracle's dense N.  The step's scalar nu multiplies the increment;
for a lone body its mean is 1 and its variance (about 3e-3 here) shifts these moments by
less than their statistical tolerance (4 standard errors).
"""
import numpy as np
import pytest

from oracle import geometry as G
from oracle.gdc import Params, body_mobility_at
from synthetic import shapes
from synthetic import workloads as WL

pytestmark = pytest.mark.gpu


def _replicas(template, n, seed):
    rng = np.random.default_rng(seed)
    q = WL.random_unit_quaternions(rng, n) if seed is not None else np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    return WL.Workload("free_replicas", [template], np.zeros(n, dtype=np.int32), np.arange(n + 1, dtype=np.int64),
                       np.zeros((n, 3)), q, dict(WL.c1().params), np.ones(n))


def _ctx(lib, wl, dt, kT):
    return lib.context_from_workload(wl, precision=1, dt=dt, kT=kT, lanczos_tol=1e-4, lanczos_max_iter=16,
                                     gmres_tol=1e-6, gmres_restart=10, gmres_max_iter=100, rfd_delta=1e-3,
                                     seed=2024, rep_A=0.0)


def _axes(q):
    return np.array([G.rotation_matrix(x) for x in q])   # columns: body axes in the lab frame


def test_free_icosahedron_msd_and_orientation_autocorrelation(lib):
    n_rep, dt, kT = 16384, 0.76, 1.0
    wl = _replicas(shapes.icosahedron(), n_rep, seed=5)
    lay = G.Layout([shapes.icosahedron()], [0])
    N = body_mobility_at(lay, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), Params())
    mu_t, mu_r = N[0, 0], N[3, 3]
    ctx = _ctx(lib, wl, dt, kT)
    Y0, q0, _ = ctx.get_state()
    A0 = _axes(q0)
    s2 = 2 * kT * mu_r * dt
    f = 1.0 / 3.0 + 2.0 / 3.0 * (1 - s2) * np.exp(-s2 / 2)
    done = 0
    for chunk in (75, 75, 150):
        ctx.step(chunk, info=False)
        done += chunk
        Y, q, step = ctx.get_state()
        assert step == done
        d2 = ((Y - Y0) ** 2).sum(axis=1)
        msd, se = d2.mean(), d2.std() / np.sqrt(n_rep)
        expect = 6 * kT * mu_t * done * dt
        assert abs(msd - expect) < 4 * se + 5e-3 * expect, (done, msd, expect, se)
        corr = np.einsum("nia,nia->na", _axes(q), A0)   # e_a(t) . e_a(0) per replica and axis
        c, se_c = corr.mean(), corr.mean(axis=1).std() / np.sqrt(n_rep)
        assert abs(c - f ** done) < 4 * se_c + 5e-3 * f ** done, (done, c, f ** done, se_c)
        # the continuum rate: f^n and exp(-2 kT mu_r t) differ by O(n s^4)
        assert abs(f ** done - np.exp(-2 * kT * mu_r * done * dt)) < done * s2 ** 2
    assert f ** done < 0.35   # the correlation has decayed well away from 1


def test_free_rods_reach_uniform_axes(lib):
    from scipy import stats
    n_rep, kT = 16384, 1.0
    tmpl = shapes.rod(10)
    lay = G.Layout([tmpl], [0])
    N = body_mobility_at(lay, np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]), Params())
    mu_r = N[3, 3]                        # rotation about an axis across the rod
    dt = 0.02 / (2 * kT * mu_r)           # per-step angular variance 0.02 per component
    wl = _replicas(tmpl, n_rep, seed=None)   # every rod starts along z
    ctx = _ctx(lib, wl, dt, kT)
    ctx.step(400, info=False)             # angular variance 8 per component in all: P1 ~ e^-8
    Y, q, _ = ctx.get_state()
    cos_t = _axes(q)[:, 2, 2]             # z component of the rod axis (template along z)
    se = 1.0 / np.sqrt(3 * n_rep)
    assert abs(cos_t.mean()) < 4 * se
    assert abs((cos_t ** 2).mean() - 1.0 / 3.0) < 4 * np.sqrt(4.0 / 45.0 / n_rep)
    assert stats.kstest(cos_t, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
