"""Pins of the matrix-free CPU twin (oracle/twin.py, oracle/twin.c) against the dense oracle.

The twin is the timed CPU baseline at sizes the dense oracle cannot store; here, on
suspensions small enough for both, its pair-by-pair FP64 products equal the dense RPY
matrix times lambda, its forces equal the dense oracle's, and its whole gDC step (Lanczos
at the benchmark's tolerance, GMRES with the block preconditioner) equals the dense step
with the same Lanczos iterate and an exact (LU) solve.
"""
import numpy as np
import pytest

from oracle import forces, geometry as G, philox, rpy, twin
from oracle import gdc as ogdc
from synthetic import workloads as WL


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_twin_product_equals_the_dense_rpy_matrix():
    rng = np.random.default_rng(3)
    r = rng.uniform(0.0, 7.0, size=(300, 3))
    r[7] = r[3]                      # coincident blobs take the self term
    lam = rng.standard_normal(900)
    u = twin.rpy_product(r, lam, 1.3, 0.7)
    assert _rel(u, rpy.rpy_matrix(r, 1.3, 0.7) @ lam) < 1e-13


def test_twin_forces_equal_the_dense_oracle():
    wl = WL.c2(seed=4, n_rods=40, box=25.0)
    lay = G.Layout(wl.templates, wl.body_tmpl)
    r = G.blob_positions(lay, wl.Y, wl.q)
    f = twin.soft_forces(r, lay.blob_body, 4.0, 0.1, 1.0)
    ref = forces.blob_forces(r, lay.blob_body, 4.0, 0.1, 1.0)
    assert np.abs(ref).max() > 0
    assert np.abs(f - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["mixed", "rods"])
def test_twin_step_equals_the_dense_step(which):
    wl = WL.mixed_small(12, seed=1) if which == "mixed" else WL.c2(seed=2, n_rods=30, box=30.0)
    lay = G.Layout(wl.templates, wl.body_tmpl)
    W = philox.normals(5, 0, 0, 0, 3 * lay.n_blobs)
    Wt = philox.normals(5, 0, 0, 1, 6 * lay.n_bodies)
    ora = ogdc.gdc_step(lay, wl.Y, wl.q, W, Wt, ogdc.Params.from_dict(dict(wl.params, rfd_delta=1e-4,
                                                                           sqrt_lanczos_tol=1e-4)))
    tw = twin.gdc_step(lay, wl.Y, wl.q, W, Wt, twin.TwinParams.from_dict(dict(wl.params, rfd_delta=1e-4,
                                                                           lanczos_tol=1e-4, gmres_tol=1e-12)))
    assert (tw["k0"], tw["k_mid"]) == (ora["k0"], ora["k_mid"])
    assert _rel(tw["vb0"], ora["vb0"]) < 1e-12 and _rel(tw["vb"], ora["vb"]) < 1e-12
    assert _rel(tw["calV"], ora["calV"]) < 1e-12
    assert abs(tw["nu"] - ora["nu"]) < 1e-10
    assert tw["residual"] <= 1e-12
    assert _rel(tw["V"], ora["V"]) < 1e-9
    assert _rel(tw["Y1"] - wl.Y, ora["Y1"] - wl.Y) < 1e-9
    assert tw["products"] == 2 * tw["k0"] + tw["k_mid"] + tw["gmres_iters"] + tw["gmres_cycles"]
