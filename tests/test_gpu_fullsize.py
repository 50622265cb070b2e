"""GPU checks at the benchmark's full size (65,520 blobs) and on the other workload shapes.

At full size the dense oracle cannot run (M would need 309 GB), so the RPY product is
checked on sampled rows that the oracle evaluates one by one (oracle.matfree), and the
mobility solve and the step are checked through properties that hold at any size.
The library runs in the configuration bench.py times (FP32-mixed, autotuned tiling).
"""
import numpy as np
import pytest

from oracle import geometry as G, matfree, philox, rigid
from oracle import gdc as ogdc
from synthetic import workloads as WL

from gpu_common import dense_state, oracle_params, rel, rot_err, susp_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl65():
    return WL.c3_65k()


@pytest.fixture(scope="module")
def ctx65(lib, wl65):
    return lib.context_from_workload(wl65, precision=lib.FP32_MIXED, rfd_delta=1e-3, gmres_tol=1e-6,
                                     lanczos_tol=1e-4, lanczos_max_iter=128)


def _host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_rpy_sampled_rows_65k(lib, wl65, ctx65, prec):
    rng = np.random.default_rng(21)
    lam = rng.standard_normal(3 * wl65.n_blobs)
    u = _host(ctx65.rpy_apply(lam, prec)).reshape(-1, 3)
    r = _host(ctx65.blob_positions()).reshape(-1, 3)
    lay, Y, q = susp_layout(wl65, 0)
    np.testing.assert_allclose(r, G.blob_positions(lay, Y, q), rtol=0, atol=1e-11)
    rows = np.concatenate([[0, 1, wl65.n_blobs - 1], rng.choice(wl65.n_blobs, 61, replace=False)])
    ref = matfree.rpy_rows(r, lam.reshape(-1, 3), rows, 1.0, 1.0)
    err = np.abs(u[rows] - ref).max() / np.abs(ref).max()
    assert err < {0: 1e-12, 1: 1e-5, 2: 1e-11}[prec], err


def test_rpy_sampled_rows_327k(lib):
    """The 327,680-blob rod suspension (640 tiles of 512): the symmetric FP32 kernel and the
    symmetric double-float kernel, whose work items widen to 10 source tiles beyond 128
    tiles per suspension, on sampled rows."""
    wl = WL.c5()
    ctx = lib.context_from_workload(wl, precision=lib.FP32_MIXED, autotune=0, pair_kernel=2)
    assert ctx.profile_read()["df_kernel"] == 4
    rng = np.random.default_rng(23)
    lam = rng.standard_normal(3 * wl.n_blobs)
    r = _host(ctx.blob_positions()).reshape(-1, 3)
    rows = np.concatenate([[0, 1, wl.n_blobs - 1], rng.choice(wl.n_blobs, 61, replace=False)])
    ref = matfree.rpy_rows(r, lam.reshape(-1, 3), rows, 1.0, 1.0)
    for prec, tol in ((1, 1e-5), (2, 1e-11)):
        u = _host(ctx.rpy_apply(lam, prec)).reshape(-1, 3)
        err = np.abs(u[rows] - ref).max() / np.abs(ref).max()
        assert err < tol, (prec, err)


def test_mobility_solve_65k(lib, wl65, ctx65):
    rng = np.random.default_rng(22)
    FT = np.zeros(6 * wl65.n_bodies)
    vb = rng.standard_normal(3 * wl65.n_blobs)
    V, lam, info = ctx65.mobility_solve(FT, vb, want_lambda=True)
    assert info["converged"] and info["residual"] <= 1e-6
    assert info["matvecs_fp64"] >= 1          # the reported residual is an FP64 one
    # independent check of the blob equations on sampled rows: M lambda - K V = -vbrev
    lam = _host(lam).reshape(-1, 3)
    V = _host(V).reshape(-1, 6)
    r = _host(ctx65.blob_positions()).reshape(-1, 3)
    lay, Y, q = susp_layout(wl65, 0)
    rows = rng.choice(wl65.n_blobs, 48, replace=False)
    Ml = matfree.rpy_rows(r, lam, rows, 1.0, 1.0)
    p = lay.blob_body[rows]
    KV = V[p, :3] + np.cross(V[p, 3:], r[rows] - Y[p])
    resid = Ml - KV + vb.reshape(-1, 3)[rows]
    assert np.abs(resid).max() <= 1e-6 * np.linalg.norm(vb)


def test_gdc_step_65k_properties(lib, wl65, ctx65):
    info = ctx65.step(1)[0]
    Y1, q1, stp = ctx65.get_state()
    assert info["solve"]["converged"] and info["solve"]["residual"] <= 1e-6
    assert np.isfinite(Y1).all() and np.isfinite(q1).all()
    assert np.abs(np.linalg.norm(q1, axis=1) - 1.0).max() < 1e-13
    disp = np.linalg.norm(Y1 - wl65.Y, axis=1)
    # a step of dt = 0.005 moves bodies by a fraction of a blob radius
    assert 0 < disp.max() < 1.0
    assert 0.0 < info["nu_min"] <= info["nu_max"] < 3.0
    assert info["lanczos_err"] < 1e-4


def test_shear_flow_step_parity(lib):
    # Config-5 physics (rods in linear shear u = (gamma_dot y, 0, 0)) at a size the oracle can run.
    wl = WL.c2(seed=4, n_rods=24, box=26.0)
    wl.params.update(shear_rate=1.0, dt=0.002)
    seed = 9
    ctx = lib.context_from_workload(wl, precision=lib.FP64, rfd_delta=1e-6, seed=seed, gmres_tol=1e-12,
                                    lanczos_tol=1e-11, lanczos_max_iter=128, gmres_max_iter=1000)
    ctx.step(1)
    Y1, q1, _ = ctx.get_state()
    lay, Y, q = susp_layout(wl, 0)
    W = philox.normals(seed, 0, 0, 0, 3 * lay.n_blobs)
    Wt = philox.normals(seed, 0, 0, 1, 6 * lay.n_bodies)
    ora = ogdc.gdc_step(lay, Y, q, W, Wt, oracle_params(wl))
    assert rel(Y1 - Y, ora["Y1"] - Y) < 1e-6
    assert rot_err(q1, ora["q1"]) < 1e-9
    # the flow drags bodies along x in proportion to their height
    ctx2 = lib.context_from_workload(wl, precision=lib.FP64, kT=0.0, rep_A=0.0, gmres_tol=1e-12)
    V, _, _ = ctx2.mobility_solve(np.zeros(6 * wl.n_bodies))
    V = _host(V).reshape(-1, 6)
    slope = np.polyfit(wl.Y[:, 1], V[:, 0], 1)[0]
    assert 0.5 < slope < 1.5


def test_batch_of_uneven_suspensions_matches_per_suspension_runs(lib):
    # Batching: a context of several uneven suspensions gives each one the result of a context of
    # its own.  kT = 0 removes the draws (which are keyed by the suspension index), so the
    # deterministic step (repulsion + mobility solve + update) must agree to solver precision.
    wl = WL.batch_small(5, seed=8, nmin=2, nmax=6)
    kw = dict(precision=lib.FP64, kT=0.0, rep_A=4.0, rep_b=0.5, gmres_tol=1e-13, gmres_max_iter=1000, autotune=0)
    big = lib.context_from_workload(wl, **kw)
    big.step(2)
    Yb, qb, _ = big.get_state()
    moved = 0.0
    for s in range(wl.n_susp):
        ctx = lib.context_from_workload(wl.subset([s]), **kw)
        ctx.step(2)
        Ys, qs, _ = ctx.get_state()
        o, e = wl.susp_body_off[s], wl.susp_body_off[s + 1]
        np.testing.assert_allclose(Yb[o:e], Ys, rtol=0, atol=1e-11)
        np.testing.assert_allclose(qb[o:e], qs, rtol=0, atol=1e-11)
        moved = max(moved, np.abs(Ys - wl.Y[o:e]).max())
    assert moved > 0.0
