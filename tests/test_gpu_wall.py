"""GPU parity of the wall mode (blobs above a no-slip wall, Sec. 4.1 and Sec. 6.2) against the
oracle's wall-corrected mobility (oracle/wall.py: the Faxen-regularised image system, built
by symbolic differentiation) and its gDC step.

Workload: 15-blob boomerangs at blob spacing a (Sec. 6.2) in independent suspensions above
the wall, with the Sec. 6.2 wall repulsion (V0 = 23 kT, b = 0.5a) and weight (0.18 kT/a).
Tolerances as for the unbounded mobility: FP64 products to rounding, FP32 products 2e-6,
steps to the solver tolerances.
"""
import numpy as np
import pytest

from oracle import forces, geometry as G, philox, rigid, wall
from oracle import gdc as ogdc
from synthetic import workloads as WL

from gpu_common import blob_slices, oracle_params, rel, rot_err, susp_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl():
    return WL.boomerang_wall(3, 3, seed=2)


def _dense(wl, s):
    lay, Y, q = susp_layout(wl, s)
    r = G.blob_positions(lay, Y, q)
    M = wall.wall_matrix(r, 1.0, 1.0)
    K = rigid.k_matrix(r, Y, lay.blob_body)
    return lay, Y, q, r, M, K, rigid.rigid_basis(K, lay.n_bodies)


def _host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_wall_product(lib, wl, prec):
    ctx = lib.context_from_workload(wl)
    lam = np.random.default_rng(1).standard_normal(3 * wl.n_blobs)
    u = _host(ctx.rpy_apply(lam, prec))
    for s, (a, b) in enumerate(blob_slices(wl)):
        lay, Y, q, r, M, K, B = _dense(wl, s)
        ref = M @ lam[3 * a:3 * b]
        assert rel(u[3 * a:3 * b], ref) < {0: 1e-13, 1: 2e-6, 2: 1e-11}[prec], (s, rel(u[3 * a:3 * b], ref))


def test_wall_preconditioner(lib, wl):
    ctx = lib.context_from_workload(wl)
    rvec = np.random.default_rng(2).standard_normal(int(ctx.saddle_off[-1]))
    z = _host(ctx.precond_apply(rvec))
    for s in range(wl.n_susp):
        lay, Y, q, r, M, K, B = _dense(wl, s)
        o = int(ctx.saddle_off[s])
        nl = 3 * lay.n_blobs
        for p in range(lay.n_bodies):
            i0, i1 = lay.blob_off[p], lay.blob_off[p + 1]
            Mp, Kp = M[3 * i0:3 * i1, 3 * i0:3 * i1], K[3 * i0:3 * i1, 6 * p:6 * p + 6]
            lp, vp = rigid.saddle_solve(Mp, Kp, np.eye(6), -rvec[o + 3 * i0:o + 3 * i1],
                                        -rvec[o + nl + 6 * p:o + nl + 6 * p + 6])
            assert rel(z[o + 3 * i0:o + 3 * i1], lp) < 1e-10
            assert rel(z[o + nl + 6 * p:o + nl + 6 * p + 6], vp) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_wall_brownian_slip(lib, wl, prec):
    tol = 1e-11 if prec == 0 else 1e-6
    ctx = lib.context_from_workload(wl, precision=prec, lanczos_tol=tol, lanczos_max_iter=128)
    W = np.random.default_rng(3).standard_normal(3 * wl.n_blobs)
    vb, iters, err = ctx.brownian_slip(W)
    vb = _host(vb)
    scale = np.sqrt(2 * wl.params["kT"] / wl.params["dt"])
    for s, (a, b) in enumerate(blob_slices(wl)):
        lay, Y, q, r, M, K, B = _dense(wl, s)
        ref = scale * rigid.sqrtm_block(M, rigid.block_factor_lab(lay, M)) @ W[3 * a:3 * b]
        assert rel(vb[3 * a:3 * b], ref) < (1e-9 if prec == 0 else 2e-5)


def test_wall_forces(lib, wl):
    ctx = lib.context_from_workload(wl, rep_A=4.0, rep_b=0.1)
    FT = _host(ctx.forces())
    for s in range(wl.n_susp):
        lay, Y, q, r, M, K, B = _dense(wl, s)
        o, e = int(wl.susp_body_off[s]), int(wl.susp_body_off[s + 1])
        f = forces.blob_forces(r, lay.blob_body, 4.0, 0.1, 1.0) + wall.blob_wall_forces(
            r, lay.blob_body, lay.n_bodies, 23.0, 0.5, 1.0, 0.18)
        ref = forces.body_force_torque(r, Y, lay.blob_body, f)
        assert rel(FT[6 * o:6 * e], ref) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_wall_step_parity(lib, wl, prec):
    seed = 17
    delta = 1e-6 if prec == 0 else 1e-3
    kw = dict(precision=prec, seed=seed, rfd_delta=delta, lanczos_max_iter=128, gmres_max_iter=1000)
    kw.update(dict(gmres_tol=1e-12, lanczos_tol=1e-11) if prec == 0 else dict(gmres_tol=1e-6, lanczos_tol=1e-7))
    ctx = lib.context_from_workload(wl, **kw)
    tr = ctx.set_trace(True)
    info = ctx.step(1)[0]
    Y1, q1, _ = ctx.get_state()
    assert info["solve"]["converged"]
    op = oracle_params(wl, rfd_delta=delta)
    assert op.wall and op.wall_V0 == 23.0 and op.body_weight == 0.18
    nu = _host(tr["nu"])
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        o, e = int(wl.susp_body_off[s]), int(wl.susp_body_off[s + 1])
        W = philox.normals(seed, s, 0, 0, 3 * lay.n_blobs)
        Wt = philox.normals(seed, s, 0, 1, 6 * lay.n_bodies)
        ora = ogdc.gdc_step(lay, Y, q, W, Wt, op)
        disp = rel(Y1[o:e] - Y, ora["Y1"] - Y)
        if prec == 0:
            assert disp < 1e-7 and rot_err(q1[o:e], ora["q1"]) < 1e-9 and abs(nu[s] - ora["nu"]) < 1e-6, disp
        else:
            assert disp < 1e-3 and rot_err(q1[o:e], ora["q1"]) < 1e-5 and abs(nu[s] - ora["nu"]) < 1e-3, disp
            assert np.abs(Y1[o:e] - ora["Y1"]).max() / np.abs(ora["Y1"]).max() < 1e-5


def test_wall_step_at_the_paper_settings_graph_equals_host(lib):
    """Sec. 6.2's solver settings (GMRES and Lanczos 1e-4, RFD delta 1e-6 in FP64) over a few
    steps of 36 single-boomerang suspensions (the paper's 36 runs in one batch): the graph
    replay equals the host-driven steps bit for bit, every blob stays above the wall."""
    wl = WL.boomerang_wall(36, 1, seed=4)
    outs = []
    for graph in (1, 0):
        ctx = lib.context_from_workload(wl, precision=0, graph=graph, seed=5)
        infos = ctx.step(4)
        Y, q, _ = ctx.get_state()
        outs.append((Y, q))
        assert all(i["solve"]["residual"] <= 1e-4 for i in infos)
        r = _host(ctx.blob_positions()).reshape(-1, 3)
        assert r[:, 2].min() > 1.0
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_wall_rejects_a_blob_below_its_radius(lib):
    wl = WL.boomerang_wall(1, 2, seed=6)
    Y = wl.Y.copy()
    Y[0, 2] = 0.5       # the body's lowest blobs are now below z = a
    bad = WL.Workload("low", wl.templates, wl.body_tmpl, wl.susp_body_off, Y, wl.q, wl.params, wl.box)
    with pytest.raises(lib.GdcError) as ei:
        lib.context_from_workload(bad)
    assert ei.value.status == 4
