"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on seeded inputs.

Tolerances: FP64 paths agree with the oracle to rounding and solver tolerance; the
FP32-mixed path must meet the target of one-step positions and orientations to
relative 1e-5 with mobility-solve residual <= 1e-6 (checked with the oracle's
dense FP64 operator).  Sizes span several 256-target tiles with ragged tails.
"""
import numpy as np
import pytest

from oracle import forces, geometry as G, philox, rigid, rpy
from oracle import gdc as ogdc
from synthetic import workloads as WL

from gpu_common import blob_slices, dense_state, oracle_params, rel, rot_err, susp_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl_mix():
    return WL.mixed_small(40, seed=1)


@pytest.fixture(scope="module")
def wl_batch():
    return WL.batch_small(6, seed=3)


@pytest.fixture(scope="module")
def wl_rod():
    return WL.c2(seed=2, n_rods=60, box=37.0)


@pytest.fixture(scope="module")
def wl_c1():
    return WL.c1()


def ctx_for(lib, wl, **kw):
    return lib.context_from_workload(wl, **kw)


def _host(t):
    return t.detach().cpu().numpy()


def test_normals_match_oracle(lib, wl_batch):
    ctx = ctx_for(lib, wl_batch, seed=1234567890123)
    sl = blob_slices(wl_batch)
    for step in (0, 7):
        W = _host(ctx.draw_normals(step, 0))
        Wt = _host(ctx.draw_normals(step, 1))
        for s in range(wl_batch.n_susp):
            lay, _, _ = susp_layout(wl_batch, s)
            a, b = sl[s]
            ref = philox.normals(1234567890123, s, step, 0, 3 * lay.n_blobs)
            np.testing.assert_allclose(W[3 * a:3 * b], ref, rtol=0, atol=1e-13)
            o = int(wl_batch.susp_body_off[s])
            ref_t = philox.normals(1234567890123, s, step, 1, 6 * lay.n_bodies)
            np.testing.assert_allclose(Wt[6 * o:6 * o + 6 * lay.n_bodies], ref_t, rtol=0, atol=1e-13)


def test_blob_positions(lib, wl_mix):
    ctx = ctx_for(lib, wl_mix)
    lay, Y, q = susp_layout(wl_mix, 0)
    np.testing.assert_allclose(_host(ctx.blob_positions()).reshape(-1, 3), G.blob_positions(lay, Y, q),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("which", ["mix", "batch"])
def test_rpy_apply(lib, wl_mix, wl_batch, prec, which):
    # prec 2: the double-float product the FP32-mixed solve checks its residuals with
    wl = wl_mix if which == "mix" else wl_batch
    ctx = ctx_for(lib, wl)
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(3 * wl.n_blobs)
    u = _host(ctx.rpy_apply(lam, prec))
    sl = blob_slices(wl)
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        a, b = sl[s]
        r, M, _, _ = dense_state(lay, Y, q)
        ref = M @ lam[3 * a:3 * b]
        if prec == 0:
            assert rel(u[3 * a:3 * b], ref) < 1e-13
        elif prec == 2:
            assert rel(u[3 * a:3 * b], ref) < 1e-11
            assert np.abs(u[3 * a:3 * b] - ref).max() < 1e-11 * np.abs(ref).max()
        else:
            assert rel(u[3 * a:3 * b], ref) < 2e-6
            assert np.abs(u[3 * a:3 * b] - ref).max() < 1e-5 * np.abs(ref).max()


def _oracle_saddle(wl):
    out = []
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        out.append(dense_state(lay, Y, q) + (lay,))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_saddle_apply(lib, wl_batch, prec):
    ctx = ctx_for(lib, wl_batch)
    rng = np.random.default_rng(12)
    n = int(ctx.saddle_off[-1])
    x = rng.standard_normal(n)
    y = _host(ctx.saddle_apply(x, prec))
    for s, (r, M, K, B, lay) in enumerate(_oracle_saddle(wl_batch)):
        o = int(ctx.saddle_off[s])
        lam, V = x[o:o + 3 * lay.n_blobs], x[o + 3 * lay.n_blobs:o + 3 * lay.n_blobs + 6 * lay.n_bodies]
        y1, y2 = rigid.saddle_apply(M, K, lam, V)
        got = y[o:o + 3 * lay.n_blobs + 6 * lay.n_bodies]
        tol = 1e-13 if prec == 0 else 2e-6
        assert rel(got, np.concatenate([y1, y2])) < tol


def test_precond_apply(lib, wl_mix, wl_rod):
    for wl in (wl_mix, wl_rod):
        ctx = ctx_for(lib, wl)
        rng = np.random.default_rng(13)
        n = int(ctx.saddle_off[-1])
        rvec = rng.standard_normal(n)
        z = _host(ctx.precond_apply(rvec))
        lay, Y, q = susp_layout(wl, 0)
        r, M, K, B = dense_state(lay, Y, q)
        nl = 3 * lay.n_blobs
        ref_l = np.zeros(nl)
        ref_v = np.zeros(6 * lay.n_bodies)
        for p in range(lay.n_bodies):
            i0, i1 = lay.blob_off[p], lay.blob_off[p + 1]
            Mp = M[3 * i0:3 * i1, 3 * i0:3 * i1]
            Kp = K[3 * i0:3 * i1, 6 * p:6 * p + 6]
            Bp = rigid.rigid_basis(Kp, 1)
            rv = Bp @ (Bp.T @ rvec[nl + 6 * p:nl + 6 * p + 6])
            lp, vp = rigid.saddle_solve(Mp, Kp, Bp, -rvec[3 * i0:3 * i1], -rv)
            ref_l[3 * i0:3 * i1] = lp
            ref_v[6 * p:6 * p + 6] = vp
        # rods: the axial torque component is not in the range of K^T and is dropped
        assert rel(z[:nl], ref_l) < 1e-10
        assert rel(z[nl:], ref_v) < 1e-10


def test_lsq_velocity(lib, wl_mix, wl_rod):
    for wl in (wl_mix, wl_rod):
        ctx = ctx_for(lib, wl)
        rng = np.random.default_rng(14)
        vb = rng.standard_normal(3 * wl.n_blobs)
        got = _host(ctx.lsq_velocity(vb))
        lay, Y, q = susp_layout(wl, 0)
        r, M, K, B = dense_state(lay, Y, q)
        assert rel(got, rigid.lsq_velocity(K, B, vb)) < 1e-12


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_brownian_slip_lanczos(lib, wl_mix, prec, precond):
    """Lanczos converges to the symmetric root M^(1/2) W (precond 0) or to the block-preconditioned
    root L (L^-1 M L^-T)^(1/2) W of Chow & Saad (precond 1), computed densely by the oracle."""
    tol = 1e-11 if prec == 0 else 1e-6
    ctx = ctx_for(lib, wl_mix, precision=prec, lanczos_tol=tol, lanczos_max_iter=128, kT=1.3, dt=0.02,
                  lanczos_precond=precond)
    rng = np.random.default_rng(15)
    W = rng.standard_normal(3 * wl_mix.n_blobs)
    vb, iters, err = ctx.brownian_slip(W)
    lay, Y, q = susp_layout(wl_mix, 0)
    r, M, K, B = dense_state(lay, Y, q)
    S = rigid.sqrtm_block(M, rigid.block_factor(lay, q, 1.0, 1.0)) if precond else rigid.sqrtm_sym(M)
    ref = np.sqrt(2 * 1.3 / 0.02) * S @ W
    assert 2 <= iters <= 128
    assert rel(_host(vb), ref) < (1e-9 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_brownian_slip_many_bodies(lib, prec):
    """About 6,300 bodies in 1,400 small suspensions, enough for the factor products of the
    preconditioned Lanczos to group several bodies of one template per block: the roots of 40
    sampled suspensions against the oracle's dense block-preconditioned root."""
    wl = WL.batch_small(1400, seed=3, nmin=4, nmax=5)
    assert wl.n_bodies >= 6000
    tol = 1e-11 if prec == 0 else 1e-6
    ctx = ctx_for(lib, wl, precision=prec, lanczos_tol=tol, lanczos_max_iter=128, kT=1.3, dt=0.02,
                  lanczos_precond=1, autotune=0)
    rng = np.random.default_rng(16)
    W = rng.standard_normal(3 * wl.n_blobs)
    vb = _host(ctx.brownian_slip(W)[0])
    sl = blob_slices(wl)
    for s in rng.choice(wl.n_susp, 40, replace=False):
        lay, Y, q = susp_layout(wl, s)
        r, M, K, B = dense_state(lay, Y, q)
        a, b = sl[s]
        ref = np.sqrt(2 * 1.3 / 0.02) * rigid.sqrtm_block(M, rigid.block_factor(lay, q, 1.0, 1.0)) @ W[3 * a:3 * b]
        assert rel(vb[3 * a:3 * b], ref) < (1e-9 if prec == 0 else 2e-5), (s, rel(vb[3 * a:3 * b], ref))


def test_precond_and_solve_many_bodies(lib):
    """About 6,300 bodies, enough for the block preconditioner to group several bodies of one
    template per block: its application against the oracle's per-body saddle solves on
    sampled bodies, and mobility solves in FP64 and FP32-mixed (whose inner cycles apply the
    template M^-1 in FP32) against the oracle's LU on sampled suspensions, with iteration
    counts that show the FP32 preconditioner preconditions as well."""
    wl = WL.batch_small(1400, seed=3, nmin=4, nmax=5)
    rng = np.random.default_rng(17)
    ctx = ctx_for(lib, wl, precision=0, gmres_tol=1e-12, gmres_max_iter=800, autotune=0)
    n = int(ctx.saddle_off[-1])
    rvec = rng.standard_normal(n)
    z = _host(ctx.precond_apply(rvec))
    picks = rng.choice(wl.n_susp, 30, replace=False)
    for s in picks[:10]:
        lay, Y, q = susp_layout(wl, s)
        r, M, K, B = dense_state(lay, Y, q)
        o = int(ctx.saddle_off[s])
        nl = 3 * lay.n_blobs
        for p in range(lay.n_bodies):
            i0, i1 = lay.blob_off[p], lay.blob_off[p + 1]
            Mp = M[3 * i0:3 * i1, 3 * i0:3 * i1]
            Kp = K[3 * i0:3 * i1, 6 * p:6 * p + 6]
            Bp = rigid.rigid_basis(Kp, 1)
            rv = Bp @ (Bp.T @ rvec[o + nl + 6 * p:o + nl + 6 * p + 6])
            lp, vp = rigid.saddle_solve(Mp, Kp, Bp, -rvec[o + 3 * i0:o + 3 * i1], -rv)
            assert rel(z[o + 3 * i0:o + 3 * i1], lp) < 1e-10
            assert rel(z[o + nl + 6 * p:o + nl + 6 * p + 6], vp) < 1e-10
    FT = rng.standard_normal(6 * wl.n_bodies).reshape(-1, 6)
    vb = rng.standard_normal(3 * wl.n_blobs)
    # physical torques only: none on the collinear rods (their axial spin is not a DOF)
    collinear = [np.linalg.matrix_rank(t - t.mean(0), tol=1e-9) <= 1 for t in wl.templates]
    FT[np.array([collinear[t] for t in wl.body_tmpl]), 3:] = 0.0
    FT = FT.reshape(-1)
    iters = {}
    for prec, tol, check in ((0, 1e-12, True), (0, 1e-6, False), (1, 1e-6, True)):
        c2 = ctx_for(lib, wl, precision=prec, gmres_tol=tol, gmres_max_iter=800, autotune=0)
        V, lam, info = c2.mobility_solve(FT, vb, want_lambda=True)
        V, lam = _host(V), _host(lam)
        assert info["converged"] and info["residual"] <= tol
        iters[(prec, tol)] = info["iterations"]
        if not check:
            continue
        sl = blob_slices(wl)
        for s in picks:
            lay, Y, q = susp_layout(wl, s)
            r, M, K, B = dense_state(lay, Y, q)
            a, b = sl[s]
            o = int(wl.susp_body_off[s])
            Fs = FT[6 * o:6 * o + 6 * lay.n_bodies]
            ls, Vs = rigid.saddle_solve(M, K, B, vb[3 * a:3 * b], Fs)
            assert rel(V[6 * o:6 * o + 6 * lay.n_bodies], Vs) < (1e-9 if prec == 0 else 1e-4)
    # the FP32-mixed solve (FP32 preconditioner product) needs about the FP64 solve's iterations
    assert iters[(1, 1e-6)] <= 1.25 * iters[(0, 1e-6)] + 3, iters


@pytest.mark.parametrize("prec", [0, 1])
def test_mobility_solve(lib, wl_mix, wl_rod, wl_batch, prec):
    for wl in (wl_mix, wl_rod, wl_batch):
        tol = 1e-12 if prec == 0 else 1e-6
        ctx = ctx_for(lib, wl, precision=prec, gmres_tol=tol, gmres_max_iter=800)
        rng = np.random.default_rng(16)
        FT = rng.standard_normal(6 * wl.n_bodies)
        vb = rng.standard_normal(3 * wl.n_blobs)
        dense = _oracle_saddle(wl)
        for s, (r, M, K, B, lay) in enumerate(dense):
            o = int(wl.susp_body_off[s])
            # rod axial torques are outside the range of K^T: physical torques never have them
            FT[6 * o:6 * o + 6 * lay.n_bodies] = B @ (B.T @ FT[6 * o:6 * o + 6 * lay.n_bodies])
        V, lam, info = ctx.mobility_solve(FT, vb, want_lambda=True)
        V, lam = _host(V), _host(lam)
        assert info["converged"] and info["residual"] <= tol
        sl = blob_slices(wl)
        for s, (r, M, K, B, lay) in enumerate(dense):
            a, b = sl[s]
            o = int(wl.susp_body_off[s])
            Fs = FT[6 * o:6 * o + 6 * lay.n_bodies]
            ls, Vs = rigid.saddle_solve(M, K, B, vb[3 * a:3 * b], Fs)
            Vg = V[6 * o:6 * o + 6 * lay.n_bodies]
            lg = lam[3 * a:3 * b]
            # FP64 residual of the GPU solution with the oracle's dense operator
            y1, y2 = rigid.saddle_apply(M, K, lg, Vg)
            res = np.linalg.norm(np.concatenate([y1 + vb[3 * a:3 * b], y2 + Fs])) / np.linalg.norm(
                np.concatenate([vb[3 * a:3 * b], Fs]))
            assert res <= 2 * tol, res
            assert rel(Vg, Vs) < (1e-9 if prec == 0 else 1e-4)


@pytest.mark.parametrize("prec", [0, 1])
def test_forces(lib, wl_mix, prec):
    ctx = ctx_for(lib, wl_mix, precision=prec)
    got = _host(ctx.forces())
    lay, Y, q = susp_layout(wl_mix, 0)
    r = G.blob_positions(lay, Y, q)
    f = forces.blob_forces(r, lay.blob_body, wl_mix.params["rep_A"], wl_mix.params["rep_b"], 1.0)
    ref = forces.body_force_torque(r, Y, lay.blob_body, f)
    assert np.abs(ref).max() > 0
    assert rel(got, ref) < (1e-12 if prec == 0 else 1e-5)


def _oracle_step(wl, s, seed, step, op, div="rfd", scheme="gdc"):
    lay, Y, q = susp_layout(wl, s)
    W = philox.normals(seed, s, step, 0, 3 * lay.n_blobs)
    Wt = philox.normals(seed, s, step, 1, 6 * lay.n_bodies)
    if scheme == "em":
        return ogdc.em_step(lay, Y, q, W, op)
    return ogdc.gdc_step(lay, Y, q, W, Wt, op, div=div)


def _step_case(lib, wl, prec, div=0, scheme=0):
    seed = 77
    delta = 1e-6 if prec == 0 else 1e-3
    kw = dict(precision=prec, seed=seed, rfd_delta=delta, divmode=div, scheme=scheme, lanczos_max_iter=128)
    if prec == 0:
        kw.update(gmres_tol=1e-12, lanczos_tol=1e-11, gmres_max_iter=1000)
    else:
        kw.update(gmres_tol=1e-6, lanczos_tol=1e-7, gmres_max_iter=1000)
    ctx = ctx_for(lib, wl, **kw)
    tr = ctx.set_trace(True)
    info = ctx.step(1)[0]
    Y1, q1, stp = ctx.get_state()
    assert stp == 1
    op = oracle_params(wl, rfd_delta=delta)
    out = []
    for s in range(wl.n_susp):
        o, e = int(wl.susp_body_off[s]), int(wl.susp_body_off[s + 1])
        ora = _oracle_step(wl, s, seed, 0, op, div="rfd" if div == 0 else "fd", scheme="gdc" if scheme == 0 else "em")
        out.append((s, o, e, ora))
    return ctx, tr, info, Y1, q1, out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", ["c1", "mix", "rod", "batch"])
def test_gdc_step_parity(lib, wl_c1, wl_mix, wl_rod, wl_batch, prec, which):
    wl = dict(c1=wl_c1, mix=wl_mix, rod=wl_rod, batch=wl_batch)[which]
    ctx, tr, info, Y1, q1, out = _step_case(lib, wl, prec)
    assert info["solve"]["converged"]
    nu = _host(tr["nu"])
    calV = _host(tr["calV"]).reshape(-1, 6)
    Vm = _host(tr["Vm"]).reshape(-1, 6)
    for s, o, e, ora in out:
        Y0 = wl.Y[o:e]
        pos_err = np.abs(Y1[o:e] - ora["Y1"]).max() / np.abs(ora["Y1"]).max()
        disp_err = rel(Y1[o:e] - Y0, ora["Y1"] - Y0)
        r_err = rot_err(q1[o:e], ora["q1"])
        if prec == 0:
            assert pos_err < 1e-11 and r_err < 1e-9 and disp_err < 1e-6, (pos_err, r_err, disp_err)
            assert rel(calV[o:e], ora["calV"]) < 1e-8
            assert abs(nu[s] - ora["nu"]) < 1e-6
            assert rel(Vm[o:e], ora["V"]) < 1e-7
        else:
            assert pos_err < 1e-5 and r_err < 1e-5, (pos_err, r_err, disp_err)
            assert disp_err < 1e-3, disp_err
            assert rel(calV[o:e], ora["calV"]) < 1e-4
            assert abs(nu[s] - ora["nu"]) < 1e-3


def test_em_step_parity(lib, wl_mix):
    ctx, tr, info, Y1, q1, out = _step_case(lib, wl_mix, 0, scheme=1)
    for s, o, e, ora in out:
        assert rel(Y1[o:e] - wl_mix.Y[o:e], ora["Y1"] - wl_mix.Y[o:e]) < 1e-7
        assert rot_err(q1[o:e], ora["q1"]) < 1e-9


def test_fd_divergence_parity(lib, wl_c1):
    ctx, tr, info, Y1, q1, out = _step_case(lib, wl_c1, 0, div=1)
    nu = _host(tr["nu"])
    for s, o, e, ora in out:
        assert abs(nu[s] - ora["nu"]) < 1e-6
        assert rel(Y1[o:e] - wl_c1.Y[o:e], ora["Y1"] - wl_c1.Y[o:e]) < 1e-6


def test_checkpoint_resume_is_bitwise(lib, wl_batch):
    ctx = ctx_for(lib, wl_batch, precision=1, rfd_delta=1e-3)
    Y0, q0, _ = ctx.get_state()
    ctx.step(2)
    Ya, qa, sa = ctx.get_state()
    ctx.set_state(Y0, q0, 0)
    ctx.step(1)
    Yh, qh, sh = ctx.get_state()
    ctx.set_state(Yh, qh, sh)
    ctx.step(1)
    Yb, qb, sb = ctx.get_state()
    assert sa == sb == 2
    np.testing.assert_array_equal(Ya, Yb)
    np.testing.assert_array_equal(qa, qb)


def test_errors_are_reported(lib, wl_c1):
    ctx = ctx_for(lib, wl_c1)
    Y, q, _ = ctx.get_state()
    bad = q.copy()
    bad[1] *= 1.5
    with pytest.raises(lib.GdcError) as ei:
        ctx.set_state(Y, bad, 0)
    assert ei.value.status == 1
    Yn = Y.copy()
    Yn[0, 0] = np.nan
    with pytest.raises(lib.GdcError):
        ctx.set_state(Yn, q, 0)
    ctx2 = ctx_for(lib, wl_c1, gmres_tol=1e-15, gmres_max_iter=2)
    with pytest.raises(lib.GdcError) as ei:
        ctx2.mobility_solve(np.ones(6 * wl_c1.n_bodies))
    assert ei.value.status == 3
    ctx3 = ctx_for(lib, wl_c1, lanczos_tol=1e-15, lanczos_max_iter=2)
    with pytest.raises(lib.GdcError) as ei:
        ctx3.brownian_slip(np.ones(3 * wl_c1.n_blobs))
    assert ei.value.status == 3
    # the context stays usable after an error
    V, _, info = ctx.mobility_solve(np.ones(6 * wl_c1.n_bodies))
    assert info["converged"]


def _overlapping_workload(kind):
    """Bodies whose blobs come closer than 2a to blobs of other bodies.

    "pairs": a mixed suspension with a few bodies moved onto their neighbours (a handful of
    overlapping pairs per blob, held in the near-pair list).  "pile": twelve 42-blob
    icospheres around nearly the same centre (more than 32 blobs within 2a of most blobs,
    which the FP32 product corrects by searching the suspension).
    """
    if kind == "pairs":
        wl = WL.mixed_small(40, seed=5)
        Y = wl.Y.copy()
        for p in range(0, 12, 2):
            Y[p + 1] = Y[p] + np.array([0.9, 0.4, -0.3]) * (1 + p / 12)
        return WL.Workload("overlap_pairs", wl.templates, wl.body_tmpl, wl.susp_body_off, Y, wl.q, wl.params, wl.box)
    from synthetic import shapes
    rng = np.random.default_rng(8)
    n = 12
    Y = rng.uniform(-0.3, 0.3, size=(n, 3))
    q = WL.random_unit_quaternions(rng, n)
    return WL.Workload("overlap_pile", [shapes.icosphere42()], np.zeros(n, dtype=np.int32),
                       np.array([0, n], dtype=np.int64), Y, q, dict(WL.c1().params), np.array([10.0]))


@pytest.mark.parametrize("kind", ["pairs", "pile"])
def test_rpy32_with_overlapping_bodies(lib, kind):
    """FP32 product and saddle operator when blobs of different bodies overlap.

    The FP32 kernel evaluates every pair at the clamped distance max(r, 2a); the epilogue
    corrects the self pair and every pair closer than 2a in FP64.
    """
    wl = _overlapping_workload(kind)
    lay, Y, q = susp_layout(wl, 0)
    r, M, K, B = dense_state(lay, Y, q)
    d = np.linalg.norm(r[:, None, :] - r[None, :, :], axis=-1)
    other = lay.blob_body[:, None] != lay.blob_body[None, :]
    near_other = ((d < 2.0) & other).sum(axis=1)
    if kind == "pairs":
        assert near_other.max() >= 1
    else:
        assert (((d < 2.0).sum(axis=1) - 1) > 32).mean() > 0.5
    ctx = ctx_for(lib, wl, autotune=0)
    rng = np.random.default_rng(17)
    lam = rng.standard_normal(3 * wl.n_blobs)
    u = _host(ctx.rpy_apply(lam, 1))
    ref = M @ lam
    assert rel(u, ref) < 2e-6
    assert np.abs(u - ref).max() < 1e-5 * np.abs(ref).max()
    n = int(ctx.saddle_off[-1])
    x = rng.standard_normal(n)
    y = _host(ctx.saddle_apply(x, 1))
    y1, y2 = rigid.saddle_apply(M, K, x[:3 * wl.n_blobs], x[3 * wl.n_blobs:])
    assert rel(y, np.concatenate([y1, y2])) < 2e-6


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("which", ["mix120", "batch_multi_tile", "overlap_pile"])
def test_rpy32_ordered_and_symmetric_kernels(lib, kernel, which):
    """Both FP32 pair kernels against the dense oracle, on suspensions of several 512-blob
    tiles (diagonal and off-diagonal tiles, ragged last tiles, work items of several tiles)."""
    if which == "mix120":
        wl = WL.mixed_small(120, seed=4)
    elif which == "batch_multi_tile":
        wl = WL.c4(seed=6, n_susp=5, nmin=20, nmax=70)
    else:
        wl = _overlapping_workload("pile")
    ctx = ctx_for(lib, wl, autotune=0, pair_kernel=kernel)
    rng = np.random.default_rng(19)
    lam = rng.standard_normal(3 * wl.n_blobs)
    u = _host(ctx.rpy_apply(lam, 1))
    n = int(ctx.saddle_off[-1])
    x = rng.standard_normal(n)
    y = _host(ctx.saddle_apply(x, 1))
    # the double-float residual product of the same kernel family (ordered or symmetric)
    udf = _host(ctx.rpy_apply(lam, 2))
    ydf = _host(ctx.saddle_apply(x, 2))
    sl = blob_slices(wl)
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        a, b = sl[s]
        r, M, K, B = dense_state(lay, Y, q)
        ref = M @ lam[3 * a:3 * b]
        assert rel(u[3 * a:3 * b], ref) < 2e-6, (s, rel(u[3 * a:3 * b], ref))
        assert np.abs(u[3 * a:3 * b] - ref).max() < 1e-5 * np.abs(ref).max()
        assert rel(udf[3 * a:3 * b], ref) < 1e-11, (s, rel(udf[3 * a:3 * b], ref))
        o = int(ctx.saddle_off[s])
        lam_s, V_s = x[o:o + 3 * lay.n_blobs], x[o + 3 * lay.n_blobs:o + 3 * lay.n_blobs + 6 * lay.n_bodies]
        y1, y2 = rigid.saddle_apply(M, K, lam_s, V_s)
        assert rel(y[o:o + 3 * lay.n_blobs + 6 * lay.n_bodies], np.concatenate([y1, y2])) < 2e-6
        assert rel(ydf[o:o + 3 * lay.n_blobs + 6 * lay.n_bodies], np.concatenate([y1, y2])) < 1e-11


@pytest.mark.parametrize("which", ["mix120", "batch_multi_tile", "overlap_pile"])
def test_double_float_kernels(lib, which):
    """The double-float residual product by each of its kernels (ordered; symmetric compiled
    for 3 and for 4 blocks per SM) against the dense oracle; the two symmetric builds run the
    same arithmetic in the same order, so they agree bit for bit."""
    if which == "mix120":
        wl = WL.mixed_small(120, seed=4)
    elif which == "batch_multi_tile":
        wl = WL.c4(seed=6, n_susp=5, nmin=20, nmax=70)
    else:
        wl = _overlapping_workload("pile")
    rng = np.random.default_rng(23)
    lam = rng.standard_normal(3 * wl.n_blobs)
    out = {}
    for dk in (1, 3, 4):
        ctx = ctx_for(lib, wl, autotune=0, pair_kernel=2, df_kernel=dk)
        assert ctx.profile_read()["df_kernel"] == (0 if dk == 1 else dk)
        n = int(ctx.saddle_off[-1])
        x = np.random.default_rng(29).standard_normal(n)
        out[dk] = (_host(ctx.rpy_apply(lam, 2)), _host(ctx.saddle_apply(x, 2)), x)
    assert np.array_equal(out[3][0], out[4][0]) and np.array_equal(out[3][1], out[4][1])
    sl = blob_slices(wl)
    for s in range(wl.n_susp):
        lay, Y, q = susp_layout(wl, s)
        a, b = sl[s]
        r, M, K, B = dense_state(lay, Y, q)
        ref = M @ lam[3 * a:3 * b]
        for dk, (udf, ydf, x) in out.items():
            assert rel(udf[3 * a:3 * b], ref) < 1e-11, (dk, s, rel(udf[3 * a:3 * b], ref))
            o = int(ctx.saddle_off[s])
            m = 3 * lay.n_blobs + 6 * lay.n_bodies
            y1, y2 = rigid.saddle_apply(M, K, x[o:o + 3 * lay.n_blobs], x[o + 3 * lay.n_blobs:o + m])
            assert rel(ydf[o:o + m], np.concatenate([y1, y2])) < 1e-11, (dk, s)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fp32_step_parity_each_pair_kernel(lib, wl_mix, kernel):
    wl = wl_mix
    _, _, _, _, _, out = _step_case(lib, wl, 1)
    ctx2 = ctx_for(lib, wl, precision=1, seed=77, rfd_delta=1e-3, lanczos_max_iter=128, gmres_tol=1e-6,
                   lanczos_tol=1e-7, gmres_max_iter=1000, autotune=0, pair_kernel=kernel)
    ctx2.step(1)
    Y2, q2, _ = ctx2.get_state()
    for s, o, e, ora in out:
        assert np.abs(Y2[o:e] - ora["Y1"]).max() / np.abs(ora["Y1"]).max() < 1e-5
        assert rot_err(q2[o:e], ora["q1"]) < 1e-5


def test_fp32_refinement_with_residual_updates(lib, wl_mix):
    """FP32-mixed GMRES with short restarts: cycles that start from a residual below 1e-3 update
    it with the FP32 product of their correction instead of an accurate product; the final
    residual, checked with the oracle's dense FP64 operator, still meets gmres_tol."""
    wl = wl_mix
    tol = 1e-6
    ctx = ctx_for(lib, wl, precision=1, gmres_tol=tol, gmres_max_iter=800, gmres_restart=4)
    rng = np.random.default_rng(21)
    vb = rng.standard_normal(3 * wl.n_blobs)
    FT = np.zeros(6 * wl.n_bodies)
    V, lam, info = ctx.mobility_solve(FT, vb, want_lambda=True)
    assert info["converged"] and info["residual"] <= tol
    assert info["cycles"] >= 3 and info["matvecs_fp64"] < info["cycles"] + 1, info   # some updated residuals
    (r, M, K, B, lay), = _oracle_saddle(wl)
    y1, y2 = rigid.saddle_apply(M, K, _host(lam), _host(V))
    res = np.linalg.norm(np.concatenate([y1 + vb, y2])) / np.linalg.norm(vb)
    assert res <= 1.2 * tol, res


@pytest.mark.parametrize("kernel", [1, 2])
def test_rpy32_ragged_suspension_sizes(lib, kernel):
    """Both FP32 pair kernels on a batch of free-blob suspensions of 1, 2, 31, 511, 512, 513
    and 1025 blobs: single-blob and sub-warp suspensions, sizes on both sides of the 256- and
    512-blob tiles, in one launch; random clouds, so blobs of different bodies overlap."""
    sizes = [1, 2, 31, 511, 512, 513, 1025]
    rng = np.random.default_rng(23)
    Y = np.concatenate([rng.uniform(0.0, 1.8 * n ** (1.0 / 3.0) + 1.0, size=(n, 3)) for n in sizes])
    nb = sum(sizes)
    wl = WL.Workload("ragged_free_blobs", [np.zeros((1, 3))], np.zeros(nb, dtype=np.int32),
                     np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64), Y,
                     np.tile([1.0, 0.0, 0.0, 0.0], (nb, 1)), dict(WL.c1().params), np.ones(len(sizes)))
    ctx = ctx_for(lib, wl, autotune=0, pair_kernel=kernel)
    lam = rng.standard_normal(3 * nb)
    u = _host(ctx.rpy_apply(lam, 1))
    off = 0
    for n in sizes:
        ref = rpy.rpy_matrix(Y[off:off + n], 1.0, 1.0) @ lam[3 * off:3 * (off + n)]
        got = u[3 * off:3 * (off + n)]
        assert rel(got, ref) < 2e-6, (n, rel(got, ref))
        off += n


def test_largest_template_bodies(lib):
    """Bodies of the largest template the library takes (340 blobs: a 7 x 7 x 7 lattice of
    blobs 2a apart without three corners; 1,020 rows per template block): products, the
    block preconditioner, the preconditioned Lanczos root and a mobility solve in FP64
    against the dense oracle, three such bodies in one suspension."""
    g = np.arange(7) * 2.0
    cube = np.array([[x, y, z] for x in g for y in g for z in g])[3:]
    cube = cube - cube.mean(axis=0)
    assert cube.shape == (340, 3)
    rng = np.random.default_rng(31)
    Y = np.array([[0.0, 0.0, 0.0], [25.0, 1.0, -2.0], [-3.0, 25.0, 4.0]])   # > 2 x 10.4a apart: no overlap
    q = WL.random_unit_quaternions(rng, 3)
    wl = WL.Workload("cubes340", [cube], np.zeros(3, dtype=np.int32), np.array([0, 3], dtype=np.int64), Y, q,
                     dict(WL.c1().params), np.array([60.0]))
    ctx = ctx_for(lib, wl, precision=0, lanczos_tol=1e-11, lanczos_max_iter=128, gmres_tol=1e-12,
                  gmres_max_iter=800, kT=1.0, dt=0.01, lanczos_precond=1)
    lay, Yl, ql = susp_layout(wl, 0)
    r, M, K, B = dense_state(lay, Yl, ql)
    lam = rng.standard_normal(3 * wl.n_blobs)
    assert rel(_host(ctx.rpy_apply(lam, 0)), M @ lam) < 1e-12
    assert rel(_host(ctx.rpy_apply(lam, 1)), M @ lam) < 2e-6
    W = rng.standard_normal(3 * wl.n_blobs)
    vb = _host(ctx.brownian_slip(W)[0])
    ref = np.sqrt(2 * 1.0 / 0.01) * rigid.sqrtm_block(M, rigid.block_factor(lay, ql, 1.0, 1.0)) @ W
    assert rel(vb, ref) < 1e-9
    FT = rng.standard_normal(6 * wl.n_bodies)
    V, lamv, info = ctx.mobility_solve(FT, W, want_lambda=True)
    assert info["converged"]
    ls, Vs = rigid.saddle_solve(M, K, B, W, FT)
    assert rel(_host(V), Vs) < 1e-9


def _degenerate_workload():
    """Single blobs (3 DOF: no rotation moves a blob at its body's centre, L_p read as a),
    2-blob dumbbells (5 DOF) and icosahedra in one suspension."""
    from synthetic import shapes
    rng = np.random.default_rng(41)
    tmpl = [np.zeros((1, 3)), np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]), shapes.icosahedron()]
    bt = np.array([0, 0, 1, 1, 2, 0, 1, 2], dtype=np.int32)
    Y = np.array([[0, 0, 0], [4.0, 0, 0], [0, 5.0, 0], [5.0, 5.0, 1.0], [-6.0, 0, 0], [0, -4.0, 2.0], [0, 0, 6.0],
                  [7.0, -6.0, 0]])
    q = WL.random_unit_quaternions(rng, len(bt))
    return WL.Workload("degenerate", tmpl, bt, np.array([0, len(bt)], dtype=np.int64), Y, q, dict(WL.c1().params),
                       np.array([20.0]))


@pytest.mark.parametrize("prec", [0, 1])
def test_degenerate_bodies_step(lib, prec):
    """One gDC step of single blobs, dumbbells and icosahedra against the oracle: positions,
    the dumbbells' axes and the icosahedra's rotations (a single blob's orientation carries
    no information)."""
    wl = _degenerate_workload()
    ctx, tr, info, Y1, q1, out = _step_case(lib, wl, prec)
    assert info["solve"]["converged"]
    (s, o, e, ora), = out
    pos_err = np.abs(Y1 - ora["Y1"]).max() / np.abs(ora["Y1"]).max()
    disp_err = rel(Y1 - wl.Y, ora["Y1"] - wl.Y)
    ico = wl.body_tmpl == 2
    dumb = wl.body_tmpl == 1
    axis = lambda qq: np.array([G.rotation_matrix(x)[:, 0] for x in qq])
    ax_err = np.abs(axis(q1[dumb]) - axis(ora["q1"][dumb])).max()
    r_err = rot_err(q1[ico], ora["q1"][ico])
    if prec == 0:
        assert pos_err < 1e-11 and disp_err < 1e-6 and ax_err < 1e-9 and r_err < 1e-9, (pos_err, disp_err, ax_err, r_err)
    else:
        assert pos_err < 1e-5 and disp_err < 1e-3 and ax_err < 1e-5 and r_err < 1e-5, (pos_err, disp_err, ax_err, r_err)
