"""GPU: fluctuating FCM of Sec. 4.2 in a periodic cube, through the C ABI, against the oracle.

The library's grid arithmetic is FP32: spreading sums, three FFT passes of log2 N radix-2
stages each way and the averaging rows carry relative rounding errors of a few 1e-7 each,
so products agree with the FP64 oracle to about 1e-6; the tests allow 2e-5.  The stress
draws are the same Philox numbers on both sides (stream 2), so the Brownian velocities are
compared sample for sample.
"""
import numpy as np
import pytest

from oracle import fcm

from gpu_common import rel

pytestmark = pytest.mark.gpu

SIGMA = 1.0 / np.sqrt(np.pi)     # a = 1
TOL = 2e-5

# (N, L, R_t, blobs): two binning cells per side, a few, many; sigma/h from 1.8 to 1.8 at 128^3
CASES = [(16, 5.0, 2.0, 7), (32, 10.0, 3.0, 40), (64, 20.0, 3.0, 300), (128, 40.0, 3.0, 3000)]


def _host(t):
    return t.detach().cpu().numpy()


def _positions(n, L, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, L, size=(n, 3))
    r[: n // 5] += L * rng.integers(-2, 3, size=(n // 5, 3))    # outside the cube: wrapped by both sides
    return r


@pytest.mark.parametrize("N,L,R_t,n", CASES)
def test_fcm_product_matches_oracle(lib, N, L, R_t, n):
    r = _positions(n, L, N)
    lam = np.random.default_rng(N + 1).standard_normal((n, 3))
    F = lib.Fcm(N, L, SIGMA, R_t, max_blobs=n)
    u = _host(F.apply(r, lam))
    ref = fcm.mobility_apply(fcm.Grid(N, L, SIGMA, R_t), r, lam)
    assert rel(u, ref) < TOL, rel(u, ref)
    # deterministic: the gather and the fixed summation orders repeat bit for bit
    np.testing.assert_array_equal(_host(F.apply(r, lam)), u)


@pytest.mark.parametrize("N,L", [(256, 80.0), (512, 150.0)])
def test_fcm_product_matches_oracle_large_grids(lib, N, L):
    """The 256- and 512-point transforms (1,024-thread blocks in the strided passes and in the
    fused z passes with the solve; 512^3 is the benchmark's grid) against the oracle (about
    30 s of numpy FFTs on the host at 512^3)."""
    R_t, n = 3.0, 60
    rng = np.random.default_rng(N)
    r = rng.uniform(0.0, L, size=(n, 3))
    lam = rng.standard_normal((n, 3))
    F = lib.Fcm(N, L, SIGMA, R_t, max_blobs=n)
    u = _host(F.apply(r, lam))
    ref = fcm.mobility_apply(fcm.Grid(N, L, SIGMA, R_t), r, lam)
    assert rel(u, ref) < TOL, rel(u, ref)


@pytest.mark.parametrize("N,L,R_t,n", CASES[:3])
def test_fcm_brownian_matches_oracle(lib, N, L, R_t, n):
    g = fcm.Grid(N, L, SIGMA, R_t)
    r = _positions(n, L, N + 2)
    seed, owner, step, kT, dt = 2024, 3, 17, 1.3, 0.01
    F = lib.Fcm(N, L, SIGMA, R_t, max_blobs=n)
    v = _host(F.brownian(r, seed, owner, step, kT, dt))
    ref, u_ref = fcm.brownian_velocity(g, r, seed, owner, step, kT, dt)
    assert rel(v, ref) < TOL, rel(v, ref)
    # the field stays on the grid: re-averaging at moved positions (Sec. 5) needs no new solve
    r2 = r + 0.4 * np.random.default_rng(5).standard_normal(r.shape)
    v2 = _host(F.average(r2))
    assert rel(v2, fcm.average(g, r2, u_ref)) < TOL
    # a deterministic product in between leaves the fluctuating field alone
    F.apply(r, np.ones((n, 3)))
    np.testing.assert_array_equal(_host(F.average(r2)), v2)


def test_fcm_rejects_bad_input(lib):
    with pytest.raises(lib.GdcError):
        lib.Fcm(24, 10.0, SIGMA, 3.0)            # not a power of two
    with pytest.raises(lib.GdcError):
        lib.Fcm(32, 10.0, SIGMA, 5.0)            # truncation reaches the periodic image
    F = lib.Fcm(32, 10.0, SIGMA, 3.0, max_blobs=4)
    with pytest.raises(lib.GdcError):
        F.average(np.zeros((2, 3)))              # no fluctuating field yet
    with pytest.raises(lib.GdcError):
        F.apply(np.zeros((5, 3)), np.zeros((5, 3)))   # more blobs than max_blobs
    before = F.launches
    F.apply(np.ones((3, 3)), np.ones((3, 3)))
    assert F.launches > before


# ---- the gDC step with the FCM mobility (Sec. 3 with Sec. 4.2, periodic cube) ----------

def _fcm_case(lib, div, graph=0, oracle=True):
    from oracle import gdc as ogdc, philox
    from synthetic import workloads as WL
    from gpu_common import oracle_params, rot_err, susp_layout
    wl = WL.c1()                       # four icosahedra, 48 blobs, no pair forces
    L, N, seed = 20.0, 64, 77          # sigma / h = 1.80
    ctx = lib.context_from_workload(wl, precision=0, mobility=1, box_L=L, fcm_N=N, seed=seed, rfd_delta=1e-3,
                                    gmres_tol=1e-7, gmres_max_iter=1000, divmode=div, graph=graph)
    tr = ctx.set_trace(True)
    info = ctx.step(1)[0]
    Y1, q1, _ = ctx.get_state()
    lay, Y, q = susp_layout(wl, 0)
    if not oracle:
        return ctx, tr, info, Y, Y1, q1, None, rot_err
    Wt = philox.normals(seed, 0, 0, 1, 6 * lay.n_bodies)
    ora = ogdc.gdc_step_fcm(lay, Y, q, Wt, fcm.Grid(N, L, SIGMA, 3.0), oracle_params(wl, rfd_delta=1e-3), seed, 0, 0,
                            div="rfd" if div == 0 else "fd")
    return ctx, tr, info, Y, Y1, q1, ora, rot_err


@pytest.mark.parametrize("div", [0, 1])
def test_fcm_gdc_step_matches_oracle(lib, div):
    ctx, tr, info, Y, Y1, q1, ora, rot_err = _fcm_case(lib, div)
    assert info["solve"]["converged"] and info["lanczos_iters"] == [0, 0, 0]
    assert rel(_host(tr["vb_n"]), ora["vb0"]) < TOL
    assert rel(_host(tr["calV"]).reshape(-1, 6), ora["calV"]) < TOL
    assert abs(_host(tr["nu"])[0] - ora["nu"]) < 1e-3
    assert rel(_host(tr["vb_m"]), ora["vb"]) < TOL          # the same field, averaged at x^m
    assert rel(Y1 - Y, ora["Y1"] - Y) < 1e-4
    assert rot_err(q1, ora["q1"]) < 1e-6


def test_fcm_step_runs_host_driven_with_graph_requested(lib):
    a = _fcm_case(lib, 0, graph=1, oracle=False)
    b = _fcm_case(lib, 0, graph=0, oracle=False)
    np.testing.assert_array_equal(a[4], b[4])
    np.testing.assert_array_equal(a[5], b[5])


def test_fcm_slip_follows_parameter_changes(lib):
    """v-breve at a fixed step scales as sqrt(kT/dt): a parameter change between two slips of
    the same step draws the field again with the new scale."""
    import dataclasses
    from synthetic import workloads as WL
    wl = WL.c1()
    ctx = lib.context_from_workload(wl, precision=0, mobility=1, box_L=20.0, fcm_N=32, seed=3)
    W = np.zeros(3 * wl.n_blobs)      # unused with FCM: the stress is drawn on the grid
    v1 = _host(ctx.brownian_slip(W)[0])
    again = _host(ctx.brownian_slip(W)[0])       # same step: the stored field, averaged again
    np.testing.assert_array_equal(again, v1)
    ctx.set_params(dataclasses.replace(ctx.params, kT=4.0 * ctx.params.kT))
    v2 = _host(ctx.brownian_slip(W)[0])
    np.testing.assert_allclose(v2, 2.0 * v1, rtol=1e-5, atol=1e-12 * np.abs(v1).max())


def _periodic_workload(**params):
    import dataclasses
    from synthetic import workloads as WL
    wl = WL.c1()
    Y = wl.Y.copy()
    Y[0] += np.array([20.0, 0.0, 0.0])          # one cube side away: forces need the minimum image
    Y[1] += np.array([0.0, -20.0, 20.0])
    return dataclasses.replace(wl, Y=Y, params=dict(wl.params, **params))


@pytest.mark.parametrize("prec", [0, 1])
def test_fcm_mode_forces_use_minimum_images(lib, prec):
    from oracle import forces, geometry as G
    from gpu_common import susp_layout
    wl = _periodic_workload(rep_A=4.0, rep_b=0.1, potential=2, well_A=5.0, well_lambda=0.5)
    ctx = lib.context_from_workload(wl, precision=prec, mobility=1, box_L=20.0, fcm_N=32)
    got = _host(ctx.forces())
    lay, Y, q = susp_layout(wl, 0)
    r = G.blob_positions(lay, Y, q)
    pp = wl.params
    f = forces.blob_forces(r, lay.blob_body, pp["rep_A"], pp["rep_b"], 1.0, 2, 5.0, 0.5, box=20.0)
    ref = forces.body_force_torque(r, Y, lay.blob_body, f)
    unwrapped = forces.body_force_torque(r, Y, lay.blob_body, forces.blob_forces(r, lay.blob_body, pp["rep_A"],
                                                                                 pp["rep_b"], 1.0, 2, 5.0, 0.5))
    assert rel(unwrapped, ref) > 0.1                 # the images matter in this configuration
    assert rel(got, ref) < (1e-12 if prec == 0 else 1e-5), rel(got, ref)


def test_fcm_gdc_step_with_wells_matches_oracle(lib):
    from oracle import gdc as ogdc, philox
    from gpu_common import oracle_params, rot_err, susp_layout
    wl = _periodic_workload(rep_A=4.0, rep_b=0.1, potential=1, well_A=5.0, well_lambda=0.5)
    L, N, seed = 20.0, 64, 91
    ctx = lib.context_from_workload(wl, precision=0, mobility=1, box_L=L, fcm_N=N, seed=seed, rfd_delta=1e-3,
                                    gmres_tol=1e-7, gmres_max_iter=1000)
    tr = ctx.set_trace(True)
    info = ctx.step(1)[0]
    assert info["solve"]["converged"]
    Y1, q1, _ = ctx.get_state()
    lay, Y, q = susp_layout(wl, 0)
    Wt = philox.normals(seed, 0, 0, 1, 6 * lay.n_bodies)
    ora = ogdc.gdc_step_fcm(lay, Y, q, Wt, fcm.Grid(N, L, SIGMA, 3.0), oracle_params(wl, rfd_delta=1e-3), seed, 0, 0)
    assert np.abs(ora["FT"]).max() > 0.1
    assert rel(_host(tr["FTm"]), ora["FT"]) < 1e-6      # x^m carries the FP32 grid's rounding through calV
    assert rel(Y1 - Y, ora["Y1"] - Y) < 1e-4
    assert rot_err(q1, ora["q1"]) < 1e-6
