"""Pins of the oracle's gDC step: exact identities, limits and the moments of App. E."""
import numpy as np
import pytest

from oracle import forces, geometry as G, rigid, rpy
from oracle.gdc import (Params, body_mobility_at, brownian_slip, em_step, fd_divergence, gdc_step,
                        mobility_divergence, perturbed_state, projected_velocity, rfd_divergence)
from synthetic import shapes


def _state(templates, body_tmpl, Y, seed=0):
    rng = np.random.default_rng(seed)
    lay = G.Layout(templates, body_tmpl)
    g = rng.standard_normal((lay.n_bodies, 4))
    return lay, np.asarray(Y, dtype=float), g / np.linalg.norm(g, axis=1, keepdims=True)


def _energy(r, blob_body, A, b, a):
    """Soft-sphere energy of Eq. (soft_sphere_potential) with U0 = A b (so that -dU/dr = A e^{-(r-2a)/b})."""
    e = 0.0
    for i in range(r.shape[0]):
        for j in range(i + 1, r.shape[0]):
            if blob_body[i] == blob_body[j]:
                continue
            d = np.linalg.norm(r[i] - r[j])
            e += A * b * np.exp(-(d - 2 * a) / b) if d >= 2 * a else A * b * (1 + (2 * a - d) / b)
    return e


def test_repulsion_is_minus_energy_gradient():
    lay, Y, q = _state([shapes.triangle(), shapes.rod(3)], [0, 1], [[0, 0, 0], [2.5, 1.0, 0.5]], seed=1)
    p = dict(A=4.0, b=0.1, a=1.0)
    r = G.blob_positions(lay, Y, q)
    f = forces.blob_forces(r, lay.blob_body, **p)
    h = 1e-6
    for i in range(r.shape[0]):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, c] += h
            rm[i, c] -= h
            g = (_energy(rp, lay.blob_body, **p) - _energy(rm, lay.blob_body, **p)) / (2 * h)
            assert abs(f[i, c] + g) < 1e-6 * (1 + abs(g))
    # body torque is minus the derivative of the energy under a rigid rotation exp(h e) * q
    FT = forces.body_force_torque(r, Y, lay.blob_body, f).reshape(-1, 6)
    for k in range(3):
        du = np.zeros((2, 3))
        du[0, k] = h
        ep = _energy(G.blob_positions(lay, *perturbed_state(lay, Y, q, np.zeros((2, 3)), du)), lay.blob_body, **p)
        em = _energy(G.blob_positions(lay, *perturbed_state(lay, Y, q, np.zeros((2, 3)), -du)), lay.blob_body, **p)
        assert abs(FT[0, 3 + k] + (ep - em) / (2 * h)) < 1e-6 * (1 + abs(FT[0, 3 + k]))
    np.testing.assert_allclose(FT[:, :3].sum(0), 0, atol=1e-12)  # Newton's third law


def test_covariance_identity_exact():
    # App. E: <calV_j V_i> = (2 kT / dt) N_ij, computed exactly from the linear maps W -> calV, W -> V.
    lay, Y, q = _state([shapes.boomerang(), shapes.rod(4), shapes.triangle()], [0, 1, 2],
                       [[0, 0, 0], [7, 1, 0], [2, 6, 1]], seed=2)
    p = Params(dt=0.01, kT=1.3)
    r, M, K, B, _ = brownian_slip(lay, Y, q, np.zeros(3 * lay.n_blobs), p)
    S = np.sqrt(2 * p.kT / p.dt) * rigid.sqrtm_sym(M)
    A_cal = np.column_stack([rigid.lsq_velocity(K, B, S[:, k]) for k in range(S.shape[1])])
    zero_F = np.zeros(6 * lay.n_bodies)
    A_V = np.column_stack([rigid.saddle_solve(M, K, B, S[:, k], zero_F)[1] for k in range(S.shape[1])])
    N = rigid.body_mobility(M, K, B)
    np.testing.assert_allclose(A_V @ A_cal.T, 2 * p.kT / p.dt * N, rtol=1e-8, atol=1e-10)
    # fluctuation-dissipation of the full solve: <V V^T> = (2 kT/dt) N
    np.testing.assert_allclose(A_V @ A_V.T, 2 * p.kT / p.dt * N, rtol=1e-8, atol=1e-10)
    # the Cholesky root gives the same covariance
    Sc = np.sqrt(2 * p.kT / p.dt) * rigid.sqrtm_chol(M)
    A_Vc = np.column_stack([rigid.saddle_solve(M, K, B, Sc[:, k], zero_F)[1] for k in range(Sc.shape[1])])
    np.testing.assert_allclose(A_Vc @ A_Vc.T, 2 * p.kT / p.dt * N, rtol=1e-8, atol=1e-10)


def test_deterministic_limit_is_forward_euler():
    # kT = 0: v-breve = 0, calV = 0, nu = 1, x^m = x^n, so gDC is x + dt N F.
    lay, Y, q = _state([shapes.icosahedron(), shapes.rod(5)], [0, 1], [[0, 0, 0], [4.6, 0.5, 0.0]], seed=3)
    p = Params(kT=0.0, dt=0.05, rep_A=4.0, rep_b=0.5)
    W = np.random.default_rng(0).standard_normal(3 * lay.n_blobs)
    Wt = np.random.default_rng(1).standard_normal(6 * lay.n_bodies)
    out = gdc_step(lay, Y, q, W, Wt, p)
    assert out["nu"] == 1.0
    np.testing.assert_array_equal(out["Ym"], Y)
    r = G.blob_positions(lay, Y, q)
    f = forces.blob_forces(r, lay.blob_body, p.rep_A, p.rep_b, p.a)
    FT = forces.body_force_torque(r, Y, lay.blob_body, f)
    V = (body_mobility_at(lay, Y, q, p) @ FT).reshape(-1, 6)
    assert np.abs(V).max() > 1e-3
    Y1, q1 = G.advance(Y, q, V, p.dt)
    np.testing.assert_allclose(out["Y1"], Y1, atol=1e-13)
    np.testing.assert_allclose(out["q1"], q1, atol=1e-13)


def test_rfd_is_unbiased_for_fd():
    # Eq. (rfd_div): averaging the RFD estimator over W-tilde gives the FD divergence of Eq. (FD).
    # The identity holds for any smooth map x -> calV(x); the symmetric root of M gives this
    # W a divergence large enough for 400 draws to resolve it.
    lay, Y, q = _state([shapes.triangle(), shapes.triangle()], [0, 0], [[0, 0, 0], [3.2, 0.8, 0.4]], seed=4)
    p = Params(dt=0.01, rfd_delta=1e-5, sqrt_mode="sym")
    W = np.random.default_rng(5).standard_normal(3 * lay.n_blobs)
    calV = projected_velocity(lay, Y, q, W, p)
    fd = fd_divergence(lay, Y, q, W, calV, p)
    rng = np.random.default_rng(6)
    est = np.array([rfd_divergence(lay, Y, q, W, rng.standard_normal(6 * lay.n_bodies), calV, p)
                    for _ in range(400)])
    se = est.std() / np.sqrt(est.size)
    assert abs(fd) > 5 * se  # the test has power
    assert abs(est.mean() - fd) < 4 * se


def test_one_step_invariants():
    lay, Y, q = _state([shapes.icosahedron()], [0, 0], [[0, 0, 0], [5.0, 0, 0]], seed=7)
    p = Params(dt=0.01)
    rng = np.random.default_rng(8)
    out = gdc_step(lay, Y, q, rng.standard_normal(3 * lay.n_blobs), rng.standard_normal(12), p)
    assert np.abs(np.linalg.norm(out["q1"], axis=1) - 1).max() < 1e-14
    a1, a2 = rigid.saddle_apply(out["M"], out["K"], out["lam"], out["V"].reshape(-1))
    np.testing.assert_allclose(a1, -out["slip"], atol=1e-10)
    np.testing.assert_allclose(a2, -out["FT"], atol=1e-10)
    # translation invariance of the whole step
    out2 = gdc_step(lay, Y + 100.0, q, rng.standard_normal(3 * lay.n_blobs), rng.standard_normal(12), p)
    assert np.isfinite(out2["Y1"]).all()


@pytest.mark.slow
def test_first_and_second_moments_and_em_control():
    # App. E: <dx> = kT dt div N and <dx dx^T> = 2 kT dt N to first order; Euler-Maruyama has no drift.
    # A 3-blob rod and a triangle close together (strong hydrodynamic coupling, so the drift is
    # resolvable); antithetic pairs (W, Wt), (-W, -Wt) cancel the odd terms of the increment.
    lay, Y, q = _state([shapes.rod(3), shapes.triangle()], [0, 1], [[0, 0, 0], [1.8, 0.3, 0.4]], seed=9)
    p = Params(dt=2e-3, kT=1.0, rfd_delta=1e-6)
    divN = mobility_divergence(lay, Y, q, p)
    N = body_mobility_at(lay, Y, q, p)
    rng = np.random.default_rng(10)
    n_pairs = 3000
    nd = 6 * lay.n_bodies
    mean_g, mean_e, second = [], [], np.zeros((nd, nd))
    for _ in range(n_pairs):
        W = rng.standard_normal(3 * lay.n_blobs)
        Wt = rng.standard_normal(nd)
        acc_g, acc_e = np.zeros(nd), np.zeros(nd)
        for s in (1.0, -1.0):
            o = gdc_step(lay, Y, q, s * W, s * Wt, p)
            dx = np.concatenate([o["Y1"] - Y, _log_rel(o["q1"], q)], axis=1).reshape(-1)
            acc_g += 0.5 * dx
            second += np.outer(dx, dx)
            e = em_step(lay, Y, q, s * W, p)
            acc_e += 0.5 * np.concatenate([e["Y1"] - Y, _log_rel(e["q1"], q)], axis=1).reshape(-1)
        mean_g.append(acc_g)
        mean_e.append(acc_e)
    mean_g = np.array(mean_g)
    mg = mean_g.mean(0)
    se = mean_g.std(0) / np.sqrt(n_pairs)
    target = p.kT * p.dt * divN
    # per component: the gDC mean matches kT dt div N
    z = (mg - target) / se
    assert np.abs(z).max() < 4.5, z
    # along the drift direction the signal is resolvable, gDC recovers it and EM does not
    g = target / np.linalg.norm(target)
    proj = mean_g @ g
    se_p = proj.std() / np.sqrt(n_pairs)
    assert np.linalg.norm(target) > 5 * se_p, "the drift must be resolvable for the test to have power"
    assert abs(proj.mean() - np.linalg.norm(target)) < 4 * se_p
    proj_em = np.array(mean_e) @ g
    assert abs(proj_em.mean() - np.linalg.norm(target)) > 4 * se_p
    cov = second / (2 * n_pairs)
    ref = 2 * p.kT * p.dt * N
    np.testing.assert_allclose(cov, ref, atol=0.12 * np.abs(np.diag(ref)).max())


def _log_rel(q1, q0):
    """Rotation vector u with q1 = exp(u) * q0 (body by body)."""
    out = []
    for a, b in zip(q1, q0):
        d = G.quat_mul(a, b * np.array([1, -1, -1, -1]))
        if d[0] < 0:
            d = -d
        s = np.linalg.norm(d[1:])
        ang = 2 * np.arctan2(s, d[0])
        out.append(d[1:] * (ang / s if s > 0 else 2.0))
    return np.array(out)
