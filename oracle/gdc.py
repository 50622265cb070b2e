"""Oracle gDC time step (Sec. 3) and Euler-Maruyama step (App. D).  TEST INFRASTRUCTURE ONLY.

Everything is dense FP64 for one suspension: M is assembled, its square root
is taken densely -- by default L (L^-1 M L^-T)^(1/2) with the body-block Cholesky
factor L (the root that block-preconditioned Lanczos converges to), or the
symmetric root (eigendecomposition, the limit of unpreconditioned Lanczos), or
the Cholesky factor of M -- the saddle point is solved by LU, and step 2 is solved as
the least-squares problem it is.  The random vectors W (3M normals) and
W-tilde (6N normals) are inputs, so the same draws can be fed to any
implementation.

Readings of points the paper leaves open (each is also listed with the design notes):

* Y_p is the blob centroid (templates are centred on it).
* The Brownian slip velocity is v-breve = sqrt(2 kT / dt) M^(1/2) W with the
  same W at the start and at the mid-step (Eqs. unconst and step5).
* M^(1/2) W (Eq. v_brown_RMB) is taken, as Sec. 4.1 does, by Lanczos in the
  preconditioned form of Chow & Saad, whose limit is L (L^-1 M L^-T)^(1/2) W with
  L the body-block Cholesky factor of rigid.block_factor: a square root of M
  (S S^T = M) that moves with each body's rotation.
* RFD (Eq. rfd_div with the footnote's L_p): the perturbed state is
  Y + delta L_p W~_t, exp(delta W~_r) * q; the estimator is
  sum_p [W~_t . (V~_t - V_t) / (delta L_p) + W~_r . (V~_r - V_r) / delta],
  and nu = 1 + dt/2 * estimator is one scalar for the whole suspension.
  A single-blob body has L_p = 0; it uses L_p = a instead.
* FD (Eq. FD): the same sum over unit perturbations of each body coordinate.
* Background shear u(r) = (shear_rate * y, 0, 0) enters the slip as
  M lambda - K V = -v-breve - u(r) at the mid-step solve only.
* Forces are the soft blob repulsion of forces.py evaluated at the mid-step (and, above a
  wall, the wall repulsion and the body weights of wall.py).
* Above a wall (Params.wall) M is the wall-corrected mobility of wall.py and the
  block-preconditioned root uses the lab-frame Cholesky factor of each body's block.
* The update x^(n+1) = x^n + nu dt V^m uses Omega^m directly as du/dt,
  which is exact because u^n = 0 and D^-1 at 0 is I (App. A).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import forces, geometry, lanczos, rigid, rpy, wall


@dataclasses.dataclass
class Params:
    eta: float = 1.0
    kT: float = 1.0
    a: float = 1.0
    dt: float = 0.01
    rfd_delta: float = 1e-6
    rep_A: float = 0.0
    rep_b: float = 0.1
    potential: int = 0          # forces.py: 0 soft sphere, 1 repel-attract, 2 repel-attract-repel
    well_A: float = 0.0         # Gaussian well amplitude (Sec. 6.4: 5 kT)
    well_lambda: float = 0.5    # Gaussian well width, a length (Sec. 6.4: 0.5 a)
    shear_rate: float = 0.0
    sqrt_mode: str = "block"    # "block" (preconditioned Lanczos root), "sym" (eigh) or "chol"
    # 0: the dense root of sqrt_mode; > 0: the Lanczos iterate at that tolerance (named apart
    # from a workload's lanczos_tol, which configures the library, not the oracle)
    sqrt_lanczos_tol: float = 0.0
    sqrt_lanczos_max_iter: int = 128
    wall: bool = False          # blobs above a no-slip wall at z = 0 (wall.py)
    wall_V0: float = 0.0        # wall repulsion strength V0 (Sec. 6.2: 23 kT), 0 = off
    wall_b: float = 0.5         # its range b, a length (Sec. 6.2: 0.5 a)
    body_weight: float = 0.0    # mg of every body, along -z (Sec. 6.2: 0.18 kT/a)

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        names = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})


def _lengths(layout: geometry.Layout, a: float) -> np.ndarray:
    return np.where(layout.L > 0.0, layout.L, a)


def sqrt_apply(M: np.ndarray, W: np.ndarray, mode: str, L: np.ndarray = None) -> np.ndarray:
    """S W for the square root S of M named by mode (S S^T = M in every mode)."""
    if mode == "sym":
        S = rigid.sqrtm_sym(M)
    elif mode == "chol":
        S = rigid.sqrtm_chol(M)
    elif mode == "block":
        S = rigid.sqrtm_block(M, L)
    else:
        raise ValueError(mode)
    return S @ W


def mobility_matrix(r: np.ndarray, p: Params) -> np.ndarray:
    """The dense blob mobility M: unbounded RPY (Sec. 4.1), or wall-corrected (wall.py)."""
    return wall.wall_matrix(r, p.a, p.eta) if p.wall else rpy.rpy_matrix(r, p.a, p.eta)


def brownian_slip_k(layout, Y, q, W, p: Params, fixed_k: int = None):
    """Blob positions, M, K, B, v-breve = sqrt(2kT/dt) M^(1/2) W at state (Y, q), and the
    Lanczos iteration count (None for a dense root).

    With p.sqrt_lanczos_tol > 0 the root is the Lanczos iterate of lanczos.py at that tolerance
    (or with exactly fixed_k iterations) on the operator of sqrt_mode: A = L^-1 M L^-T with
    the result multiplied by L ("block"), or M itself ("sym")."""
    r = geometry.blob_positions(layout, Y, q)
    M = mobility_matrix(r, p)
    K = rigid.k_matrix(r, Y, layout.blob_body)
    B = rigid.rigid_basis(K, layout.n_bodies)
    L = None
    if p.sqrt_mode == "block":
        L = rigid.block_factor_lab(layout, M) if p.wall else rigid.block_factor(layout, q, p.a, p.eta)
    scale = np.sqrt(2.0 * p.kT / p.dt)
    k = None
    if p.sqrt_lanczos_tol > 0.0 and p.sqrt_mode in ("block", "sym"):
        if p.sqrt_mode == "block":
            Linv = np.linalg.inv(L)
            A = Linv @ M @ Linv.T
            y, k, _ = lanczos.lanczos_sqrt(0.5 * (A + A.T), W, p.sqrt_lanczos_tol, p.sqrt_lanczos_max_iter, fixed_k)
            vb = scale * (L @ y)
        else:
            y, k, _ = lanczos.lanczos_sqrt(M, W, p.sqrt_lanczos_tol, p.sqrt_lanczos_max_iter, fixed_k)
            vb = scale * y
    else:
        vb = scale * sqrt_apply(M, W, p.sqrt_mode, L)
    return r, M, K, B, vb, k


def brownian_slip(layout, Y, q, W, p: Params):
    """Blob positions, M, K, B and v-breve = sqrt(2kT/dt) M^(1/2) W at state (Y, q)."""
    return brownian_slip_k(layout, Y, q, W, p)[:5]


def projected_velocity(layout, Y, q, W, p: Params, fixed_k: int = None) -> np.ndarray:
    """Step 2: the least-squares rigid velocity of v-breve at state (Y, q), shape (N, 6)."""
    _, _, K, B, vb, _ = brownian_slip_k(layout, Y, q, W, p, fixed_k)
    return rigid.lsq_velocity(K, B, vb).reshape(-1, 6)


def perturbed_state(layout, Y, q, dY: np.ndarray, du: np.ndarray):
    """(Y + dY, exp(du) * q) body by body."""
    Yp = Y + dY
    qp = np.array([geometry.quat_mul(geometry.quat_exp(du[k]), q[k]) for k in range(Y.shape[0])])
    return Yp, qp


def rfd_divergence(layout, Y, q, W, Wt, calV, p: Params, project=None) -> float:
    """Step 3(b): one-sample random finite difference of div(calV) (Eq. rfd_div and its footnote).

    project(Y, q) gives calV at another state (default: step 2 with the RPY slip of W)."""
    project = project or (lambda Ys, qs: projected_velocity(layout, Ys, qs, W, p))
    d = p.rfd_delta
    L = _lengths(layout, p.a)
    Wt = Wt.reshape(-1, 6)
    Yt, qt = perturbed_state(layout, Y, q, d * L[:, None] * Wt[:, :3], d * Wt[:, 3:])
    calVt = project(Yt, qt)
    dV = calVt - calV
    return float(((Wt[:, :3] * dV[:, :3]).sum(axis=1) / (d * L)).sum()
                 + (Wt[:, 3:] * dV[:, 3:]).sum() / d)


def fd_divergence(layout, Y, q, W, calV, p: Params, project=None) -> float:
    """Step 3(a): one-sided finite differences over every body coordinate (Eq. FD)."""
    project = project or (lambda Ys, qs: projected_velocity(layout, Ys, qs, W, p))
    d = p.rfd_delta
    L = _lengths(layout, p.a)
    total = 0.0
    for k in range(layout.n_bodies):
        for c in range(6):
            dY = np.zeros((layout.n_bodies, 3))
            du = np.zeros((layout.n_bodies, 3))
            if c < 3:
                dY[k, c] = d * L[k]
            else:
                du[k, c - 3] = d
            Vp = project(*perturbed_state(layout, Y, q, dY, du))
            total += (Vp[k, c] - calV[k, c]) / (d * L[k] if c < 3 else d)
    return float(total)


def midpoint_solve(layout, Ym, qm, W, p: Params):
    """Step 5: full mobility solve at the mid-step with the same W (Eq. step5)."""
    r, M, K, B, vb, k = brownian_slip_k(layout, Ym, qm, W, p)
    f = forces.blob_forces(r, layout.blob_body, p.rep_A, p.rep_b, p.a, p.potential, p.well_A, p.well_lambda)
    if p.wall:
        f = f + wall.blob_wall_forces(r, layout.blob_body, layout.n_bodies, p.wall_V0, p.wall_b, p.a, p.body_weight)
    FT = forces.body_force_torque(r, Ym, layout.blob_body, f)
    slip = vb.copy()
    if p.shear_rate != 0.0:
        uinf = np.zeros_like(r)
        uinf[:, 0] = p.shear_rate * r[:, 1]
        slip = slip + uinf.reshape(-1)
    lam, V = rigid.saddle_solve(M, K, B, slip, FT)
    return dict(r=r, M=M, K=K, B=B, vb=vb, FT=FT, slip=slip, lam=lam, V=V.reshape(-1, 6), k_mid=k)


def gdc_step(layout, Y, q, W, Wt, p: Params, div: str = "rfd") -> dict:
    """One gDC step (Sec. 3, steps 2-6) from (Y, q) with given W (3M) and W-tilde (6N)."""
    # step 2
    r0, M0, K0, B0, vb0, k0 = brownian_slip_k(layout, Y, q, W, p)
    calV = rigid.lsq_velocity(K0, B0, vb0).reshape(-1, 6)
    # step 3: the perturbed Lanczos runs take the iteration count of the run at x^n

    def project(Ys, qs):
        return projected_velocity(layout, Ys, qs, W, p, fixed_k=k0)

    if div == "rfd":
        dv = rfd_divergence(layout, Y, q, W, Wt, calV, p, project)
    elif div == "fd":
        dv = fd_divergence(layout, Y, q, W, calV, p, project)
    else:
        raise ValueError(div)
    nu = 1.0 + 0.5 * p.dt * dv
    # step 4
    Ym, qm = geometry.advance(Y, q, calV, 0.5 * p.dt)
    # step 5
    mid = midpoint_solve(layout, Ym, qm, W, p)
    # step 6
    Y1, q1 = geometry.advance(Y, q, mid["V"], nu * p.dt)
    return dict(r0=r0, vb0=vb0, calV=calV, div=dv, nu=nu, Ym=Ym, qm=qm, Y1=Y1, q1=q1, k0=k0, **mid)


def gdc_step_fcm(layout, Y, q, Wt, grid, p: Params, seed: int, susp: int, step: int, div: str = "rfd") -> dict:
    """One gDC step with the fluctuating FCM of Sec. 4.2 in a periodic cube (oracle.fcm.Grid).

    The Brownian slip is v-breve = J L^-1 D W (already in the velocity form): the stress of
    (seed, susp, step) gives one fluctuating field u-breve per step, averaged at x^n, at the
    perturbed states of step 3 and at the mid-step x^m -- the same W throughout, and the
    re-averaging Sec. 5 describes.  The mobility solve of step 5 uses the dense M_FCM at x^m,
    with the pair forces of forces.py at x^m at minimum-image distances in the cube."""
    from . import fcm
    r0 = geometry.blob_positions(layout, Y, q)
    vb0, ufield = fcm.brownian_velocity(grid, r0, seed, susp, step, p.kT, p.dt)
    vb0 = vb0.reshape(-1)

    def project(Ys, qs):
        rs = geometry.blob_positions(layout, Ys, qs)
        Ks = rigid.k_matrix(rs, Ys, layout.blob_body)
        return rigid.lsq_velocity(Ks, rigid.rigid_basis(Ks, layout.n_bodies),
                                  fcm.average(grid, rs, ufield).reshape(-1)).reshape(-1, 6)

    calV = project(Y, q)
    if div == "rfd":
        dv = rfd_divergence(layout, Y, q, None, Wt, calV, p, project)
    elif div == "fd":
        dv = fd_divergence(layout, Y, q, None, calV, p, project)
    else:
        raise ValueError(div)
    nu = 1.0 + 0.5 * p.dt * dv
    Ym, qm = geometry.advance(Y, q, calV, 0.5 * p.dt)
    rm = geometry.blob_positions(layout, Ym, qm)
    n3 = rm.size
    M = np.zeros((n3, n3))
    for c in range(n3):
        e = np.zeros(n3)
        e[c] = 1.0
        M[:, c] = fcm.mobility_apply(grid, rm, e).reshape(-1)
    K = rigid.k_matrix(rm, Ym, layout.blob_body)
    B = rigid.rigid_basis(K, layout.n_bodies)
    vbm = fcm.average(grid, rm, ufield).reshape(-1)
    f = forces.blob_forces(rm, layout.blob_body, p.rep_A, p.rep_b, p.a, p.potential, p.well_A, p.well_lambda,
                           box=grid.L)
    FT = forces.body_force_torque(rm, Ym, layout.blob_body, f)
    lam, V = rigid.saddle_solve(M, K, B, vbm, FT)
    Y1, q1 = geometry.advance(Y, q, V.reshape(-1, 6), nu * p.dt)
    return dict(r0=r0, vb0=vb0, calV=calV, div=dv, nu=nu, Ym=Ym, qm=qm, M=M, vb=vbm, FT=FT, lam=lam,
                V=V.reshape(-1, 6), Y1=Y1, q1=q1)


def em_step(layout, Y, q, W, p: Params) -> dict:
    """Euler-Maruyama (App. D): one full solve at x^n, then x^(n+1) = x^n + dt V^n."""
    sol = midpoint_solve(layout, Y, q, W, p)
    Y1, q1 = geometry.advance(Y, q, sol["V"], p.dt)
    return dict(Y1=Y1, q1=q1, **sol)


def body_mobility_at(layout, Y, q, p: Params) -> np.ndarray:
    """Dense N(x) = (K^T M^-1 K)^-1 at state (Y, q) (Eq. body_mob)."""
    r = geometry.blob_positions(layout, Y, q)
    M = mobility_matrix(r, p)
    K = rigid.k_matrix(r, Y, layout.blob_body)
    B = rigid.rigid_basis(K, layout.n_bodies)
    return rigid.body_mobility(M, K, B)


def mobility_divergence(layout, Y, q, p: Params, h: float = 1e-5) -> np.ndarray:
    """(div N)_i = sum_j d N_ij / d x_j by central differences in x = (Y, u) with u = 0 (App. E)."""
    n = layout.n_bodies
    out = np.zeros(6 * n)
    for k in range(n):
        for c in range(6):
            dY = np.zeros((n, 3))
            du = np.zeros((n, 3))
            if c < 3:
                dY[k, c] = h
            else:
                du[k, c - 3] = h
            Np = body_mobility_at(layout, *perturbed_state(layout, Y, q, dY, du), p)
            Nm = body_mobility_at(layout, *perturbed_state(layout, Y, q, -dY, -du), p)
            out += (Np[:, 6 * k + c] - Nm[:, 6 * k + c]) / (2.0 * h)
    return out


def draw_W(seed: int, susp: int, step: int, n_blobs: int) -> np.ndarray:
    from . import philox
    return philox.normals(seed, susp, step, philox.STREAM_W, 3 * n_blobs)


def draw_Wt(seed: int, susp: int, step: int, n_bodies: int) -> np.ndarray:
    from . import philox
    return philox.normals(seed, susp, step, philox.STREAM_WTILDE, 6 * n_bodies)
