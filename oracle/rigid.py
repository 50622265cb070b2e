"""Oracle rigid-body algebra: K, K^T K, the saddle point, N and step-2 least squares.

TEST INFRASTRUCTURE ONLY.  Dense FP64 restatements of Sec. 2.2 (Eqs. rigid_body_cond to v_brown_RMB),
Sec. 3 step 2 (Eqs. unconst, sol_unconst) and Sec. 5 (the closed form of (K^T K)^(p)).

Rank-deficient bodies.  A body whose blobs are collinear (a rod) cannot be
spun about its own axis by any blob velocity: K_p has a null vector, so
K_p^T K_p, K^T M^-1 K and the saddle matrix are singular.  The paper's
bodies never meet this.  Reading used here: such a body has only the rigid
motions that move some blob; the axial spin is defined to be zero.  Every
solve below is therefore done in the reduced basis B_p (the eigenvectors of
K_p^T K_p with non-zero eigenvalue), and results are mapped back with
V_p = B_p V_red, which equals applying the Moore-Penrose pseudo-inverse.
"""
from __future__ import annotations

import numpy as np

from . import rpy
from .geometry import cross_matrix, rotation_matrix


def k_matrix(r: np.ndarray, Y: np.ndarray, blob_body: np.ndarray) -> np.ndarray:
    """K (3M x 6N): block (i, p) = [I_3, [x (r_i - Y_p)]] if blob i is in body p, else 0 (the K block of Sec. 2.2).

    [x v] = -[v x], so [x (r_i - Y_p)] Omega = Omega x (r_i - Y_p) (Eq. rigid_body_cond).
    """
    m = r.shape[0]
    n = Y.shape[0]
    K = np.zeros((3 * m, 6 * n))
    for i in range(m):
        p = int(blob_body[i])
        K[3 * i:3 * i + 3, 6 * p:6 * p + 3] = np.eye(3)
        K[3 * i:3 * i + 3, 6 * p + 3:6 * p + 6] = -cross_matrix(r[i] - Y[p])
    return K


def ktk_closed_form(r: np.ndarray, Y: np.ndarray, blob_body: np.ndarray, p: int) -> np.ndarray:
    """(K^T K)^(p) as printed in Sec. 5: [[N_b I, sum [x d]], [sum [d x], -sum [d x]^2]], d = r_i - Y_p."""
    idx = np.nonzero(blob_body == p)[0]
    out = np.zeros((6, 6))
    out[:3, :3] = len(idx) * np.eye(3)
    for i in idx:
        c = cross_matrix(r[i] - Y[p])
        out[:3, 3:] += -c
        out[3:, :3] += c
        out[3:, 3:] += -(c @ c)
    return out


def rigid_basis(K: np.ndarray, n_bodies: int, rel_tol: float = 1e-10) -> np.ndarray:
    """Block-diagonal basis B (6N x n_red) of the rigid motions that move some blob.

    For each body, the eigenvectors of K_p^T K_p whose eigenvalue exceeds
    rel_tol times the largest one.  B = I for every body that is not collinear.
    """
    cols = []
    for p in range(n_bodies):
        Kp = K[:, 6 * p:6 * p + 6]
        g = Kp.T @ Kp
        w, v = np.linalg.eigh(g)
        keep = w > rel_tol * w.max()
        if keep.all():
            v = np.eye(6)
        else:
            v = v[:, keep]
        blk = np.zeros((6 * n_bodies, v.shape[1]))
        blk[6 * p:6 * p + 6] = v
        cols.append(blk)
    return np.hstack(cols)


def saddle_solve(M: np.ndarray, K: np.ndarray, B: np.ndarray, slip: np.ndarray, F: np.ndarray):
    """Solve [[M, -K], [-K^T, 0]] [lambda; V] = [-slip; -F] by dense LU (Eqs. saddle_point_sys, lin_sys_RMB).

    slip is the blob velocity on the right-hand side (the Brownian velocity
    v-breve, plus the background flow where there is one); F stacks [F_p; T_p]
    per body.  Returns (lambda, V) with V in the full 6N coordinates.
    """
    m3 = M.shape[0]
    KB = K @ B
    nr = KB.shape[1]
    A = np.zeros((m3 + nr, m3 + nr))
    A[:m3, :m3] = M
    A[:m3, m3:] = -KB
    A[m3:, :m3] = -KB.T
    rhs = np.concatenate([-slip, -(B.T @ F)])
    sol = np.linalg.solve(A, rhs)
    return sol[:m3], B @ sol[m3:]


def saddle_apply(M: np.ndarray, K: np.ndarray, lam: np.ndarray, V: np.ndarray):
    """The saddle operator applied to [lambda; V]: [M lambda - K V; -K^T lambda]."""
    return M @ lam - K @ V, -(K.T @ lam)


def body_mobility(M: np.ndarray, K: np.ndarray, B: np.ndarray) -> np.ndarray:
    """N = (K^T M^-1 K)^-1 (Eq. body_mob), in the reduced basis: N = B (B^T K^T M^-1 K B)^-1 B^T."""
    KB = K @ B
    G = KB.T @ np.linalg.solve(M, KB)
    return B @ np.linalg.inv(G) @ B.T


def lsq_velocity(K: np.ndarray, B: np.ndarray, vb: np.ndarray) -> np.ndarray:
    """Step 2 (Eq. sol_unconst): V = (K^T K)^-1 K^T v-breve, i.e. argmin ||K V - v-breve||."""
    KB = K @ B
    return B @ np.linalg.solve(KB.T @ KB, KB.T @ vb)


def sqrtm_sym(M: np.ndarray) -> np.ndarray:
    """Principal (symmetric) square root Q diag(sqrt(mu)) Q^T of the SPD matrix M."""
    w, Q = np.linalg.eigh(M)
    if w.min() <= 0.0:
        raise np.linalg.LinAlgError("M is not positive definite")
    return (Q * np.sqrt(w)) @ Q.T


def sqrtm_chol(M: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor L with L L^T = M (another valid M^(1/2), Eq. v_brown_RMB)."""
    return np.linalg.cholesky(M)


def block_factor(layout, q: np.ndarray, a: float, eta: float) -> np.ndarray:
    """The block-diagonal factor L = diag_p(R-hat_p L_t(p)) of the body blocks of M.

    L_t is the lower Cholesky factor of the template's RPY block in the body frame
    (L_t L_t^T = M_t, Sec. 4.1 blob mobility at the template's own blob positions) and
    R-hat_p = diag(R(q_p), ..., R(q_p)) rotates each blob of body p (Eq.
    quaternion_rotation_matrix).  Because RPY is rotation covariant and intra-body
    distances are fixed, L_p L_p^T = R-hat_p M_t R-hat_p^T is body p's diagonal block of M:
    L L^T is the block-diagonal preconditioner matrix of Sec. 2.2 (without the K rows).
    """
    n3 = 3 * layout.n_blobs
    L = np.zeros((n3, n3))
    chol = {}
    for p in range(layout.n_bodies):
        t = int(layout.body_tmpl[p])
        if t not in chol:
            chol[t] = np.linalg.cholesky(rpy.rpy_matrix(layout.templates[t], a, eta))
        nb = layout.templates[t].shape[0]
        Rhat = np.kron(np.eye(nb), rotation_matrix(q[p]))
        i0, i1 = 3 * layout.blob_off[p], 3 * layout.blob_off[p + 1]
        L[i0:i1, i0:i1] = Rhat @ chol[t]
    return L


def block_factor_lab(layout, M: np.ndarray) -> np.ndarray:
    """diag_p(chol(M_pp)): the lower Cholesky factor of each body's diagonal block of M, in the
    lab frame.  Used when M_pp is not a rotated template block (above a wall, where the
    mobility of a body depends on its height and orientation)."""
    L = np.zeros_like(M)
    for p in range(layout.n_bodies):
        i0, i1 = 3 * layout.blob_off[p], 3 * layout.blob_off[p + 1]
        L[i0:i1, i0:i1] = np.linalg.cholesky(M[i0:i1, i0:i1])
    return L


def sqrtm_block(M: np.ndarray, L: np.ndarray) -> np.ndarray:
    """S = L (L^-1 M L^-T)^(1/2): the square root that preconditioned Lanczos converges to.

    Sec. 4.1 takes M^(1/2) W by the Lanczos method of Chow & Saad, who precondition the
    Krylov space with a factor L of an approximation L L^T of M: Lanczos then builds the
    Krylov space of A = L^-1 M L^-T from W and returns L A^(1/2) W.  S S^T = L A L^T = M,
    so v-breve has the covariance of Eq. v_brown_RMB whatever L is.  Here L is
    block_factor's body-block factor.
    """
    Linv = np.linalg.inv(L)
    A = Linv @ M @ Linv.T
    A = 0.5 * (A + A.T)
    return L @ sqrtm_sym(A)
