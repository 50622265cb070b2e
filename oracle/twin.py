"""Matrix-free FP64 CPU twin of the gDC step.  TEST INFRASTRUCTURE ONLY.

The dense oracle (gdc.py) stores M and cannot go beyond a few thousand blobs (65,520 blobs
would need a 309 GB matrix).  This twin computes the same step without storing M: every
RPY product u = M lambda is evaluated pair by pair in FP64 by plain C (twin.c, one OpenMP
loop over targets), and the linear algebra follows the steps of the method directly:

* M^(1/2) W by Lanczos (Sec. 4.1; lanczos.py) on the block-preconditioned operator
  A = L^-1 M L^-T with L = diag_p(R-hat_p L_t), L_t the Cholesky factor of the template's
  RPY block (the root rigid.sqrtm_block defines), then v-breve = sqrt(2 kT/dt) L y;
* step 2 (Eq. sol_unconst) per body with the closed-form (K^T K)^(p) of Sec. 5;
* the RFD divergence (Eq. rfd_div with its footnote's L_p) with the same W and the
  iteration count of the run at x^n; nu one scalar for the suspension;
* the mid-step mobility solve (Eq. step5) by GMRES, right-preconditioned with the exact
  per-body saddle solve P of Sec. 2.2 (block diagonal), restart 50, x0 = 0, classical
  Gram-Schmidt twice, stopped when the true relative residual ||b - A x|| / ||b|| of the
  unpreconditioned system is at most gmres_tol (checked with a product at every restart);
* the soft repulsion of Sec. 6.3 at the mid-step (twin.c).

Per-body operations are vectorised over the bodies of each template.  Collinear bodies use
pseudo-inverses, as the dense oracle's reduced basis does.  It serves as the timed CPU
baseline at the benchmark's size and is cross-checked against the dense oracle's step on
suspensions small enough for both.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import time

import numpy as np

from . import geometry, lanczos, rigid, rpy

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "twin.c")
LIB = os.path.join(HERE, "_build", "libtwin.so")

_lib = None


def build() -> str:
    """Compile twin.c (gcc -O2 -fopenmp) into oracle/_build/libtwin.so."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.twin_rpy_product.argtypes = [ctypes.c_long, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.twin_rpy_product.restype = None
        lib.twin_soft_forces.argtypes = [ctypes.c_long, dp, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, dp]
        lib.twin_soft_forces.restype = None
        lib.twin_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def rpy_product(r: np.ndarray, lam: np.ndarray, a: float, eta: float) -> np.ndarray:
    """u = M lambda for blob positions r (M, 3), pair by pair in FP64 (twin.c)."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
    u = np.empty_like(lam)
    _load().twin_rpy_product(lam.size // 3, _dp(r), _dp(lam), a, eta, _dp(u))
    return u


def soft_forces(r: np.ndarray, blob_body: np.ndarray, A: float, b: float, a: float) -> np.ndarray:
    """Soft-sphere blob forces between different bodies (twin.c), shape (M, 3)."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    bb = np.ascontiguousarray(blob_body, dtype=np.int32)
    f = np.zeros_like(r)
    if A != 0.0:
        _load().twin_soft_forces(r.size // 3, _dp(r), bb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), A, b, a,
                                 _dp(f))
    return f.reshape(-1, 3)


def threads() -> int:
    return int(_load().twin_threads())


@dataclasses.dataclass
class TwinParams:
    eta: float = 1.0
    kT: float = 1.0
    a: float = 1.0
    dt: float = 0.01
    rfd_delta: float = 1e-6
    rep_A: float = 0.0
    rep_b: float = 0.1
    lanczos_tol: float = 1e-4
    lanczos_max_iter: int = 128
    gmres_tol: float = 1e-6
    gmres_restart: int = 50
    gmres_max_iter: int = 1000

    @classmethod
    def from_dict(cls, d: dict) -> "TwinParams":
        names = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})


class _Template:
    """Body-frame quantities of one template (Sec. 2.2, Sec. 5)."""

    def __init__(self, b: np.ndarray, a: float, eta: float):
        self.b = b                                   # centred blob coordinates, (n, 3)
        self.n = b.shape[0]
        Mt = rpy.rpy_matrix(b, a, eta)
        self.Lt = np.linalg.cholesky(Mt)
        self.Lt_inv = np.linalg.inv(self.Lt)
        self.Mt_inv = np.linalg.inv(Mt)
        Kt = rigid.k_matrix(b, np.zeros((1, 3)), np.zeros(self.n, dtype=np.int64))
        self.Gt = self.Mt_inv @ Kt                   # M_t^-1 K_t, (3n, 6)
        self.Nt = np.linalg.pinv(Kt.T @ self.Gt, rcond=1e-10, hermitian=True)
        self.KtK_pinv = np.linalg.pinv(rigid.ktk_closed_form(b, np.zeros((1, 3)), np.zeros(self.n, np.int64), 0),
                                       rcond=1e-10, hermitian=True)


class Suspension:
    """One suspension at a state (Y, q): positions, rotations and the per-body operators."""

    def __init__(self, layout: geometry.Layout, templates, Y: np.ndarray, q: np.ndarray, p: TwinParams):
        self.lay, self.tm, self.p = layout, templates, p
        self.Y, self.q = Y, q
        self.R = np.array([geometry.rotation_matrix(x) for x in q])          # (N, 3, 3)
        self.groups = []
        for t, tmpl in enumerate(templates):
            bodies = np.nonzero(layout.body_tmpl == t)[0]
            if bodies.size == 0:
                continue
            blobs = layout.blob_off[bodies][:, None] + np.arange(tmpl.n)[None, :]
            self.groups.append((tmpl, bodies, blobs))
        self.r = np.zeros((layout.n_blobs, 3))
        for tmpl, bodies, blobs in self.groups:
            self.r[blobs] = Y[bodies][:, None, :] + np.einsum("pij,kj->pki", self.R[bodies], tmpl.b)
        self.d = self.r - Y[layout.blob_body]                                 # r_i - Y_p
        self.products = 0

    # -- blob vectors (3 per blob) --
    def M(self, lam: np.ndarray) -> np.ndarray:
        self.products += 1
        return rpy_product(self.r, lam, self.p.a, self.p.eta)

    def _blockwise(self, x: np.ndarray, mat: str, before: str, after: str) -> np.ndarray:
        """Per body: out = [R] F [R^T] x_p for the template matrix F (rotations as named)."""
        x = x.reshape(-1, 3)
        out = np.zeros_like(x)
        for tmpl, bodies, blobs in self.groups:
            R = self.R[bodies]
            v = x[blobs]                                                         # (nb, n, 3)
            if before == "RT":
                v = np.einsum("pij,pki->pkj", R, v)
            F = getattr(tmpl, mat)
            w = (v.reshape(len(bodies), -1) @ F.T).reshape(len(bodies), tmpl.n, 3)
            if after == "R":
                w = np.einsum("pij,pkj->pki", R, w)
            out[blobs] = w
        return out.reshape(-1)

    def L(self, x):            # R-hat L_t x
        return self._blockwise(x, "Lt", "", "R")

    def L_invT(self, x):       # L^-T x = R-hat L_t^-T x
        x = x.reshape(-1, 3)
        out = np.zeros_like(x)
        for tmpl, bodies, blobs in self.groups:
            w = (x[blobs].reshape(len(bodies), -1) @ tmpl.Lt_inv).reshape(len(bodies), tmpl.n, 3)
            out[blobs] = np.einsum("pij,pkj->pki", self.R[bodies], w)
        return out.reshape(-1)

    def L_inv(self, x):        # L^-1 x = L_t^-1 R-hat^T x
        return self._blockwise(x, "Lt_inv", "RT", "")

    # -- rigid-body maps (Sec. 2.2) --
    def KT(self, lam: np.ndarray) -> np.ndarray:
        lam = lam.reshape(-1, 3)
        F = np.zeros((self.lay.n_bodies, 6))
        np.add.at(F[:, :3], self.lay.blob_body, lam)
        np.add.at(F[:, 3:], self.lay.blob_body, np.cross(self.d, lam))
        return F.reshape(-1)

    def K(self, V: np.ndarray) -> np.ndarray:
        V = V.reshape(-1, 6)[self.lay.blob_body]
        return (V[:, :3] + np.cross(V[:, 3:], self.d)).reshape(-1)

    def lsq(self, vb: np.ndarray) -> np.ndarray:
        """Step 2 (Eq. sol_unconst): (K^T K)^+ K^T v-breve per body, in the body frame."""
        g = self.KT(vb).reshape(-1, 6)
        out = np.zeros_like(g)
        for tmpl, bodies, _ in self.groups:
            R = self.R[bodies]
            gb = np.concatenate([np.einsum("pij,pi->pj", R, g[bodies, :3]), np.einsum("pij,pi->pj", R, g[bodies, 3:])],
                                axis=1)
            vb_ = gb @ tmpl.KtK_pinv.T
            out[bodies] = np.concatenate([np.einsum("pij,pj->pi", R, vb_[:, :3]), np.einsum("pij,pj->pi", R, vb_[:, 3:])],
                                         axis=1)
        return out.reshape(-1)

    # -- the saddle system of Eq. lin_sys_RMB, vectors [lambda (3 per blob); V (6 per body)] --
    def split(self, x):
        nl = 3 * self.lay.n_blobs
        return x[:nl], x[nl:]

    def saddle(self, x: np.ndarray) -> np.ndarray:
        lam, V = self.split(x)
        return np.concatenate([self.M(lam) - self.K(V), -self.KT(lam)])

    def precond(self, x: np.ndarray) -> np.ndarray:
        """The exact per-body solve of [M_pp -K_p; -K_p^T 0] (block-diagonal P of Sec. 2.2):
        a = M_pp^-1 r_lam, V = -N_p (r_V + K_p^T a), lam = a + M_pp^-1 K_p V, in the body frame."""
        rl, rV = self.split(x)
        rl = rl.reshape(-1, 3)
        rV = rV.reshape(-1, 6)
        lam = np.zeros_like(rl)
        V = np.zeros_like(rV)
        for tmpl, bodies, blobs in self.groups:
            R = self.R[bodies]
            nb = len(bodies)
            rho = np.einsum("pij,pki->pkj", R, rl[blobs]).reshape(nb, -1)
            a = rho @ tmpl.Mt_inv.T
            a3 = a.reshape(nb, tmpl.n, 3)
            g = np.concatenate([a3.sum(axis=1), np.cross(tmpl.b[None, :, :], a3).sum(axis=1)], axis=1)
            rVb = np.concatenate([np.einsum("pij,pi->pj", R, rV[bodies, :3]), np.einsum("pij,pi->pj", R, rV[bodies, 3:])],
                                 axis=1)
            Vb = -(rVb + g) @ tmpl.Nt.T
            lb = (a + Vb @ tmpl.Gt.T).reshape(nb, tmpl.n, 3)
            lam[blobs] = np.einsum("pij,pkj->pki", R, lb)
            V[bodies] = np.concatenate([np.einsum("pij,pj->pi", R, Vb[:, :3]), np.einsum("pij,pj->pi", R, Vb[:, 3:])],
                                       axis=1)
        return np.concatenate([lam.reshape(-1), V.reshape(-1)])


def gmres(S: Suspension, b: np.ndarray, tol: float, m: int, max_iter: int):
    """Right-preconditioned restarted GMRES for the saddle system, x0 = 0 (see module doc).
    Returns (x, inner iterations, restart cycles, final true relative residual)."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0, 0.0
    r = b.copy()
    total = cycles = 0
    while True:
        beta = np.linalg.norm(r)
        res = beta / bn
        if res <= tol or total >= max_iter:
            return x, total, cycles, res
        cycles += 1
        V = np.zeros((b.size, m + 1))
        H = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        j_used = 0
        for j in range(m):
            w = S.saddle(S.precond(V[:, j]))
            h = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].T @ w
            w = w - V[:, :j + 1] @ h2
            H[:j + 1, j] = h + h2
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t1 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t1
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / rr, H[j + 1, j] / rr) if rr > 0 else (1.0, 0.0)
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_used = j + 1
            wn = np.linalg.norm(w)
            if abs(g[j + 1]) / bn <= tol or total >= max_iter or wn == 0.0:
                break
            V[:, j + 1] = w / wn
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        x = x + S.precond(V[:, :j_used] @ y)
        r = b - S.saddle(x)


def brownian_slip(S: Suspension, W: np.ndarray, fixed_k: int = None):
    """v-breve = sqrt(2 kT/dt) L A^(1/2) W by Lanczos on A = L^-1 M L^-T; returns (v-breve, k)."""
    p = S.p
    y, k, _ = lanczos.lanczos_sqrt(lambda x: S.L_inv(S.M(S.L_invT(x))), W, p.lanczos_tol, p.lanczos_max_iter, fixed_k)
    return np.sqrt(2.0 * p.kT / p.dt) * S.L(y), k


def gdc_step(layout: geometry.Layout, Y: np.ndarray, q: np.ndarray, W: np.ndarray, Wt: np.ndarray, p: TwinParams,
             templates=None) -> dict:
    """One gDC step (Sec. 3 steps 2-6), matrix-free; also returns product counts and times."""
    t0 = time.perf_counter()
    tm = templates or [_Template(t, p.a, p.eta) for t in layout.templates]
    S0 = Suspension(layout, tm, Y, q, p)
    vb0, k0 = brownian_slip(S0, W)
    calV = S0.lsq(vb0).reshape(-1, 6)
    # step 3: random finite difference with the same W and the iteration count of x^n
    d = p.rfd_delta
    Lp = np.where(layout.L > 0.0, layout.L, p.a)
    Wt6 = Wt.reshape(-1, 6)
    Yt = Y + d * Lp[:, None] * Wt6[:, :3]
    qt = np.array([geometry.quat_mul(geometry.quat_exp(d * Wt6[k, 3:]), q[k]) for k in range(Y.shape[0])])
    St = Suspension(layout, tm, Yt, qt, p)
    vbt, _ = brownian_slip(St, W, fixed_k=k0)
    dV = St.lsq(vbt).reshape(-1, 6) - calV
    div = float(((Wt6[:, :3] * dV[:, :3]).sum(axis=1) / (d * Lp)).sum() + (Wt6[:, 3:] * dV[:, 3:]).sum() / d)
    nu = 1.0 + 0.5 * p.dt * div
    # step 4
    Ym, qm = geometry.advance(Y, q, calV, 0.5 * p.dt)
    # step 5
    Sm = Suspension(layout, tm, Ym, qm, p)
    f = soft_forces(Sm.r, layout.blob_body, p.rep_A, p.rep_b, p.a)
    FT = Sm.KT(f.reshape(-1))
    vbm, km = brownian_slip(Sm, W)
    b = np.concatenate([-vbm, -FT])
    x, iters, cycles, res = gmres(Sm, b, p.gmres_tol, p.gmres_restart, p.gmres_max_iter)
    V = Sm.split(x)[1].reshape(-1, 6)
    # step 6
    Y1, q1 = geometry.advance(Y, q, V, nu * p.dt)
    products = S0.products + St.products + Sm.products
    return dict(vb0=vb0, calV=calV, nu=nu, div=div, Ym=Ym, qm=qm, vb=vbm, FT=FT, V=V, lam=Sm.split(x)[0],
                Y1=Y1, q1=q1, k0=k0, k_mid=km, gmres_iters=iters, gmres_cycles=cycles, residual=res,
                products=products, seconds=time.perf_counter() - t0)
