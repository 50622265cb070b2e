"""Oracle fluctuating force-coupling method (FCM) in a periodic cube.  TEST INFRASTRUCTURE ONLY.

Sec. 4.2 writes the FCM mobility as three operators, M_FCM = J L^-1 S, and the Brownian
velocities as v-breve = J L^-1 D W:

  S (Eq. spreading)   f(x) = sum_i lambda_i Delta_i(x), Gaussian envelopes
                      Delta_i(x) = (2 pi sigma^2)^(-3/2) exp(-|x - r_i|^2 / (2 sigma^2)),
                      sigma = a / sqrt(pi) for RPY-matching self-mobility;
  L^-1                the Stokes solve of Eqs. fluc_stokes1-2 (grad p - eta lap u = f, div u = 0);
  J = S* (Eq. averaging)  v_i = integral of u Delta_i;
  D W                 the divergence of the fluctuating stress, whose entries are
                      delta-correlated with <W_ab W_cd> = 2 eta kT (d_ac d_bd + d_ad d_bc).

Discretisation (Sec. 4.2, last paragraph, and Sec. 6.1): a periodic cube of side L with
N^3 points x_g = g h, h = L/N; envelopes evaluated on the grid at the minimum-image
distance and truncated beyond R_t (Sec. 6.1 uses 3a); a Fourier spectral Stokes solve,
u_hat = (I - k k^T / k^2) f_hat / (eta k^2), with the mean (k = 0) and every mode with a
Nyquist component set to zero (even N: those modes have no consistent derivative); the
averaging integral by the trapezoidal rule, v_i = h^3 sum_g u(x_g) Delta_i(x_g); the stress
as six independent N(0,1) per grid point, diagonal entries scaled by 2 sqrt(kT eta / (h^3
dt)) and off-diagonal ones by sqrt(2 kT eta / (h^3 dt)) (Sec. 6.1), its divergence
(D W)_a = d_b W_ab taken spectrally (i k_b W_hat_ab).  With the Delta t^(-1/2) in the stress,
v-breve has the covariance (2 kT / dt) M_FCM of the velocity form sqrt(2 kT/dt) M^(1/2) W.

Grid arrays are indexed [component, z, y, x], so the flat point index is x + N (y + N z).
The six stress normals of point g are normals 6g .. 6g + 5 of Philox stream 2 (oracle.philox),
in the order xx, yy, zz, xy, xz, yz.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import philox

STREAM_FCM = 2


@dataclasses.dataclass(frozen=True)
class Grid:
    N: int          # points per side (even)
    L: float        # side of the periodic cube
    sigma: float    # envelope width (a / sqrt(pi) for RPY-matching self-mobility)
    R_t: float      # envelope truncation radius (Sec. 6.1: 3a); must be below L / 2
    eta: float = 1.0

    @property
    def h(self) -> float:
        return self.L / self.N


def envelopes(g: Grid, r: np.ndarray) -> list:
    """Per particle: (flat indices, Delta_i values) of the grid points within R_t.

    Distances are minimum-image: for each axis the candidate grid indices are those within
    R_t of the particle (the whole axis when that covers it), d = x_g - r - L round((x_g - r)/L).
    """
    assert g.R_t < g.L / 2, "the truncated envelope must not meet its periodic image"
    norm = (2.0 * np.pi * g.sigma ** 2) ** -1.5
    xs = np.arange(g.N) * g.h
    m = int(np.ceil(g.R_t / g.h)) + 1
    out = []
    for ri in np.asarray(r, dtype=float).reshape(-1, 3):
        axes = []
        for d in range(3):
            if 2 * m + 2 >= g.N:
                idx = np.arange(g.N)
            else:
                idx = (int(np.floor(ri[d] / g.h)) - m + np.arange(2 * m + 2)) % g.N
            dd = xs[idx] - ri[d]
            dd -= g.L * np.round(dd / g.L)
            axes.append((idx, dd))
        (ix, dx), (iy, dy), (iz, dz) = axes
        d2 = (dx[None, None, :] ** 2 + dy[None, :, None] ** 2) + dz[:, None, None] ** 2
        flat = ix[None, None, :] + g.N * (iy[None, :, None] + g.N * iz[:, None, None])
        sel = d2 <= g.R_t ** 2
        out.append((flat[sel], norm * np.exp(-d2[sel] / (2.0 * g.sigma ** 2))))
    return out


def spread(g: Grid, r: np.ndarray, lam: np.ndarray, env=None) -> np.ndarray:
    """f = S lambda on the grid, (3, N, N, N)."""
    env = envelopes(g, r) if env is None else env
    f = np.zeros((3, g.N ** 3))
    for (idx, w), li in zip(env, np.asarray(lam, dtype=float).reshape(-1, 3)):
        f[:, idx] += li[:, None] * w[None, :]
    return f.reshape(3, g.N, g.N, g.N)


def average(g: Grid, r: np.ndarray, u: np.ndarray, env=None) -> np.ndarray:
    """v = J u: h^3 sum_g u(x_g) Delta_i(x_g), (n, 3)."""
    env = envelopes(g, r) if env is None else env
    uf = u.reshape(3, -1)
    return np.array([g.h ** 3 * (uf[:, idx] * w[None, :]).sum(axis=1) for idx, w in env])


def wavenumbers(g: Grid):
    """(kz, ky, kx) broadcastable arrays and the mask of the modes the solve keeps."""
    m = np.fft.fftfreq(g.N) * g.N                      # 0, 1, .., N/2 - 1, -N/2, .., -1
    k = 2.0 * np.pi * m / g.L
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    nyq = np.abs(m) == g.N // 2
    mz, my, mx = np.meshgrid(nyq, nyq, nyq, indexing="ij")
    keep = ~(mz | my | mx)
    keep[0, 0, 0] = False
    return kz, ky, kx, keep


def stokes_solve_hat(g: Grid, fh: np.ndarray) -> np.ndarray:
    """u_hat = (I - k k^T/k^2) f_hat / (eta k^2) on the kept modes, zero elsewhere."""
    kz, ky, kx, keep = wavenumbers(g)
    k = [kx, ky, kz]
    k2 = np.where(keep, kx * kx + ky * ky + kz * kz, 1.0)
    kf = (kx * fh[0] + ky * fh[1] + kz * fh[2]) / k2
    return np.stack([np.where(keep, (fh[a] - k[a] * kf) / (g.eta * k2), 0.0) for a in range(3)])


def stokes_solve(g: Grid, f: np.ndarray) -> np.ndarray:
    """u = L^-1 f for a real force density on the grid (3, N, N, N)."""
    fh = np.fft.fftn(f, axes=(1, 2, 3))
    return np.real(np.fft.ifftn(stokes_solve_hat(g, fh), axes=(1, 2, 3)))


def mobility_apply(g: Grid, r: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """u = M_FCM lambda = J L^-1 S lambda, (n, 3)."""
    env = envelopes(g, r)
    return average(g, r, stokes_solve(g, spread(g, r, lam, env)), env)


def stress(g: Grid, normals6: np.ndarray, kT: float, dt: float) -> np.ndarray:
    """The symmetric stress from six N(0,1) per point: (3, 3, N, N, N)."""
    n = np.asarray(normals6, dtype=float).reshape(g.N ** 3, 6)
    dv = g.h ** 3
    sd = 2.0 * np.sqrt(kT * g.eta / (dv * dt))        # diagonal
    so = np.sqrt(2.0 * kT * g.eta / (dv * dt))        # off-diagonal
    W = np.zeros((3, 3, g.N ** 3))
    for a in range(3):
        W[a, a] = sd * n[:, a]
    for c, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        W[a, b] = W[b, a] = so * n[:, 3 + c]
    return W.reshape(3, 3, g.N, g.N, g.N)


def fluctuating_field(g: Grid, W: np.ndarray) -> np.ndarray:
    """u-breve = L^-1 D W on the grid, D W taken spectrally."""
    kz, ky, kx, keep = wavenumbers(g)
    k = [kx, ky, kz]
    Wh = np.fft.fftn(W, axes=(2, 3, 4))
    DWh = np.stack([1j * sum(k[b] * Wh[a, b] for b in range(3)) for a in range(3)])
    return np.real(np.fft.ifftn(stokes_solve_hat(g, DWh), axes=(1, 2, 3)))


def brownian_velocity(g: Grid, r: np.ndarray, seed: int, susp: int, step: int, kT: float, dt: float):
    """v-breve = J L^-1 D W with the stress drawn from Philox stream 2; also returns u-breve."""
    W = stress(g, philox.normals(seed, susp, step, STREAM_FCM, 6 * g.N ** 3), kT, dt)
    u = fluctuating_field(g, W)
    return average(g, r, u), u


def lattice_mobility(L: float, sigma: float, r: np.ndarray, eta: float = 1.0, kmax_sigma: float = 6.5) -> np.ndarray:
    """The FCM mobility of Gaussian envelopes in a periodic cube as a reciprocal-lattice sum,
    M_ij = (1/(eta L^3)) sum_{k != 0} (I - k k^T/k^2) exp(-k^2 sigma^2) cos(k . (r_i - r_j)) / k^2,
    without grid, truncation or FFT (the continuous S, L^-1 and J of Sec. 4.2).  Dense 3n x 3n."""
    r = np.asarray(r, dtype=float).reshape(-1, 3)
    mmax = int(np.ceil(kmax_sigma * L / (2.0 * np.pi * sigma)))
    m = np.arange(-mmax, mmax + 1)
    K = 2.0 * np.pi / L * np.stack(np.meshgrid(m, m, m, indexing="ij"), axis=-1).reshape(-1, 3)
    K = K[np.any(K != 0, axis=1)]
    k2 = (K * K).sum(axis=1)
    wgt = np.exp(-k2 * sigma ** 2) / k2
    keep = wgt > 1e-18 * wgt.max()
    K, k2, wgt = K[keep], k2[keep], wgt[keep]
    P = np.eye(3)[None] - K[:, :, None] * K[:, None, :] / k2[:, None, None]
    n = r.shape[0]
    M = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for j in range(i, n):
            c = np.cos(K @ (r[i] - r[j])) * wgt
            blk = np.einsum("k,kab->ab", c, P) / (eta * L ** 3)
            M[3 * i:3 * i + 3, 3 * j:3 * j + 3] = blk
            M[3 * j:3 * j + 3, 3 * i:3 * i + 3] = blk.T
    return M
