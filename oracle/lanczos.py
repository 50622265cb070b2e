"""Oracle Lanczos approximation of A^(1/2) W (Sec. 4.1).  TEST INFRASTRUCTURE ONLY.

Sec. 4.1 obtains M^(1/2) W by the Lanczos method: the Krylov space
span{W, A W, A^2 W, ...} is enlarged one vector at a time, and after k vectors
the approximation is y_k = ||W|| V_k T_k^(1/2) e_1, with V_k the orthonormal
basis and T_k the tridiagonal matrix of the recurrence.  The paper fixes the
operator's role and the tolerance but not the details, which are read here as:

* full reorthogonalisation (every new vector is orthogonalised against the
  whole basis, twice), so V_k stays orthonormal to rounding;
* T_k^(1/2) e_1 from the eigendecomposition of T_k (numpy's eigh);
* stop at the smallest k >= 2 with ||c_k - c_(k-1)|| / ||c_k|| < tol, where
  c_k = ||W|| T_k^(1/2) e_1 and c_(k-1) is padded with a zero (the change of y_k,
  since the basis is orthonormal);
* stop also when the space is exhausted (k equals the dimension) or the new
  vector vanishes numerically (beta_k <= 1e-14 max(|alpha_1|, |alpha_k|));
* fixed_k: stop at exactly k = fixed_k (or earlier if the space is exhausted),
  used for the perturbed state of the RFD step (Sec. 3 step 3), whose two
  Lanczos runs take the same number of iterations so that x -> v-breve is smooth.

With tol -> 0 the iterate tends to A^(1/2) W, which pins this module against the
dense square roots of rigid.py.
"""
from __future__ import annotations

import numpy as np


def lanczos_sqrt(A, W: np.ndarray, tol: float, kmax: int = 128, fixed_k: int = None):
    """(y, k, change): the Lanczos approximation y of A^(1/2) W for the SPD operator A, a
    matrix or a function that returns A x."""
    apply = A if callable(A) else (lambda x: A @ x)
    W = np.asarray(W, dtype=np.float64)
    n = W.size
    wn = float(np.linalg.norm(W))
    if wn == 0.0:
        return np.zeros(n), 0, 0.0
    basis = [W / wn]
    alpha, beta = [], []
    c_prev = None
    for k in range(1, kmax + 1):
        Vk = np.array(basis).T
        w = apply(basis[-1])
        h = Vk.T @ w
        w = w - Vk @ h
        h2 = Vk.T @ w
        w = w - Vk @ h2
        alpha.append(float(h[-1] + h2[-1]))
        b = float(np.linalg.norm(w))
        exhausted = k >= n or b <= 1e-14 * max(abs(alpha[0]), abs(alpha[-1]))
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        theta, Q = np.linalg.eigh(T)
        c = wn * (Q @ (np.sqrt(np.maximum(theta, 0.0)) * Q[0]))
        change = 1.0
        if c_prev is not None:
            change = float(np.linalg.norm(c - np.append(c_prev, 0.0)) / np.linalg.norm(c))
        if exhausted:
            change = 0.0
        if fixed_k is not None:
            done = k >= fixed_k or exhausted or k == kmax
        else:
            done = exhausted or (k >= 2 and change < tol) or k == kmax
        if done:
            return Vk @ c, k, change
        beta.append(b)
        basis.append(w / b)
        c_prev = c
    raise AssertionError("unreachable")
