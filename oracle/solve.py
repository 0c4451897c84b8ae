"""Solving and projecting (oracle; test infrastructure only).

Eq. covIterative1 with the aperture mask (Eq. SAap1):
    W_s (Sigma_ss + Sigma_eta_eta) W_s^T zeta = s
and Eq. covIterative2 / SAap2:
    phi_hat = W_phi Sigma_phi_beta_s W_s^T zeta.
The MMSE reconstructor itself is Eq. covBasedReconstructors1.  The matrix is
symmetric positive definite once Sigma_eta_eta > 0, so zeta is unique and is
obtained here by FP64 Cholesky (the plain definition), by textbook conjugate
gradients or by MINRES (Sec. 2.G names both among the solvers used).
"""

import numpy as np
import scipy.linalg as sla


def solve_cholesky(A, s):
    """zeta = A^{-1} s via FP64 Cholesky; ``s`` may be (N,) or (N, B)."""
    c = sla.cho_factor(A, lower=True, check_finite=False)
    return sla.cho_solve(c, s, check_finite=False)


def relative_residual(A, s, zeta):
    """||s - A zeta||_2 / ||s||_2 in FP64, per column when ``s`` is (N, B)."""
    r = s - A @ zeta
    return np.linalg.norm(r, axis=0) / np.linalg.norm(s, axis=0)


def cg(A, s, tol=1e-4, maxit=10000, x0=None):
    """Textbook conjugate gradients on SPD ``A`` (FP64), zero start by default.

    Stops when the recursively updated residual satisfies ||r|| <= tol ||s||.
    Returns (x, iterations).
    """
    x = np.zeros_like(s) if x0 is None else x0.astype(np.float64).copy()
    r = s - A @ x
    p = r.copy()
    rr = r @ r
    stop = (tol * np.linalg.norm(s)) ** 2
    it = 0
    while rr > stop and it < maxit:
        Ap = A @ p
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def minres(A, s, tol=1e-4, maxit=10000, x0=None):
    """MINRES of Paige and Saunders on symmetric ``A`` (FP64), zero start by
    default (Sec. 2.G names MINRES among the solvers used).

    Lanczos builds an orthonormal basis V_k of the Krylov space with
    A V_k = V_{k+1} T_k, T_k tridiagonal (diagonal delta_j, off-diagonal
    gamma_j); x_k = x_0 + V_k y_k minimises ||gamma_1 e_1 - T_k y||, solved by
    a QR factorisation of T_k that Givens rotations update one column at a
    time; the search vectors w_j = V_k R_k^{-1} e_j update x by short
    recurrences.  |eta| after step k equals ||s - A x_k||.  Stops when it is
    <= tol ||s||.  Returns (x, iterations).
    """
    x = np.zeros_like(s) if x0 is None else x0.astype(np.float64).copy()
    r = s - A @ x
    gamma = np.linalg.norm(r)           # gamma_1
    stop = tol * np.linalg.norm(s)
    if gamma == 0.0:
        return x, 0
    v_prev = np.zeros_like(r)
    v = r / gamma
    w_prev2 = np.zeros_like(r)          # w_{j-2}
    w_prev = np.zeros_like(r)           # w_{j-1}
    c_prev2, s_prev2 = 1.0, 0.0         # rotation j-2
    c_prev, s_prev = 1.0, 0.0           # rotation j-1
    eta = gamma
    it = 0
    while abs(eta) > stop and it < maxit:
        Av = A @ v
        delta = v @ Av
        v_next = Av - delta * v - gamma * v_prev
        gamma_next = np.linalg.norm(v_next)
        # column j of T: gamma_j (row j-1), delta_j (row j), gamma_{j+1} (row j+1);
        # rotations j-2 and j-1 act on it, then rotation j zeroes gamma_{j+1}
        eps = s_prev2 * gamma
        t = c_prev2 * gamma
        rho2 = c_prev * t + s_prev * delta
        rho1_bar = -s_prev * t + c_prev * delta
        rho1 = np.hypot(rho1_bar, gamma_next)
        c, sn = rho1_bar / rho1, gamma_next / rho1
        w = (v - eps * w_prev2 - rho2 * w_prev) / rho1
        x = x + (c * eta) * w
        eta = -sn * eta
        it += 1
        if gamma_next == 0.0:
            break
        v_prev, v = v, v_next / gamma_next
        gamma = gamma_next
        w_prev2, w_prev = w_prev, w
        c_prev2, s_prev2, c_prev, s_prev = c_prev, s_prev, c, sn
    return x, it


def reconstructor(F, A):
    """Explicit reconstructor R = F A^{-1} (Eq. covBasedReconstructors1) for the
    projection F (n_vphi x N) and the SPD system matrix A, by Cholesky
    (R^T = A^{-1} F^T since A is symmetric)."""
    return solve_cholesky(A, F.T).T


def remove_piston(phi):
    """Subtract the mean over the (valid) phase points; slopes do not see piston."""
    return phi - phi.mean(axis=0, keepdims=True)
