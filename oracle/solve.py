"""Solving and projecting (oracle; test infrastructure only).

Eq. covIterative1 with the aperture mask (Eq. SAap1):
    W_s (Sigma_ss + Sigma_eta_eta) W_s^T zeta = s
and Eq. covIterative2 / SAap2:
    phi_hat = W_phi Sigma_phi_beta_s W_s^T zeta.
The MMSE reconstructor itself is Eq. covBasedReconstructors1.  The matrix is
symmetric positive definite once Sigma_eta_eta > 0, so zeta is unique and is
obtained here by FP64 Cholesky (the plain definition) or by textbook conjugate
gradients (Sec. 2.G names CG among the solvers used).
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


def remove_piston(phi):
    """Subtract the mean over the (valid) phase points; slopes do not see piston."""
    return phi - phi.mean(axis=0, keepdims=True)
