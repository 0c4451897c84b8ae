"""Pins of the oracle's solve (Eq. covIterative1 / SAap1) and projection helpers."""
import numpy as np
import pytest

from oracle import covariance as cov
from oracle import solve
from conftest import small_cfg


@pytest.fixture(scope="module")
def system():
    cfg = small_cfg(n=6, lgs=True, obstruction=0.2)
    A = cov.system_matrix(cfg)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((A.shape[0], 3))
    return cfg, A, s


def test_cholesky_residual(system):
    _, A, s = system
    z = solve.solve_cholesky(A, s)
    assert solve.relative_residual(A, s, z).max() < 1e-12


def test_cg_matches_cholesky(system):
    _, A, s = system
    z = solve.solve_cholesky(A, s[:, 0])
    x, it = solve.cg(A, s[:, 0], tol=1e-13, maxit=20000)
    assert np.linalg.norm(x - z) / np.linalg.norm(z) < 1e-9
    assert it > 0


def test_cg_finite_termination():
    # on a well-conditioned SPD matrix CG terminates in at most N steps
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Q @ np.diag(np.linspace(1, 3, 12)) @ Q.T
    b = rng.standard_normal(12)
    x, it = solve.cg(A, b, tol=1e-12, maxit=100)
    assert it <= 12 and np.allclose(A @ x, b, atol=1e-10)


def test_rows_helpers_match_full():
    cfg = small_cfg(n=5, lgs=True, obstruction=0.2, targets=((1e-5, 0.0),))
    C = cov.css_dense(cfg)
    rows = [0, 7, len(C) - 1]
    assert np.allclose(cov.css_rows(cfg, rows), C[rows], rtol=0, atol=1e-12 * np.abs(C).max())
    F = cov.cos_interp(cfg, 0)
    r2 = [0, 5, F.shape[0] - 1]
    assert np.allclose(cov.cos_interp_rows(cfg, 0, r2), F[r2], rtol=0, atol=1e-12 * np.abs(F).max())


def test_remove_piston():
    phi = np.arange(10.0)[:, None] + np.array([[1.0, 5.0]])
    out = solve.remove_piston(phi)
    assert np.allclose(out.mean(axis=0), 0.0)
    assert np.allclose(out[:, 0], out[:, 1])


def _krylov_min_residual(A, b, k):
    """argmin ||b - A x|| over span{b, A b, ..., A^{k-1} b}, by brute force."""
    K = [b / np.linalg.norm(b)]
    for _ in range(k - 1):
        K.append(A @ K[-1])
        K[-1] /= np.linalg.norm(K[-1])
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    return Q @ y


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_minres_minimises_the_residual_over_the_krylov_space(system, k):
    # the defining property of MINRES, checked against an explicit Krylov basis
    _, A, s = system
    b = s[:, 1]
    x, it = solve.minres(A, b, tol=0.0, maxit=k)
    assert it == k
    ref = _krylov_min_residual(A, b, k)
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)


def test_minres_residual_monotone_and_below_cg(system):
    _, A, s = system
    b = s[:, 2]
    prev = np.inf
    for k in range(1, 40, 3):
        xm, _ = solve.minres(A, b, tol=0.0, maxit=k)
        xc, _ = solve.cg(A, b, tol=0.0, maxit=k)
        rm, rc = np.linalg.norm(b - A @ xm), np.linalg.norm(b - A @ xc)
        assert rm <= prev * (1 + 1e-12)
        assert rm <= rc * (1 + 1e-9)
        prev = rm


def test_minres_matches_cholesky_and_scipy(system):
    import scipy.sparse.linalg as spla
    _, A, s = system
    z = solve.solve_cholesky(A, s[:, 0])
    x, it = solve.minres(A, s[:, 0], tol=1e-12, maxit=20000)
    assert np.linalg.norm(x - z) / np.linalg.norm(z) < 1e-8
    # scipy's MINRES after the same number of steps gives the same iterate
    x12, _ = solve.minres(A, s[:, 0], tol=0.0, maxit=12)
    xs, _ = spla.minres(A, s[:, 0], rtol=1e-30, maxiter=12)
    assert np.linalg.norm(x12 - xs) <= 1e-8 * np.linalg.norm(xs)


def test_minres_singular_consistent_system():
    # semi-definite, consistent: MINRES from zero converges to the minimum-norm solution
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    A = Q @ np.diag(np.r_[np.linspace(1, 4, 8), 0.0, 0.0]) @ Q.T
    b = A @ rng.standard_normal(10)
    x, _ = solve.minres(A, b, tol=1e-13, maxit=100)
    assert np.allclose(x, np.linalg.pinv(A) @ b, atol=1e-10)


def test_reconstructor_definition(system):
    # R A = F and R s = F A^{-1} s (the direct MVM reproduces the iterative estimate)
    cfg, A, s = system
    F = cov.cos_interp(cfg, 0)
    R = solve.reconstructor(F, A)
    assert R.shape == F.shape
    assert np.abs(R @ A - F).max() <= 1e-9 * np.abs(F).max()
    z = solve.solve_cholesky(A, s)
    assert np.allclose(R @ s, F @ z, rtol=1e-9, atol=1e-9 * np.abs(F @ z).max())
