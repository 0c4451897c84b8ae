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
