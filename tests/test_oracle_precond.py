"""Pins of the FP64 block-circulant preconditioner reference (oracle/precond.py)."""
import numpy as np

from conftest import small_cfg
from oracle import covariance as cov
from oracle import precond


def test_periodised_generator_agrees_with_dense_covariance():
    # on lags |di|, |dj| <= n-1 the periodised generator is the 2RBT generator:
    # it must equal entries of the dense Sigma_ss
    from oracle import geometry as geo
    cfg = small_cfg(n=5, lgs=True, obstruction=0.0)
    P = 12
    t = precond.periodised_generators(cfg, P)
    C = cov.css_dense(cfg)
    v = geo.valid_list(geo.subaperture_mask(5, 0.0))
    nv = len(v)
    # slope (p, a) vs (q, b): lag = a - b in (row, col)
    for p, q in [(0, 0), (1, 2), (5, 3)]:
        for a, b in [(0, 0), (7, 3), (nv - 1, 0), (12, 18)]:
            di, dj = v[a, 0] - v[b, 0], v[a, 1] - v[b, 1]
            assert abs(C[p * nv + a, q * nv + b] - t[p, q, di + P // 2, dj + P // 2]) <= 1e-12 * abs(C).max()


def test_preconditioner_is_symmetric_positive_definite():
    cfg = small_cfg(n=6, lgs=True, obstruction=0.2)
    P = 12
    M = precond.spectra(cfg, P)
    N = cov.system_matrix(cfg).shape[0]
    E = precond.apply(cfg, np.eye(N), P, M=M)          # rows: M^{-1} e_i
    assert np.abs(E - E.T).max() <= 1e-10 * np.abs(E).max()
    assert np.linalg.eigvalsh(0.5 * (E + E.T)).min() > 0


def test_preconditioner_approximates_the_inverse():
    # on a pupil without obstruction the circulant approximation clusters the spectrum
    cfg = small_cfg(n=8, lgs=True, obstruction=0.0, noise=0.3)
    A = cov.system_matrix(cfg)
    N = A.shape[0]
    E = precond.apply(cfg, np.eye(N), 16)
    w = np.sort(np.real(np.linalg.eigvals(E @ A)))
    wa = np.linalg.eigvalsh(A)
    assert w[-1] / w[0] < 0.5 * wa[-1] / wa[0]
