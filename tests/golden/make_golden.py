"""Writes tests/golden/<name>.npz: oracle results on seeded inputs.

Calls only ``oracle/`` (for every expected value) and the seeded input
generator ``paper_1806_07938_gb300.workloads``.  Run from the repo root:

    python tests/golden/make_golden.py [ngs8m] [lgs_mid]

Stored per system: the plain-number config, noise sigmas, 2 seeded random
vectors x and y = A x (A of Eq. SAap1), Sigma_phi_s x (LGS: the new-grid
interpolated form), 4 seeded slope frames s, zeta = A^{-1} s by FP64
Cholesky, and phi_hat = Sigma_phi_s zeta (exact and new-grid forms).
"""
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import covariance as cov  # noqa: E402
from oracle import geometry as geo  # noqa: E402
from oracle import solve  # noqa: E402
from paper_1806_07938_gb300 import workloads as W  # noqa: E402


def _rows(args):
    cfg, rows = args
    return cov.css_rows(cfg, rows)


def make(name, workers=8):
    cfg = W.config(name)
    full, sigma = W.slope_frames(cfg, 4, seed=1)
    cfg["noise_sigma"] = [float(s) for s in sigma]
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    s = full[..., mask].reshape(4, -1)
    N = s.shape[1]
    blocks = [np.arange(a, min(N, a + 128)) for a in range(0, N, 128)]
    with ProcessPoolExecutor(workers) as ex:
        C = np.concatenate(list(ex.map(_rows, [(cfg, b) for b in blocks])))
    A = C.copy()
    A[np.diag_indices_from(A)] += cov.noise_variance(cfg)
    rng = np.random.default_rng(20240601)
    x = rng.standard_normal((2, N))
    y = x @ A.T
    zeta = solve.solve_cholesky(A, s.T).T
    Fi = cov.cos_interp(cfg, 0)
    Fe = cov.cos_exact(cfg, 0)
    out = dict(config=json.dumps(cfg), noise_sigma=np.array(sigma), x=x, y=y, ycos=x @ Fi.T, s=s, zeta=zeta,
               phi_interp=zeta @ Fi.T, phi_exact=zeta @ Fe.T,
               relres=solve.relative_residual(A, s.T, zeta.T))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.npz")
    np.savez_compressed(path, **out)
    print(path, "N =", N, "max relres", out["relres"].max())


if __name__ == "__main__":
    for nm in (sys.argv[1:] or ["ngs8m", "lgs_mid"]):
        make(nm)
