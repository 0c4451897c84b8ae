"""Elongated laser spots (Sec. 2.F): Sigma_eta_eta with one 2 x 2 block per
subaperture coupling its x- and y-slope noise, against the oracle's dense
matrices.  Every block of the side-launch model is sigma^2 (I + e^2 v v^T),
whose smaller eigenvalue is sigma^2, so A >= sigma^2 I still bounds the error
of a solve by its residual over sigma^2."""
import numpy as np
import pytest

from conftest import small_cfg
from oracle import covariance as cov
from oracle import solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA = 0.15


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    tomo.lib()
    return tomo


def elongated(n=8, k=3.0, **kw):
    from paper_1806_07938_gb300 import workloads as W
    cfg = small_cfg(n=n, lgs=True, obstruction=0.2, D=0.6 * n, noise=SIGMA, **kw)
    cfg["noise_cov"] = W.elongated_noise(cfg, SIGMA, k)
    return cfg


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def relL2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def css(T, h, x, f64=False):
    dt = torch.float64 if f64 else torch.float32
    xd = dev(x, dt)
    yd = torch.empty_like(xd)
    (T.tomo_apply_css_f64 if f64 else T.tomo_apply_css)(h, xd, yd, x.shape[0])
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


def solve_gpu(T, h, s, **opts):
    info_l, _, _ = T.tomo_layout(h)
    sd = dev(s)
    zd = torch.zeros_like(sd)
    phi = torch.empty((s.shape[0], info_l.n_targets, info_l.n_vphi), dtype=torch.float32, device="cuda")
    info = T.tomo_solve(h, sd, s.shape[0], T.solve_opts(**opts), zd, phi)
    torch.cuda.synchronize()
    return zd.double().cpu().numpy(), phi.double().cpu().numpy(), info


@pytest.mark.parametrize("n", [7, 12])
def test_elongated_products(T, n):
    cfg = elongated(n)
    Css = cov.css_dense(cfg)
    S = cov.noise_matrix(cfg)
    A = Css + S
    x = np.random.default_rng(n).standard_normal((3, A.shape[0]))
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        y = css(T, h, x)                                 # chunked: batch 3 > max_batch 2
        assert relL2(y, x @ A.T) <= 1e-5
        y64 = css(T, h, x, f64=True)
        assert relL2(y64, x @ A.T) <= 1e-11
        # the noise term alone: |Sigma_eta_eta x| is ~1e-3 of |A x| here, so the
        # FP64 product resolves it to ~1e-8; white noise would be 0.4 off
        assert relL2(y64 - x @ Css.T, x @ S.T) <= 1e-7
        assert relL2(x @ np.diag(np.diag(S)), x @ S.T) > 0.1
    finally:
        T.tomo_destroy(h)


@pytest.mark.parametrize("method,pcg", [("cg", False), ("cg", True), ("minres", False), ("block", True)])
def test_elongated_solves(T, method, pcg):
    cfg = elongated(8, targets=((0.0, 0.0), (12e-6, 0.0)))
    A = cov.system_matrix(cfg)
    s = np.random.default_rng(3).standard_normal((4, A.shape[0]))
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=4, precond=pcg)
    try:
        z, phi, info = solve_gpu(T, h, s, tol=3e-5, max_iter=20000, max_refine=5, precond=pcg, method=method)
        print("elongated", method, pcg, info)
        assert (info["status"] == 0).all() and (info["relres"] <= 3e-5).all()
        zs = solve.solve_cholesky(A, s.T).T
        bound = info["relres"] * np.linalg.norm(s, axis=1) / SIGMA ** 2
        assert (np.linalg.norm(z - zs, axis=1) <= bound).all()
        for t in range(2):
            assert relL2(phi[:, t], zs @ cov.cos_interp(cfg, t).T) <= 2e-3
        # the noise model changes the estimate
        zd = solve.solve_cholesky(cov.system_matrix(dict(cfg, noise_cov=None)), s.T).T
        assert relL2(zd, zs) > 0.05
    finally:
        T.tomo_destroy(h)


def test_elongated_per_frame_r0_and_noise_scale(T):
    cfg = elongated(7)
    r0 = np.array([0.10, 0.15, 0.2])
    nu = np.array([0.5, 1.0, 3.0])
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=3)
    try:
        info_l, _, _ = T.tomo_layout(h)
        s = np.random.default_rng(8).standard_normal((3, info_l.N))
        sd = dev(s)
        zd = torch.zeros_like(sd)
        info = T.tomo_solve_r0(h, sd, 3, r0, T.solve_opts(tol=3e-5, max_iter=20000, max_refine=5), zd,
                               noise_scale=nu)
        torch.cuda.synchronize()
        z = zd.double().cpu().numpy()
        assert (info["status"] == 0).all() and (info["relres"] <= 3e-5).all()
        for f in range(3):
            zs = solve.solve_cholesky(cov.system_matrix_r0(cfg, r0[f], nu[f]), s[f])
            assert np.linalg.norm(z[f] - zs) <= info["relres"][f] * np.linalg.norm(s[f]) / (nu[f] * SIGMA ** 2)
    finally:
        T.tomo_destroy(h)


@pytest.mark.parametrize("method", ["cg", "minres"])
def test_elongated_with_mode_removal(T, method):
    # both per-WFS passes after the row-inverse pass: the noise blocks, then the
    # tip/tilt/focus projection, each rewriting the solver's partial sums
    from oracle import modes
    cfg = elongated(8, targets=((0.0, 0.0), (12e-6, 0.0)))
    A = cov.system_matrix(cfg)
    s = np.random.default_rng(21).standard_normal((3, A.shape[0]))
    zs, phis = modes.reconstruct(cfg, s.T, A)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=3, mode_removal=True)
    try:
        z, phi, info = solve_gpu(T, h, s, tol=3e-5, max_iter=20000, max_refine=5, method=method)
        assert (info["status"] == 0).all() and (info["relres"] <= 3e-5).all()
        Ms = modes.slope_removal(cfg)
        assert (modes.relative_residual(cfg, A, s.T, z.T) <= 3.5e-5).all()
        bound = info["relres"] * np.linalg.norm(s @ Ms, axis=1) / SIGMA ** 2
        assert (np.linalg.norm(z - zs.T, axis=1) <= bound).all()
        for t in range(2):
            assert relL2(phi[:, t], phis[t].T) <= 2e-3
    finally:
        T.tomo_destroy(h)


def test_elongated_wfe_matches_oracle(T):
    # Eq. analytical1 holds for any Sigma_eta_eta inside A
    from oracle import wfe
    cfg = elongated(8, targets=((0.0, 0.0), (10e-6, 5e-6)))
    ref = wfe.analytic_wfe(cfg, 1)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=16)
    try:
        info, _, _ = T.tomo_layout(h)
        rinfo, w = T.tomo_reconstructor(h, 1, T.solve_opts(tol=1e-6, max_iter=20000, max_refine=5), None,
                                        n_rows=info.n_vphi, wfe=True)
        assert (rinfo["status"] == 0).all()
        assert abs(w[0] ** 2 - ref) <= 1e-3 * ref
    finally:
        T.tomo_destroy(h)


def test_elongated_rejects_indefinite_blocks(T):
    cfg = elongated(6)
    from oracle import geometry as geo
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    bad = cfg["noise_cov"].copy()
    i, j = np.argwhere(mask)[0]
    bad[1, i, j, 2] = 1.01 * np.sqrt(bad[1, i, j, 0] * bad[1, i, j, 1])     # |s_xy| > sqrt(s_xx s_yy)
    with pytest.raises(T.TomoError):
        T.tomo_create(dict(cfg, noise_cov=bad), stream=torch.cuda.current_stream())
    # entries outside the pupil are never read
    if (~mask).any():
        ok = cfg["noise_cov"].copy()
        i, j = np.argwhere(~mask)[0]
        ok[0, i, j] = (-1.0, -1.0, 5.0)
        h = T.tomo_create(dict(cfg, noise_cov=ok), stream=torch.cuda.current_stream())
        T.tomo_destroy(h)


@pytest.fixture(scope="module")
def row_group_system():
    from paper_1806_07938_gb300 import workloads as W
    cfg = small_cfg(n=36, n_gs=2, lgs=True, obstruction=0.2, D=0.5 * 36, layers=((8000.0, 1.0),), noise=0.2)
    cfg["noise_cov"] = W.elongated_noise(cfg, 0.2, 3.0)
    return cfg, cov.system_matrix(cfg)


@pytest.mark.parametrize("method,modes_on", [("cg", False), ("minres", False), ("cg", True)])
def test_elongated_with_row_groups(T, row_group_system, method, modes_on):
    # n = 36 has 18 row pairs: a small batch runs the row passes as two blocks
    # per plane, whose partial sums the per-WFS passes (noise blocks, then the
    # mode projection) must rewrite for every row group
    from oracle import modes
    cfg, A = row_group_system
    s = np.random.default_rng(36).standard_normal((2, A.shape[0]))
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2, mode_removal=modes_on)
    try:
        tol = 1.5e-4                    # cond(A) ~ 4e4: the FP32 floor is near 6e-5 here
        z, _, info = solve_gpu(T, h, s, tol=tol, max_iter=20000, max_refine=5, method=method)
        print("row groups", method, modes_on, info)
        assert (info["status"] == 0).all() and (info["relres"] <= tol).all()
        if modes_on:
            zs, _ = modes.reconstruct(cfg, s.T, A)
            Ms = modes.slope_removal(cfg)
            bound = info["relres"] * np.linalg.norm(s @ Ms, axis=1) / 0.2 ** 2
            assert (np.linalg.norm(z - zs.T, axis=1) <= bound).all()
        else:
            zs = solve.solve_cholesky(A, s.T).T
            bound = info["relres"] * np.linalg.norm(s, axis=1) / 0.2 ** 2
            assert (np.linalg.norm(z - zs, axis=1) <= bound).all()
    finally:
        T.tomo_destroy(h)
