"""Block conjugate gradients over the frames of a batch, against the oracle."""
import json
import os

import numpy as np
import pytest

from conftest import ROOT, small_cfg
from oracle import covariance as cov
from oracle import solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NM_PER_RAD = 500.0 / (2 * np.pi)


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    tomo.lib()
    return tomo


def golden(name):
    g = dict(np.load(os.path.join(ROOT, "tests", "golden", f"{name}.npz")))
    g["cfg"] = json.loads(str(g["config"]))
    return g


def run(T, h, s, **opts):
    info_l, _, _ = T.tomo_layout(h)
    sd = torch.tensor(np.ascontiguousarray(s), dtype=torch.float32, device="cuda")
    zd = torch.zeros_like(sd)
    phi = torch.empty((s.shape[0], info_l.n_targets, info_l.n_vphi), dtype=torch.float32, device="cuda")
    info = T.tomo_solve(h, sd, s.shape[0], T.solve_opts(**opts), zd, phi)
    torch.cuda.synchronize()
    return zd.double().cpu().numpy(), phi.double().cpu().numpy(), info


@pytest.mark.parametrize("name,pcg", [("ngs8m", False), ("ngs8m", True), ("lgs_mid", False), ("lgs_mid", True)])
def test_block_cg_golden(T, name, pcg):
    g = golden(name)
    h = T.tomo_create(g["cfg"], stream=torch.cuda.current_stream(), max_batch=4, precond=True)
    try:
        z, phi, info = run(T, h, g["s"], tol=1e-5, max_iter=20000, max_refine=3, precond=pcg, method="block")
        _, _, cg = run(T, h, g["s"], tol=1e-5, max_iter=20000, max_refine=3, precond=pcg)
        print(name, "block", "PCG" if pcg else "CG", info, "single-frame iters", cg["iters"])
        assert (info["status"] == 0).all() and (info["relres"] <= 1e-5).all()
        err = np.linalg.norm(z - g["zeta"], axis=1)
        bound = info["relres"] * np.linalg.norm(g["s"], axis=1) / min(g["noise_sigma"]) ** 2
        assert (err <= bound).all()
        ref = solve.remove_piston(g["phi_interp"].T).T
        rms = [NM_PER_RAD * np.sqrt(np.mean((solve.remove_piston(phi[f, 0]) - ref[f]) ** 2)) for f in range(4)]
        assert max(rms) <= 0.1, rms
        assert info["iters"].max() < cg["iters"].mean()
    finally:
        T.tomo_destroy(h)


def test_block_cg_many_frames_zero_frame_and_modes(T):
    # 40 frames of the 16 x 16 system in one block (N = 2304), one of them zero;
    # then the same with tip/tilt/focus removal against the oracle
    from oracle import modes
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("lgs_mid")
    full, sigma = W.slope_frames(cfg, 40, seed=31)
    cfg["noise_sigma"] = [float(x) for x in sigma]
    A = cov.system_matrix(cfg)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=40, precond=True)
    try:
        _, sub, _ = T.tomo_layout(h)
        s = T.valid_slopes(full, sub)
        s[7] = 0.0
        z, _, info = run(T, h, s, tol=1e-5, max_iter=20000, max_refine=3, precond=True, method="block")
        print("40 frames block PCG", info["iters"][0], info["relres"].max())
        assert (info["status"] == 0).all() and (info["relres"] <= 1e-5).all()
        assert np.abs(z[7]).max() == 0.0
        zs = solve.solve_cholesky(A, s.T).T
        bound = info["relres"] * np.linalg.norm(s, axis=1) / min(cfg["noise_sigma"]) ** 2
        assert (np.linalg.norm(z - zs, axis=1) <= bound + 1e-30).all()
    finally:
        T.tomo_destroy(h)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=8, precond=True, mode_removal=True)
    try:
        s8 = s[:8].copy()
        z, phi, info = run(T, h, s8, tol=3e-5, max_iter=20000, max_refine=5, precond=True, method="block")
        assert (info["status"] == 0).all() and (info["relres"] <= 3e-5).all()
        zs, phis = modes.reconstruct(cfg, s8.T, A)
        Ms = modes.slope_removal(cfg)
        bound = info["relres"] * np.linalg.norm(s8 @ Ms, axis=1) / min(cfg["noise_sigma"]) ** 2
        assert (np.linalg.norm(z - zs.T, axis=1) <= bound + 1e-30).all()
    finally:
        T.tomo_destroy(h)


@pytest.mark.parametrize("kappa", [1.0, 0.5])
def test_block_cg_proportional_operators(T, kappa):
    # four seeings in one block: nu_f = kappa c_f makes A_f = c_f (Sigma_ss + kappa Sigma_eta_eta)
    cfg = small_cfg(n=7, lgs=True, obstruction=0.2, D=4.2, noise=0.15, targets=((0.0, 0.0), (10e-6, -5e-6)))
    r0 = np.array([0.10, 0.133, 0.167, 0.20])
    c = (r0 / cfg["r0"]) ** (-5.0 / 3.0)
    nu = kappa * c
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=4, precond=True)
    try:
        info_l, _, _ = T.tomo_layout(h)
        s = np.random.default_rng(6).standard_normal((4, info_l.N))
        sd = torch.tensor(s, dtype=torch.float32, device="cuda")
        zd = torch.zeros_like(sd)
        phi = torch.empty((4, 2, info_l.n_vphi), dtype=torch.float32, device="cuda")
        info = T.tomo_solve_r0(h, sd, 4, r0, T.solve_opts(tol=3e-5, max_iter=20000, max_refine=5, precond=True,
                                                          method="block"), zd, phi, noise_scale=nu)
        torch.cuda.synchronize()
        z, phi = zd.double().cpu().numpy(), phi.double().cpu().numpy()
        print("proportional block", info)
        assert (info["status"] == 0).all() and (info["relres"] <= 3e-5).all()
        sig2 = min(cfg["noise_sigma"]) ** 2
        for f in range(4):
            A = cov.system_matrix_r0(cfg, r0[f], nu[f])
            zs = solve.solve_cholesky(A, s[f])
            assert np.linalg.norm(z[f] - zs) <= info["relres"][f] * np.linalg.norm(s[f]) / (nu[f] * sig2)
            for t in range(2):
                ref = cov.cos_interp(dict(cfg, r0=r0[f]), t) @ zs
                assert float(np.linalg.norm(phi[f, t] - ref) / np.linalg.norm(ref)) <= 2e-3
    finally:
        T.tomo_destroy(h)


def test_block_cg_rejected_where_invalid(T):
    cfg = small_cfg(n=6, lgs=True)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        info, _, _ = T.tomo_layout(h)
        sd = torch.ones((2, info.N), dtype=torch.float32, device="cuda")
        zd = torch.zeros_like(sd)
        with pytest.raises(T.TomoError):        # fixed noise, two seeings: no common Krylov space
            T.tomo_solve_r0(h, sd, 2, np.array([0.1, 0.2]), T.solve_opts(method="block"), zd)
    finally:
        T.tomo_destroy(h)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=65)
    try:
        info, _, _ = T.tomo_layout(h)
        sd = torch.ones((2, info.N), dtype=torch.float32, device="cuda")
        zd = torch.zeros_like(sd)
        with pytest.raises(T.TomoError):        # blocks of at most 64 frames
            T.tomo_solve(h, sd, 2, T.solve_opts(method="block"), zd)
    finally:
        T.tomo_destroy(h)
