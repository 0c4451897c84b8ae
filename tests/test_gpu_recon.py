"""Adjoint projection, explicit reconstructor and its GEMM against the oracle."""
import numpy as np
import pytest

from conftest import small_cfg
from oracle import covariance as cov
from oracle import solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    tomo.lib()
    return tomo


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def relL2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("lgs", [False, True])
def test_cos_adjoint_matches_oracle(T, lgs):
    targets = ((0.0, 0.0), (15e-6, -5e-6), (-30e-6, 20e-6))
    cfg = small_cfg(n=7, lgs=lgs, obstruction=0.2, targets=targets)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        info, _, _ = T.tomo_layout(h)
        rng = np.random.default_rng(4)
        phi = rng.standard_normal((3, 3, info.n_vphi))           # batch 3 > max_batch 2: chunked
        z = torch.empty((3, info.N), dtype=torch.float32, device="cuda")
        T.tomo_apply_cos_adjoint(h, dev(phi), z, 3)
        zeta = rng.standard_normal((3, info.N))
        y = torch.empty((3, 3, info.n_vphi), dtype=torch.float32, device="cuda")
        T.tomo_apply_cos(h, dev(zeta), y, 3)
        torch.cuda.synchronize()
        z, y = z.double().cpu().numpy(), y.double().cpu().numpy()
        ref = sum(phi[:, t] @ cov.cos_interp(cfg, t) for t in range(3))
        assert relL2(z, ref) <= 1e-5
        # <Cos zeta, phi> = <zeta, Cos^T phi>
        lhs, rhs = float((y * phi).sum()), float((zeta * z).sum())
        assert abs(lhs - rhs) <= 1e-5 * np.abs(y * phi).sum()
    finally:
        T.tomo_destroy(h)


def test_reconstructor_matches_oracle(T):
    import json
    import os
    from conftest import ROOT
    g = dict(np.load(os.path.join(ROOT, "tests", "golden", "lgs_mid.npz")))
    cfg = json.loads(str(g["config"]))
    A = cov.system_matrix(cfg)
    F = cov.cos_interp(cfg, 0)
    R_ref = solve.reconstructor(F, A)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=64, precond=True)
    try:
        info, _, _ = T.tomo_layout(h)
        R = torch.empty((info.n_vphi, info.N), dtype=torch.float32, device="cuda")
        rinfo = T.tomo_reconstructor(h, 0, T.solve_opts(tol=1e-5, max_iter=20000, max_refine=3, precond=True), R)
        torch.cuda.synchronize()
        print("reconstructor rows", info.n_vphi, "iters mean", rinfo["iters"].mean())
        assert (rinfo["status"] == 0).all() and (rinfo["relres"] <= 1e-5).all()
        Rn = R.double().cpu().numpy()
        # row v solves A x = F[v] to relres_v: ||x - x*|| <= relres_v ||F[v]|| / sigma_min^2
        err = np.linalg.norm(Rn - R_ref, axis=1)
        bound = rinfo["relres"] * np.linalg.norm(F, axis=1) / min(cfg["noise_sigma"]) ** 2
        print("R relL2", relL2(Rn, R_ref), "max err/bound", (err / bound).max())
        assert (err <= bound).all()
        assert relL2(Rn, R_ref) <= 1e-2
        # the direct MVM on the golden frames reproduces the Cholesky wave-front
        s = g["s"]
        out = torch.empty((s.shape[0], info.n_vphi), dtype=torch.float32, device="cuda")
        T.tomo_apply_reconstructor(h, R, dev(s), s.shape[0], out)
        torch.cuda.synchronize()
        phi = out.double().cpu().numpy()
        ref = solve.remove_piston(g["phi_interp"].T).T
        rms = np.sqrt(np.mean((solve.remove_piston(phi.T).T - ref) ** 2, axis=1)) * 500 / (2 * np.pi)
        print("direct MVM wave-front rms diff [nm]", rms)
        assert rms.max() <= 0.5
    finally:
        T.tomo_destroy(h)


@pytest.mark.parametrize("rows,batch,n,n_gs", [(200, 70, 6, 2), (64, 1, 24, 6), (4160, 3, 16, 3), (100, 64, 30, 6)])
def test_apply_reconstructor_gemm(T, rows, batch, n, n_gs):
    # the GEMM alone: ragged tiles, a batch above one tile, a single frame, and
    # reduction lengths with and without the split over N
    cfg = small_cfg(n=n, n_gs=n_gs, D=0.5 * n)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        info, _, _ = T.tomo_layout(h)
        Nh = info.N
        rng = np.random.default_rng(rows)
        R = rng.standard_normal((rows, Nh))
        s = rng.standard_normal((batch, Nh))
        out = torch.empty((batch, rows), dtype=torch.float32, device="cuda")
        T.tomo_apply_reconstructor(h, dev(R), dev(s), batch, out)
        torch.cuda.synchronize()
        assert relL2(out.double().cpu().numpy(), s @ R.T) <= 1e-5
    finally:
        T.tomo_destroy(h)


@pytest.mark.parametrize("lgs", [False, True])
def test_analytic_wfe_matches_oracle(T, lgs):
    # Eq. analytical1 for the MMSE reconstructor, from the reconstructor build
    from oracle import wfe
    cfg = small_cfg(n=8, lgs=lgs, obstruction=0.2, D=4.0, noise=0.2, targets=((0.0, 0.0), (10e-6, 5e-6)))
    ref = wfe.analytic_wfe(cfg, 1)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=16)
    try:
        info, _, _ = T.tomo_layout(h)
        rinfo, w = T.tomo_reconstructor(h, 1, T.solve_opts(tol=1e-6, max_iter=20000, max_refine=5), None,
                                        n_rows=info.n_vphi, wfe=True)
        print("wfe", w, "oracle", ref, "rms rad", np.sqrt(ref))
        assert (rinfo["status"] == 0).all()
        assert abs(w[0] ** 2 - ref) <= 1e-3 * ref
        assert abs(w[0] ** 2 - (w[1] - w[2])) <= 1e-12 * w[1]
    finally:
        T.tomo_destroy(h)
