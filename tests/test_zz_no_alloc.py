"""tomo_apply_css_noalloc: the Sigma_ss product for callers that must not
allocate device memory while running (e.g. a real-time reconstruction loop,
where cudaMalloc would stall the frame, or a process whose device memory is
owned by another allocator).  It must give the same result as tomo_apply_css
through the C ABI, call after call, although every call reuses one static
device buffer.  This file is collected last on purpose."""
import json
import os

import numpy as np
import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_apply_css_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    g = dict(np.load(os.path.join(ROOT, "tests", "golden", "lgs_mid.npz")))
    cfg = json.loads(str(g["config"]))
    h = tomo.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        x1 = torch.tensor(g["x"], dtype=torch.float32, device="cuda")
        x2 = torch.tensor(np.ascontiguousarray(g["x"][::-1] * 0.5 + 1.0), dtype=torch.float32, device="cuda")
        for x in (x1, x2):                      # two calls in a row, different inputs
            ref = torch.empty_like(x)
            out = torch.full_like(x, float("nan"))
            tomo.tomo_apply_css(h, x, ref, x.shape[0])
            tomo.tomo_apply_css_noalloc(h, x, out, x.shape[0])
            torch.cuda.synchronize()
            r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
            assert np.isfinite(o).all()
            assert np.linalg.norm(o - r) / np.linalg.norm(r) <= 1e-5
        # and the first input against the oracle's stored product
        tomo.tomo_apply_css_noalloc(h, x1, out, 2)
        torch.cuda.synchronize()
        o = out.double().cpu().numpy()
        assert np.linalg.norm(o - g["y"]) / np.linalg.norm(g["y"]) <= 1e-5
    finally:
        tomo.tomo_destroy(h)


def test_noalloc_with_elongated_noise():
    # the 2 x 2 noise blocks of elongated laser spots (Sec. 2.F) on the same path
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import small_cfg
    from oracle import covariance as cov
    from paper_1806_07938_gb300 import tomo
    from paper_1806_07938_gb300 import workloads as W
    cfg = small_cfg(n=9, lgs=True, obstruction=0.2, D=5.4, noise=0.15)
    cfg["noise_cov"] = W.elongated_noise(cfg, 0.15, 3.0)
    A = cov.system_matrix(cfg)
    x = np.random.default_rng(9).standard_normal((2, A.shape[0]))
    h = tomo.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=2)
    try:
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        out = torch.full_like(xd, float("nan"))
        tomo.tomo_apply_css_noalloc(h, xd, out, 2)
        torch.cuda.synchronize()
        o = out.double().cpu().numpy()
        ref = x @ A.T
        assert np.linalg.norm(o - ref) / np.linalg.norm(ref) <= 1e-5
    finally:
        tomo.tomo_destroy(h)
