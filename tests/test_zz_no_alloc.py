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


def test_noalloc_several_chunks_elt():
    # the 74 x 74, 6-star system needs 1.08 MB of scratch per frame, so the
    # 16 MiB buffer takes 15 frames at a time: 20 frames run as two chunks
    # (15 + 5), and every element must equal tomo_apply_css's
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("elt_ltao")
    cfg["noise_sigma"] = [0.17] * len(cfg["gs"])
    h = tomo.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=20)
    try:
        info, _, _ = tomo.tomo_layout(h)
        per_frame = 2 * (2 * info.n_gs) * (info.P // 2 + 1) * info.n * 8
        assert (16 << 20) // per_frame == 15
        x = torch.tensor(np.random.default_rng(31).standard_normal((20, info.N)), dtype=torch.float32, device="cuda")
        for _ in range(2):
            ref = torch.empty_like(x)
            out = torch.full_like(x, float("nan"))
            tomo.tomo_apply_css(h, x, ref, 20)
            tomo.tomo_apply_css_noalloc(h, x, out, 20)
            torch.cuda.synchronize()
            r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
            assert np.isfinite(o).all()
            # frame by frame, so that a frame of the second chunk read or
            # written at a wrong offset cannot hide in the total
            err = np.linalg.norm(o - r, axis=1) / np.linalg.norm(r, axis=1)
            assert err.max() <= 1e-5, err
            x = x.flip(0).contiguous() * 0.5
    finally:
        tomo.tomo_destroy(h)


def test_noalloc_chunk_beyond_grid_limit():
    # one natural star on a 2 x 2 grid needs 192 B per frame, so the buffer
    # would hold 87 381 frames; a chunk is capped at 65 535 (the grid's y
    # limit), so 70 000 frames still run, as two chunks
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import small_cfg
    from oracle import covariance as cov
    from paper_1806_07938_gb300 import tomo
    cfg = small_cfg(n=2, n_gs=1, D=1.0, noise=0.1)
    A = cov.system_matrix(cfg)
    B = 70000
    x = np.random.default_rng(5).standard_normal((B, A.shape[0]))
    h = tomo.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=4096)
    try:
        info, _, _ = tomo.tomo_layout(h)
        assert info.N == A.shape[0] == 8
        assert (16 << 20) // (2 * 2 * (info.P // 2 + 1) * info.n * 8) > 65535
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        ref = torch.empty_like(xd)
        out = torch.full_like(xd, float("nan"))
        tomo.tomo_apply_css(h, xd, ref, B)
        tomo.tomo_apply_css_noalloc(h, xd, out, B)
        torch.cuda.synchronize()
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        assert np.isfinite(o).all()
        err = np.linalg.norm(o - r, axis=1) / np.linalg.norm(r, axis=1)
        assert err.max() <= 1e-5, err.max()
        y = x @ A.T
        assert np.linalg.norm(o - y) / np.linalg.norm(y) <= 1e-5
    finally:
        tomo.tomo_destroy(h)
