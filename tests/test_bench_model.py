"""The work model behind bench.py's roofline figures (no GPU needed)."""
import importlib.util
import os

from conftest import ROOT


def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class Layout:
    n, P, n_gs, N = 74, 150, 6, 47664       # the 74 x 74, 6-star system, 3972 valid subapertures


def test_kernel_model_counts():
    # per frame-iteration: 444 packed row FFTs of 150 points per row pass
    # (5 L log2 L flops each), 912 + 912 column FFTs and the 76 x 150 blocks of
    # 12 x 12 complex multiply-adds (8 flops) in the column pass
    import math
    b = bench()
    m = b.kernel_model(Layout)
    f150 = 5 * 150 * math.log2(150)
    assert abs(m["rows_fwd"]["flops"] - 12 * 37 * f150) < 1e-6
    assert abs(m["cols_mul"]["flops"] - (2 * 12 * 76 * f150 + 76 * 150 * 144 * 8)) < 1e-6
    assert m["cols_mul"]["bytes"] == 2 * 12 * 76 * 74 * 8
    assert m["cols_mul"]["per_launch_bytes"] == 76 * 150 * 78 * 8      # K_qp = conj K_pq: 78 of 144 blocks


def test_whole_product_fraction():
    # 64 frames, 1982.45 iterations, 447.5 ms per step at 6689.5 GB/s: the solve
    # runs at 17.7 % of the product's HBM-bound time, below the FP32 ridge
    b = bench()
    w = b.whole_product(b.kernel_model(Layout), 64, 447.513, 1982.453125, 6689.5, 80.54784)
    assert abs(w["bytes_per_frame_iter"] / 1e6 - 4.177) < 1e-3
    assert w["flop_per_byte"] < w["ridge_flop_per_byte"]
    assert abs(w["frac_of_hbm_bound"] - 0.177) < 1e-3
    assert abs(w["hbm_bound_us"] / w["solve_us_per_frame_iter"] - w["frac_of_hbm_bound"]) < 1e-12
    # below the ridge the HBM bound is the larger one
    assert w["alu_bound_us"] < w["hbm_bound_us"] and w["frac_of_roofline"] == w["frac_of_hbm_bound"]
    assert abs(w["alu_bound_us"] - 27.836217216e6 / 80.54784e12 * 1e6) < 1e-9
