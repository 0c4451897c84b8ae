"""The paper's operation-count model (Sec. 2.E), reported by bench.py beside this
design's own work model, against the reduction factors the paper prints for
n = 80 with N_gs = 6, N_layer = 9, n' = 1.2 n and a = 5 (caption of the
operation-count figure): 8e-3 for Sigma_ss zeta, 4e-2 for Sigma_phi_s zeta with
natural stars, 0.1 with laser stars.  The one-digit values are bracketed to
the next digit; a base-e logarithm, a dropped N_gs product term or a dropped
layer product term falls outside them."""
import importlib.util
import os

from conftest import ROOT


def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reduction_factors_printed_by_the_paper():
    o = bench().paper_opcounts(80, 6, 9, 1.2 * 80)
    assert 8e-3 <= o["sigma_ss"] / o["sigma_ss_full"] < 9e-3
    assert 4e-2 <= o["sigma_phi_s_ngs"] / o["sigma_phi_s_full"] < 5e-2
    assert 0.1 <= o["sigma_phi_s_lgs"] / o["sigma_phi_s_full"] < 0.11


def test_full_mvm_counts_are_the_matrix_sizes():
    # a full MVM costs one operation per matrix entry: Sigma_ss is 2 N_gs n^2
    # square, Sigma_phi_s (n+1)^2 x 2 N_gs n^2 on the square grid
    for n, g in ((20, 3), (74, 6)):
        o = bench().paper_opcounts(n, g, 9, 1.2 * n)
        assert o["sigma_ss_full"] == (2 * g * n * n) ** 2
        assert o["sigma_phi_s_full"] == (n + 1) ** 2 * 2 * g * n * n
