import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libtomo.so")


def small_cfg(n=6, n_gs=3, lgs=False, layers=((0.0, 0.6), (6000.0, 0.4)), D=3.0, obstruction=0.0,
              radius_arcsec=20.0, noise=0.1, targets=((0.0, 0.0),)):
    """A small system for oracle pins (plain numbers only)."""
    from paper_1806_07938_gb300 import workloads as W
    H = 90e3 if lgs else 0.0
    return dict(name="small", D=D, obstruction=obstruction, n=n, r0=0.15, L0=25.0,
                layers=[tuple(l) for l in layers], gs=W.ring(n_gs, radius_arcsec * W.ARCSEC, H),
                targets=[tuple(t) for t in targets], noise_sigma=[noise] * n_gs, noise_frac=0.05)


@pytest.fixture
def small():
    return small_cfg
