"""Pins of the von Karman covariance (Appendix A.2 structure function, A.1 PSD)."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import turbulence as turb


def test_variance_closed_form():
    # B(0) = c_v (L0/r0)^{5/3} with c_v = 0.0863143 (value of the constant)
    assert turb.C_V == pytest.approx(0.0863143, abs=5e-8)
    r0, L0 = 0.15, 25.0
    assert turb.vk_covariance(0.0, r0, L0) == pytest.approx(0.0863143 * (L0 / r0) ** (5 / 3), rel=1e-6)
    # continuity at rho -> 0 (x^nu K_nu(x) -> 2^{nu-1} Gamma(nu))
    assert turb.vk_covariance(1e-9, r0, L0) == pytest.approx(turb.vk_covariance(0.0, r0, L0), rel=1e-10)


def test_structure_function_prefactor_of_the_paper():
    # the paper rounds 2 c_v to 0.17253; the exact value differs by < 1e-3 relative
    assert 2 * turb.C_V == pytest.approx(0.17253, rel=1e-3)
    assert turb.vk_structure_function(0.0, 0.15, 25.0) == 0.0


def _psd_hankel(rho, r0, L0):
    # B(rho) = 2 pi int_0^inf Phi(f) J0(2 pi f rho) f df, Phi = 0.0228956 r0^{-5/3} (f^2 + L0^-2)^{-11/6}
    c = (24 / 5 * special.gamma(6 / 5)) ** (5 / 6) * special.gamma(11 / 6) ** 2 / (2 * np.pi ** (11 / 3))
    f = lambda u: c * r0 ** (-5 / 3) * (u * u + L0 ** -2) ** (-11 / 6) * special.j0(2 * np.pi * u * rho) * u
    val, _ = integrate.quad(f, 0, np.inf, limit=2000, epsabs=0, epsrel=1e-10)
    return 2 * np.pi * val


@pytest.mark.parametrize("rho", [0.0, 0.1, 1.0, 7.5, 30.0])
def test_covariance_is_the_hankel_transform_of_the_psd(rho):
    # an independent route (the PSD of Appendix A.1) to the same covariance
    r0, L0 = 0.129, 25.0
    if rho == 0.0:
        ref = _psd_hankel(0.0, r0, L0)
    else:
        # oscillatory tail: integrate J0 piecewise via the weight option
        c = (24 / 5 * special.gamma(6 / 5)) ** (5 / 6) * special.gamma(11 / 6) ** 2 / (2 * np.pi ** (11 / 3))
        g = lambda u: c * r0 ** (-5 / 3) * (u * u + L0 ** -2) ** (-11 / 6) * u * special.j0(2 * np.pi * u * rho)
        pieces = np.concatenate([[0.0], (np.arange(1, 4000) / (2 * rho))])
        ref = 2 * np.pi * sum(integrate.quad(g, a, b, epsabs=0, epsrel=1e-12)[0] for a, b in zip(pieces[:-1], pieces[1:]))
    assert turb.vk_covariance(rho, r0, L0) == pytest.approx(ref, rel=2e-5, abs=1e-6 * turb.vk_covariance(0, r0, L0))


def test_small_separation_series():
    # From the ascending series of K_nu (nu = 5/6):
    #   x^nu K_nu(x) = 2^{nu-1} Gamma(nu) [1 + x^2/(4(1-nu))] + 2^{-nu-1} Gamma(-nu) x^{2nu} + O(x^{2+2nu}),
    # so D(r) = 2 B(0) [-2^{-2nu} Gamma(-nu)/Gamma(nu) x^{2nu} - x^2/(4(1-nu))] + O(x^{11/3}), x = 2 pi r/L0.
    nu = 5 / 6
    r0, L0 = 0.15, 25.0
    B0 = turb.vk_covariance(0.0, r0, L0)
    for r in [0.01, 0.03, 0.08]:
        x = 2 * np.pi * r / L0
        series = 2 * B0 * (-2 ** (-2 * nu) * special.gamma(-nu) / special.gamma(nu) * x ** (2 * nu)
                           - x * x / (4 * (1 - nu)))
        assert turb.vk_structure_function(r, r0, L0) == pytest.approx(series, rel=5 * x * x + 1e-9)


def test_kolmogorov_coefficient():
    # the leading term is the Kolmogorov structure function 6.88 (r/r0)^{5/3}
    nu = 5 / 6
    coef = 2 * turb.C_V * (-2 ** (-2 * nu) * special.gamma(-nu) / special.gamma(nu)) * (2 * np.pi) ** (5 / 3)
    assert coef == pytest.approx(6.8839, rel=2e-4)


def test_layer_fractions_combine():
    # sum_k r0_k^{-5/3} = r0^{-5/3}
    fr = np.array([0.4, 0.12, 0.1, 0.09, 0.08, 0.07, 0.06, 0.05, 0.03])
    r0 = 0.129
    assert np.sum(turb.layer_r0(r0, fr) ** (-5 / 3)) == pytest.approx(r0 ** (-5 / 3), rel=1e-12)
