"""von Karman turbulence statistics (oracle side; test infrastructure only).

Appendix A.2, structure-function equation (von Karman D_phi with K_{5/6}).
The printed equation is garbled (it shows (r0/L0)^{5/6} where the bracket can
only vanish at r = 0 with (r/L0)^{5/6}, and rounds the prefactor to 0.17253).
This module uses the standard von Karman phase covariance

    B(rho) = c_v (L0/r0)^{5/3} * 2^{1/6}/Gamma(5/6) * x^{5/6} K_{5/6}(x),
    x = 2 pi rho / L0,
    c_v = (24/5 Gamma(6/5))^{5/6} Gamma(11/6) Gamma(5/6) / (2 pi^{8/3}),

with B(0) = c_v (L0/r0)^{5/3} and D_phi(rho) = 2 (B(0) - B(rho)); 2 c_v is
the prefactor the paper rounds to 0.17253.  K_{5/6} is scipy's kv.

Per layer k of a Cn^2 profile with fractions f_k (sum 1):
r0_k = r0 f_k^{-3/5}, i.e. (L0/r0_k)^{5/3} = f_k (L0/r0)^{5/3}.
"""

import numpy as np
from scipy.special import gamma, kv

NU = 5.0 / 6.0
C_V = (24.0 / 5.0 * gamma(6.0 / 5.0)) ** (5.0 / 6.0) * gamma(11.0 / 6.0) * gamma(5.0 / 6.0) \
    / (2.0 * np.pi ** (8.0 / 3.0))


def layer_r0(r0, frac):
    """Fried parameter of one layer carrying Cn^2 fraction ``frac``."""
    return r0 * frac ** (-3.0 / 5.0)


def vk_covariance(rho, r0, L0):
    """von Karman phase covariance B(rho) in rad^2 (rho in metres, array ok)."""
    rho = np.asarray(rho, dtype=np.float64)
    amp = C_V * (L0 / r0) ** (5.0 / 3.0)
    out = np.full(rho.shape, amp, dtype=np.float64)
    nz = rho > 0.0
    x = 2.0 * np.pi * rho[nz] / L0
    out[nz] = amp * (2.0 ** (1.0 / 6.0) / gamma(NU)) * x ** NU * kv(NU, x)
    return out


def vk_structure_function(rho, r0, L0):
    """D_phi(rho) = 2 (B(0) - B(rho)) in rad^2."""
    return 2.0 * (C_V * (L0 / r0) ** (5.0 / 3.0) - vk_covariance(rho, r0, L0))
