"""Plain FP64 CPU oracle for the spatio-angular MMSE tomographic reconstructor.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
anything in this package.  The product path (the CUDA library behind
``include/tomo.h`` and its Python binding) never does; the two share no code.

What it computes (Ono et al., "Fast iterative tomographic wave-front estimation
with recursive Toeplitz reconstructor structure"):

* ``geometry``   -- valid-subaperture and valid-phase-point masks (Sec. 2.F,
                    "Non-square aperture"), index maps in row-major order
                    k(i, j) = i*n + j (Sec. 2.E, step 1 of the 2RBT MVM).
* ``turbulence`` -- von Karman phase covariance / structure function
                    (Appendix A.2, structure-function equation; scipy's K_nu).
* ``covariance`` -- dense slope-slope covariance Sigma_ss and phase-slope
                    covariance Sigma_phi_s from point covariances of the
                    Hudgin-like two-point slope model (Appendix A.2), with the
                    LGS cone compression per layer (Sec. 2.D), plus the LGS
                    "new phase grid + bilinear interpolation" form of
                    Sigma_phi_s (Sec. 2.D, Eq. interp and the sum over layers).
* ``solve``      -- Eq. covIterative1 / SAap1 by FP64 Cholesky and by textbook
                    CG; Eq. covIterative2 / SAap2 projection.

Every entry is formed directly from point coordinates; no Toeplitz generator,
no FFT and no closed-form Hudgin expression is used, so the structure the GPU
path exploits is a property the oracle is tested for, not one it assumes.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, special cases and brute force); none is unpinned.
"""

from . import geometry, turbulence, covariance, solve  # noqa: F401
