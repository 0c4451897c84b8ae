"""Pupil geometry of a Shack-Hartmann WFS (oracle side; test infrastructure only).

Sec. 2.D (geometry of the n x n subapertures and the (n+1) x (n+1) phase
points of one SH-WFS) and Sec. 2.F "Non-square aperture" (W_s, W_phi remove
vignetted subapertures and phase points).

Conventions (plain reading; the figure that shows them is missing):
* subaperture (i, j): i is the row (y), j the column (x); its centre is at
  x = (j + 1/2 - n/2) d, y = (i + 1/2 - n/2) d with d = D / n.
* a subaperture is valid iff its centre lies inside the annular pupil:
  r <= D/2 and r >= obstruction * D/2.  In integers, with
  q = (2j + 1 - n)^2 + (2i + 1 - n)^2, this is q <= n^2 and q >= (eps n)^2.
* phase point (i, j), 0 <= i, j <= n, sits at the subaperture corner
  ((j - n/2) d, (i - n/2) d); it is valid iff it is a corner of at least one
  valid subaperture.
* valid entries are listed in row-major order k(i, j) = i*n + j (Sec. 2.E).
"""

import numpy as np


def subaperture_mask(n, obstruction):
    """Boolean n x n mask of valid subapertures (centre inside the annulus)."""
    mask = np.zeros((n, n), dtype=bool)
    thr = (obstruction * n) * (obstruction * n)
    for i in range(n):
        for j in range(n):
            q = (2 * j + 1 - n) ** 2 + (2 * i + 1 - n) ** 2
            mask[i, j] = (q <= n * n) and (q >= thr)
    return mask


def phase_point_mask(n, obstruction):
    """Boolean (n+1) x (n+1) mask: corners of at least one valid subaperture."""
    sub = subaperture_mask(n, obstruction)
    pm = np.zeros((n + 1, n + 1), dtype=bool)
    for i in range(n):
        for j in range(n):
            if sub[i, j]:
                pm[i, j] = pm[i + 1, j] = pm[i, j + 1] = pm[i + 1, j + 1] = True
    return pm


def valid_list(mask):
    """Row-major list of (i, j) of the True entries of ``mask``."""
    ii, jj = np.nonzero(mask)          # np.nonzero walks a C array row-major
    return np.stack([ii, jj], axis=1)


def subaperture_centres(n, D, obstruction):
    """(n_vs, 2) array of (x, y) centres of the valid subapertures, metres."""
    d = D / n
    v = valid_list(subaperture_mask(n, obstruction))
    x = (v[:, 1] + 0.5 - n / 2.0) * d
    y = (v[:, 0] + 0.5 - n / 2.0) * d
    return np.stack([x, y], axis=1)


def phase_points(n, D, obstruction):
    """(n_vphi, 2) array of (x, y) of the valid phase points, metres."""
    d = D / n
    v = valid_list(phase_point_mask(n, obstruction))
    x = (v[:, 1] - n / 2.0) * d
    y = (v[:, 0] - n / 2.0) * d
    return np.stack([x, y], axis=1)
