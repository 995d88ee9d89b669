"""Host-side helpers for the paper's measurements (Sec. 3-4): Young-Laplace fit
(Eq. 12), equivalent radius of a droplet from its volume, drift velocity.
The field reductions themselves run on the GPU (lbm_pressure_jump,
lbm_droplet_stats, lbm_reduce)."""
import math

import numpy as np


def equivalent_radius(volume, quasi_2d, hemisphere=False):
    """Radius of the disc (quasi-2D) or sphere (3D) or hemisphere of this volume."""
    if quasi_2d:
        return math.sqrt(volume / math.pi)
    if hemisphere:
        return (3.0 * volume / (2.0 * math.pi)) ** (1.0 / 3.0)
    return (3.0 * volume / (4.0 * math.pi)) ** (1.0 / 3.0)


def laplace_fit(radii, dps, dims=2):
    """Least-squares fit dp = s / R + c.  Eq. 12 is the 2D form dp = sigma / R;
    in 3D dp = 2 sigma / R.  Returns (sigma, intercept, max residual)."""
    R = np.asarray(radii, dtype=float)
    dp = np.asarray(dps, dtype=float)
    A = np.vstack([1.0 / R, np.ones_like(R)]).T
    (s, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    resid = float(np.max(np.abs(A @ np.array([s, c]) - dp)))
    return (s if dims == 2 else s / 2.0), float(c), resid


def drift_velocity(com_a, com_b, steps):
    """Centre-of-mass displacement per step between two measurements."""
    d = np.asarray(com_b, dtype=float) - np.asarray(com_a, dtype=float)
    return d / float(steps)
