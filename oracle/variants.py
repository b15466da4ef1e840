"""Correlation kernels X of the MV-RL variants listed in Supp. Note 2 sec. 1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The update of every variant is psi <- psi * prod_v [(phi_v / (psi * P_v)) * X_v]
(Supp. Note 2 sec. 1); "independent" is X_v = P_v^*, the plain MV-RL update.
The printed formulas for the others leave points open; the readings taken:
  * W_v = all views other than v;
  * juxtaposition and the product over w multiply kernels pixel by pixel over
    the K x K support of P_v^*; '*' is convolution, cropped to that support
    (same centre);
  * "optimization I" reads  X_v = P_v^* . prod_{w in W_v} (P_v^* * P_w)
    (the printed index 'v in W_v' read as 'w in W_v');
  * "optimization II" reads X_v = P_v^* . prod_{w in W_v} P_w^*;
  * every X_v is normalised to unit sum (a constant ratio of 1 then yields a
    correction of 1 away from the borders, so noise-free data stay a fixed
    point under the circular boundary).
With a single view every variant is the independent update.
"""

from __future__ import annotations

import numpy as np
from scipy.signal import convolve2d

from .rl import flip_psf

VARIANTS = ("independent", "efficient_bayesian", "optimization_1", "optimization_2")


def _conv_same(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full 2D convolution of two K x K kernels cropped to the K x K centre."""
    K = a.shape[0]
    full = convolve2d(a, b)                      # (2K-1) x (2K-1), centre at K-1
    R = (K - 1) // 2
    return full[K - 1 - R:K + R, K - 1 - R:K + R]


def correlation_kernels(psfs: np.ndarray, variant: str) -> np.ndarray:
    """X_v for every view (FP64, [V][K][K]); the update convolves the ratio
    with X_v (the independent variant: X_v = P_v^*)."""
    psfs = np.asarray(psfs, dtype=np.float64)
    V = psfs.shape[0]
    flips = np.stack([flip_psf(p) for p in psfs])
    out = []
    for v in range(V):
        x = flips[v].copy()
        for w in range(V):
            if w == v or variant == "independent":
                continue
            if variant == "efficient_bayesian":
                x *= _conv_same(_conv_same(flips[v], psfs[w]), flips[w])
            elif variant == "optimization_1":
                x *= _conv_same(flips[v], psfs[w])
            elif variant == "optimization_2":
                x *= flips[w]
            else:
                raise ValueError(f"unknown variant {variant!r}")
        out.append(x / x.sum())
    return np.stack(out)
