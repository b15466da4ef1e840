"""3D multi-view RL for views turned about the rotation axis, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The plane-wise method (Results; Fig. 1a) deconvolves every plane orthogonal
to the rotation axis with a 2D PSF.  A view turned about that axis keeps its
PSF profile along the axis, so its 3D PSF factorises as

    P3_v(y, z, x) = a_v(y) P_v(z, x)

with a_v the profile along the rotation axis (y, the plane index) and P_v the
in-plane PSF the plane-wise method uses.  The 3D update (the same Supp.
Note 1 equation with 3D convolutions) is

    psi <- psi * prod_v [ (phi_v / (psi * P3_v)) (*) P3_v^* ],

and with a_v = delta it is the plane-wise update on every plane.  Used to
measure what the plane-wise approximation loses (Supp. Figs. 3 and 4 compare
it with 3D deconvolution).  Arrays are in plane layout [Y][Z][X].
"""

from __future__ import annotations

import numpy as np

from .rl import CIRCULAR, ZERO, convolve, correlate, init_mean


def _axial(vol: np.ndarray, a: np.ndarray, boundary: str, flip: bool) -> np.ndarray:
    """out[y] = sum_i a[i] vol[y -/+ (i - R)]: convolution (flip False) or
    correlation (flip True) along the plane axis, zero or wrapped outside."""
    vol = np.asarray(vol, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    Ka = a.shape[0]
    if Ka % 2 != 1:
        raise ValueError("axial profile must have odd length")
    R = (Ka - 1) // 2
    Y = vol.shape[0]
    out = np.zeros_like(vol)
    for i in range(Ka):
        if a[i] == 0.0:
            continue
        s = (i - R) if flip else -(i - R)         # out[y] += a[i] vol[y + s]
        if boundary == CIRCULAR:
            out += a[i] * vol[(np.arange(Y) + s) % Y]
        elif boundary == ZERO:
            y0, y1 = max(0, -s), min(Y, Y - s)
            if y0 < y1:
                out[y0:y1] += a[i] * vol[y0 + s:y1 + s]
        else:
            raise ValueError(f"unknown boundary {boundary!r}")
    return out


def convolve3d(vol, P, a, boundary=ZERO):
    """vol * P3 with P3(y, z, x) = a(y) P(z, x): in-plane convolution of every
    plane, then along the plane axis."""
    planes = np.stack([convolve(p, P, boundary) for p in np.asarray(vol, dtype=np.float64)])
    return _axial(planes, a, boundary, flip=False)


def correlate3d(vol, P, a, boundary=ZERO):
    """Correlation with P3, i.e. convolution with the flipped P3."""
    planes = np.stack([correlate(p, P, boundary) for p in np.asarray(vol, dtype=np.float64)])
    return _axial(planes, a, boundary, flip=True)


def rl3d(phi, psfs, axial, iters, boundary=ZERO, eps=1e-6, psi0=None, order="simultaneous"):
    """3D MV-RL on views in plane layout.

    phi:   [V][Y][Z][X] data, one volume per view (planes y along the axis)
    psfs:  [V][K][K] in-plane PSFs; axial: [V][Ka] profiles along the axis
    psi0:  None -> per-plane mean of all views' pixels (as the plane-wise
           method starts), else [Y][Z][X]
    Returns psi [Y][Z][X] after `iters` updates (simultaneous product, or the
    views one after another for order="sequential").
    """
    phi = np.asarray(phi, dtype=np.float64)
    V = phi.shape[0]
    if psi0 is None:
        means = init_mean(phi)
        psi = np.broadcast_to(means[:, None, None], phi.shape[1:]).copy()
    else:
        psi = np.asarray(psi0, dtype=np.float64).copy()
    for _ in range(iters):
        if order == "sequential":
            for v in range(V):
                blur = convolve3d(psi, psfs[v], axial[v], boundary)
                psi = psi * correlate3d(phi[v] / np.maximum(blur, eps), psfs[v], axial[v], boundary)
        elif order == "simultaneous":
            update = np.ones_like(psi)
            for v in range(V):
                blur = convolve3d(psi, psfs[v], axial[v], boundary)
                update *= correlate3d(phi[v] / np.maximum(blur, eps), psfs[v], axial[v], boundary)
            psi = psi * update
        else:
            raise ValueError(f"unknown update order {order!r}")
    return psi
