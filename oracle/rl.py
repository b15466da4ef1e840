"""Forward plane-wise multi-view Richardson-Lucy, written out in FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the
library imports this module.

What is computed (paper: Supp. Note 1, the multi-view RL update equation;
Results and Fig. 1a for the plane-wise approximation and reslicing):

    psi^{t+1} = psi^t * prod_{v in V} [ (phi_v / (psi^t * P_v)) (*) P_v^* ]

with P_v^* the flipped PSF of view v (Supp. Note 2 section 1, symbol list).
Every plane orthogonal to the rotation axis is processed independently with
one 2D PSF per view.

Readings of points the paper leaves open:
  * all views use the same psi^t (simultaneous product, as printed);
  * each view's ratio is correlated with its own flipped PSF before the
    product over views;
  * division guard: r = phi / max(b, eps);
  * ZERO boundary = linear convolution cropped to the plane ("same"), which
    is what padding by the PSF size for the Fourier route implements
    (Supp. Table 1 caption); CIRCULAR = indices taken modulo the plane size;
  * odd K only, PSF centre at (R, R) with R = (K-1)/2, and
    P^*(i, j) = P(K-1-i, K-1-j);
  * initial estimate = per-plane mean over the pixels of all views (FP64);
  * rotation axis = the stack's middle axis: a stack [Z][Y][X] becomes
    planes [Y][Z][X].

Index convention used throughout (i, j in [0, K), di = i-R, dj = j-R):
    convolve : b(y, x) = sum_ij P[i, j] * img(y - di, x - dj)
    correlate: c(y, x) = sum_ij P[i, j] * img(y + di, x + dj)
"""

from __future__ import annotations

import numpy as np

ZERO = "zero"
CIRCULAR = "circular"

# Weighted MV-RL: where a view's weighted footprint n_v = w_v (*) P_v is below
# this floor the view leaves psi unchanged (its factor is 1).
NORM_FLOOR = 1e-6


def _check_psf(P: np.ndarray) -> int:
    P = np.asarray(P)
    if P.ndim != 2 or P.shape[0] != P.shape[1] or P.shape[0] % 2 != 1:
        raise ValueError("PSF must be K x K with odd K")
    return (P.shape[0] - 1) // 2


def flip_psf(P: np.ndarray) -> np.ndarray:
    """P^*(i, j) = P(K-1-i, K-1-j): the flipped PSF (Supp. Note 2, sec. 1)."""
    return np.asarray(P)[::-1, ::-1].copy()


def _shifted(img: np.ndarray, sy: int, sx: int, boundary: str) -> np.ndarray:
    """out(y, x) = img(y + sy, x + sx); zero or wrapped outside the plane."""
    H, W = img.shape
    if boundary == CIRCULAR:
        ys = (np.arange(H) + sy) % H
        xs = (np.arange(W) + sx) % W
        return img[np.ix_(ys, xs)]
    if boundary != ZERO:
        raise ValueError(f"unknown boundary {boundary!r}")
    out = np.zeros_like(img)
    y0, y1 = max(0, -sy), min(H, H - sy)
    x0, x1 = max(0, -sx), min(W, W - sx)
    if y0 < y1 and x0 < x1:
        out[y0:y1, x0:x1] = img[y0 + sy:y1 + sy, x0 + sx:x1 + sx]
    return out


def convolve(img: np.ndarray, P: np.ndarray, boundary: str = ZERO) -> np.ndarray:
    """Direct "same"-size 2D convolution psi * P by shift-and-add over K^2 taps.

    b(y, x) = sum_{i,j} P[i, j] img(y - (i-R), x - (j-R)).
    """
    R = _check_psf(P)
    img = np.asarray(img, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    out = np.zeros_like(img)
    K = P.shape[0]
    for i in range(K):
        for j in range(K):
            if P[i, j] != 0.0:
                out += P[i, j] * _shifted(img, -(i - R), -(j - R), boundary)
    return out


def correlate(img: np.ndarray, P: np.ndarray, boundary: str = ZERO) -> np.ndarray:
    """Direct "same"-size correlation with P, i.e. convolution with P^*.

    c(y, x) = sum_{i,j} P[i, j] img(y + (i-R), x + (j-R)).
    """
    R = _check_psf(P)
    img = np.asarray(img, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    out = np.zeros_like(img)
    K = P.shape[0]
    for i in range(K):
        for j in range(K):
            if P[i, j] != 0.0:
                out += P[i, j] * _shifted(img, i - R, j - R, boundary)
    return out


def _fft_conv(img: np.ndarray, P: np.ndarray, boundary: str) -> np.ndarray:
    """Convolution in the Fourier domain (Supp. Note 2, sec. 4).

    ZERO: the plane is padded by the PSF size so that the cyclic product of
    spectra equals the linear convolution (Supp. Table 1 caption), then the
    "same" window is cropped.  CIRCULAR: the PSF is wrapped onto the plane
    grid with its centre at the origin.
    """
    R = _check_psf(P)
    img = np.asarray(img, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    H, W = img.shape
    K = P.shape[0]
    if boundary == ZERO:
        Hp, Wp = H + K - 1, W + K - 1
        F = np.fft.rfft2(img, s=(Hp, Wp)) * np.fft.rfft2(P, s=(Hp, Wp))
        full = np.fft.irfft2(F, s=(Hp, Wp))
        return full[R:R + H, R:R + W].copy()
    if boundary == CIRCULAR:
        ker = np.zeros((H, W))
        for i in range(K):
            for j in range(K):
                ker[(i - R) % H, (j - R) % W] += P[i, j]
        F = np.fft.rfft2(img) * np.fft.rfft2(ker)
        return np.fft.irfft2(F, s=(H, W))
    raise ValueError(f"unknown boundary {boundary!r}")


def convolve_fft(img, P, boundary=ZERO):
    """Fourier-route psi * P; equal to :func:`convolve` up to rounding."""
    return _fft_conv(img, P, boundary)


def correlate_fft(img, P, boundary=ZERO):
    """Fourier-route correlation = convolution with the flipped PSF."""
    return _fft_conv(img, flip_psf(P), boundary)


def init_mean(phi: np.ndarray) -> np.ndarray:
    """Uniform initial estimate: per-plane mean of all views' pixels, FP64.

    phi: [V][P][H][W] -> [P] (one scalar per plane).
    """
    phi = np.asarray(phi, dtype=np.float64)
    return phi.mean(axis=(0, 2, 3))


def rl_step(psi, phi_planes, psfs, boundary=ZERO, eps=1e-6, route="direct",
            order="simultaneous", corr_kernels=None, weights=None):
    """One MV-RL update of one plane (Supp. Note 1, update equation).

    psi: [H][W]; phi_planes: [V][H][W]; psfs: [V][K][K].

    weights: optional [V][H][W] per-pixel view weights (the "weights" array
    of the memory table in Supp. Note 1).  The paper gives no formula for
    them; the reading taken is the EM update of a Poisson likelihood whose
    pixels count with weight w_v: each view's factor becomes
        c_v = ((w_v phi_v / (psi * P_v)) (*) P_v^*) / n_v,   n_v = w_v (*) P_v^*,
    and c_v = 1 where n_v < NORM_FLOOR (no weighted pixel in reach).  Unit
    weights with normalised PSFs under the circular boundary give n_v = 1,
    i.e. the unweighted update.

    order="simultaneous": every view's ratio uses the same psi and the
    views' corrections are multiplied, as the equation is printed.
    order="sequential": the views update psi one after another, each with
    the single-view factor of the same equation evaluated at the current
    psi (the sequential scheme of the multi-view RL literature the paper
    builds on, Supp. Note 2 sec. 1).
    """
    conv = convolve if route == "direct" else convolve_fft
    corr = correlate if route == "direct" else correlate_fft
    if corr_kernels is not None:
        # variant kernels X_v (Supp. Note 2 sec. 1): the ratio is convolved with
        # X_v, i.e. correlated with its flip
        xs = [flip_psf(x) for x in corr_kernels]
        corr_of = lambda img, v, b: corr(img, xs[v], b)  # noqa: E731
    else:
        corr_of = lambda img, v, b: corr(img, psfs[v], b)  # noqa: E731
    psi = np.asarray(psi, dtype=np.float64)

    def factor(v, psi_now):
        blur = conv(psi_now, psfs[v], boundary)
        data = np.asarray(phi_planes[v], dtype=np.float64)
        if weights is None:
            return corr_of(data / np.maximum(blur, eps), v, boundary)
        w = np.asarray(weights[v], dtype=np.float64)
        n = corr_of(w, v, boundary)
        c = corr_of(w * data / np.maximum(blur, eps), v, boundary)
        return np.where(n >= NORM_FLOOR, c / np.where(n >= NORM_FLOOR, n, 1.0), 1.0)

    if order == "sequential":
        for v in range(len(psfs)):
            psi = psi * factor(v, psi)
        return psi
    if order != "simultaneous":
        raise ValueError(f"unknown update order {order!r}")
    update = np.ones_like(psi)
    for v in range(len(psfs)):
        update *= factor(v, psi)
    return psi * update


def rl_planes(phi, psfs, iters, boundary=ZERO, eps=1e-6, psi0=None,
              route="direct", planes=None, order="simultaneous", corr_kernels=None, weights=None):
    """Plane-wise MV-RL over a stack of planes.

    phi:  [V][P][H][W] data (any real dtype; used as FP64)
    psfs: [V][K][K]
    psi0: None -> per-plane mean initial estimate; else [P][H][W]
    planes: optional iterable of plane indices to compute (others skipped;
            the result then holds only those planes, in that order)
    order:  "simultaneous" (default, as printed) or "sequential" (see rl_step)
    corr_kernels: optional [V][K][K] kernels X_v of a variant (oracle.variants);
            the ratio of view v is then convolved with X_v instead of being
            correlated with P_v
    weights: optional [V][P][H][W] per-pixel view weights (see rl_step)
    Returns the estimate after ``iters`` updates, FP64 [n][H][W].
    """
    phi = np.asarray(phi)
    V, P, H, W = phi.shape
    psfs = np.asarray(psfs, dtype=np.float64)
    if psfs.shape[0] != V:
        raise ValueError("one PSF per view")
    idx = list(range(P)) if planes is None else list(planes)
    means = None if psi0 is not None else init_mean(phi[:, idx])
    out = np.empty((len(idx), H, W))
    for n, p in enumerate(idx):
        if psi0 is None:
            psi = np.full((H, W), means[n])
        else:
            psi = np.asarray(psi0[p], dtype=np.float64).copy()
        for _ in range(iters):
            psi = rl_step(psi, phi[:, p], psfs, boundary, eps, route, order, corr_kernels,
                          None if weights is None else np.asarray(weights)[:, p])
        out[n] = psi
    return out


def reslice(stack: np.ndarray) -> np.ndarray:
    """Reslice a registered view stack into planes orthogonal to the
    rotation axis (Abstract; Fig. 1a).  [Z][Y][X] -> [Y][Z][X]."""
    return np.ascontiguousarray(np.transpose(np.asarray(stack), (1, 0, 2)))


def embed_padded(phi, pad):
    """Padded-domain estimate (Supp. Table 1 caption: data padded by the PSF
    size): planes [V][P][H][W] -> zero-padded planes [V][P][H+2pad][W+2pad]
    and weights that are 1 on the data and 0 in the padding."""
    phi = np.asarray(phi)
    V, P, H, W = phi.shape
    out = np.zeros((V, P, H + 2 * pad, W + 2 * pad), dtype=phi.dtype)
    out[:, :, pad:pad + H, pad:pad + W] = phi
    w = np.zeros(out.shape, dtype=np.float64)
    w[:, :, pad:pad + H, pad:pad + W] = 1.0
    return out, w


def crop_padded(est, pad):
    """[P][H+2pad][W+2pad] -> [P][H][W] (the data region of the estimate)."""
    est = np.asarray(est)
    return est[:, pad:est.shape[1] - pad, pad:est.shape[2] - pad].copy()
