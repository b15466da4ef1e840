"""Seeded synthetic inputs shaped like the paper's light-sheet data.

This module makes inputs only: ground-truth blob images, sampled Gaussian
PSFs and noisy view data.  It holds none of the deconvolution's arithmetic
(the forward blur used to make the data is a library call:
``scipy.signal.fftconvolve`` on the host, ``torch.nn.functional.conv1d``
on a device), so both the CUDA path and the FP64 oracle can be fed from it.

Recipes (Supp. Fig. 2 caption: views blurred by PSFs elongated along z and x;
Validation section: axial sigma about 8 px, lateral 1.5-1.8 px):
  * truth = background + sum of Gaussian blobs (sigma 1 px, peak amplitude
    uniform in [100, 1000]), centres uniform in the plane / volume;
  * PSF of a view = sampled 2D Gaussian exp(-dr^2/2sr^2 - dc^2/2sc^2) at
    integer offsets from the centre of a K x K grid, normalised to sum 1 in
    FP64 and cast to FP32.  A view turned by 90 degrees swaps (sr, sc);
  * view data = truth blurred plane-wise with the view's PSF (zero outside
    the plane), Poisson noise, clipped to [0, 65535].
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def gaussian_psf(K: int, sigma_rows: float, sigma_cols: float,
                 angle_deg: float = 0.0) -> np.ndarray:
    """Sampled, normalised K x K Gaussian PSF (FP32).

    ``angle_deg`` turns the PSF in the plane; multiples of 90 degrees are
    exact swaps/flips of the axes, other angles rotate the covariance.
    """
    if K % 2 != 1 or K < 1:
        raise ValueError("K must be odd and positive")
    R = (K - 1) // 2
    d = np.arange(-R, R + 1, dtype=np.float64)
    dr, dc = np.meshgrid(d, d, indexing="ij")
    a = angle_deg % 360.0
    if a in (0.0, 180.0):
        sr, sc = sigma_rows, sigma_cols
        g = np.exp(-dr**2 / (2 * sr**2) - dc**2 / (2 * sc**2))
    elif a in (90.0, 270.0):
        sr, sc = sigma_cols, sigma_rows
        g = np.exp(-dr**2 / (2 * sr**2) - dc**2 / (2 * sc**2))
    else:
        t = math.radians(a)
        u = math.cos(t) * dr + math.sin(t) * dc
        w = -math.sin(t) * dr + math.cos(t) * dc
        g = np.exp(-u**2 / (2 * sigma_rows**2) - w**2 / (2 * sigma_cols**2))
    g /= g.sum()
    return g.astype(np.float32)


def gaussian_1d(K: int, sigma: float) -> np.ndarray:
    """Normalised sampled 1D Gaussian (FP64), used to blur volumes."""
    R = (K - 1) // 2
    d = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-d**2 / (2 * sigma**2))
    return g / g.sum()


def blob_plane(H: int, W: int, n_blobs: int, rng: np.random.Generator,
               sigma: float = 1.0, amp=(100.0, 1000.0),
               background: float = 10.0) -> np.ndarray:
    """FP64 [H][W] truth: background + Gaussian blobs."""
    cy = rng.uniform(0, H, n_blobs)
    cx = rng.uniform(0, W, n_blobs)
    A = rng.uniform(amp[0], amp[1], n_blobs)
    img = np.full((H, W), background, dtype=np.float64)
    foot = int(math.ceil(4 * sigma))
    for y0, x0, a in zip(cy, cx, A):
        ys = np.arange(max(0, int(y0) - foot), min(H, int(y0) + foot + 2))
        xs = np.arange(max(0, int(x0) - foot), min(W, int(x0) + foot + 2))
        gy = np.exp(-(ys + 0.0 - y0) ** 2 / (2 * sigma**2))
        gx = np.exp(-(xs + 0.0 - x0) ** 2 / (2 * sigma**2))
        img[np.ix_(ys, xs)] += a * np.outer(gy, gx)
    return img


def blur_plane_library(truth: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Zero-boundary "same" blur with scipy (library routine, FP64)."""
    from scipy.signal import fftconvolve
    out = fftconvolve(truth, np.asarray(psf, dtype=np.float64), mode="same")
    return np.maximum(out, 0.0)


@dataclass
class PlaneCase:
    truth: np.ndarray        # [P][H][W] float64
    psfs: np.ndarray         # [V][K][K] float32
    phi: np.ndarray          # [V][P][H][W] float32 or uint16
    iters: int
    eps: float
    boundary: str


def plane_case(seed: int = 0, H: int = 128, W: int = 128, n_planes: int = 1,
               n_blobs: int = 200, K: int = 17, sigma_axial: float = 6.0,
               sigma_lateral: float = 1.5, angles=(0.0, 90.0), iters: int = 10,
               eps: float = 1e-6, boundary: str = "zero", dtype=np.float32,
               noise: bool = True) -> PlaneCase:
    """Planes of blobs seen by len(angles) views (default: the 2-view,
    one 128x128 plane, 17x17 PSF case with sigma (1.5, 6) px)."""
    rng = np.random.default_rng(seed)
    psfs = np.stack([gaussian_psf(K, sigma_axial, sigma_lateral, a) for a in angles])
    truth = np.stack([blob_plane(H, W, n_blobs, rng) for _ in range(n_planes)])
    phi = np.empty((len(angles), n_planes, H, W), dtype=dtype)
    for v in range(len(angles)):
        for p in range(n_planes):
            lam = blur_plane_library(truth[p], psfs[v])
            img = rng.poisson(lam).astype(np.float64) if noise else lam
            phi[v, p] = np.clip(img, 0, 65535).astype(dtype)
    return PlaneCase(truth, psfs, phi, iters, eps, boundary)


def volume_stacks(Z: int, Y: int, X: int, K: int, sigma_axial: float,
                  sigma_lateral: float, angles, density: float, seed: int,
                  device="cpu", background: float = 10.0):
    """Registered view stacks [V][Z][Y][X] uint16 (torch) of 3D blobs.

    Each view is the truth blurred plane-wise in the (z, x) planes that are
    orthogonal to the rotation axis y, by that view's axis-aligned PSF, with
    Poisson noise.  Returns (stacks, psfs [V][K][K] float32 numpy).
    """
    import torch
    import torch.nn.functional as F

    rng = np.random.default_rng(seed)
    n = int(round(density * Z * Y * X))
    cz = rng.uniform(0, Z, n)
    cy = rng.uniform(0, Y, n)
    cx = rng.uniform(0, X, n)
    A = rng.uniform(100.0, 1000.0, n)
    dev = torch.device(device)
    truth = torch.full((Z * Y * X,), background, dtype=torch.float32, device=dev)
    foot = 4
    off = torch.arange(-foot, foot + 1, device=dev)
    oz, oy, ox = torch.meshgrid(off, off, off, indexing="ij")
    oz, oy, ox = oz.reshape(1, -1), oy.reshape(1, -1), ox.reshape(1, -1)
    chunk = 1 << 16
    for s in range(0, n, chunk):
        tz = torch.as_tensor(cz[s:s + chunk], device=dev).reshape(-1, 1)
        ty = torch.as_tensor(cy[s:s + chunk], device=dev).reshape(-1, 1)
        tx = torch.as_tensor(cx[s:s + chunk], device=dev).reshape(-1, 1)
        ta = torch.as_tensor(A[s:s + chunk], device=dev).reshape(-1, 1)
        iz = tz.floor().long() + oz
        iy = ty.floor().long() + oy
        ix = tx.floor().long() + ox
        val = ta * torch.exp(-((iz - tz) ** 2 + (iy - ty) ** 2 + (ix - tx) ** 2) / 2.0)
        ok = (iz >= 0) & (iz < Z) & (iy >= 0) & (iy < Y) & (ix >= 0) & (ix < X)
        lin = (iz * Y + iy) * X + ix
        truth.index_put_((lin[ok],), val[ok].float(), accumulate=True)
    truth = truth.reshape(Z, Y, X)

    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    R = (K - 1) // 2
    psfs, stacks = [], []
    for a in angles:
        psfs.append(gaussian_psf(K, sigma_axial, sigma_lateral, a))
        if a % 90.0 != 0.0:
            # oblique view: blur every (z, x) plane with the full 2D PSF
            ker = torch.as_tensor(psfs[-1], dtype=torch.float32, device=dev).flip(0, 1).reshape(1, 1, K, K)
            t = truth.permute(1, 0, 2).reshape(Y, 1, Z, X)
            t = F.conv2d(t, ker, padding=R).reshape(Y, Z, X).permute(1, 0, 2).contiguous().clamp_(min=0)
            noisy = torch.poisson(t, generator=gen).clamp_(0, 65535)
            stacks.append(noisy.to(torch.int32).to(torch.uint16))
            del t, noisy
            continue
        rot = (a % 180.0) == 90.0
        s_rows, s_cols = (sigma_lateral, sigma_axial) if rot else (sigma_axial, sigma_lateral)
        kr = torch.as_tensor(gaussian_1d(K, s_rows), dtype=torch.float32, device=dev)
        kc = torch.as_tensor(gaussian_1d(K, s_cols), dtype=torch.float32, device=dev)
        # along x (plane columns)
        t = F.conv1d(truth.reshape(Z * Y, 1, X), kc.reshape(1, 1, K), padding=R)
        t = t.reshape(Z, Y, X)
        # along z (plane rows)
        t = t.permute(1, 2, 0).reshape(Y * X, 1, Z)
        t = F.conv1d(t, kr.reshape(1, 1, K), padding=R)
        t = t.reshape(Y, X, Z).permute(2, 0, 1).contiguous().clamp_(min=0)
        noisy = torch.poisson(t, generator=gen).clamp_(0, 65535)
        stacks.append(noisy.to(torch.int32).to(torch.uint16))
        del t, noisy
    return torch.stack(stacks), np.stack(psfs)


def uneven_volumes(n: int, seed: int, side=(96, 768), planes=(16, 256), views=(2, 6), psf=(9, 41),
                   sigma_lateral=(1.0, 2.0), sigma_axial=(4.0, 12.0), iters=(5, 20), density=5e-5,
                   device="cpu", only=None, shapes_only=False):
    """Independent volumes of uneven shape for batched runs.

    Volume i uses seed + i: square planes of side U{side}, U{planes} planes,
    U{views} views at angles k*180/V degrees, an odd PSF side U{psf},
    Gaussian sigmas (U(lateral), U(axial)) px and U{iters} iterations.
    Returns a list of dicts (stacks [V][H][P][W] uint16 on `device`, psfs,
    iters, shape).  `only`: indices of the volumes to return (the others are
    skipped; a volume depends on seed + i alone).  shapes_only: no data
    (stacks and psfs None)."""
    out = []
    keep = None if only is None else set(only)
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        s = int(rng.integers(side[0], side[1] + 1))
        p = int(rng.integers(planes[0], planes[1] + 1))
        v = int(rng.integers(views[0], views[1] + 1))
        k = int(rng.integers((psf[0] - 1) // 2, (psf[1] - 1) // 2 + 1)) * 2 + 1
        sl = float(rng.uniform(*sigma_lateral))
        sa = float(rng.uniform(*sigma_axial))
        it = int(rng.integers(iters[0], iters[1] + 1))
        angles = tuple(180.0 * j / v for j in range(v))
        if keep is not None and i not in keep:
            continue
        if shapes_only:
            stacks = psfs = None
        else:
            stacks, psfs = volume_stacks(s, p, s, k, sa, sl, angles, density, seed=seed + i, device=device)
        out.append({"stacks": stacks, "psfs": psfs, "iters": it, "H": s, "W": s, "P": p, "views": v, "K": k})
    return out


def volume3d_case(Y: int, Z: int, X: int, K: int, sigma_axial: float, sigma_lateral: float, sigma_y: float,
                  angles=(0.0, 90.0), n_blobs: int = 100, seed: int = 0, background: float = 10.0,
                  noise: bool = True):
    """Views of a 3D blob volume blurred in 3D: view v's PSF is
    a(y) P_v(z, x) with P_v the in-plane Gaussian PSF (sigma_axial,
    sigma_lateral, turned by the view's angle) and a a Gaussian of sigma_y
    along the rotation axis y (the plane index), odd length covering
    +-3 sigma_y; Poisson noise.  Plane layout.  Returns a dict with truth
    [Y][Z][X] (FP64), phi [V][Y][Z][X] (uint16), psfs [V][K][K] (FP32),
    axial [V][Ka] (FP32)."""
    from scipy.ndimage import convolve1d
    from scipy.signal import fftconvolve

    rng = np.random.default_rng(seed)
    truth = np.full((Y, Z, X), background, dtype=np.float64)
    cy, cz, cx = rng.uniform(0, Y, n_blobs), rng.uniform(0, Z, n_blobs), rng.uniform(0, X, n_blobs)
    A = rng.uniform(100.0, 1000.0, n_blobs)
    yy, zz, xx = np.meshgrid(np.arange(Y), np.arange(Z), np.arange(X), indexing="ij")
    for y0, z0, x0, a in zip(cy, cz, cx, A):
        truth += a * np.exp(-((yy - y0) ** 2 + (zz - z0) ** 2 + (xx - x0) ** 2) / 2.0)
    Ra = max(1, int(math.ceil(3 * sigma_y)))
    axial = gaussian_1d(2 * Ra + 1, sigma_y)
    psfs, phis = [], []
    for ang in angles:
        P = gaussian_psf(K, sigma_axial, sigma_lateral, ang)
        psfs.append(P)
        planes = np.stack([fftconvolve(truth[y], P.astype(np.float64), mode="same") for y in range(Y)])
        blurred = convolve1d(planes, axial, axis=0, mode="constant", cval=0.0)
        img = rng.poisson(np.maximum(blurred, 0)) if noise else np.round(blurred)
        phis.append(np.clip(img, 0, 65535).astype(np.uint16))
    return {"truth": truth, "phi": np.stack(phis), "psfs": np.stack(psfs).astype(np.float32),
            "axial": np.stack([axial] * len(angles)).astype(np.float32)}
