"""Reverse-mode PSF gradient through unrolled MV-RL iterations, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The forward map is the update of Supp. Note 1 (see ``oracle.rl``) run for
T iterations from the per-plane mean; the loss is the Poisson negative
log-likelihood of each view's data under the forward-blurred estimate,

    y_v = P_v * psi^T,    L = sum_v sum_x [ y_v - phi_v log max(y_v, eps) ]

(constants dropped).  The paper has no calibration step: this is the
differentiation axis built on top of its iteration.  Gradients are taken
with respect to the raw PSF entries; projecting onto non-negative,
normalised kernels belongs to the optimiser step.  psi^0 (the data mean)
does not depend on the PSFs.

Reverse sweep for one iteration, given psibar = dL/dpsi^{t+1}:
    psibar_t   = psibar * prod_v c_v
    cbar_v     = psibar * psi^t * prod_{w != v} c_w
    rbar_v     = P_v * cbar_v              (adjoint of the correlation)
    Pbar_v[k] += sum_x cbar_v(x) r_v(x + d_k)
    bbar_v     = -rbar_v * phi_v / b_v^2   where b_v > eps, else 0
    psibar_t  += P_v (*) bbar_v            (adjoint of the convolution)
    Pbar_v[k] += sum_x bbar_v(x) psi^t(x - d_k)
with d_k = (i-R, j-R) the offset of tap k = (i, j).
"""

from __future__ import annotations

import numpy as np

from .rl import ZERO, _check_psf, _shifted, convolve, correlate


def _lag_sum_forward(g: np.ndarray, img: np.ndarray, K: int, boundary: str) -> np.ndarray:
    """G[i, j] = sum_x g(x) img(x - d_ij): derivative of convolve() wrt P."""
    R = (K - 1) // 2
    G = np.empty((K, K))
    for i in range(K):
        for j in range(K):
            G[i, j] = np.sum(g * _shifted(img, -(i - R), -(j - R), boundary))
    return G


def _lag_sum_backward(g: np.ndarray, img: np.ndarray, K: int, boundary: str) -> np.ndarray:
    """G[i, j] = sum_x g(x) img(x + d_ij): derivative of correlate() wrt P."""
    R = (K - 1) // 2
    G = np.empty((K, K))
    for i in range(K):
        for j in range(K):
            G[i, j] = np.sum(g * _shifted(img, i - R, j - R, boundary))
    return G


def poisson_nll(y: np.ndarray, phi: np.ndarray, eps: float) -> float:
    """sum_x [ y - phi log max(y, eps) ] (Poisson NLL without constants)."""
    y = np.asarray(y, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    return float(np.sum(y - phi * np.log(np.maximum(y, eps))))


def _forward(phi_plane, psfs, iters, boundary, eps):
    V, H, W = phi_plane.shape
    psi = np.full((H, W), np.asarray(phi_plane, dtype=np.float64).mean())
    tape = []
    for _ in range(iters):
        b = [convolve(psi, psfs[v], boundary) for v in range(V)]
        r = [phi_plane[v] / np.maximum(b[v], eps) for v in range(V)]
        c = [correlate(r[v], psfs[v], boundary) for v in range(V)]
        tape.append((psi, b, r, c))
        nxt = psi.copy()
        for v in range(V):
            nxt = nxt * c[v]
        psi = nxt
    return psi, tape


def rl_loss(phi, psfs, iters, boundary=ZERO, eps=1e-6) -> float:
    """Loss summed over planes: phi [V][P][H][W], psfs [V][K][K]."""
    phi = np.asarray(phi, dtype=np.float64)
    psfs = np.asarray(psfs, dtype=np.float64)
    V, P, H, W = phi.shape
    total = 0.0
    for p in range(P):
        psi, _ = _forward(phi[:, p], psfs, iters, boundary, eps)
        for v in range(V):
            total += poisson_nll(convolve(psi, psfs[v], boundary), phi[v, p], eps)
    return total


def rl_loss_and_psf_grad(phi, psfs, iters, boundary=ZERO, eps=1e-6):
    """Loss and dL/dP_v for all views; sums over planes.

    Returns (loss, grad [V][K][K], psi_T [P][H][W]).
    """
    phi = np.asarray(phi, dtype=np.float64)
    psfs = np.asarray(psfs, dtype=np.float64)
    V, P, H, W = phi.shape
    K = psfs.shape[1]
    _check_psf(psfs[0])
    grad = np.zeros((V, K, K))
    loss = 0.0
    psis = np.empty((P, H, W))
    for p in range(P):
        ph = phi[:, p]
        psi_T, tape = _forward(ph, psfs, iters, boundary, eps)
        psis[p] = psi_T
        # terminal data fit
        psibar = np.zeros((H, W))
        for v in range(V):
            y = convolve(psi_T, psfs[v], boundary)
            loss += poisson_nll(y, ph[v], eps)
            ybar = np.where(y > eps, 1.0 - ph[v] / np.maximum(y, eps), 1.0)
            psibar += correlate(ybar, psfs[v], boundary)
            grad[v] += _lag_sum_forward(ybar, psi_T, K, boundary)
        # unrolled iterations, last first
        for psi, b, r, c in reversed(tape):
            prod_all = np.ones((H, W))
            for v in range(V):
                prod_all = prod_all * c[v]
            nbar = psibar * prod_all
            for v in range(V):
                others = np.ones((H, W))
                for w in range(V):
                    if w != v:
                        others = others * c[w]
                cbar = psibar * psi * others
                rbar = convolve(cbar, psfs[v], boundary)
                grad[v] += _lag_sum_backward(cbar, r[v], K, boundary)
                bbar = np.where(b[v] > eps, -rbar * ph[v] / np.maximum(b[v], eps) ** 2, 0.0)
                nbar = nbar + correlate(bbar, psfs[v], boundary)
                grad[v] += _lag_sum_forward(bbar, psi, K, boundary)
            psibar = nbar
    return loss, grad, psis
