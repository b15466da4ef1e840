"""Pins for the FP64 oracle against things other than itself.

Each check is chosen so that a plausible mistake in the oracle (a flipped
PSF, an off-by-one centre, a dropped view, a wrong boundary, a wrong sign in
the adjoint) fails at least one of them:

  brute force   quadruple-loop convolution on tiny planes
  library       scipy.signal.convolve2d / correlate2d, numpy FFT
  closed forms  hand-derived one-iteration results, Gaussian*Gaussian
  invariants    flux conservation (V=1), fixed point, adjointness, symmetry
  textbook RL   matrix form psi <- psi * prod_v A_v^T (phi_v / A_v psi)
  gradients     FP64 central finite differences
"""

import json
import os

import numpy as np
import pytest
from scipy.signal import convolve2d, correlate2d

import oracle
from paper_1503_07998_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_convolve(img, P, boundary):
    H, W = img.shape
    K = P.shape[0]
    R = K // 2
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            s = 0.0
            for i in range(K):
                for j in range(K):
                    yy, xx = y - (i - R), x - (j - R)
                    if boundary == "circular":
                        yy, xx = yy % H, xx % W
                    elif not (0 <= yy < H and 0 <= xx < W):
                        continue
                    s += P[i, j] * img[yy, xx]
            out[y, x] = s
    return out


def conv_matrix(P, H, W, boundary):
    """A with (A psi)(y,x) = sum_ij P[i,j] psi(y-di, x-dj), built entrywise."""
    K = P.shape[0]
    R = K // 2
    A = np.zeros((H * W, H * W))
    for y in range(H):
        for x in range(W):
            for i in range(K):
                for j in range(K):
                    yy, xx = y - (i - R), x - (j - R)
                    if boundary == "circular":
                        yy, xx = yy % H, xx % W
                    elif not (0 <= yy < H and 0 <= xx < W):
                        continue
                    A[y * W + x, yy * W + xx] += P[i, j]
    return A


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("shape,K", [((7, 5), 3), ((8, 8), 5), ((6, 9), 1), ((5, 5), 5)])
def test_convolve_matches_brute_force_and_scipy(boundary, shape, K):
    rng = np.random.default_rng(1)
    img = rng.random(shape)
    P = rng.random((K, K))  # deliberately not symmetric
    b = oracle.convolve(img, P, boundary)
    np.testing.assert_allclose(b, brute_convolve(img, P, boundary), rtol=1e-13, atol=1e-13)
    sb = "fill" if boundary == "zero" else "wrap"
    np.testing.assert_allclose(b, convolve2d(img, P, mode="same", boundary=sb), rtol=1e-12, atol=1e-13)
    c = oracle.correlate(img, P, boundary)
    np.testing.assert_allclose(c, correlate2d(img, P, mode="same", boundary=sb), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(c, brute_convolve(img, oracle.flip_psf(P), boundary), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("shape,K", [((32, 40), 7), ((17, 23), 9), ((16, 16), 15)])
def test_fft_route_equals_direct_route(boundary, shape, K):
    rng = np.random.default_rng(2)
    img = rng.random(shape)
    P = rng.random((K, K))
    for f_direct, f_fft in ((oracle.convolve, oracle.convolve_fft),
                            (oracle.correlate, oracle.correlate_fft)):
        d = f_direct(img, P, boundary)
        f = f_fft(img, P, boundary)
        assert np.linalg.norm(d - f) <= 1e-12 * np.linalg.norm(d)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_correlate_is_adjoint_of_convolve(boundary):
    rng = np.random.default_rng(3)
    x = rng.random((11, 13))
    y = rng.random((11, 13))
    P = rng.random((5, 5))
    lhs = np.sum(oracle.convolve(x, P, boundary) * y)
    rhs = np.sum(x * oracle.correlate(y, P, boundary))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_hand_derived_one_iteration():
    """Golden values worked out by hand from the update equation."""
    with open(os.path.join(GOLDEN, "hand_1x3.json")) as f:
        case = json.load(f)
    phi = np.array(case["phi"], dtype=np.float64)[:, None]      # [V][P=1][H][W]
    psf = np.array(case["psf"], dtype=np.float64)
    out = oracle.rl_planes(phi, psf, case["iters"], boundary=case["boundary"], eps=1e-6)
    expected = np.array([[n / d for n, d in row] for row in case["expected"]])
    np.testing.assert_allclose(out[0], expected, rtol=1e-14)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_delta_psf_one_iteration(boundary):
    """Delta PSF: psi^1 = psi0^(1-V) prod_v phi_v (exactly phi for V = 1)."""
    rng = np.random.default_rng(4)
    for V, K in ((1, 1), (1, 5), (2, 3), (3, 1)):
        phi = rng.uniform(5, 50, size=(V, 2, 6, 7))
        delta = np.zeros((K, K))
        delta[K // 2, K // 2] = 1.0
        psfs = np.stack([delta] * V)
        out = oracle.rl_planes(phi, psfs, 1, boundary=boundary)
        psi0 = oracle.init_mean(phi)
        expect = np.prod(phi, axis=0) * psi0[:, None, None] ** (1 - V)
        np.testing.assert_allclose(out, expect, rtol=1e-13)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_flux_conserved_single_view(boundary):
    """V = 1: sum psi^{t+1} = sum phi for every t (adjoint pair, b > eps)."""
    rng = np.random.default_rng(5)
    phi = rng.uniform(1, 100, size=(1, 1, 12, 10))
    P = rng.random((5, 5)) + 0.05     # positive, non-symmetric, not normalised
    psi = np.full((12, 10), phi.mean())
    for _ in range(4):
        psi = oracle.rl_step(psi, phi[:, 0], P[None], boundary)
        assert abs(psi.sum() - phi.sum()) <= 1e-11 * phi.sum()


def test_fixed_point_noise_free_circular():
    """phi_v = P_v * psi exactly and psi0 = psi: psi stays psi (any V)."""
    rng = np.random.default_rng(6)
    psi_true = rng.uniform(10, 100, size=(16, 12))
    psfs = np.stack([synth.gaussian_psf(5, 2.0, 0.7, a).astype(np.float64) for a in (0, 90, 45)])
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = np.stack([convolve2d(psi_true, P, mode="same", boundary="wrap") for P in psfs])[:, None]
    out = oracle.rl_planes(phi, psfs, 5, boundary="circular", psi0=psi_true[None])
    np.testing.assert_allclose(out[0], psi_true, rtol=1e-12)


def test_gaussian_closed_form_and_constant():
    """Sampled Gaussian (s1) blurred by a normalised sampled Gaussian PSF (s2)
    is close to a Gaussian of variance s1^2 + s2^2, centred at the same place."""
    H = W = 64
    s1, s2 = 4.0, 2.0
    yy, xx = np.mgrid[0:H, 0:W]
    c = 31.0
    img = np.exp(-((yy - c) ** 2 + (xx - c) ** 2) / (2 * s1**2))
    P = synth.gaussian_psf(21, s2, s2).astype(np.float64)
    P /= P.sum()
    s = np.sqrt(s1**2 + s2**2)
    expect = (s1**2 / s**2) * np.exp(-((yy - c) ** 2 + (xx - c) ** 2) / (2 * s**2))
    out = oracle.convolve(img, P, "zero")
    assert np.max(np.abs(out - expect)) < 1e-3 * expect.max()
    assert np.unravel_index(np.argmax(out), out.shape) == (31, 31)
    const = np.full((9, 11), 7.5)
    np.testing.assert_allclose(oracle.convolve(const, P[8:13, 8:13] / P[8:13, 8:13].sum(), "circular"),
                               const, rtol=1e-14)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_matches_textbook_matrix_rl(boundary):
    """psi <- psi * prod_v A_v^T (phi_v / max(A_v psi, eps)) with A_v built
    entry by entry: pins the grouping (ratio per view, correlate, product)."""
    rng = np.random.default_rng(7)
    H, W, V, K = 5, 6, 3, 3
    psfs = rng.random((V, K, K)) + 0.1
    phi = rng.uniform(1, 20, size=(V, 1, H, W))
    A = [conv_matrix(psfs[v], H, W, boundary) for v in range(V)]
    psi = np.full(H * W, phi.mean())
    for _ in range(3):
        upd = np.ones(H * W)
        for v in range(V):
            upd *= A[v].T @ (phi[v, 0].ravel() / np.maximum(A[v] @ psi, 1e-6))
        psi = psi * upd
    out = oracle.rl_planes(phi, psfs, 3, boundary=boundary)
    np.testing.assert_allclose(out[0].ravel(), psi, rtol=1e-12)


def test_symmetries():
    rng = np.random.default_rng(8)
    phi = rng.uniform(1, 30, size=(2, 1, 9, 7))
    psfs = rng.random((2, 5, 5)) + 0.1
    a = oracle.rl_planes(phi, psfs, 3)
    b = oracle.rl_planes(phi[::-1], psfs[::-1], 3)          # swap the views
    np.testing.assert_allclose(a, b, rtol=1e-13)
    c = oracle.rl_planes(np.swapaxes(phi, 2, 3), np.swapaxes(psfs, 1, 2), 3)
    np.testing.assert_allclose(c[0], a[0].T, rtol=1e-13)     # transpose everything


def test_init_mean_and_fft_route_planes():
    rng = np.random.default_rng(9)
    phi = rng.uniform(0, 10, size=(3, 4, 5, 6))
    m = oracle.init_mean(phi)
    for p in range(4):
        assert abs(m[p] - sum(phi[v, p].sum() for v in range(3)) / (3 * 30)) < 1e-12
    psfs = rng.random((3, 3, 3)) + 0.1
    d = oracle.rl_planes(phi + 1, psfs, 2, route="direct")
    f = oracle.rl_planes(phi + 1, psfs, 2, route="fft")
    np.testing.assert_allclose(f, d, rtol=1e-11)
    sub = oracle.rl_planes(phi + 1, psfs, 2, planes=[3, 1])
    np.testing.assert_allclose(sub, d[[3, 1]], rtol=1e-14)


def test_reslice_is_the_axis_swap():
    stack = np.arange(4 * 3 * 5).reshape(4, 3, 5)
    out = oracle.reslice(stack)
    assert out.shape == (3, 4, 5)
    for z in range(4):
        for y in range(3):
            for x in range(5):
                assert out[y, z, x] == stack[z, y, x]


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_psf_gradient_matches_central_differences(boundary):
    rng = np.random.default_rng(10)
    V, H, W, K, T = 2, 7, 6, 3, 3
    psfs = rng.random((V, K, K)) + 0.2
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = rng.uniform(2, 40, size=(V, 2, H, W))
    loss, grad, _ = oracle.rl_loss_and_psf_grad(phi, psfs, T, boundary)
    assert abs(loss - oracle.rl_loss(phi, psfs, T, boundary)) <= 1e-12 * abs(loss)
    h = 1e-5
    fd = np.zeros_like(grad)
    for v in range(V):
        for i in range(K):
            for j in range(K):
                p = psfs.copy(); p[v, i, j] += h
                m = psfs.copy(); m[v, i, j] -= h
                fd[v, i, j] = (oracle.rl_loss(phi, p, T, boundary) - oracle.rl_loss(phi, m, T, boundary)) / (2 * h)
    assert np.linalg.norm(grad - fd) <= 1e-6 * np.linalg.norm(fd)


@pytest.mark.slow
def test_psf_gradient_at_the_calibration_setting():
    """The PSF-calibration setting itself: two views of blob data made with
    sigma (1.5, 7) px, free 31x31 PSFs at sigma (1.2, 5), 10 unrolled
    iterations, a 32x32 crop; the reverse-sweep gradient against FP64
    central differences with h = 1e-4 on 48 seeded taps of both views.  The
    finite differences carry an O(h^2) truncation error: halving h must cut
    the gap to the gradient about four-fold, so what is left is truncation
    and not a wrong term (a dropped or wrong term would leave a gap that does
    not shrink with h)."""
    case = synth.plane_case(seed=71, H=32, W=32, n_planes=1, n_blobs=6, K=31, sigma_axial=7.0,
                            sigma_lateral=1.5, dtype=np.float64)
    psfs = np.stack([synth.gaussian_psf(31, 5.0, 1.2, a) for a in (0, 90)]).astype(np.float64)
    _, grad, _ = oracle.rl_loss_and_psf_grad(case.phi, psfs, 10, "zero")
    taps = np.random.default_rng(5).choice(psfs.size, 48, replace=False)

    def fd(h):
        out = []
        for k in taps:
            v, i, j = np.unravel_index(k, psfs.shape)
            p = psfs.copy(); p[v, i, j] += h
            m = psfs.copy(); m[v, i, j] -= h
            out.append((oracle.rl_loss(case.phi, p, 10, "zero") - oracle.rl_loss(case.phi, m, 10, "zero")) / (2 * h))
        return np.array(out)

    g = grad.reshape(-1)[taps]
    gap1 = np.linalg.norm(fd(1e-4) - g) / np.linalg.norm(g)
    gap2 = np.linalg.norm(fd(5e-5) - g) / np.linalg.norm(g)
    assert gap1 <= 1e-5, (gap1, gap2)
    assert 2.5 <= gap1 / gap2 <= 6.0, (gap1, gap2)


def test_gradient_zero_iterations_is_data_fit_only():
    """T = 0: L = sum_v NLL(P_v * mean, phi_v) and its gradient has the
    closed form dL/dP_v[i,j] = sum_x (1 - phi/y)(x) * m * [x - d_ij in plane]."""
    rng = np.random.default_rng(11)
    V, H, W, K = 1, 5, 5, 3
    psfs = rng.random((V, K, K)) + 0.1
    phi = rng.uniform(1, 9, size=(V, 1, H, W))
    loss, grad, _ = oracle.rl_loss_and_psf_grad(phi, psfs, 0, "circular")
    m = phi.mean()
    y = np.full((H, W), m * psfs[0].sum())          # circular: P * const = const * sum P
    assert abs(loss - np.sum(y - phi[0, 0] * np.log(y))) < 1e-10 * abs(loss)
    expect = np.full((K, K), np.sum(1 - phi[0, 0] / y) * m)
    np.testing.assert_allclose(grad[0], expect, rtol=1e-10)


def test_gaussian_psf_recipe():
    P = synth.gaussian_psf(17, 6.0, 1.5)
    assert P.dtype == np.float32 and P.shape == (17, 17)
    assert abs(P.astype(np.float64).sum() - 1) < 1e-6
    np.testing.assert_allclose(synth.gaussian_psf(17, 6.0, 1.5, 90.0), P.T, rtol=1e-7)
    assert np.argmax(P) == 8 * 17 + 8
    # elongated along rows (axial) for the first view
    assert P[0, 8] > P[8, 0]


@pytest.mark.parametrize("name", ["small_zero", "small_circular"])
def test_golden_fixtures_reproduce(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        case = json.load(f)
    out = oracle.rl_planes(np.array(case["phi"], dtype=np.float64),
                           np.array(case["psf"], dtype=np.float64),
                           case["iters"], boundary=case["boundary"], eps=case["eps"])
    np.testing.assert_allclose(out, np.array(case["expected"]), rtol=1e-13)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_sequential_order_matches_textbook_and_conserves_last_view_flux(boundary):
    """Sequential order: each view applies a single-view RL step to the
    current estimate, so after a full iteration sum(psi) = sum(phi_last)."""
    rng = np.random.default_rng(12)
    H, W, V, K = 5, 6, 3, 3
    psfs = rng.random((V, K, K)) + 0.1
    phi = rng.uniform(1, 20, size=(V, 1, H, W))
    A = [conv_matrix(psfs[v], H, W, boundary) for v in range(V)]
    psi = np.full(H * W, phi.mean())
    for _ in range(3):
        for v in range(V):
            psi = psi * (A[v].T @ (phi[v, 0].ravel() / np.maximum(A[v] @ psi, 1e-6)))
        assert abs(psi.sum() - phi[V - 1].sum()) <= 1e-11 * phi[V - 1].sum()
    out = oracle.rl_planes(phi, psfs, 3, boundary=boundary, order="sequential")
    np.testing.assert_allclose(out[0].ravel(), psi, rtol=1e-12)
    one = oracle.rl_planes(phi[:1], psfs[:1], 3, boundary=boundary, order="sequential")
    np.testing.assert_allclose(one, oracle.rl_planes(phi[:1], psfs[:1], 3, boundary=boundary), rtol=1e-14)


def brute_conv_same(A, B):
    """c[i, j] = sum_{a,b} A[a, b] B[i+R-a, j+R-b] over in-range indices."""
    K = A.shape[0]
    R = (K - 1) // 2
    c = np.zeros((K, K))
    for i in range(K):
        for j in range(K):
            for a in range(K):
                for b in range(K):
                    m, n = i + R - a, j + R - b
                    if 0 <= m < K and 0 <= n < K:
                        c[i, j] += A[a, b] * B[m, n]
    return c


def test_variant_kernels_brute_force():
    """Each X_v written out with loops from its definition (Supp. Note 2
    sec. 1, readings in oracle.variants) on random non-symmetric PSFs."""
    rng = np.random.default_rng(13)
    V, K = 3, 5
    psfs = rng.random((V, K, K)) + 0.05
    fl = psfs[:, ::-1, ::-1]
    for variant in oracle.VARIANTS:
        X = oracle.correlation_kernels(psfs, variant)
        for v in range(V):
            x = fl[v].copy()
            for w in range(V):
                if w == v:
                    continue
                if variant == "efficient_bayesian":
                    x = x * brute_conv_same(brute_conv_same(fl[v], psfs[w]), fl[w])
                elif variant == "optimization_1":
                    x = x * brute_conv_same(fl[v], psfs[w])
                elif variant == "optimization_2":
                    x = x * fl[w]
            np.testing.assert_allclose(X[v], x / x.sum(), rtol=1e-12, err_msg=variant)


def test_variant_kernels_gaussian_closed_form():
    """Isotropic Gaussians (sigma_1, sigma_2), wide support: convolutions add
    variances and products add precisions, so X_1 of each variant is a
    Gaussian of known width."""
    K, s1, s2 = 41, 1.6, 2.2
    r = np.arange(K) - (K - 1) / 2
    r2 = r[:, None] ** 2 + r[None, :] ** 2

    def g(s):
        e = np.exp(-r2 / (2 * s * s))
        return e / e.sum()

    psfs = np.stack([g(s1), g(s2)])
    widths = {
        "independent": [s1 * s1],
        "efficient_bayesian": [s1 * s1, s1 * s1 + 2 * s2 * s2],
        "optimization_1": [s1 * s1, s1 * s1 + s2 * s2],
        "optimization_2": [s1 * s1, s2 * s2],
    }
    for variant, variances in widths.items():
        var = 1.0 / sum(1.0 / q for q in variances)
        X = oracle.correlation_kernels(psfs, variant)
        np.testing.assert_allclose(X[0], g(np.sqrt(var)), atol=1e-9, err_msg=variant)


@pytest.mark.parametrize("variant", ["efficient_bayesian", "optimization_1", "optimization_2"])
def test_variants_single_view_delta_and_fixed_point(variant):
    """One view: every variant is plain RL.  Delta PSFs: X = delta.  Noise-free
    circular data: psi stays a fixed point (X_v has unit sum)."""
    rng = np.random.default_rng(14)
    phi1 = rng.uniform(1, 30, size=(1, 2, 9, 8))
    P1 = rng.random((1, 5, 5)) + 0.1
    X1 = oracle.correlation_kernels(P1, variant)
    np.testing.assert_allclose(X1[0], P1[0, ::-1, ::-1] / P1[0].sum(), rtol=1e-14)
    P1n = P1 / P1.sum()
    np.testing.assert_allclose(oracle.rl_planes(phi1, P1n, 3, corr_kernels=X1), oracle.rl_planes(phi1, P1n, 3),
                               rtol=1e-13)
    delta = np.zeros((3, 5, 5))
    delta[:, 2, 2] = 1.0
    np.testing.assert_allclose(oracle.correlation_kernels(delta, variant), delta, atol=0)
    psi_true = rng.uniform(10, 100, size=(16, 12))
    psfs = np.stack([synth.gaussian_psf(5, 2.0, 0.7, a).astype(np.float64) for a in (0, 90, 45)])
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    phi = np.stack([convolve2d(psi_true, P, mode="same", boundary="wrap") for P in psfs])[:, None]
    X = oracle.correlation_kernels(psfs, variant)
    for order in ("simultaneous", "sequential"):
        out = oracle.rl_planes(phi, psfs, 4, boundary="circular", psi0=psi_true[None], order=order, corr_kernels=X)
        np.testing.assert_allclose(out[0], psi_true, rtol=1e-11)


def weighted_textbook(phi, psfs, w, iters, boundary, order):
    """psi <- psi * prod_v A_v^T(w_v phi_v / max(A_v psi, eps)) / A_v^T w_v,
    factor 1 where A_v^T w_v < floor; A_v built entry by entry."""
    V, _, H, W = phi.shape
    A = [conv_matrix(psfs[v], H, W, boundary) for v in range(V)]
    psi = np.full(H * W, phi.mean())
    for _ in range(iters):
        fac = []
        for v in range(V):
            wv, pv = w[v, 0].ravel(), phi[v, 0].ravel()
            n = A[v].T @ wv

            def f(ps, v=v, wv=wv, pv=pv, n=n):
                c = A[v].T @ (wv * pv / np.maximum(A[v] @ ps, 1e-6))
                out = np.ones_like(ps)
                ok = n >= oracle.NORM_FLOOR
                out[ok] = c[ok] / n[ok]
                return out
            fac.append(f)
        if order == "sequential":
            for v in range(V):
                psi = psi * fac[v](psi)
        else:
            upd = np.ones_like(psi)
            for v in range(V):
                upd *= fac[v](psi)
            psi = psi * upd
    return psi


@pytest.mark.parametrize("boundary", ["zero", "circular"])
@pytest.mark.parametrize("order", ["simultaneous", "sequential"])
def test_weighted_matches_textbook_em(boundary, order):
    """Weighted MV-RL against the matrix-form EM update with the footprint
    normaliser, on random weights with a zero block wide enough that the
    guard (factor 1 where no weighted pixel is in reach) is exercised."""
    rng = np.random.default_rng(15)
    H, W, V, K = 9, 10, 2, 3
    psfs = rng.random((V, K, K)) + 0.1
    phi = rng.uniform(1, 20, size=(V, 1, H, W))
    w = rng.uniform(0.2, 1.0, size=(V, 1, H, W))
    w[0, 0, 1:6, 2:7] = 0.0                      # interior 3x3 block has n_0 = 0
    out = oracle.rl_planes(phi, psfs, 3, boundary=boundary, order=order, weights=w)
    want = weighted_textbook(phi, psfs, w, 3, boundary, order)
    np.testing.assert_allclose(out[0].ravel(), want, rtol=1e-12)


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_weighted_em_invariant_single_view(boundary):
    """One view, weights > 0: sum_x (P (*) w)(x) psi'(x) = sum_x w(x) phi(x)
    after every update (any PSF, either boundary)."""
    rng = np.random.default_rng(16)
    phi = rng.uniform(1, 30, size=(1, 1, 11, 13))
    P = rng.random((1, 5, 5)) + 0.05
    w = rng.uniform(0.1, 1.0, size=phi.shape)
    n = oracle.correlate(w[0, 0], P[0], boundary)
    for it in (1, 2, 3):
        psi = oracle.rl_planes(phi, P, it, boundary=boundary, weights=w)[0]
        assert abs((n * psi).sum() - (w * phi).sum()) <= 1e-11 * (w * phi).sum()


def test_weighted_unit_weights_and_zero_weight_view():
    """Unit weights with normalised PSFs under the circular boundary give the
    unweighted update; a view with all-zero weights changes nothing."""
    rng = np.random.default_rng(17)
    phi = rng.uniform(1, 30, size=(2, 2, 12, 9))
    psfs = rng.random((2, 5, 5)) + 0.1
    psfs /= psfs.sum(axis=(1, 2), keepdims=True)
    ones = np.ones(phi.shape)
    np.testing.assert_allclose(oracle.rl_planes(phi, psfs, 3, boundary="circular", weights=ones),
                               oracle.rl_planes(phi, psfs, 3, boundary="circular"), rtol=1e-12)
    w = ones.copy()
    w[1] = 0.0
    psi0 = rng.uniform(5, 10, size=(2, 12, 9))
    np.testing.assert_allclose(oracle.rl_planes(phi, psfs, 3, psi0=psi0, weights=w),
                               oracle.rl_planes(phi[:1], psfs[:1], 3, psi0=psi0, weights=w[:1]), rtol=1e-13)


def test_padded_domain_fixed_point_and_embedding():
    """The estimate on the data+PSF-padded domain (Supp. Table 1 caption):
    noise-free data phi_v = (P_v * psi_true) seen only on the data region,
    embedded with zero weights in the padding, leave psi_true fixed (any V,
    zero boundary); embed/crop are each other's inverse on the data."""
    rng = np.random.default_rng(18)
    K, R, H, W = 7, 3, 14, 11
    psfs = np.stack([synth.gaussian_psf(K, 2.0, 0.8, a).astype(np.float64) for a in (0, 90, 45)])
    psi_true = rng.uniform(10, 100, size=(H + 2 * R, W + 2 * R))
    phi = np.stack([oracle.convolve(psi_true, P, "zero")[R:R + H, R:R + W] for P in psfs])[:, None]
    pphi, w = oracle.embed_padded(phi, R)
    assert pphi.shape == (3, 1, H + 2 * R, W + 2 * R) and w.sum() == 3 * H * W
    np.testing.assert_array_equal(oracle.crop_padded(pphi[0], R), phi[0])
    out = oracle.rl_planes(pphi, psfs, 4, boundary="zero", psi0=psi_true[None], weights=w, order="sequential")
    np.testing.assert_allclose(out[0], psi_true, rtol=1e-11)


def brute3d(vol, P, a, boundary, corr):
    Y, Z, X = vol.shape
    K, Ka = P.shape[0], a.shape[0]
    R, Ra = (K - 1) // 2, (Ka - 1) // 2
    out = np.zeros_like(vol)
    sg = 1 if corr else -1
    for y in range(Y):
        for z in range(Z):
            for x in range(X):
                s = 0.0
                for i in range(Ka):
                    for j in range(K):
                        for k in range(K):
                            yy, zz, xx = y + sg * (i - Ra), z + sg * (j - R), x + sg * (k - R)
                            if boundary == "circular":
                                yy, zz, xx = yy % Y, zz % Z, xx % X
                            elif not (0 <= yy < Y and 0 <= zz < Z and 0 <= xx < X):
                                continue
                            s += a[i] * P[j, k] * vol[yy, zz, xx]
                out[y, z, x] = s
    return out


@pytest.mark.parametrize("boundary", ["zero", "circular"])
def test_convolve3d_brute_force_scipy_and_adjoint(boundary):
    """3D convolution with a(y) P(z, x) against a sextuple loop and (zero
    boundary) scipy's 3D convolution; correlation is its adjoint."""
    from scipy.signal import convolve as sconv
    rng = np.random.default_rng(19)
    vol = rng.random((5, 6, 7))
    P = rng.random((3, 3))
    a = rng.random(5)
    np.testing.assert_allclose(oracle.convolve3d(vol, P, a, boundary), brute3d(vol, P, a, boundary, False),
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.correlate3d(vol, P, a, boundary), brute3d(vol, P, a, boundary, True),
                               rtol=1e-12)
    if boundary == "zero":
        k3 = a[:, None, None] * P[None]
        np.testing.assert_allclose(oracle.convolve3d(vol, P, a, "zero"), sconv(vol, k3, mode="same"), rtol=1e-12)
    u = rng.random(vol.shape)
    lhs = (oracle.convolve3d(vol, P, a, boundary) * u).sum()
    rhs = (vol * oracle.correlate3d(u, P, a, boundary)).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_rl3d_reduces_to_planewise_and_conserves_flux():
    """A delta axial profile gives the plane-wise result on every plane; one
    view with normalised kernels under the circular boundary conserves flux."""
    rng = np.random.default_rng(20)
    phi = rng.uniform(1, 30, size=(2, 4, 9, 8))
    psfs = rng.random((2, 5, 5)) + 0.1
    delta = np.zeros((2, 3))
    delta[:, 1] = 1.0
    for order in ("simultaneous", "sequential"):
        np.testing.assert_allclose(oracle.rl3d(phi, psfs, delta, 3, order=order),
                                   oracle.rl_planes(phi, psfs, 3, order=order), rtol=1e-13)
    P = psfs[:1] / psfs[:1].sum()
    a = rng.random((1, 5))
    a /= a.sum()
    for it in (1, 2, 3):
        psi = oracle.rl3d(phi[:1], P, a, it, boundary="circular")
        assert abs(psi.sum() - phi[0].sum()) <= 1e-11 * phi[0].sum()
