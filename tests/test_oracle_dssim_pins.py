"""Pins of the oracle's L1 + D-SSIM loss (Eq. loss3dgs) to things other than itself: a library
Gaussian filter, closed forms for constant images (borders included), the maximum of SSIM at
identical images, symmetry, a tap-by-tap evaluation of the map at every pixel, and FP64
central differences of the gradient."""
import math

import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def test_window_means_are_scipy_gaussian_filter():
    # the local means under the 11x11 window, sigma 1.5, zero outside the image, are a
    # Gaussian filter truncated at radius 5 in constant (0) mode
    rng = np.random.default_rng(1)
    x = rng.random((3, 23, 31))
    _, m = oracle.ssim_maps(x, np.zeros_like(x))
    for c in range(3):
        ref = scipy_ndimage.gaussian_filter(x[c], 1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)
        np.testing.assert_allclose(m["mu_x"][c], ref, rtol=1e-12, atol=1e-15)
    w = oracle.ssim_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15


def one_d_partial_sums(n):
    """s[y] = weight of the 1D normalised window (sigma 1.5, radius 5) that falls inside [0, n)."""
    k = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    k /= k.sum()
    return np.array([sum(k[t + 5] for t in range(-5, 6) if 0 <= y + t < n) for y in range(n)])


def test_constant_images_closed_form():
    # x = a, y = b everywhere: with s(p) the window weight inside the image (a product of 1D
    # partial sums), mu_x = a s, E[x^2] = a^2 s, so var_x = a^2 s (1 - s), cov = a b s (1 - s)
    a, b, H, W = 0.7, 0.2, 14, 19
    x = np.full((1, H, W), a)
    y = np.full((1, H, W), b)
    S, _ = oracle.ssim_maps(x, y)
    s = np.outer(one_d_partial_sums(H), one_d_partial_sums(W))
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ref = ((2 * a * b * s * s + C1) * (2 * a * b * s * (1 - s) + C2)
           / (((a * a + b * b) * s * s + C1) * ((a * a + b * b) * s * (1 - s) + C2)))
    np.testing.assert_allclose(S[0], ref, rtol=1e-9, atol=1e-12)
    # away from the border s = 1 and the map is the luminance term alone
    assert abs(S[0, 7, 9] - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12


def test_identical_images_are_the_maximum():
    rng = np.random.default_rng(2)
    x = rng.random((3, 17, 22))
    S, _ = oracle.ssim_maps(x, x)
    np.testing.assert_allclose(S, 1.0, rtol=0, atol=1e-12)
    loss, (g,) = oracle.l1_dssim([x], [x.copy()])
    assert abs(loss) < 1e-12
    np.testing.assert_allclose(g, 0.0, atol=1e-15)     # SSIM's maximum, sign(0) = 0
    y = x + 0.05 * rng.standard_normal(x.shape)
    S2, _ = oracle.ssim_maps(x, y)
    S3, _ = oracle.ssim_maps(y, x)
    np.testing.assert_allclose(S2, S3, rtol=1e-13)      # symmetric in its arguments
    assert np.all(S2 < 1.0)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(3)
    V = 2
    imgs = [rng.random((3, 9, 13)), rng.random((3, 12, 7))]
    tgts = [rng.random(i.shape) for i in imgs]
    for i, t in zip(imgs, tgts):                       # keep |x - y| clear of the L1 kink
        close = np.abs(i - t) < 1e-3
        i[close] += 2e-3
    _, gs = oracle.l1_dssim(imgs, tgts, lam)
    h = 1e-6
    for v in range(V):
        fd = np.zeros_like(imgs[v])
        for idx in np.ndindex(imgs[v].shape):
            p = [a.copy() for a in imgs]
            m = [a.copy() for a in imgs]
            p[v][idx] += h
            m[v][idx] -= h
            fd[idx] = (oracle.l1_dssim(p, tgts, lam)[0] - oracle.l1_dssim(m, tgts, lam)[0]) / (2 * h)
        np.testing.assert_allclose(gs[v], fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())


def test_loss_weights_and_view_mean():
    # lam = 0: the L1 loss of the same views; lam = 1: mean over views of 1 - SSIM
    rng = np.random.default_rng(4)
    imgs = [rng.random((3, 10, 12)), rng.random((3, 6, 20))]
    tgts = [rng.random(i.shape) for i in imgs]
    l1, g1 = oracle.l1(imgs, tgts)
    l0, g0 = oracle.l1_dssim(imgs, tgts, 0.0)
    assert math.isclose(l0, l1, rel_tol=1e-12)
    for a, b in zip(g0, g1):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    ls, _ = oracle.l1_dssim(imgs, tgts, 1.0)
    ref = np.mean([1.0 - oracle.ssim_maps(i, t)[0].mean() for i, t in zip(imgs, tgts)])
    assert math.isclose(ls, ref, rel_tol=1e-12)


def test_ssim_map_equals_brute_force_per_pixel():
    # every output pixel summed tap by tap from the definition, with its own window weights
    rng = np.random.default_rng(6)
    H, W = 7, 9
    x = rng.random((2, H, W))
    y = rng.random((2, H, W))
    g1 = [math.exp(-(t * t) / (2 * 1.5 ** 2)) for t in range(-5, 6)]
    z = sum(a * b for a in g1 for b in g1)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    S, _ = oracle.ssim_maps(x, y)
    for c in range(2):
        for py in range(H):
            for px in range(W):
                mx = my = exx = eyy = exy = 0.0
                for i in range(-5, 6):
                    for j in range(-5, 6):
                        qy, qx = py + i, px + j
                        if not (0 <= qy < H and 0 <= qx < W):
                            continue
                        wgt = g1[i + 5] * g1[j + 5] / z
                        a, b = x[c, qy, qx], y[c, qy, qx]
                        mx += wgt * a
                        my += wgt * b
                        exx += wgt * a * a
                        eyy += wgt * b * b
                        exy += wgt * a * b
                vx, vy, cov = exx - mx * mx, eyy - my * my, exy - mx * my
                ref = ((2 * mx * my + C1) * (2 * cov + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
                assert abs(S[c, py, px] - ref) < 1e-12, (c, py, px)
