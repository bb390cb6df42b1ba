"""Pins of the FP64 oracle to things other than itself.

- the SH basis against scipy's complex spherical harmonics (a library routine of a different
  form), and its derivative against finite differences;
- a single isotropic Gaussian on the optical axis: Sigma', radius, every pixel and the
  gradients in closed form (Eq. 1, Eq. 2);
- two overlapping Gaussians: C = c1 a1 + c2 a2 (1 - a1) (Eq. 2);
- brute-force compositing over all Gaussians equals the tiled renderer, for every tile size;
- finite differences of the oracle forward against its analytic gradient;
- invariants: T monotone and >= 1e-4, C = sum c a T, permutation invariance, masked Gaussian
  == deleted Gaussian, masked SH band == zeroed band, rotation invariance of isotropic
  Gaussians, zero gradient of masked coefficients;
- the key oracle against an independent numpy lexsort.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_14534_gb300 import synth

scipy_special = pytest.importorskip("scipy.special")


def direct_camera(z_offset, W, H, f, R=None, campos=None):
    """Camera whose frame is the world frame shifted by z_offset along z."""
    vm = np.eye(4)
    if R is not None:
        vm[:3, :3] = R
    vm[2, 3] = z_offset
    cp = np.array([0.0, 0.0, -z_offset]) if campos is None else campos
    return synth.Camera(viewmat=vm, campos=cp, fx=f, fy=f, cx=W / 2.0, cy=H / 2.0,
                        width=W, height=H)


def one_gaussian(mu, log_scale, opacity_logit, dc, quat=(1.0, 0.0, 0.0, 0.0), rest=None,
                 mask=None, shmask=None):
    s = dict(means=np.array([mu], float), log_scales=np.array([log_scale], float),
             quats=np.array([quat], float), opacity_logits=np.array([opacity_logit], float),
             sh_dc=np.array([dc], float), sh_rest=None if rest is None else np.array([rest]),
             mask_logits=None if mask is None else np.array([mask], float),
             sh_mask_logits=None if shmask is None else np.array([shmask], float),
             sh_degree=None)
    if rest is None:
        s["deg_max"] = 0
    return s


def concat_scenes(a, b):
    out = {}
    for k in a:
        if k == "deg_max":
            out[k] = a[k]
        elif a[k] is None:
            out[k] = None
        else:
            out[k] = np.concatenate([a[k], b[k]])
    return out


# ---------------------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------------------

def real_sh_from_scipy(l, m, theta, phi):
    """Real SH in the sign convention of the rasterizer, from scipy's complex SH (which
    carries the Condon-Shortley phase): m<0 -> sqrt2 Im Y_l^|m|, m>0 -> sqrt2 Re Y_l^m."""
    if m == 0:
        return scipy_special.sph_harm_y(l, 0, theta, phi).real
    Y = scipy_special.sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2.0) * (Y.imag if m < 0 else Y.real)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, _ = oracle.sh_basis(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = real_sh_from_scipy(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, k], ref, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform in phi integrates degree <= 6 polynomials exactly
    x, w = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * (2 * np.pi / 16)
    d, wt = [], []
    for xi, wi in zip(x, w):
        for p in phis:
            s = math.sqrt(1 - xi * xi)
            d.append((s * math.cos(p), s * math.sin(p), xi))
            wt.append(wi * 2 * np.pi / 16)
    Y, _ = oracle.sh_basis(np.array(d))
    gram = (Y * np.array(wt)[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_basis_derivative_fd():
    rng = np.random.default_rng(4)
    d = rng.normal(size=(20, 3))
    _, dY = oracle.sh_basis(d)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        Yp, _ = oracle.sh_basis(d + e)
        Ym, _ = oracle.sh_basis(d - e)
        np.testing.assert_allclose(dY[:, :, c], (Yp - Ym) / (2 * h), atol=1e-7)


# ---------------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------------

def single_closed_form(W, H, f, z, sigma, o_logit, dc, s=0.3):
    """Image of one isotropic Gaussian at (0, 0, z) in camera space, degree-0 colour."""
    v = (f * sigma / z) ** 2 + s
    r = math.ceil(3.0 * math.sqrt(v + math.sqrt(0.1)))
    mx, my = W / 2.0 - 0.5, H / 2.0 - 0.5
    o = 1.0 / (1.0 + math.exp(-o_logit))
    c = np.maximum(0.0, 0.5 + np.asarray(dc) / (2.0 * math.sqrt(math.pi)))
    py, px = np.mgrid[0:H, 0:W].astype(float)
    dx, dy = mx - px, my - py
    a = o * np.exp(-(dx * dx + dy * dy) / (2 * v))
    inside = (np.abs(dx) <= r) & (np.abs(dy) <= r)
    a = np.where(inside, np.minimum(0.99, a), 0.0)
    a = np.where(a < 1 / 255, 0.0, a)
    img = c[:, None, None] * a[None]
    return img, 1.0 - a, v, r, a, dx, dy, o, c


@pytest.mark.parametrize("z,sigma,o_logit", [(4.0, 0.05, 0.3), (3.0, 0.02, 2.0),
                                             (6.0, 0.2, -1.0), (5.0, 0.001, 5.0)])
def test_single_gaussian_closed_form(z, sigma, o_logit):
    W, H, f = 64, 48, 100.0
    dc = (0.3, -0.2, 0.9)
    scene = one_gaussian((0.0, 0.0, 0.0), [math.log(sigma)] * 3, o_logit, dc)
    cam = direct_camera(z, W, H, f)
    st = oracle.Settings(tile=16)
    out = oracle.render(scene, cam, st)
    img, T, v, r, *_ = single_closed_form(W, H, f, z, sigma, o_logit, dc)
    sp = out["splats"]
    assert sp["radius"][0] == r
    np.testing.assert_allclose(sp["conic"][0], [1 / v, 0.0, 1 / v], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(sp["mean2d"][0], [W / 2 - 0.5, H / 2 - 0.5], atol=1e-12)
    np.testing.assert_allclose(out["image"], img, atol=1e-13)
    np.testing.assert_allclose(out["T_final"], T, atol=1e-13)


def test_single_gaussian_gradient_closed_form():
    W, H, f, z, sigma, o_logit = 48, 40, 90.0, 4.0, 0.06, 0.4
    dc = (0.3, 0.1, 0.7)
    scene = one_gaussian((0.0, 0.0, 0.0), [math.log(sigma)] * 3, o_logit, dc)
    cam = direct_camera(z, W, H, f)
    st = oracle.Settings(tile=16)
    rng = np.random.default_rng(11)
    wimg = rng.normal(size=(3, H, W))
    grads, stats, g9 = oracle.grad(scene, [cam], st, [wimg])
    img, T, v, r, a, dx, dy, o, c = single_closed_form(W, H, f, z, sigma, o_logit, dc)
    on = a > 0
    wc = (wimg * c[:, None, None]).sum(0)          # sum_ch w_ch c_ch per pixel
    # opacity logit: a = sigma(o) G, dL/do = sum w c G sigma(1 - sigma)
    g_o = (wc * np.where(on, a * (1 - o), 0)).sum()
    # log-scale x: Sigma'_00 = (f s_x / z)^2 + s, d a / d Sigma'_00 = a dx^2 / (2 Sigma'_00^2)
    u = (f * sigma / z) ** 2
    g_lx = (wc * np.where(on, a * dx * dx / (2 * v * v), 0)).sum() * 2 * u
    g_ly = (wc * np.where(on, a * dy * dy / (2 * v * v), 0)).sum() * 2 * u
    # mean x: d mean2d_x / d mu_x = f / z; d a / d mean2d_x = -a dx / v
    g_mx = (wc * np.where(on, -a * dx / v, 0)).sum() * f / z
    g_my = (wc * np.where(on, -a * dy / v, 0)).sum() * f / z
    # mean z: Sigma' diagonal changes by -2 u / z per unit z; mean2d does not move
    g_mz = (wc * np.where(on, a * (dx * dx + dy * dy) / (2 * v * v), 0)).sum() * (-2 * u / z)
    # colour: dL/dc_ch = sum w_ch a, dc coefficient Y00 = 1 / (2 sqrt(pi))
    g_dc = (wimg * a[None]).reshape(3, -1).sum(1) / (2 * math.sqrt(math.pi))
    np.testing.assert_allclose(grads["opacity_logits"][0], g_o, rtol=1e-10)
    np.testing.assert_allclose(grads["log_scales"][0], [g_lx, g_ly, 0.0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(grads["means"][0], [g_mx, g_my, g_mz], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(grads["sh_dc"][0], g_dc, rtol=1e-10)
    # densification statistic: |dL/dmean2d| in pixel units
    np.testing.assert_allclose(stats["accum"][0], math.hypot(g_mx, g_my) * z / f, rtol=1e-9)
    assert stats["count"][0] == 1 and stats["max_radius"][0] == r


def test_two_gaussians_blend_closed_form():
    W, H, f = 32, 32, 80.0
    a = one_gaussian((0.0, 0.0, 0.0), [math.log(0.05)] * 3, 0.5, (0.9, 0.1, 0.1))
    b = one_gaussian((0.02, -0.01, 1.0), [math.log(0.07)] * 3, 1.0, (0.1, 0.2, 0.9))
    scene = concat_scenes(a, b)
    cam = direct_camera(4.0, W, H, f)
    st = oracle.Settings(tile=16)
    out = oracle.render(scene, cam, st)
    sp = out["splats"]
    py, px = np.mgrid[0:H, 0:W].astype(float)

    def alpha(i):
        dx, dy = sp["mean2d"][i, 0] - px, sp["mean2d"][i, 1] - py
        cn = sp["conic"][i]
        x = sp["opacity"][i] * np.exp(-0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy)
        rc = sp["rect"][i]
        inside = (px >= rc[0]) & (px <= rc[1]) & (py >= rc[2]) & (py <= rc[3])
        x = np.where(inside, np.minimum(0.99, x), 0.0)
        return np.where(x < 1 / 255, 0.0, x)

    a1, a2 = alpha(0), alpha(1)        # Gaussian 0 is nearer (depth 4 < 5)
    c1, c2 = sp["rgb"][0], sp["rgb"][1]
    expect = c1[:, None, None] * a1 + c2[:, None, None] * a2 * (1 - a1)
    np.testing.assert_allclose(out["image"], expect, atol=1e-13)
    np.testing.assert_allclose(out["T_final"], (1 - a1) * (1 - a2), atol=1e-13)


# ---------------------------------------------------------------------------------------
# brute force, tile-size invariance, invariants
# ---------------------------------------------------------------------------------------

def tiny_scene(n, seed, masks=True, degree=False):
    sc = synth.blob_scene(n, 4, seed, log_scale=(-2.6, 0.5), masks=masks,
                          per_gaussian_degree=degree)
    return sc


def tiny_cam(W=48, H=40, angle=0.3):
    return synth.ring_cameras(1, [(W, H)], radius=4.0, height=0.5, phase=angle)[0]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_equals_tiled_all_tile_sizes(seed):
    scene = tiny_scene(300, seed)
    cam = tiny_cam(61, 45)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    brute = oracle.render(scene, cam, st, brute=True)
    for tile in (8, 16, 32):
        st.tile = tile
        t = oracle.render(scene, cam, st)
        assert np.array_equal(t["image"], brute["image"])
        assert np.array_equal(t["T_final"], brute["T_final"])
        assert np.array_equal(t["n_contrib"], brute["n_contrib"])
    assert (brute["n_contrib"] > 0).mean() > 0.1


def test_alpha_support_equals_brute_force_without_box():
    scene = tiny_scene(200, 5)
    cam = tiny_cam(40, 40)
    st = oracle.Settings(tile=8, support=oracle.SUPPORT_ALPHA, eps_mask=0.5, eps_sh=0.5)
    out = oracle.render(scene, cam, st)
    # In the alpha-exact support the box never removes a fragment that would count:
    # widen every rect to the whole image and compare.
    sp = dict(out["splats"])
    sp["rect"] = sp["rect"].copy()
    vis = sp["radius"] > 0
    sp["rect"][vis] = [0, cam.width - 1, 0, cam.height - 1]
    wide = oracle.blend(sp, cam.width, cam.height, tile=8, brute=True)
    np.testing.assert_allclose(wide["image"], out["image"], atol=1e-15)


def test_transmittance_and_colour_invariants():
    scene = tiny_scene(400, 7)
    cam = tiny_cam(48, 40)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5, bg=(0.0, 0.0, 0.0))
    out = oracle.render(scene, cam, st)
    sp = out["splats"]
    T = out["T_final"]
    assert (T >= 1e-4).all() and (T <= 1.0).all()
    # recompute each pixel from the brute-force order: C = sum c a T, T monotone
    order = np.lexsort((np.arange(len(sp["depth"])), sp["depth"].astype(np.float32).view(np.uint32)))
    order = [i for i in order if sp["radius"][i] > 0]
    for (py, px) in [(5, 7), (20, 24), (33, 40), (0, 0), (39, 47)]:
        Tp, Cp, Ts = 1.0, np.zeros(3), []
        for i in order:
            rc = sp["rect"][i]
            if not (rc[0] <= px <= rc[1] and rc[2] <= py <= rc[3]):
                continue
            dx, dy = sp["mean2d"][i, 0] - px, sp["mean2d"][i, 1] - py
            cn = sp["conic"][i]
            pw = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy
            a = min(0.99, sp["opacity"][i] * math.exp(pw))
            if pw > 0 or a < 1 / 255:
                continue
            if Tp * (1 - a) < 1e-4:
                break
            Cp += sp["rgb"][i] * a * Tp
            Tp *= 1 - a
            Ts.append(Tp)
        assert all(x >= y for x, y in zip([1.0] + Ts, Ts))
        np.testing.assert_allclose(out["image"][:, py, px], Cp, atol=1e-13)
        np.testing.assert_allclose(T[py, px], Tp, atol=1e-15)
    # background: image = C + T_final * bg
    st2 = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5, bg=(0.2, 0.5, 1.0))
    out2 = oracle.render(scene, cam, st2)
    np.testing.assert_allclose(out2["image"], out["image"] + T[None] * np.array(st2.bg)[:, None, None],
                               atol=1e-13)


def test_permutation_invariance():
    scene = tiny_scene(250, 9)
    cam = tiny_cam()
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    ref = oracle.render(scene, cam, st)
    perm = np.random.default_rng(0).permutation(250)
    ps = {k: (None if v is None else v[perm]) for k, v in scene.items()}
    out = oracle.render(ps, cam, st)
    np.testing.assert_allclose(out["image"], ref["image"], atol=1e-13)


def test_masked_gaussian_equals_deleted():
    scene = tiny_scene(200, 10)
    cam = tiny_cam()
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    m = scene["mask_logits"].copy()
    drop = np.arange(0, 200, 3)
    m[drop] = -5.0
    masked = dict(scene, mask_logits=m)
    keep = np.setdiff1d(np.arange(200), drop)
    deleted = {k: (None if v is None else v[keep]) for k, v in masked.items()}
    a = oracle.render(masked, cam, st)
    b = oracle.render(deleted, cam, st)
    np.testing.assert_allclose(a["image"], b["image"], atol=1e-14)
    # masked Gaussians receive exactly zero gradient
    w = np.random.default_rng(1).normal(size=(3, cam.height, cam.width))
    g, _, _ = oracle.grad(masked, [cam], st, [w])
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest", "mask_logits"):
        assert np.all(g[k][drop] == 0.0), k


def test_masked_band_equals_zeroed_band():
    scene = tiny_scene(150, 12)
    cam = tiny_cam()
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    shm = scene["sh_mask_logits"].copy()
    shm[:, :] = 3.0
    shm[::2, 1] = -3.0      # band 2 masked on even Gaussians
    a = oracle.render(dict(scene, sh_mask_logits=shm), cam, st)
    rest = scene["sh_rest"].copy()
    rest[::2, 3:8, :] = 0.0
    b = oracle.render(dict(scene, sh_mask_logits=np.full_like(shm, 3.0), sh_rest=rest), cam, st)
    np.testing.assert_allclose(a["image"], b["image"], atol=1e-14)
    w = np.random.default_rng(2).normal(size=(3, cam.height, cam.width))
    g, _, _ = oracle.grad(dict(scene, sh_mask_logits=shm), [cam], st, [w])
    assert np.all(g["sh_rest"][::2, 3:8, :] == 0.0)
    assert np.any(g["sh_mask_logits"][::2, 1] != 0.0)   # straight-through still flows


def test_per_gaussian_degree_equals_zeroed_bands():
    scene = tiny_scene(150, 13, masks=False, degree=True)
    cam = tiny_cam()
    st = oracle.Settings(tile=16)
    a = oracle.render(scene, cam, st)
    b = oracle.render(dict(scene, sh_degree=None), cam, st)   # coefficients above are zero
    np.testing.assert_allclose(a["image"], b["image"], atol=1e-14)


def test_rotation_invariance_isotropic():
    scene = tiny_scene(150, 14, masks=False)
    ls = scene["log_scales"].copy()
    ls[:, 1] = ls[:, 0]
    ls[:, 2] = ls[:, 0]
    base = dict(scene, log_scales=ls, sh_rest=np.zeros_like(scene["sh_rest"]))
    q = np.random.default_rng(5).normal(size=(150, 4))
    rot = dict(base, quats=q)
    cam = tiny_cam()
    st = oracle.Settings(tile=16)
    np.testing.assert_allclose(oracle.render(base, cam, st)["image"],
                               oracle.render(rot, cam, st)["image"], atol=1e-12)


def test_threads_do_not_change_results():
    scene = tiny_scene(300, 15)
    cam = tiny_cam(64, 48)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    sp = oracle.preprocess(scene, cam, st)
    a = oracle.blend(sp, 64, 48, 16, nthreads=1)
    b = oracle.blend(sp, 64, 48, 16, nthreads=4)
    assert np.array_equal(a["image"], b["image"])
    w = np.random.default_rng(3).normal(size=(3, 48, 64))
    g1 = oracle.blend_backward(sp, 64, 48, w, 16, nthreads=1)
    g4 = oracle.blend_backward(sp, 64, 48, w, 16, nthreads=4)
    np.testing.assert_allclose(g1, g4, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------------------
# keys
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("tile", [8, 16, 32])
def test_key_oracle_against_lexsort(tile):
    scene = tiny_scene(400, 16)
    cam = tiny_cam(70, 50)
    st = oracle.Settings(tile=tile, eps_mask=0.5, eps_sh=0.5)
    sp = oracle.preprocess(scene, cam, st)
    keys, vals, ranges = oracle.keys(sp["radius"], sp["rect"], sp["depth"], 70, 50, tile,
                                     tile_offset=7, value_offset=1000)
    gx = (70 + tile - 1) // tile
    tiles, ids, db = [], [], []
    for i in range(400):
        if sp["radius"][i] <= 0:
            continue
        x0, x1, y0, y1 = sp["rect"][i]
        for ty in range(y0 // tile, y1 // tile + 1):
            for tx in range(x0 // tile, x1 // tile + 1):
                tiles.append(7 + ty * gx + tx)
                ids.append(1000 + i)
                db.append(np.float32(sp["depth"][i]).view(np.uint32))
    tiles, ids, db = map(np.array, (tiles, ids, db))
    o = np.lexsort((ids, db, tiles))
    ek = (tiles[o].astype(np.uint64) << np.uint64(32)) | db[o].astype(np.uint64)
    assert np.array_equal(keys, ek)
    assert np.array_equal(vals, ids[o].astype(np.uint32))
    for t in range(ranges.shape[0]):
        sel = np.nonzero(tiles[o] == 7 + t)[0]
        if len(sel) == 0:
            assert tuple(ranges[t]) == (0, 0)
        else:
            assert tuple(ranges[t]) == (sel[0], sel[-1] + 1)


# ---------------------------------------------------------------------------------------
# finite differences
# ---------------------------------------------------------------------------------------

def _loss(scene, cams, st, ws):
    tot = 0.0
    fps = []
    for cam, w in zip(cams, ws):
        out = oracle.render(scene, cam, st)
        tot += float((out["image"] * w).sum())
        fps.append((out["n_contrib"].copy(), out["last"].copy(), out["splats"]["rect"].copy()))
    return tot, fps


def _same(fa, fb):
    return all(np.array_equal(x, y) for a, b in zip(fa, fb) for x, y in zip(a, b))


def _fd_check(scene, cams, st, n_checks, seed, keys=None, rtol=2e-5):
    rng = np.random.default_rng(seed)
    scene = {k: (None if v is None or k in ("sh_degree", "deg_max") else
                 np.array(v, dtype=np.float64)) if k not in ("sh_degree", "deg_max") else v
             for k, v in scene.items()}
    ws = [rng.normal(size=(3, c.height, c.width)) for c in cams]
    grads, _, _ = oracle.grad(scene, cams, st, ws)
    L0, f0 = _loss(scene, cams, st, ws)
    # The straight-through mask gradients are not derivatives of the (piecewise constant)
    # forward; they are pinned by test_straight_through_* instead.
    keys = keys or [k for k in oracle.GRAD_KEYS
                    if scene.get(k) is not None and k not in ("mask_logits", "sh_mask_logits")]
    checked = skipped = 0
    worst = 0.0
    for _ in range(n_checks):
        k = keys[rng.integers(len(keys))]
        idx = tuple(rng.integers(0, s) for s in scene[k].shape)
        x = scene[k][idx]
        h = 1e-6 * max(1.0, abs(x))
        scene[k][idx] = x + h
        Lp, fp = _loss(scene, cams, st, ws)
        scene[k][idx] = x - h
        Lm, fm = _loss(scene, cams, st, ws)
        scene[k][idx] = x
        fwd, bwd = (Lp - L0) / h, (L0 - Lm) / h
        if not (_same(f0, fp) and _same(f0, fm)) or abs(fwd - bwd) > 1e-4 * (abs(fwd) + 1e-3):
            skipped += 1
            continue
        fd = (Lp - Lm) / (2 * h)
        g = grads[k][idx]
        err = abs(fd - g) / (abs(fd) + 1e-3)
        worst = max(worst, err)
        assert err < rtol, (k, idx, fd, g)
        checked += 1
    return checked, skipped, worst


def test_fd_gradient_masked_scene():
    scene = tiny_scene(60, 21)
    cams = [tiny_cam(40, 32, 0.2), tiny_cam(32, 24, 1.9)]
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    checked, skipped, _ = _fd_check(scene, cams, st, 160, 1)
    assert checked >= 120


def test_fd_gradient_every_parameter_kind():
    scene = tiny_scene(40, 22)
    scene["quats"] = scene["quats"] * 1.7        # non-unit quaternions exercise normalisation
    cams = [tiny_cam(36, 28, 0.7)]
    st = oracle.Settings(tile=8, eps_mask=0.5, eps_sh=0.5, bg=(0.3, 0.1, 0.6))
    for j, k in enumerate(oracle.GRAD_KEYS[:6]):
        checked, _, _ = _fd_check(scene, cams, st, 25, 100 + j, keys=[k])
        assert checked >= 15, k


def test_fd_gradient_alpha_support_and_degree():
    scene = tiny_scene(50, 23, masks=False, degree=True)
    cams = [tiny_cam(36, 30, 2.5)]
    st = oracle.Settings(tile=16, support=oracle.SUPPORT_ALPHA)
    checked, _, _ = _fd_check(scene, cams, st, 80, 5)
    assert checked >= 60


def test_fd_gradient_jacobian_clamp_active():
    # wide Gaussians whose centres lie beyond 1.3 x the half field of view
    W, H, f = 40, 32, 20.0
    rng = np.random.default_rng(8)
    n = 6
    sc = dict(means=np.column_stack([rng.uniform(3.2, 3.8, n) * rng.choice([-1, 1], n),
                                     rng.uniform(-0.5, 0.5, n), rng.uniform(-0.3, 0.3, n)]),
              log_scales=rng.normal(-0.2, 0.2, (n, 3)), quats=rng.normal(size=(n, 4)),
              opacity_logits=rng.normal(1.0, 0.5, n), sh_dc=rng.uniform(0, 1, (n, 3)),
              sh_rest=rng.normal(0, 0.1, (n, 15, 3)), mask_logits=None, sh_mask_logits=None,
              sh_degree=None)
    cam = direct_camera(2.0, W, H, f)
    st = oracle.Settings(tile=8)
    sp = oracle.preprocess(sc, cam, st)
    tx = sc["means"][:, 0] / (sc["means"][:, 2] + 2.0)
    assert np.all(np.abs(tx) > 1.3 * W / (2 * f))       # clamp active for every Gaussian
    assert np.all(sp["radius"] > 0)                        # and each still touches the image
    checked, _, _ = _fd_check(sc, [cam], st, 60, 9, keys=["means", "log_scales", "quats"])
    assert checked >= 40


def test_l1_loss_and_sign_convention():
    img = [np.array([[[0.5, 0.2], [0.3, 0.3]]] * 3)]
    tgt = [np.array([[[0.4, 0.2], [0.5, 0.3]]] * 3)]
    loss, g = oracle.l1(img, tgt)
    np.testing.assert_allclose(loss, (0.1 + 0.2) * 3 / 12)
    np.testing.assert_array_equal(np.sign(g[0][0]), [[1, 0], [-1, 0]])


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def test_straight_through_volume_mask():
    """dL/dm = sigma'(m) dL/dM, with dL/dM the derivative of the render with respect to a
    continuous M multiplying opacity and scale (mask equation). Evaluated by FD in M:
    scale by M is log-scale + log M, opacity M sigma(o) is logit(M sigma(o))."""
    scene = {k: (None if v is None else np.array(v, np.float64)) for k, v in
             tiny_scene(30, 31).items()}
    scene["mask_logits"][:] = np.abs(scene["mask_logits"]) + 0.5    # all unmasked (M = 1)
    cams = [tiny_cam(36, 28, 0.4)]
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    rng = np.random.default_rng(0)
    ws = [rng.normal(size=(3, c.height, c.width)) for c in cams]
    grads, _, _ = oracle.grad(scene, cams, st, ws)
    checked = 0
    for i in range(30):
        def L(M):
            sc = dict(scene)
            sc["log_scales"] = scene["log_scales"].copy()
            sc["log_scales"][i] += math.log(M)
            sc["opacity_logits"] = scene["opacity_logits"].copy()
            p = M * _sig(scene["opacity_logits"][i])
            sc["opacity_logits"][i] = math.log(p / (1 - p))
            return _loss(sc, cams, st, ws)
        h = 1e-6
        (Lp, fp), (Lm, fm), (L0, f0) = L(1 + h), L(1 - h), L(1.0)
        if not (_same(f0, fp) and _same(f0, fm)):
            continue
        dLdM = (Lp - Lm) / (2 * h)
        m = scene["mask_logits"][i]
        expect = dLdM * _sig(m) * (1 - _sig(m))
        np.testing.assert_allclose(grads["mask_logits"][i], expect, rtol=2e-5, atol=1e-9)
        checked += 1
    assert checked >= 20


def test_straight_through_sh_band_masks():
    """dL/dm^l = sigma'(m^l) dL/dM^l for masked and unmasked bands, with dL/dM^l the
    derivative with respect to a continuous factor on band l's coefficients (Eq. sh-masks)."""
    scene = {k: (None if v is None else np.array(v, np.float64)) for k, v in
             tiny_scene(30, 32).items()}
    scene["mask_logits"][:] = 5.0
    shm = np.where(np.random.default_rng(1).uniform(size=(30, 3)) < 0.4, -2.0, 2.0)
    scene["sh_mask_logits"] = shm
    cams = [tiny_cam(36, 28, 1.1)]
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    rng = np.random.default_rng(2)
    ws = [rng.normal(size=(3, c.height, c.width)) for c in cams]
    grads, _, _ = oracle.grad(scene, cams, st, ws)
    bands = [(1, slice(0, 3)), (2, slice(3, 8)), (3, slice(8, 15))]
    checked = 0
    for i in range(30):
        for l, sl in bands:
            base = dict(scene, sh_mask_logits=np.full_like(shm, 2.0))   # every band on
            M0 = 1.0 if shm[i, l - 1] > 0 else 0.0

            def L(M):
                sc = dict(base)
                sc["sh_rest"] = scene["sh_rest"].copy()
                # other bands of this Gaussian keep their hard mask value
                for l2, sl2 in bands:
                    if l2 != l and shm[i, l2 - 1] < 0:
                        sc["sh_rest"][i, sl2] = 0.0
                sc["sh_rest"][i, sl] *= M
                for j in range(30):
                    if j != i:
                        for l2, sl2 in bands:
                            if shm[j, l2 - 1] < 0:
                                sc["sh_rest"][j, sl2] = 0.0
                return _loss(sc, cams, st, ws)
            h = 1e-6
            (Lp, fp), (Lm, fm), (L0, f0) = L(M0 + h), L(M0 - h), L(M0)
            if not (_same(f0, fp) and _same(f0, fm)):
                continue
            dLdM = (Lp - Lm) / (2 * h)
            m = shm[i, l - 1]
            expect = dLdM * _sig(m) * (1 - _sig(m))
            np.testing.assert_allclose(grads["sh_mask_logits"][i, l - 1], expect, rtol=2e-5,
                                       atol=1e-9)
            checked += 1
    assert checked >= 60


@pytest.mark.parametrize("tile", [8, 16])
def test_tile_masked_blend_equals_full_blend_on_those_tiles(tile):
    scene = tiny_scene(600, 41)
    cam = tiny_cam(75, 53, 0.6)
    st = oracle.Settings(tile=tile, eps_mask=0.5, eps_sh=0.5, bg=(0.1, 0.0, 0.3))
    sp = oracle.preprocess(scene, cam, st)
    full = oracle.blend(sp, 75, 53, tile, st.bg, margins=True)
    gx, gy = (75 + tile - 1) // tile, (53 + tile - 1) // tile
    mask = np.zeros(gx * gy, np.uint8)
    mask[np.random.default_rng(0).choice(gx * gy, size=gx * gy // 3, replace=False)] = 1
    part = oracle.blend(sp, 75, 53, tile, st.bg, margins=True, tile_mask=mask)
    pix = np.repeat(np.repeat(mask.reshape(gy, gx), tile, 0), tile, 1)[:53, :75].astype(bool)
    for k in ("T_final", "last", "n_contrib", "n_examined", "n_eval", "margin"):
        assert np.array_equal(part[k][pix], full[k][pix]), k
    assert np.array_equal(part["image"][:, pix], full["image"][:, pix])
    w = np.random.default_rng(1).normal(size=(3, 53, 75)) * pix[None]
    g_full = oracle.blend_backward(sp, 75, 53, w, tile, st.bg)
    g_part = oracle.blend_backward(sp, 75, 53, w, tile, st.bg, tile_mask=mask)
    np.testing.assert_allclose(g_part, g_full, rtol=1e-12, atol=1e-15)


def test_blend_with_given_lists_equals_blend():
    scene = tiny_scene(500, 43)
    cam = tiny_cam(70, 50, 1.3)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    sp = oracle.preprocess(scene, cam, st)
    _, vals, ranges = oracle.keys(sp["radius"], sp["rect"], sp["depth"], 70, 50, 16)
    a = oracle.blend(sp, 70, 50, 16)
    b = oracle.blend(sp, 70, 50, 16, lists=(vals, ranges))
    for k in ("image", "T_final", "last", "n_examined"):
        assert np.array_equal(a[k], b[k]), k
    w = np.random.default_rng(0).normal(size=(3, 50, 70))
    np.testing.assert_array_equal(oracle.blend_backward(sp, 70, 50, w, 16),
                                  oracle.blend_backward(sp, 70, 50, w, 16, lists=(vals, ranges)))


def _cull_of(sp):
    """Float32 cull data (mean2d, conic, tau) of FP64 records, tau = 2 ln(255 o' / (1 - 1e-3))."""
    with np.errstate(divide="ignore", invalid="ignore"):
        tau = 2.0 * np.log(255.0 * sp["opacity"] / (1.0 - 1e-3))
        c32 = sp["conic"].astype(np.float32)
        bc = c32[:, 1] / c32[:, 2]
        ba = c32[:, 1] / c32[:, 0]
    return np.column_stack([sp["mean2d"], sp["conic"], tau, bc, ba]).astype(np.float32)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tile_cull_drops_only_tiles_without_a_visible_pixel(tile):
    scene = tiny_scene(500, 47)
    scene["log_scales"][:, 0] += 0.8          # strongly anisotropic footprints
    cam = tiny_cam(90, 70, 0.4)
    st = oracle.Settings(tile=tile, eps_mask=0.5, eps_sh=0.5)
    sp = oracle.preprocess(scene, cam, st)
    cull = _cull_of(sp)
    k_all, _, _ = oracle.keys(sp["radius"], sp["rect"], sp["depth"], 90, 70, tile)
    k_cul, v_cul, r_cul = oracle.keys(sp["radius"], sp["rect"], sp["depth"], 90, 70, tile, cull=cull)
    assert 0 < len(k_cul) < 0.9 * len(k_all)
    kept = set((int(k >> np.uint64(32)), int(v)) for k, v in zip(k_cul, oracle.keys(
        sp["radius"], sp["rect"], sp["depth"], 90, 70, tile, cull=cull)[1]))
    gx = (90 + tile - 1) // tile
    py, px = np.mgrid[0:70, 0:90].astype(float)
    for i in np.nonzero(sp["radius"] > 0)[0]:
        x0, x1, y0, y1 = sp["rect"][i]
        dx, dy = sp["mean2d"][i, 0] - px, sp["mean2d"][i, 1] - py
        a, b, c = sp["conic"][i]
        alpha = sp["opacity"][i] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        for ty in range(y0 // tile, y1 // tile + 1):
            for tx in range(x0 // tile, x1 // tile + 1):
                if (ty * gx + tx, i) in kept:
                    continue
                ys = slice(max(ty * tile, y0), min(ty * tile + tile - 1, y1) + 1)
                xs = slice(max(tx * tile, x0), min(tx * tile + tile - 1, x1) + 1)
                # a dropped tile holds no pixel that reaches alpha >= 1/255 (with the margin)
                assert alpha[ys, xs].max() < (1.0 - 0.5e-3) / 255.0, (i, tx, ty)
    # and the image, the transmittance and the contributor count are unchanged
    full = oracle.blend(sp, 90, 70, tile)
    cul = oracle.blend(sp, 90, 70, tile, lists=(v_cul, r_cul))
    for k in ("image", "T_final", "n_contrib"):
        assert np.array_equal(full[k], cul[k]), k


# ---------------------------------------------------------------------------------------
# significance score (Eq. significance-score)
# ---------------------------------------------------------------------------------------

def python_hits(sp, W, H):
    """Ray hits by a plain per-pixel loop over all Gaussians in (depth bits, index) order,
    written here from Eq. 2 without the oracle's tile lists: a pixel blends a Gaussian when it
    is inside its box, the exponent is <= 0, alpha = min(0.99, o G) >= 1/255 and the
    transmittance stays >= 1e-4."""
    n = sp["radius"].shape[0]
    vis = [i for i in range(n) if sp["radius"][i] > 0]
    db = np.asarray(sp["depth"], np.float32).view(np.uint32)
    order = sorted(vis, key=lambda i: (int(db[i]), i))
    hits = np.zeros(n, np.int64)
    for py in range(H):
        for px in range(W):
            T = 1.0
            for g in order:
                x0, x1, y0, y1 = sp["rect"][g]
                if not (x0 <= px <= x1 and y0 <= py <= y1):
                    continue
                dx, dy = sp["mean2d"][g][0] - px, sp["mean2d"][g][1] - py
                a, b, c = sp["conic"][g]
                power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if power > 0.0:
                    continue
                alpha = min(0.99, sp["opacity"][g] * math.exp(power))
                if alpha < 1.0 / 255.0:
                    continue
                if T * (1.0 - alpha) < 1e-4:
                    break
                hits[g] += 1
                T *= 1.0 - alpha
    return hits


def test_hits_equal_a_plain_per_pixel_loop():
    scene = tiny_scene(60, 9)
    cam = tiny_cam(24, 20)
    st = oracle.Settings(tile=8, eps_mask=0.5, eps_sh=0.5)
    sp = oracle.preprocess(scene, cam, st)
    ref = python_hits(sp, cam.width, cam.height)
    for tile in (8, 16):
        np.testing.assert_array_equal(oracle.hits(sp, cam.width, cam.height, tile=tile), ref)
    np.testing.assert_array_equal(oracle.hits(sp, cam.width, cam.height, brute=True, nthreads=3), ref)
    assert ref.sum() > 0 and (ref > 0).sum() > 3


def test_hits_of_one_gaussian_closed_form():
    # one isotropic Gaussian: alpha <= 0.99 never stops a pixel, so its hits are the pixels
    # of its box where alpha >= 1/255 (the closed-form alpha image above)
    W, H, f, z, sigma, o_logit = 64, 48, 100.0, 4.0, 0.05, 0.3
    scene = one_gaussian((0.0, 0.0, 0.0), [math.log(sigma)] * 3, o_logit, (0.3, 0.2, 0.1))
    cam = direct_camera(z, W, H, f)
    st = oracle.Settings(tile=16)
    sp = oracle.preprocess(scene, cam, st)
    *_, a, _dx, _dy, _o, _c = single_closed_form(W, H, f, z, sigma, o_logit, (0.3, 0.2, 0.1))
    assert oracle.hits(sp, W, H)[0] == int((a > 0.0).sum()) > 0
    # masked out: no hits and no score
    masked = one_gaussian((0.0, 0.0, 0.0), [math.log(sigma)] * 3, o_logit, (0.3, 0.2, 0.1), mask=-3.0)
    st_m = oracle.Settings(tile=16, eps_mask=0.5)
    spm = oracle.preprocess(masked, cam, st_m)
    hm = oracle.hits(spm, W, H)
    assert hm[0] == 0 and oracle.significance(masked, st_m, hm)[0] == 0.0


def test_significance_closed_form():
    # four Gaussians with volumes 1, 2, 4, 8 (log-scales summing to log v), opacity logits
    # 0 (o = 1/2) except the last (logit log 3: o = 3/4); the 0.9 quantile of 4 volumes is the
    # one at rank floor(0.9 * 3) = 2, i.e. 4: gamma = 1/4, 1/2, 1, 1
    vols = [1.0, 2.0, 4.0, 8.0]
    scene = dict(means=np.zeros((4, 3)),
                 log_scales=np.array([[math.log(v), 0.0, 0.0] for v in vols]),
                 quats=np.tile([1.0, 0.0, 0.0, 0.0], (4, 1)),
                 opacity_logits=np.array([0.0, 0.0, 0.0, math.log(3.0)]),
                 sh_dc=np.zeros((4, 3)), sh_rest=None, mask_logits=None, sh_mask_logits=None,
                 sh_degree=None, deg_max=0)
    hits = np.array([10, 0, 3, 7])
    got = oracle.significance(scene, oracle.Settings(), hits)
    np.testing.assert_allclose(got, [10 * 0.5 * 0.25, 0.0, 3 * 0.5 * 1.0, 7 * 0.75 * 1.0], rtol=1e-14)
    # q = 1 normalises by the largest volume (gamma = v / 8), q = 0 by the smallest (gamma = 1)
    got = oracle.significance(scene, oracle.Settings(), hits, quantile=1.0)
    np.testing.assert_allclose(got, [10 * 0.5 / 8, 0.0, 3 * 0.5 * 4 / 8, 7 * 0.75], rtol=1e-14)
    got = oracle.significance(scene, oracle.Settings(), hits, quantile=0.0)
    np.testing.assert_allclose(got, [10 * 0.5, 0.0, 3 * 0.5, 7 * 0.75], rtol=1e-14)
    # a masked Gaussian has opacity and volume 0; the quantile is taken over all n volumes
    scene["mask_logits"] = np.array([5.0, 5.0, -5.0, 5.0])
    got = oracle.significance(scene, oracle.Settings(eps_mask=0.5), hits)
    # volumes 1, 2, 0, 8 -> sorted 0, 1, 2, 8 -> rank 2: 2 -> gamma 1/2, 1, 0, 1
    np.testing.assert_allclose(got, [10 * 0.5 * 0.5, 0.0, 0.0, 7 * 0.75], rtol=1e-14)
    # q = 0 now picks the masked Gaussian's volume 0: gamma = 1 for all, the masked one still 0
    got = oracle.significance(scene, oracle.Settings(eps_mask=0.5), hits, quantile=0.0)
    np.testing.assert_allclose(got, [10 * 0.5, 0.0, 0.0, 7 * 0.75], rtol=1e-14)


def test_prune_selection_rule():
    s = np.array([3.0, 1.0, 1.0, 2.0, 0.5])
    np.testing.assert_array_equal(oracle.prune_select(s, 0.5), [False, True, False, False, True])
    np.testing.assert_array_equal(oracle.prune_select(s, 0.6), [False, True, True, False, True])
    assert not oracle.prune_select(s, 0.0).any() and oracle.prune_select(s, 1.0).all()
    rng = np.random.default_rng(3)
    x = rng.integers(0, 20, 500).astype(float)          # many ties
    sel = oracle.prune_select(x, 0.37)
    k = int(math.floor(0.37 * 500))
    ranked = sorted(range(500), key=lambda i: (x[i], i))  # the rule, by plain sorting
    assert set(np.flatnonzero(sel)) == set(ranked[:k])


# ---- compaction ----------------------------------------------------------------------------

def test_compact_keeps_order_and_drops_what_is_named():
    scene = synth.blob_scene(300, 4, 12, log_scale=(-3.0, 0.5), masks=True)
    st = oracle.Settings(eps_mask=0.5)
    rng = np.random.default_rng(5)
    remove = rng.random(300) < 0.3
    out, idx = oracle.compact(scene, st, remove)
    # by a plain loop: kept = not removed and mask logit above the float32 threshold
    tau = np.float32(math.log(0.5 / 0.5))
    want = [j for j in range(300) if not remove[j] and np.float32(scene["mask_logits"][j]) > tau]
    assert list(idx) == want
    for k in oracle.SCENE_KEYS:
        if scene.get(k) is not None:
            for new, old in enumerate(want):
                np.testing.assert_array_equal(out[k][new], scene[k][old])
    assert oracle.compact(scene, st, None, masked=False)[1].tolist() == list(range(300))
    assert oracle.compact(scene, st, np.ones(300, bool))[1].size == 0


def test_compacting_masked_gaussians_leaves_the_image_unchanged():
    # a Gaussian with M = 0 has opacity 0 and never blends (the mask equation), so removing it
    # changes no pixel
    scene = synth.blob_scene(400, 4, 13, log_scale=(-3.0, 0.5), masks=True)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    cam = synth.ring_cameras(1, [(48, 40)], radius=4.0)[0]
    out, idx = oracle.compact(scene, st)
    assert 0 < idx.size < 400
    a = oracle.render(scene, cam, st)["image"]
    b = oracle.render(out, cam, st)["image"]
    np.testing.assert_array_equal(a, b)


# ---- FP16 storage ---------------------------------------------------------------------------

def test_half_rounding_is_ieee_nearest_even():
    # binary16: 10 fraction bits, max 65504, smallest subnormal 2^-24
    x = np.array([1.0 / 3.0, 65504.0, 65519.0, 65520.0, 2.0 ** -24, 2.0 ** -26, 1.0 + 2.0 ** -11,
                  1.0 + 3.0 * 2.0 ** -11, -2.5, 1e-8], np.float64)
    want = [0.333251953125, 65504.0, 65504.0, np.inf, 2.0 ** -24, 0.0, 1.0, 1.0 + 2.0 ** -9, -2.5, 0.0]
    scene = {"means": x.reshape(-1, 1)}
    got = oracle.to_half(scene)["means"].reshape(-1)
    np.testing.assert_array_equal(got.astype(np.float64), want)


# ---- mask losses of Eq. loss3dgs ------------------------------------------------------------

def test_mask_losses_closed_forms():
    """Closed forms of the reading: sigmoid(0) = 1/2 gives L_m = L_sh = 1/2; a saturated logit
    of one band alone gives that band's share of the rest coefficients, (2l + 1) / 15 -- the
    weighting by the number of coefficients per band (Sec. "Spherical Harmonic (SH) Masking")."""
    n = 7
    zero = {"mask_logits": np.zeros(n), "sh_mask_logits": np.zeros((n, 3))}
    loss, g = oracle.mask_loss(zero, 1.0, 0.0)
    assert abs(loss - 0.5) < 1e-15
    np.testing.assert_allclose(g["mask_logits"], 0.25 / n, rtol=1e-15)
    loss, g = oracle.mask_loss(zero, 0.0, 1.0)
    assert abs(loss - 0.5) < 1e-15
    for l, coeffs in [(1, 3), (2, 5), (3, 7)]:
        b = np.full((n, 3), -60.0)
        b[:, l - 1] = 60.0
        loss, _ = oracle.mask_loss({"sh_mask_logits": b}, 0.0, 1.0)
        assert abs(loss - coeffs / 15.0) < 1e-12, (l, loss)
    # the volume mask: mean of sigmoid over the Gaussians, weight lambda_m
    m = np.array([-60.0, 60.0, 60.0, 0.0])
    loss, _ = oracle.mask_loss({"mask_logits": m}, 0.05, 0.0)
    assert abs(loss - 0.05 * 2.5 / 4) < 1e-12
    # an absent array contributes nothing
    loss, g = oracle.mask_loss({"mask_logits": None, "sh_mask_logits": None})
    assert loss == 0.0 and g["mask_logits"] is None and g["sh_mask_logits"] is None


def test_mask_losses_gradient_fd():
    rng = np.random.default_rng(17)
    sc = {"mask_logits": rng.normal(2.0, 1.5, size=9), "sh_mask_logits": rng.normal(1.0, 2.0, size=(9, 3))}
    _, g = oracle.mask_loss(sc, 0.05, 0.05)
    for key in ("mask_logits", "sh_mask_logits"):
        a = sc[key]
        for idx in np.ndindex(a.shape):
            h = 1e-6
            old = a[idx]
            a[idx] = old + h
            lp, _ = oracle.mask_loss(sc, 0.05, 0.05)
            a[idx] = old - h
            lm, _ = oracle.mask_loss(sc, 0.05, 0.05)
            a[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[key][idx]) <= 1e-9 * max(1.0, abs(fd)), (key, idx, fd, g[key][idx])


# ---- densification (clone and split) --------------------------------------------------------

def _densify_3dgs_procedure(scene, accum, count, tau_g, scale_thr, normals):
    """The same reading as 3DGS carries it out, step by step with Python lists: clone appends
    copies (their gradient statistics padded with zeros), split then selects on the extended
    set, appends the children as two stacked blocks of the selection and drops the originals."""
    keys = [k for k in oracle.SCENE_KEYS if scene.get(k) is not None]
    rows = [{k: np.array(scene[k][i], copy=True) for k in keys} for i in range(len(scene["means"]))]
    src = list(range(len(rows)))
    avg = []
    for a, c in zip(accum, count):
        avg.append(np.float32(a) / np.float32(c) if c > 0 else np.float32(0.0))
    thr = np.float32(math.log(scale_thr))
    big = lambda r: np.float32(np.max(r["log_scales"])) > thr
    n0 = len(rows)
    for i in range(n0):                                   # clone
        if avg[i] >= np.float32(tau_g) and not big(rows[i]):
            rows.append({k: v.copy() for k, v in rows[i].items()})
            src.append(i)
            avg.append(np.float32(0.0))
    sel = [i for i in range(len(rows)) if avg[i] >= np.float32(tau_g) and big(rows[i])]
    for c in range(2):                                    # split: stacked blocks of children
        for i in sel:
            r = {k: v.copy() for k, v in rows[i].items()}
            q = [float(v) for v in rows[i]["quats"]]
            nq = math.sqrt(sum(v * v for v in q))
            w, x, y, z = (v / nq for v in q)
            Rm = [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]
            s = [math.exp(float(v)) for v in rows[i]["log_scales"]]
            zz = [float(v) for v in normals[i, c]]
            r["means"] = np.array([float(rows[i]["means"][a]) + sum(Rm[a][b] * s[b] * zz[b] for b in range(3))
                                   for a in range(3)])
            r["log_scales"] = np.array([math.log(v / 1.6) for v in s])
            rows.append(r)
            src.append(src[i])
    keep = [j for j in range(len(rows)) if j not in set(sel)]
    out = {k: np.stack([rows[j][k] for j in keep]) for k in keys}
    return out, [src[j] for j in keep]


def test_densify_equals_the_3dgs_procedure():
    scene = synth.blob_scene(400, 4, 31, log_scale=(-3.0, 0.7), masks=True)
    rng = np.random.default_rng(8)
    count = rng.integers(0, 5, size=400).astype(np.int32)
    accum = (rng.exponential(0.5, size=400) * count).astype(np.float32)
    normals = rng.normal(size=(400, 2, 3))
    tau_g, thr = 0.4, math.exp(-3.0)
    out, src, n_clone, n_split = oracle.densify(scene, accum, count, tau_g, thr, normals)
    ref, ref_src = _densify_3dgs_procedure(scene, accum, count, tau_g, thr, normals)
    assert n_clone > 10 and n_split > 10
    assert list(src) == ref_src and len(src) == 400 + n_clone + n_split
    for k, v in ref.items():
        np.testing.assert_allclose(np.asarray(out[k], np.float64), v, rtol=1e-12, atol=1e-12, err_msg=k)


def test_densify_children_recover_their_normals():
    """R^T (child - parent) / scale is the caller's normal draw; log-scales drop by log 1.6; an
    axis-aligned Gaussian's children sit at mu + s * z."""
    scene = synth.blob_scene(60, 2, 32, log_scale=(-1.0, 0.3), masks=False)
    scene["quats"][0] = [1.0, 0.0, 0.0, 0.0]
    n = 60
    rng = np.random.default_rng(9)
    normals = rng.normal(size=(n, 2, 3))
    accum, count = np.ones(n, np.float32), np.ones(n, np.int32)
    out, src, n_clone, n_split = oracle.densify(scene, accum, count, 0.5, 1e-6, normals)
    assert n_clone == 0 and n_split == n and len(src) == 2 * n
    for c in range(2):
        for j in range(n):
            row = c * n + j
            q = np.asarray(scene["quats"][j], np.float64)
            Rm = oracle._rotation(q / np.linalg.norm(q))
            s = np.exp(np.asarray(scene["log_scales"][j], np.float64))
            d = out["means"][row] - np.asarray(scene["means"][j], np.float64)
            np.testing.assert_allclose(Rm.T @ d / s, normals[j, c], rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(out["log_scales"][row], np.log(s) - math.log(1.6), rtol=0, atol=1e-12)
    s0 = np.exp(np.asarray(scene["log_scales"][0], np.float64))
    np.testing.assert_allclose(out["means"][0], np.asarray(scene["means"][0], np.float64) + s0 * normals[0, 0],
                               rtol=1e-12, atol=1e-12)


def test_densify_decision_edges():
    """Zero visibility is never chosen; the gradient test is >= and the scale test strict >."""
    scene = synth.uniform_scene(4, 33)
    t = np.float32(0.25)
    scene["log_scales"][:] = np.float32(-2.0)
    accum = np.array([t, t * 2, 0.0, 5.0], np.float32)
    count = np.array([1, 2, 0, 0], np.int32)
    thr = float(np.exp(np.float64(np.float32(-2.0))))     # log(thr) rounds to the log-scale itself
    assert np.float32(np.log(np.float64(thr))) == np.float32(-2.0)
    out, src, n_clone, n_split = oracle.densify(scene, accum, count, float(t), thr, np.zeros((4, 2, 3)))
    assert (n_clone, n_split) == (2, 0) and list(src) == [0, 1, 2, 3, 0, 1]
