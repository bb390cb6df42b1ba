"""L1 + D-SSIM loss (Eq. loss3dgs) through the C ABI against the FP64 oracle: the separable
two-kernel loss and gradient on ragged image sizes, and the batched training step with the
D-SSIM term (separate forward, loss and backward launches).

Tolerances: the GPU sums the window in float32 in another order (two 1D passes), so each
window sum carries a relative rounding error of a few 1e-7; the variances come from
E[x^2] - mu^2 and enter through 1 / (sigma_x^2 + sigma_y^2 + C2) with C2 = 9e-4, which can
amplify that error by up to (x^2 / C2) ~ 1e3 where both images are flat. Hence per view a
maximum gradient error of 2e-3 of the largest gradient magnitude, and 1e-5 relative on the loss
(a mean of millions of terms)."""
import numpy as np
import pytest

import oracle
from helpers import GRAD_RTOL, IMAGE_ATOL, image_compare, rel_err
from paper_2501_14534_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available: the GPU tests cannot run")
    from paper_2501_14534_gb300 import build
    build.build()
    from paper_2501_14534_gb300 import rasterizer as R
    return R


def np_(t):
    return t.detach().cpu().numpy()


def images_for(sizes, seed, smooth=False):
    rng = np.random.default_rng(seed)
    out = []
    for (H, W) in sizes:
        if smooth:   # rendered-like: slowly varying, low local variance
            yy, xx = np.mgrid[0:H, 0:W]
            ph = rng.random((3, 1, 1)) * 6.0
            a = 0.5 + 0.2 * np.sin(0.07 * xx[None] + 0.05 * yy[None] + ph) + 0.01 * rng.standard_normal((3, H, W))
        else:
            a = rng.random((3, H, W))
        out.append(a.astype(np.float32))
    return out


def check(R, sizes, lam, seed, smooth=False):
    rast = R.Rasterizer()
    xs = images_for(sizes, seed, smooth)
    ys = images_for(sizes, seed + 100, smooth)
    loss, grads = rast.l1_dssim_loss([torch.from_numpy(x).cuda() for x in xs],
                                     [torch.from_numpy(y).cuda() for y in ys], lam)
    ref_loss, ref_g = oracle.l1_dssim(xs, ys, lam)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss) + 1e-7, (float(loss.item()), ref_loss)
    for g, r in zip(grads, ref_g):
        err = np.abs(np_(g).astype(np.float64) - r).max()
        assert err <= 2e-3 * np.abs(r).max(), (err, np.abs(r).max())
        assert rel_err(np_(g), r) <= 1e-4


@pytest.mark.parametrize("lam", [0.2, 1.0])
@pytest.mark.parametrize("sizes", [[(45, 61)], [(22, 32), (23, 33), (1, 1), (1, 70), (70, 1), (11, 5)],
                                   [(130, 97), (64, 64)]])
def test_l1_dssim_matches_oracle(R, sizes, lam):
    check(R, sizes, lam, seed=len(sizes) * 7 + int(lam * 10))


def test_l1_dssim_smooth_images(R):
    check(R, [(90, 120), (47, 33)], 0.2, seed=31, smooth=True)


def test_lambda_zero_is_the_l1_loss(R):
    # lambda = 0: the gradient is the L1 gradient exactly and the loss the L1 loss
    rast = R.Rasterizer()
    xs = [torch.from_numpy(a).cuda() for a in images_for([(40, 50), (23, 7)], 3)]
    ys = [torch.from_numpy(a).cuda() for a in images_for([(40, 50), (23, 7)], 4)]
    loss, grads = rast.l1_dssim_loss(xs, ys, 0.0)
    l1 = torch.zeros(1, device="cuda")
    for x, y, g in zip(xs, ys, grads):
        g1 = torch.empty_like(x)
        R.Rasterizer.l1_loss(x, y, 1.0 / (x.numel() * len(xs)), l1, g1)
        assert torch.equal(g, g1)
    assert abs(loss.item() - l1.item()) <= 1e-6 * l1.item()


def test_identical_images(R):
    rast = R.Rasterizer()
    x = [torch.from_numpy(a).cuda() for a in images_for([(37, 53)], 5)]
    loss, grads = rast.l1_dssim_loss(x, [t.clone() for t in x], 0.2)
    assert abs(loss.item()) < 1e-6
    assert float(grads[0].abs().max()) < 1e-9


def batched_case(n=4000):
    scene = synth.blob_scene(n, 8, 9, log_scale=(-3.0, 0.5))
    sizes = [(40, 26), (80, 52), (80, 52), (160, 104)]
    cams = synth.ring_cameras(len(sizes), sizes)
    targets = synth.target_images(17, sizes)
    return scene, cams, targets, oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)


@pytest.mark.parametrize("tile,ppt", [(16, 1), (32, 2), (8, 2)])
def test_batched_step_with_dssim_matches_oracle(R, tile, ppt):
    scene, cams, targets, st = batched_case()
    st.tile = tile
    rast = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=st.eps_mask, eps_sh=st.eps_sh, ssim_lambda=0.2)
    g = R.Gaussians.from_numpy(scene)
    tg = [torch.from_numpy(t).cuda() for t in targets]
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n)
    loss = torch.zeros(1, device="cuda")
    images = [torch.empty((3, c.height, c.width), device="cuda") for c in cams]
    rast.plan(g, cams)
    rast.train_step_batched(g, cams, tg, grads, stats, loss, images=images, dssim=True)
    rast.poll()
    refs = [oracle.render(scene, c, st, margins=True) for c in cams]
    for v in range(len(cams)):
        m, excl = image_compare(np_(images[v]), refs[v]["image"], refs[v]["margin"])
        assert m <= IMAGE_ATOL and excl < 0.05
    ref_loss, dls = oracle.l1_dssim([r["image"] for r in refs], targets, 0.2)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    ref, _, _ = oracle.grad(scene, cams, st, dls)
    for k, t in grads.items():
        e = rel_err(np_(t), ref[k])
        assert e <= GRAD_RTOL, (k, e)


def test_batched_dssim_step_equals_its_parts(R):
    # the step = forward images, then the standalone loss, then the backward of those dL/dC;
    # and a captured graph replays it
    scene, cams, targets, st = batched_case(3000)
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=st.eps_mask, eps_sh=st.eps_sh, ssim_lambda=0.3)
    g = R.Gaussians.from_numpy(scene)
    tg = [torch.from_numpy(t).cuda() for t in targets]
    rast.plan(g, cams)
    grads = rast.alloc_grads(g)
    loss = torch.zeros(1, device="cuda")
    images = [torch.empty((3, c.height, c.width), device="cuda") for c in cams]
    rast.train_step_batched(g, cams, tg, grads, None, loss, images=images, dssim=True)
    l2, dls = rast.l1_dssim_loss(images, tg, 0.3)
    parts, _ = rast.backward(g, cams, rast.forward(g, cams), dls)
    assert abs(loss.item() - l2.item()) <= 1e-6 * abs(l2.item())
    for k in grads:
        if grads[k] is not None:
            assert rel_err(np_(grads[k]), np_(parts[k])) <= 1e-4, k
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        graphed = rast.alloc_grads(g)
        loss_g = torch.zeros(1, device="cuda")
        for _ in range(3):
            rast.train_step_batched(g, cams, tg, graphed, None, loss_g, dssim=True, graph=True)
    s.synchronize()
    rast.poll()
    assert abs(loss_g.item() - loss.item()) <= 1e-6 * abs(loss.item())
    for k in grads:
        if grads[k] is not None:
            np.testing.assert_allclose(np_(graphed[k]), np_(grads[k]), rtol=1e-4, atol=1e-7)


def test_full_size_views(R):
    # 16 views of 1280x832 in one call; two sampled views against the oracle (the gradient of a
    # view depends on that view alone, the loss is the mean over views)
    V, H, W = 16, 832, 1280
    rast = R.Rasterizer()
    rng = np.random.default_rng(8)
    xs = [torch.rand((3, H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(v)) for v in range(V)]
    ys = [torch.rand((3, H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(100 + v)) for v in range(V)]
    _, grads = rast.l1_dssim_loss(xs, ys, 0.2)
    pick = [0, int(rng.integers(1, V))]
    sub_x = [np_(xs[v]) for v in pick]
    sub_y = [np_(ys[v]) for v in pick]
    ref_loss, ref_g = oracle.l1_dssim(sub_x, sub_y, 0.2)
    for v, r in zip(pick, ref_g):
        r = r * (len(pick) / V)
        got = np_(grads[v]).astype(np.float64)
        assert np.abs(got - r).max() <= 2e-3 * np.abs(r).max()
        assert rel_err(got, r) <= 1e-4
    sub_loss, _ = rast.l1_dssim_loss([xs[v] for v in pick], [ys[v] for v in pick], 0.2)
    assert abs(sub_loss.item() - ref_loss) <= 1e-5 * ref_loss
