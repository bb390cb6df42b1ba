"""FP16 storage of trained Gaussians (the paper's post-processing): the conversion kernel
against IEEE round-to-nearest-even, and the render path reading halves -- bit for bit the
float32 render of the rounded parameters, and against the oracle."""
import numpy as np
import pytest

import oracle
from helpers import IMAGE_ATOL, image_compare
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


def scene_for(n=5000, seed=31, degree=True):
    return synth.blob_scene(n, 8, seed, log_scale=(-3.0, 0.5), masks=True, per_gaussian_degree=degree)


def test_conversion_is_ieee_nearest_even(R):
    scene = scene_for(3001)
    rng = np.random.default_rng(4)
    scene["means"] = scene["means"].copy()
    special = np.array([1.0 / 3.0, 65504.0, 65519.0, 65520.0, -70000.0, 2.0 ** -24, 2.0 ** -26,
                        1.0 + 2.0 ** -11, 1.0 + 3.0 * 2.0 ** -11, 0.0, -0.0, 1e-8, 6.1e-5], np.float32)
    flat = scene["means"].reshape(-1)
    flat[:special.size] = special
    flat[special.size:special.size + 1000] = rng.standard_normal(1000).astype(np.float32) * 300.0
    g = R.Gaussians.from_numpy(scene)
    h = R.Rasterizer.to_half(g)
    ref = oracle.to_half(scene)
    for k, t in h.params().items():
        got = np_(t)
        with np.errstate(over="ignore"):
            want = np.asarray(scene[k], np.float32).astype(np.float16)
        np.testing.assert_array_equal(got.view(np.uint16), want.view(np.uint16), err_msg=k)
        np.testing.assert_array_equal(got.astype(np.float32), ref[k], err_msg=k)


@pytest.mark.parametrize("tile,ppt", [(16, 1), (32, 2), (8, 2)])
def test_fp16_render_is_the_float32_render_of_the_rounded_parameters(R, tile, ppt):
    scene = scene_for()
    cams = synth.ring_cameras(2, [(96, 72), (61, 45)])
    rast = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    h = R.Rasterizer.to_half(g)
    g32 = R.Gaussians.from_numpy(oracle.to_half(scene))
    a = rast.forward(h, cams, want_radii=True)
    b = rast.forward(g32, cams, want_radii=True)
    for x, y in zip(a, b):
        for k in ("image", "T_final", "last", "radii"):
            assert torch.equal(x[k], y[k]), k
    hits_h = rast.count_hits(h, cams)
    hits_f = rast.count_hits(g32, cams)
    assert torch.equal(hits_h, hits_f)


def test_fp16_render_matches_oracle(R):
    scene = scene_for(4000, 32)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    cams = synth.ring_cameras(2, [(80, 60), (64, 48)])
    rast = R.Rasterizer(tile=16, eps_mask=0.5, eps_sh=0.5)
    h = R.Rasterizer.to_half(R.Gaussians.from_numpy(scene))
    outs = rast.forward(h, cams)
    sh = oracle.to_half(scene)
    for o, cam in zip(outs, cams):
        ref = oracle.render(sh, cam, st, margins=True)
        m, excl = image_compare(np_(o["image"]), ref["image"], ref["margin"])
        assert m <= IMAGE_ATOL and excl < 0.05


def test_fp16_is_refused_by_the_training_paths(R):
    from paper_2501_14534_gb300 import _binding as B
    scene = scene_for(500)
    cams = synth.ring_cameras(1, [(32, 32)])
    rast = R.Rasterizer(tile=16, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    h = R.Rasterizer.to_half(g)
    tg = [torch.rand((3, 32, 32), device="cuda")]
    with pytest.raises(B.TgsError) as e1:
        rast.train_step_batched(h, cams, tg, rast.alloc_grads(g), None, torch.zeros(1, device="cuda"))
    outs = rast.forward(h, cams)
    with pytest.raises(B.TgsError) as e2:
        rast.backward(h, cams, outs, [torch.ones((3, 32, 32), device="cuda")], grads=rast.alloc_grads(g))
    with pytest.raises(B.TgsError) as e3:
        rast.compact(h)
    for e in (e1, e2, e3):
        assert e.value.status == B.TGS_ERR_NOT_SUPPORTED
