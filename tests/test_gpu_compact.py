"""Compaction of masked and pruned Gaussians through the C ABI against the oracle: the kept
rows and the index map bit for bit, edge cases, an unchanged image after removing masked
Gaussians, and a full pruning round (hits, score, selection, compaction)."""
import math

import numpy as np
import pytest

import oracle
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


def check(R, scene, st, remove, masked):
    rast = R.Rasterizer(eps_mask=st.eps_mask, eps_sh=st.eps_sh)
    g = R.Gaussians.from_numpy(scene)
    rm = torch.from_numpy(remove.astype(np.uint8)).cuda() if remove is not None else None
    kept, idx = rast.compact(g, rm, masked=masked)
    ref, ref_idx = oracle.compact(scene, st, remove, masked=masked)
    assert kept.n == ref_idx.size
    np.testing.assert_array_equal(np_(idx).astype(np.int64), ref_idx)
    for k in oracle.SCENE_KEYS:
        if scene.get(k) is None:
            continue
        got = getattr(kept, k)
        np.testing.assert_array_equal(np_(got), np.asarray(ref[k]).astype(np_(got).dtype), err_msg=k)
    return kept


@pytest.mark.parametrize("masked,with_remove", [(True, True), (True, False), (False, True), (False, False)])
def test_compact_matches_oracle(R, masked, with_remove):
    scene = synth.blob_scene(5000, 6, 21, log_scale=(-3.0, 0.5), masks=True, per_gaussian_degree=True)
    st = oracle.Settings(eps_mask=0.5, eps_sh=0.5)
    remove = np.random.default_rng(2).random(5000) < 0.4 if with_remove else None
    check(R, scene, st, remove, masked)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1023, 1024, 1025, 70_001])
def test_compact_sizes(R, n):
    scene = synth.blob_scene(n, 3, n, log_scale=(-3.0, 0.5), masks=True)
    st = oracle.Settings(eps_mask=0.5)
    rng = np.random.default_rng(n)
    for frac in (0.0, 0.5, 1.0):
        check(R, scene, st, rng.random(n) < frac, masked=False)
    check(R, scene, st, None, masked=True)


def test_removing_masked_gaussians_leaves_the_images_unchanged(R):
    scene = synth.blob_scene(6000, 8, 22, log_scale=(-3.0, 0.5), masks=True)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    cams = synth.ring_cameras(2, [(96, 64), (61, 45)])
    rast = R.Rasterizer(tile=16, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    kept, _ = rast.compact(g, None, masked=True)
    assert 0 < kept.n < g.n
    a = rast.forward(g, cams)
    b = rast.forward(kept, cams)
    for x, y in zip(a, b):
        assert torch.equal(x["image"], y["image"])


def test_pruning_round(R):
    # hits -> score -> 60 % selection -> compaction: the survivors are the 40 % highest scores
    scene = synth.blob_scene(4000, 8, 23, log_scale=(-3.0, 0.5), masks=True)
    st = oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)
    cams = synth.ring_cameras(3, [(80, 60), (64, 64), (50, 40)])
    rast = R.Rasterizer(tile=16, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    scores = rast.significance(g, rast.count_hits(g, cams), 0.9)
    prune = rast.prune_select(scores, 0.6)
    kept, idx = rast.compact(g, prune, masked=False)
    assert kept.n == g.n - math.floor(0.6 * g.n)
    s = np_(scores)
    keep_ref = ~oracle.prune_select(s.astype(np.float64), 0.6)
    np.testing.assert_array_equal(np_(idx), np.flatnonzero(keep_ref))
    np.testing.assert_array_equal(np_(kept.means), scene["means"][keep_ref])
