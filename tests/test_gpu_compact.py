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


# ---- densification (clone and split) ---------------------------------------------------------

@pytest.mark.parametrize("n,degree", [(1, False), (33, False), (1025, True), (70001, False)])
def test_densify_matches_oracle(R, n, degree):
    """tgs_densify against the oracle on seeded statistics: the same Gaussians cloned and split
    (decisions bit-exact, in float32 on both sides), the index map and every copied row bit for
    bit, the children's means and log-scales within float32 rounding of the float64 oracle."""
    scene = synth.blob_scene(n, 4, 40 + n, log_scale=(-3.0, 0.7), masks=not degree, per_gaussian_degree=degree)
    rng = np.random.default_rng(n)
    count = rng.integers(0, 6, size=n).astype(np.int32)
    accum = (rng.exponential(0.5, size=n) * count).astype(np.float32)
    normals = rng.normal(size=(n, 2, 3)).astype(np.float32)
    tau_g, thr = 0.45, math.exp(-3.0)
    rast = R.Rasterizer()
    g = R.Gaussians.from_numpy(scene)
    stats = {"grad_norm_accum": torch.from_numpy(accum).cuda(), "vis_count": torch.from_numpy(count).cuda()}
    new, src, nc, ns = rast.densify(g, stats, torch.from_numpy(normals).cuda(), tau_g, thr)
    ref, ref_src, rc, rs = oracle.densify(scene, accum, count, tau_g, thr, normals.astype(np.float64))
    assert (nc, ns) == (rc, rs) and new.n == len(ref_src)
    np.testing.assert_array_equal(np_(src).astype(np.int64), ref_src)
    if n >= 1025:
        assert nc > 0 and ns > 0
    child = np.arange(new.n) >= n - ns + nc           # rows of the split children
    for k in oracle.SCENE_KEYS:
        if scene.get(k) is None:
            continue
        got = np_(getattr(new, k) if k != "sh_degree" else new.sh_degree)
        if k in ("means", "log_scales"):
            np.testing.assert_array_equal(got[~child], np.asarray(scene[k])[ref_src[~child]])
            np.testing.assert_allclose(got[child], ref[k][child], rtol=2e-6, atol=2e-6, err_msg=k)
        else:
            np.testing.assert_array_equal(got, ref[k], err_msg=k)


def test_densify_reports_capacity(R):
    from paper_2501_14534_gb300 import _binding as B
    import ctypes as C
    scene = synth.blob_scene(500, 4, 41, log_scale=(-3.0, 0.7))
    g = R.Gaussians.from_numpy(scene)
    rast = R.Rasterizer()
    stats = {"grad_norm_accum": torch.full((500,), 10.0, device="cuda"),
             "vis_count": torch.ones(500, device="cuda", dtype=torch.int32)}
    normals = torch.zeros((500, 2, 3), device="cuda")
    out = {k: torch.empty_like(v) for k, v in g.params().items()}
    n_out, nc, ns = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    st = B.lib.tgs_densify(rast._h, C.byref(g.struct()), C.byref(rast._stats_struct(stats)),
                           C.c_void_p(normals.data_ptr()), 1.0, 0.05, C.byref(rast._grad_struct(out)), None, None,
                           500, C.byref(n_out), C.byref(nc), C.byref(ns),
                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.TGS_ERR_CAPACITY and n_out.value == 1000 and nc.value + ns.value == 500
