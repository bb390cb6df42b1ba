"""Significance pruning (Eq. significance-score) through the C ABI against the FP64 oracle:
ray hits counted in the forward blend, the score from hits, opacity and volume, and the
selection of the Gaussians a pruning round removes."""
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


def case(n=3000, views=((61, 45, 0.2), (96, 80, 2.0)), seed=5):
    scene = synth.blob_scene(n, 8, seed, log_scale=(-3.0, 0.5), masks=True)
    cams = [synth.ring_cameras(1, [(w, h)], radius=4.0, height=0.5, phase=a)[0]
            for (w, h, a) in views]
    return scene, cams, oracle.Settings(tile=16, eps_mask=0.5, eps_sh=0.5)


def make_rast(R, st, ppt=1):
    return R.Rasterizer(tile=st.tile, ppt=ppt, support=st.support, low_pass=st.low_pass,
                        eps_mask=st.eps_mask, eps_sh=st.eps_sh, near=st.near, bg=st.bg)


def np_(t):
    return t.detach().cpu().numpy()


def oracle_hits_with_slack(scene, cams, st):
    """Oracle hits summed over the views, and per Gaussian the number of pixels of its rect
    (over the views) where some blend decision is not clear of its threshold (margin < 1):
    a decision that flips between float32 and float64 changes the Gaussian's hits by at most
    one per such pixel (also through the pixel's stop, which moves every later fragment)."""
    n = np.shape(scene["means"])[0]
    hits = np.zeros(n, np.int64)
    slack = np.zeros(n, np.int64)
    for cam in cams:
        ref = oracle.render(scene, cam, st, margins=True)
        sp = ref["splats"]
        hits += oracle.hits(sp, cam.width, cam.height, tile=st.tile)
        u = (ref["margin"] < 1.0).astype(np.int64)
        I = np.zeros((cam.height + 1, cam.width + 1), np.int64)   # integral image
        I[1:, 1:] = u.cumsum(0).cumsum(1)
        vis = sp["radius"] > 0
        x0, x1, y0, y1 = (np.clip(sp["rect"][:, k], 0, (cam.width - 1, cam.width - 1,
                                                       cam.height - 1, cam.height - 1)[k])
                          for k in range(4))
        cnt = I[y1 + 1, x1 + 1] - I[y0, x1 + 1] - I[y1 + 1, x0] + I[y0, x0]
        slack += np.where(vis, cnt, 0)
    return hits, slack


@pytest.mark.parametrize("tile,ppt", [(16, 1), (32, 2), (8, 2)])
def test_count_hits_matches_oracle(R, tile, ppt):
    scene, cams, st = case()
    st.tile = tile
    rast = make_rast(R, st, ppt)
    g = R.Gaussians.from_numpy(scene)
    gpu = np_(rast.count_hits(g, cams)).astype(np.int64)
    ref, slack = oracle_hits_with_slack(scene, cams, st)
    hit = ref > 0
    assert (slack[hit] == 0).mean() > 0.3, (slack[hit] == 0).mean()
    np.testing.assert_array_equal(gpu[slack == 0], ref[slack == 0])
    assert np.all(np.abs(gpu - ref) <= slack)
    assert abs(int(gpu.sum()) - int(ref.sum())) <= 1e-3 * ref.sum()
    assert ref.sum() > 1000


def test_hits_are_the_contributing_fragments(R):
    # the same blend decisions: summed over the Gaussians, the hits are the per-pixel counts
    # of blended fragments of a forward with counters
    scene, cams, st = case(4000, ((128, 96, 0.7), (75, 41, 2.5)), seed=8)
    rast = make_rast(R, st)
    g = R.Gaussians.from_numpy(scene)
    hits = np_(rast.count_hits(g, cams)).astype(np.int64)
    outs = rast.forward(g, cams, want_counts=True)
    assert hits.sum() == sum(int(np_(o["n_contrib"]).sum()) for o in outs) > 0
    again = np_(rast.count_hits(g, cams, torch.from_numpy(hits.astype(np.int32)).cuda())).astype(np.int64)
    np.testing.assert_array_equal(again, 2 * hits)   # counts add up over calls


@pytest.mark.parametrize("fused", [True, False])
def test_batched_step_counts_the_same_hits(R, fused):
    scene, cams, st = case(3000, ((96, 64, 0.4), (61, 45, 1.9), (40, 40, 3.0)), seed=11)
    st.tile = 32
    rast = make_rast(R, st, ppt=2)
    g = R.Gaussians.from_numpy(scene)
    targets = [torch.rand((3, c.height, c.width), device="cuda") for c in cams]
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n, hits=True)
    loss = torch.zeros(1, device="cuda")
    rast.plan(g, cams)
    rast.train_step_batched(g, cams, targets, grads, stats, loss, fused=fused)
    rast.poll()
    ref = np_(rast.count_hits(g, cams))
    np.testing.assert_array_equal(np_(stats["hit_count"]), ref)
    # without the counter the step's gradients are the same
    grads2 = rast.alloc_grads(g)
    stats2 = rast.alloc_stats(g.n)
    rast.train_step_batched(g, cams, targets, grads2, stats2, loss, fused=fused)
    for k in grads:
        if grads[k] is not None:
            torch.testing.assert_close(grads2[k], grads[k], rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("quantile", [0.9, 0.0, 1.0, 0.37])
def test_significance_matches_oracle(R, quantile):
    scene, cams, st = case(2500, ((80, 60, 1.1),), seed=13)
    rast = make_rast(R, st)
    g = R.Gaussians.from_numpy(scene)
    hits = rast.count_hits(g, cams)
    got = np_(rast.significance(g, hits, quantile)).astype(np.float64)
    ref = oracle.significance(scene, st, np_(hits).astype(np.int64), quantile)
    assert (ref > 0).sum() > 100
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6 * ref.max())


def test_prune_select_rule(R):
    rast = make_rast(R, oracle.Settings())
    rng = np.random.default_rng(21)
    for n, frac, ties in [(1, 0.5, False), (1000, 0.6, False), (5000, 0.42, True), (777, 1.0, True),
                          (3000, 0.0, False), (100_003, 0.6 * 0.7, True)]:
        x = rng.integers(0, 50, n).astype(np.float32) if ties else rng.random(n).astype(np.float32)
        got = np_(rast.prune_select(torch.from_numpy(x).cuda(), frac))
        ref = oracle.prune_select(x.astype(np.float64), frac)
        np.testing.assert_array_equal(got, ref)
        assert got.sum() == math.floor(frac * n)


def test_pruning_round_on_the_benchmark_scene(R):
    # 1M Gaussians, 16 views 1280x832: the hits of a batched step equal its blended fragments,
    # and a 60 % pruning round removes exactly the lowest 60 % of the GPU's scores
    w = synth.workload(2)
    rast = R.Rasterizer(tile=32, ppt=2, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    g = R.Gaussians.from_numpy(w["scene"])
    tg = [torch.from_numpy(t).cuda() for t in w["targets"]]
    rast.plan(g, w["cams"], 1.15)
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n, hits=True)
    loss = torch.zeros(1, device="cuda")
    rast.train_step_batched(g, w["cams"], tg, grads, stats, loss)
    rast.poll()
    hits = stats["hit_count"]
    contrib = 0
    counter = R.Rasterizer(tile=32, ppt=2, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    for cam in w["cams"]:
        contrib += int(np_(counter.forward(g, [cam], want_counts=True)[0]["n_contrib"]).sum())
    assert int(np_(hits).astype(np.int64).sum()) == contrib
    scores = rast.significance(g, hits, 0.9)
    prune = np_(rast.prune_select(scores, 0.6))
    s = np_(scores).astype(np.float64)
    assert prune.sum() == math.floor(0.6 * g.n)
    np.testing.assert_array_equal(prune, oracle.prune_select(s, 0.6))
    assert s[prune].max() <= s[~prune].min()


def _keys_oracle(rec, rad, cams, n, tile):
    """The key oracle's sorted keys, ids and ranges of V views' float32 records (views
    concatenated as the library numbers them)."""
    from helpers import cull_data, splats_to_oracle
    ek, ev, er, toff = [], [], [], 0
    for v, cam in enumerate(cams):
        r_v, d_v = rec[v * n:(v + 1) * n], rad[v * n:(v + 1) * n]
        gs = splats_to_oracle(r_v, d_v)
        k, vv, r = oracle.keys(gs["radius"], gs["rect"], r_v[:, 11], cam.width, cam.height, tile,
                               tile_offset=toff, value_offset=v * n, cull=cull_data(r_v))
        base = sum(len(x) for x in ek)
        r = r.copy()
        r[r[:, 1] > 0] += base
        ek.append(k)
        ev.append(vv)
        er.append(r)
        toff += r.shape[0]
    return np.concatenate(ek), np.concatenate(ev), np.concatenate(er)


def _bin_and_compare(R, rast, g, cams, st):
    """Bins g's records in rast's context and in a fresh one; both must equal the key oracle."""
    splats, radii = rast.preprocess(g, cams)
    ids, keys, ranges, K = rast.bin(splats, radii, g.n, cams)
    fresh = make_rast(R, st)
    ids_f, keys_f, ranges_f, K_f = fresh.bin(splats, radii, g.n, cams)
    assert K == K_f > 0
    assert torch.equal(ids, ids_f) and torch.equal(keys, keys_f) and torch.equal(ranges, ranges_f)
    ek, ev, er = _keys_oracle(np_(splats), np_(radii), cams, g.n, st.tile)
    assert np.array_equal(np_(keys).view(np.uint64), ek)
    assert np.array_equal(np_(ids).view(np.uint32), ev)
    assert np.array_equal(np_(ranges).view(np.uint32), er)
    return K


def test_binning_after_significance_and_compaction_in_one_context(R):
    """The per-record scratch of a context is reused: the volumes of tgs_significance and the
    key counts of an earlier binning with more visible records must not leak into a later
    binning. One context runs a pruning round (hits, score, selection), bins again, compacts
    and bins the smaller scene; every binning equals a fresh context's and the key oracle."""
    scene, cams, st = case(3000)
    rast = make_rast(R, st)
    g = R.Gaussians.from_numpy(scene)
    K0 = _bin_and_compare(R, rast, g, cams, st)
    hits = rast.count_hits(g, cams)
    scores = rast.significance(g, hits, 0.9)
    prune = rast.prune_select(scores, 0.6)
    # the hit-counting binnings after tgs_significance reused the count scratch for volumes
    hits2 = rast.count_hits(g, cams)
    assert torch.equal(hits2, hits)
    assert _bin_and_compare(R, rast, g, cams, st) == K0
    kept, _ = rast.compact(g, prune, masked=True)
    assert 0 < kept.n < g.n
    K1 = _bin_and_compare(R, rast, kept, cams, st)
    assert K1 < K0
    # a second pruning round in the same context
    scores = rast.significance(kept, rast.count_hits(kept, cams), 0.9)
    kept2, _ = rast.compact(kept, rast.prune_select(scores, 0.6 * 0.7), masked=True)
    assert 0 < kept2.n < kept.n
    assert _bin_and_compare(R, rast, kept2, cams, st) < K1
    rast.poll()
