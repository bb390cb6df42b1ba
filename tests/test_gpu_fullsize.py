"""Parity at the workloads' full sizes, on sampled outputs the FP64 oracle computes tile by
tile (a tile's pixels depend only on that tile's list, so any subset of tiles is exact):

- 1M Gaussians, 16 views of 1280x832, batched fused step in the benchmark's launch
  configuration: images on sampled tiles, keys bit-exact for one view, the backward on
  sampled tiles (sparse dL/dimage), fused and unfused gradients equal, and every parameter
  gradient of the fused step against the oracle's blend backward + preprocess backward with
  the loss restricted to sampled tiles of all 16 views;
- 3M Gaussians, 8 views of 1600x1064, the autograd path with per-view checkpointing:
  gradients of 64 random parameters against FP64 central differences, each difference
  re-blending only the tiles the perturbed Gaussian touches;
- 300K Gaussians with per-Gaussian SH degree at 1920x1080 (render only) and 500K Gaussians
  over 16 mixed-resolution views (batched): images on sampled tiles, and for the batch every
  parameter gradient as for 1M.

The batched step computes its own L1 gradient sign(C - target) / (3 H W V). To restrict the
loss to sampled tiles, the target equals the step's own rendered image everywhere else (sign(0)
= 0 gives dL/dC = 0 there, exactly), and on the sampled tiles it sits 0.02..0.5 away from the
oracle's image, on a random side, at the pixels whose blend decisions are clear of their
thresholds (elsewhere it equals the rendered image too). The oracle's dL/dC is that random
sign times 1 / (3 H W V) on those pixels and 0 elsewhere: it never reads a GPU value.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2501_14534_gb300 import synth

from helpers import IMAGE_ATOL, check_grad, cull_data, elem_err, gpu_lists, rel_err, splats_to_oracle

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, len(os.sched_getaffinity(0))))

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


def tile_grid(cam, tile):
    return (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile


def sample_tiles(cam, tile, ranges=None, n_rand=12, n_heavy=4, seed=0):
    gx, gy = tile_grid(cam, tile)
    mask = np.zeros(gx * gy, np.uint8)
    rng = np.random.default_rng(seed)
    mask[rng.choice(gx * gy, size=min(n_rand, gx * gy), replace=False)] = 1
    if ranges is not None:
        lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
        mask[np.argsort(-lens)[:n_heavy]] = 1
    return mask


def pixel_mask(mask, cam, tile):
    gx, gy = tile_grid(cam, tile)
    return np.repeat(np.repeat(mask.reshape(gy, gx), tile, 0), tile, 1)[:cam.height, :cam.width].astype(bool)


def check_tiles(img, ref, pix):
    clear = (ref["margin"] >= 1.0) & pix
    diff = np.abs(np.asarray(img, np.float64) - ref["image"]).max(axis=0)
    assert clear.sum() > 0.95 * pix.sum()
    m = diff[clear].max()
    assert m <= IMAGE_ATOL, m
    return m


def sparse_step_gradients(R, rast, g, scene, cams, st, tile, seed, n_rand=3, n_heavy=1):
    """Runs the batched fused step with the loss restricted to sampled tiles of every view
    (see the module docstring) and returns its gradients and statistics with the oracle's.
    The oracle blends the GPU's float32 records over the key oracle's lists of them, then
    runs its float64 preprocess backward."""
    V = len(cams)
    tg0 = [torch.zeros((3, c.height, c.width), device="cuda") for c in cams]
    images = [torch.empty((3, c.height, c.width), device="cuda") for c in cams]
    loss = torch.zeros(1, device="cuda")
    rast.plan(g, cams, headroom=1.15)
    rast.train_step_batched(g, cams, tg0, rast.alloc_grads(g), None, loss, images=images)
    rast.poll()
    rng = np.random.default_rng(seed)
    targets, dls, masks, lists_of, n_px = [], [], [], [], 0
    for v, cam in enumerate(cams):
        W, H = cam.width, cam.height
        splats, radii = rast.preprocess(g, [cam])
        rec, rad = np_(splats), np_(radii)
        gs = splats_to_oracle(rec, rad)
        lists = gpu_lists(rec, rad, W, H, tile)
        mask = sample_tiles(cam, tile, lists[1], n_rand=n_rand, n_heavy=n_heavy, seed=seed + v)
        ref = oracle.blend(gs, W, H, tile, st.bg, margins=True, tile_mask=mask, lists=lists,
                           nthreads=NTHREADS)
        img = np_(images[v])
        pix = pixel_mask(mask, cam, tile)
        check_tiles(img, ref, pix)
        clear = pix & (ref["margin"] >= 1.0)
        sgn = rng.choice([-1.0, 1.0], size=(3, H, W))
        t = img.copy()
        t[:, clear] = (ref["image"] - sgn * rng.uniform(0.02, 0.5, size=(3, H, W)))[:, clear].astype(np.float32)
        dl = np.zeros((3, H, W))
        dl[:, clear] = sgn[:, clear] / (3.0 * W * H * V)
        targets.append(torch.from_numpy(t).cuda())
        dls.append(dl)
        masks.append(mask)
        lists_of.append(lists)
        n_px += int(clear.sum())
    grads = rast.alloc_grads(g)
    stats = rast.alloc_stats(g.n)
    rast.train_step_batched(g, cams, targets, grads, stats, loss)
    rast.poll()
    ref_g = oracle.zero_grads(scene)
    rstats = oracle.new_stats(g.n)
    for v, cam in enumerate(cams):
        splats, radii = rast.preprocess(g, [cam])
        rec, rad = np_(splats), np_(radii)
        gs = splats_to_oracle(rec, rad)
        g9 = oracle.blend_backward(gs, cam.width, cam.height, dls[v], tile, st.bg, nthreads=NTHREADS,
                                   tile_mask=masks[v], lists=lists_of[v])
        oracle.preprocess_backward(scene, cam, st, g9, ref_g, rstats)
    return grads, stats, ref_g, rstats, n_px


def check_sparse_gradients(grads, stats, ref_g, rstats, tag):
    for k, t in grads.items():
        got = np_(t)
        e, r = check_grad(got, ref_g[k], k)
        print(f"GRAD {tag} {k} rel={e:.3e} elem={r:.3f} nonzero={int(np.count_nonzero(ref_g[k]))}")
    cnt = np_(stats["vis_count"])
    assert np.mean(cnt != rstats["count"]) <= 1e-4
    same = cnt == rstats["count"]
    acc = np_(stats["grad_norm_accum"])[same]
    assert rel_err(acc, rstats["accum"][same]) <= 1e-3 and elem_err(acc, rstats["accum"][same]) <= 1.0


# ------------------------------------------------------------------------------------
# 1M Gaussians, 16 x 1280x832, batched fused step
# ------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2(R):
    w = synth.workload(2)
    g = R.Gaussians.from_numpy(w["scene"])
    tg = [torch.from_numpy(t).cuda() for t in w["targets"]]
    return w, g, tg


def test_1m_16views_batched_step_parameter_gradients(R, c2):
    """Every parameter gradient and statistic of the fused step in the benchmark's launch
    configuration (tile 32, 2 pixels per thread) against the oracle, the loss on 4 sampled
    tiles of each of the 16 views (the heaviest one among them)."""
    w, g, tg = c2
    cams = w["cams"]
    st = oracle.Settings(tile=32, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast = R.Rasterizer(tile=32, ppt=2, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    grads, stats, ref_g, rstats, n_px = sparse_step_gradients(R, rast, g, w["scene"], cams, st, 32, 200)
    assert n_px > 16 * 3 * 1000
    check_sparse_gradients(grads, stats, ref_g, rstats, "1M")


@pytest.mark.parametrize("tile,ppt", [(32, 2), (16, 1)])
def test_1m_16views_batched_step_sampled_tiles(R, c2, tile, ppt):
    w, g, tg = c2
    cams = w["cams"]
    st = oracle.Settings(tile=tile, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast.plan(g, cams, headroom=1.15)
    images = [torch.empty((3, c.height, c.width), device="cuda") for c in cams]
    grads = rast.alloc_grads(g)
    loss = torch.zeros(1, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):   # capture, then replay
            rast.train_step_batched(g, cams, tg, grads, None, loss, images=images, graph=True)
    s.synchronize()
    rast.poll()
    # the fused loss equals the loss of the images it wrote
    l_img = sum(float((im - t).abs().mean()) for im, t in zip(images, tg)) / len(cams)
    assert abs(loss.item() - l_img) <= 1e-5 * l_img
    # fused and unfused steps: same arithmetic, different atomic order
    g2 = rast.alloc_grads(g)
    rast.train_step_batched(g, cams, tg, g2, None, loss, fused=False)
    rast.poll()
    for k in grads:
        assert rel_err(np_(g2[k]), np_(grads[k])) <= 1e-4, k
    # images on sampled tiles of three views, against the oracle blending the same records
    for v in (0, 5, 11):
        cam = cams[v]
        splats, radii = rast.preprocess(g, [cam])
        ids, keys, ranges, K = rast.bin(splats, radii, g.n, [cam], want_keys=(v == 0))
        rec, rad = np_(splats), np_(radii)
        gs = splats_to_oracle(rec, rad)
        rg = np_(ranges).view(np.uint32)
        mask = sample_tiles(cam, tile, rg, seed=v)
        ref = oracle.blend(gs, cam.width, cam.height, tile, st.bg, margins=True, tile_mask=mask,
                           nthreads=NTHREADS)
        check_tiles(np_(images[v]), ref, pixel_mask(mask, cam, tile))
        if v == 0:
            # binning of a full view: bit-exact against the key oracle
            ek, ev, er = oracle.keys(gs["radius"], gs["rect"], rec[:, 11], cam.width, cam.height, tile,
                                     cull=cull_data(rec))
            assert np.array_equal(np_(keys).view(np.uint64), ek)
            assert np.array_equal(np_(ids).view(np.uint32), ev)
            assert np.array_equal(rg, er)
            # backward on the sampled tiles: dL/dimage nonzero only there
            pix = pixel_mask(mask, cam, tile)
            rng = np.random.default_rng(3)
            dl = (rng.normal(size=(3, cam.height, cam.width)) * pix[None]).astype(np.float32)
            outs = rast.blend_forward(splats, ids, ranges, [cam])
            sg = np_(rast.blend_backward(splats, ids, ranges, [cam], outs, [torch.from_numpy(dl).cuda()]))
            rg9 = oracle.blend_backward(gs, cam.width, cam.height, dl, tile, st.bg, nthreads=NTHREADS,
                                        tile_mask=mask)
            for name, cols in [("mean2d", [0, 1]), ("conic", [2, 3, 4]), ("opacity", [5]),
                               ("rgb", [6, 7, 8])]:
                assert rel_err(sg[:, cols], rg9[:, cols]) <= 1e-3, name


# ------------------------------------------------------------------------------------
# 3M Gaussians, 8 x 1600x1064: finite differences of 64 parameters
# ------------------------------------------------------------------------------------

def test_3m_8views_checkpointed_gradients_against_fp64_fd(R):
    w = synth.workload(5)
    scene, cams = w["scene"], w["cams"]
    st = oracle.Settings(tile=16, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast = R.Rasterizer(tile=16, ppt=1, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    g = R.Gaussians.from_numpy(scene)
    keys = ["means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest"]
    for k in keys:
        getattr(g, k).requires_grad_(True)
    rng = np.random.default_rng(55)
    ws = [rng.normal(size=(3, c.height, c.width)).astype(np.float32) for c in cams]
    imgs = R.rasterize(rast, g, cams)                      # per-view checkpointed autograd
    loss = sum((im * torch.from_numpy(wv).cuda()).sum() for im, wv in zip(imgs, ws))
    loss.backward()
    gpu = {k: np_(getattr(g, k).grad) for k in keys}
    del imgs, loss
    torch.cuda.empty_cache()

    base = [oracle.preprocess(scene, c, st) for c in cams]
    vis = np.zeros(scene["means"].shape[0], bool)
    for b in base:
        vis |= b["radius"] > 0
    cand = np.nonzero(vis)[0]
    params = {k: np.array(scene[k], dtype=np.float64) for k in keys}
    sc64 = dict(scene, **params)
    fields = ("mean2d", "depth", "conic", "opacity", "rgb", "radius", "rect")

    def record(v, i, k=None, idx=None, val=None):
        """Oracle record of Gaussian i in view v, with one parameter set to val."""
        if k is not None:
            old = params[k][(i,) + idx]
            params[k][(i,) + idx] = val
        one = {kk: (vv[i:i + 1] if isinstance(vv, np.ndarray) else vv) for kk, vv in sc64.items()}
        p1 = oracle.preprocess(one, cams[v], st)
        if k is not None:
            params[k][(i,) + idx] = old
        return {f: p1[f][0].copy() for f in fields}

    # tile coordinates of every Gaussian's rect per view; a difference then blends only the
    # Gaussians with a key in the perturbed Gaussian's tiles: the same tile lists restricted
    # to those tiles (ascending ids keep the order of depth ties)
    trect = [np.where(b["radius"][:, None] > 0, b["rect"] // 16, -1) for b in base]

    def blend_three(v, i, recs):
        """Blends of view v with Gaussian i's record replaced by each of recs, on its tiles:
        the Gaussians with a key in those tiles, in an image cropped to them (shifted by whole
        tiles, so every tile list and pixel value is unchanged)."""
        cam = cams[v]
        x0, x1, y0, y1 = (int(c) for c in recs[0]["rect"] // 16)
        tr = trect[v]
        sub = np.nonzero((tr[:, 1] >= x0) & (tr[:, 0] <= x1) & (tr[:, 3] >= y0) & (tr[:, 2] <= y1))[0]
        j = int(np.searchsorted(sub, i))
        assert sub[j] == i
        ox, oy = 16 * x0, 16 * y0
        Wc, Hc = min(cam.width, 16 * (x1 + 1)) - ox, min(cam.height, 16 * (y1 + 1)) - oy
        sp = {f: np.ascontiguousarray(base[v][f][sub]) for f in fields}
        sp["m_all"] = sp["m_edge"] = None
        wv = ws[v][:, oy:oy + Hc, ox:ox + Wc]
        outs = []
        for r in recs:
            for f in fields:
                sp[f][j] = r[f]
            # shift by whole tiles and clip each rect to the crop (a pixel of the crop is in
            # the clipped rect exactly when it is in the original one)
            rc = sp["rect"] - np.array([ox, ox, oy, oy], np.int32)
            rc = np.column_stack([np.maximum(rc[:, 0], 0), np.minimum(rc[:, 1], Wc - 1),
                                  np.maximum(rc[:, 2], 0), np.minimum(rc[:, 3], Hc - 1)])
            cs = dict(sp, mean2d=sp["mean2d"] - np.array([ox, oy], float),
                      rect=np.ascontiguousarray(rc, dtype=np.int32))
            o = oracle.blend(cs, Wc, Hc, 16, st.bg, nthreads=NTHREADS)
            outs.append((float((o["image"] * wv).sum()), o["n_contrib"].copy(), o["last"].copy()))
        return outs

    fd_vals, gpu_vals, tries = [], [], 0
    while len(fd_vals) < 64 and tries < 400:
        tries += 1
        i = int(rng.choice(cand))
        k = keys[rng.integers(len(keys))]
        idx = tuple(int(rng.integers(0, s_)) for s_ in params[k].shape[1:])
        x = params[k][(i,) + idx]
        h = 1e-6 * max(1.0, abs(x))
        dL, ok = 0.0, True
        for v, cam in enumerate(cams):
            r0 = record(v, i)
            rp, rm = record(v, i, k, idx, x + h), record(v, i, k, idx, x - h)
            if any(r["radius"] != r0["radius"] or not np.array_equal(r["rect"], r0["rect"])
                   for r in (rp, rm)):
                ok = False   # the footprint itself moves: not differentiable here
                break
            if r0["radius"] <= 0:
                continue
            o0, op, om = blend_three(v, i, (r0, rp, rm))
            if not all(np.array_equal(o[1], o0[1]) and np.array_equal(o[2], o0[2]) for o in (op, om)):
                ok = False   # a blend decision flips between x - h and x + h
                break
            lp, lm = op[0], om[0]
            dL += (lp - lm) / (2 * h)
        if not ok:
            continue
        fd_vals.append(dL)
        gpu_vals.append(float(gpu[k][(i,) + idx]))
    assert len(fd_vals) == 64, (len(fd_vals), tries)
    fd_vals, gpu_vals = np.array(fd_vals), np.array(gpu_vals)
    for a, b in zip(gpu_vals, fd_vals):
        print(f"FD3M gpu={a:.9e} fd={b:.9e}")
    e, r = check_grad(gpu_vals, fd_vals, "3M finite differences")
    print(f"FD3M rel={e:.3e} elem={r:.3f}")


# ------------------------------------------------------------------------------------
# 300K, per-Gaussian SH degree, 1920x1080 render; 500K, 16 mixed views batched
# ------------------------------------------------------------------------------------

def test_300k_1920x1080_render_sampled_tiles(R):
    w = synth.workload(4, n_views=3)
    scene, cams = w["scene"], w["cams"]
    st = oracle.Settings(tile=16, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast = R.Rasterizer(tile=16, ppt=1)
    g = R.Gaussians.from_numpy(scene)
    outs = rast.forward(g, cams)
    for v, cam in enumerate(cams):
        mask = sample_tiles(cam, 16, seed=40 + v, n_rand=24)
        # end to end against the FP64 preprocess (decision-margin exclusion)
        ref = oracle.blend(oracle.preprocess(scene, cam, st), cam.width, cam.height, 16, st.bg,
                           margins=True, depth_margin=True, tile_mask=mask, nthreads=NTHREADS)
        pix = pixel_mask(mask, cam, 16)
        clear = (ref["margin"] >= 1.0) & pix
        diff = np.abs(np_(outs[v]["image"]) - ref["image"]).max(axis=0)
        assert clear.sum() > 0.9 * pix.sum()
        assert diff[clear].max() <= IMAGE_ATOL


@pytest.mark.parametrize("tile,ppt", [(16, 1), (32, 2)])
def test_500k_16_mixed_views_batched_sampled_tiles(R, tile, ppt):
    w = synth.workload(3)
    scene, cams = w["scene"], w["cams"]
    st = oracle.Settings(tile=tile, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    rast = R.Rasterizer(tile=tile, ppt=ppt, eps_mask=w["eps_mask"], eps_sh=w["eps_sh"])
    g = R.Gaussians.from_numpy(scene)
    tg = [torch.from_numpy(t).cuda() for t in w["targets"]]
    images = [torch.empty((3, c.height, c.width), device="cuda") for c in cams]
    grads = rast.alloc_grads(g)
    loss = torch.zeros(1, device="cuda")
    rast.plan(g, cams)
    rast.train_step_batched(g, cams, tg, grads, None, loss, images=images)
    rast.poll()
    for v in (0, 5, 15):   # one view of each resolution
        cam = cams[v]
        splats, radii = rast.preprocess(g, [cam])
        gs = splats_to_oracle(np_(splats), np_(radii))
        mask = sample_tiles(cam, tile, seed=70 + v, n_rand=16)
        ref = oracle.blend(gs, cam.width, cam.height, tile, st.bg, margins=True, tile_mask=mask,
                           nthreads=NTHREADS)
        check_tiles(np_(images[v]), ref, pixel_mask(mask, cam, tile))
    # every parameter gradient with the loss on sampled tiles of all 16 views
    grads, stats, ref_g, rstats, n_px = sparse_step_gradients(R, rast, g, scene, cams, st, tile, 300 + tile)
    check_sparse_gradients(grads, stats, ref_g, rstats, f"500K tile={tile}")
