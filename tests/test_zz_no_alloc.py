"""tgs_bin_noalloc against tgs_bin.

tgs_bin_noalloc is the binning step for callers that must not allocate device memory (an
application that owns all device memory through its own allocator, a real-time loop, a
fixed memory budget): its scratch is a fixed array inside the library instead of a
context's arena. Its outputs must equal tgs_bin's bit for bit, on consecutive calls (the
array keeps the previous call's contents), and inputs beyond its fixed limits must be
refused with TGS_ERR_SCRATCH_LIMIT. Kept in its own file so that it is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2501_14534_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available: the GPU tests cannot run")
    from paper_2501_14534_gb300 import build
    build.build()
    from paper_2501_14534_gb300 import _binding as B
    from paper_2501_14534_gb300 import rasterizer as R
    return B, R


def _noalloc(B, R, splats, radii, n, cams, tile, capacity):
    T = sum(((c.width + tile - 1) // tile) * ((c.height + tile - 1) // tile) for c in cams)
    ids = torch.full((max(capacity, 1),), -1, device="cuda", dtype=torch.int32)
    keys = torch.full((max(capacity, 1),), -1, device="cuda", dtype=torch.int64)
    ranges = torch.full((T, 2), -1, device="cuda", dtype=torch.int32)
    K = C.c_int64(-1)
    st = B.lib.tgs_bin_noalloc(C.c_void_p(splats.data_ptr()), C.c_void_p(radii.data_ptr()), n,
                               R.cameras_array(cams), len(cams), tile,
                               C.c_void_p(ids.data_ptr()), C.c_void_p(keys.data_ptr()),
                               C.c_void_p(ranges.data_ptr()), capacity, C.byref(K),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, int(K.value), ids, keys, ranges


def _compare_with_bin(B, R, rast, g, cams, tile, tag):
    splats, radii = rast.preprocess(g, cams)
    ids_ref, keys_ref, ranges_ref, K = rast.bin(splats, radii, g.n, cams)
    torch.cuda.synchronize()
    assert 0 < K <= B.TGS_NOALLOC_MAX_KEYS and g.n * len(cams) <= B.TGS_NOALLOC_MAX_RECORDS
    st, K2, ids, keys, ranges = _noalloc(B, R, splats, radii, g.n, cams, tile, K)
    assert st == B.TGS_OK, B.lib.tgs_status_string(st)
    assert K2 == K, (tag, K2, K)
    assert torch.equal(ids[:K], ids_ref), tag
    assert torch.equal(keys[:K], keys_ref), tag
    assert torch.equal(ranges, ranges_ref), tag
    return K


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_noalloc_larger_then_smaller_scenes(tile):
    """The array keeps what the previous call left in it: a call with more visible records
    and keys, then calls with fewer (the same Gaussians mostly masked out, then fewer
    Gaussians), must each equal tgs_bin bit for bit."""
    B, R = _setup()
    scene = synth.blob_scene(30000, 8, 23, log_scale=(-3.2, 0.5))
    cams = synth.ring_cameras(2, [(160, 104), (96, 64)])
    rast = R.Rasterizer(tile=tile, ppt=2 if tile == 8 else 1, eps_mask=0.5, eps_sh=0.5)
    K_big = _compare_with_bin(B, R, rast, R.Gaussians.from_numpy(scene), cams, tile, "all")
    fewer = dict(scene)
    m = np.array(scene["mask_logits"], copy=True)
    m[np.random.default_rng(4).random(m.shape[0]) < 0.7] = -5.0   # 70 % masked: not visible
    fewer["mask_logits"] = m
    K_fewer = _compare_with_bin(B, R, rast, R.Gaussians.from_numpy(fewer), cams, tile, "masked")
    small = {k: (v[:7000] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    K_small = _compare_with_bin(B, R, rast, R.Gaussians.from_numpy(small), cams, tile, "fewer")
    assert K_big > K_fewer and K_big > K_small


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_noalloc_equals_bin_on_consecutive_calls(tile):
    B, R = _setup()
    scene = synth.blob_scene(30000, 8, 21, log_scale=(-3.2, 0.5))
    cams = synth.ring_cameras(2, [(160, 104), (96, 64)])
    rast = R.Rasterizer(tile=tile, ppt=2 if tile == 8 else 1, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    splats, radii = rast.preprocess(g, cams)
    ids_ref, keys_ref, ranges_ref, K = rast.bin(splats, radii, g.n, cams)
    torch.cuda.synchronize()
    assert 0 < K <= B.TGS_NOALLOC_MAX_KEYS and g.n * len(cams) <= B.TGS_NOALLOC_MAX_RECORDS
    for call in range(2):
        st, K2, ids, keys, ranges = _noalloc(B, R, splats, radii, g.n, cams, tile, K)
        assert st == B.TGS_OK, B.lib.tgs_status_string(st)
        assert K2 == K, (call, K2, K)
        assert torch.equal(ids[:K], ids_ref), call
        assert torch.equal(keys[:K], keys_ref), call
        assert torch.equal(ranges, ranges_ref), call


def test_bin_noalloc_refuses_inputs_beyond_its_limits():
    B, R = _setup()
    cams = synth.ring_cameras(2, [(64, 48), (64, 48)])
    n = B.TGS_NOALLOC_MAX_RECORDS // 2 + 1            # n * V just above the record limit
    splats = torch.zeros((1, 12), device="cuda")
    radii = torch.zeros((1,), device="cuda", dtype=torch.int32)
    st, K, *_ = _noalloc(B, R, splats, radii, n, cams, 16, 1024)
    assert st == B.TGS_ERR_SCRATCH_LIMIT and K == 0
    # more keys than the capacity the caller offers
    scene = synth.blob_scene(4000, 4, 3, log_scale=(-3.0, 0.5))
    rast = R.Rasterizer(tile=16, eps_mask=0.5, eps_sh=0.5)
    g = R.Gaussians.from_numpy(scene)
    splats, radii = rast.preprocess(g, cams)
    st, K, *_ = _noalloc(B, R, splats, radii, g.n, cams, 16, 10)
    assert st == B.TGS_ERR_CAPACITY and K > 10
