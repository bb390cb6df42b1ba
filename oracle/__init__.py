"""FP64 CPU oracle of the Trick-GS rasterizer hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It is built from ``tgs_oracle.c`` (plain C, double precision) and shares
no code with the CUDA library.

Functions follow the paper's notation: Eq. 1 (EWA projection to G'), Eq. 2 (front-to-back
blending), the straight-through volume mask and the straight-through SH-band masks (Eq.
sh-masks), the significance score of Eq. significance-score (ray hits, opacity, volume)
and the L1 + D-SSIM loss of Eq. loss3dgs (numpy). ``tgs_oracle.c`` states the conventions
the paper inherits from 3DGS.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "tgs_oracle.c")

SUPPORT_BOX3 = 0
SUPPORT_ALPHA = 1


def build(force=False):
    """Compile the oracle with gcc (no contraction of a*b+c, so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                           _SRC, "-lm", "-lpthread"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_u8p = C.POINTER(C.c_uint8)
_f32p = C.POINTER(C.c_float)


class _Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", _dp), ("log_scales", _dp), ("quats", _dp),
                ("opacity_logits", _dp), ("sh_dc", _dp), ("sh_rest", _dp),
                ("sh_degree", _u8p), ("mask_logits", _dp), ("sh_mask_logits", _dp),
                ("deg_max", C.c_int64)]


class _Grads(C.Structure):
    _fields_ = [(k, _dp) for k in ("means", "log_scales", "quats", "opacity_logits", "sh_dc",
                                   "sh_rest", "mask_logits", "sh_mask_logits")]


class _Splats(C.Structure):
    _fields_ = [("mean2d", _dp), ("depth", _dp), ("conic", _dp), ("opacity", _dp),
                ("rgb", _dp), ("radius", _i32p), ("rect", _i32p), ("m_all", _dp),
                ("m_edge", _dp)]


def _declare(L):
    L.orc_sh_basis.argtypes = [C.c_int64, _dp, _dp, _dp]
    L.orc_preprocess.argtypes = [C.POINTER(_Params), _dp, _dp, C.POINTER(_Splats)]
    L.orc_count_keys.argtypes = [C.c_int64, _i32p, _i32p, _f32p, C.c_int, C.c_int, C.c_int]
    L.orc_count_keys.restype = C.c_int64
    L.orc_keys.argtypes = [C.c_int64, _i32p, _i32p, _dp, _f32p, C.c_int, C.c_int, C.c_int,
                           C.c_uint64, C.c_uint32, _u64p, _u32p, _u32p]
    L.orc_keys.restype = C.c_int64
    L.orc_blend.argtypes = [C.c_int64, C.POINTER(_Splats), C.c_int, C.c_int, C.c_int, _dp,
                            C.c_int, C.c_int, C.c_int, _u8p, _u32p, _u32p, _dp, _dp, _i32p,
                            _i32p, _i32p, _i32p, _dp]
    L.orc_blend_backward.argtypes = [C.c_int64, C.POINTER(_Splats), C.c_int, C.c_int, C.c_int,
                                     _dp, _dp, C.c_int, _u8p, _u32p, _u32p, _dp]
    L.orc_preprocess_backward.argtypes = [C.POINTER(_Params), _dp, _dp, _dp, C.POINTER(_Grads),
                                          _dp, _i32p, _i32p]
    L.orc_l1.argtypes = [C.c_int64, _dp, _dp, C.c_double, _dp]
    L.orc_l1.restype = C.c_double
    L.orc_hits.argtypes = [C.c_int64, C.POINTER(_Splats), C.c_int, C.c_int, C.c_int, C.c_int,
                           C.c_int, _u8p, _u32p, _u32p, C.POINTER(C.c_int64)]


def _ptr(a, t=_dp):
    if a is None:
        return C.cast(None, t)
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


@dataclasses.dataclass
class Settings:
    """Rasterizer settings: tile size, footprint rule, mask thresholds, near plane, background
    and the low-pass term s of Sigma' + sI."""
    tile: int = 16
    support: int = SUPPORT_BOX3
    eps_mask: float = 0.05
    eps_sh: float = 0.1
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    low_pass: float = 0.3


def cam_vec(cam, low_pass):
    v = np.zeros(22)
    vm = np.asarray(cam.viewmat, dtype=np.float64)
    v[0:9] = vm[:3, :3].reshape(-1)
    v[9:12] = vm[:3, 3]
    v[12:15] = np.asarray(cam.campos, dtype=np.float64)
    v[15:22] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, low_pass]
    return v


def cfg_vec(st: Settings):
    return np.array([st.tile, st.support, st.eps_mask, st.eps_sh, st.near, *st.bg],
                    dtype=np.float64)


class _Scene:
    """Keeps the float64 copies alive while the C structure points at them."""

    def __init__(self, scene):
        d = lambda k: None if scene.get(k) is None else np.ascontiguousarray(
            scene[k], dtype=np.float64)
        self.arrs = {k: d(k) for k in ("means", "log_scales", "quats", "opacity_logits",
                                       "sh_dc", "sh_rest", "mask_logits", "sh_mask_logits")}
        self.deg = None if scene.get("sh_degree") is None else np.ascontiguousarray(
            scene["sh_degree"], dtype=np.uint8)
        self.n = self.arrs["means"].shape[0]
        deg_max = 3 if self.arrs["sh_rest"] is not None else 0
        if "deg_max" in scene:
            deg_max = scene["deg_max"]
        a = self.arrs
        self.c = _Params(self.n, _ptr(a["means"]), _ptr(a["log_scales"]), _ptr(a["quats"]),
                         _ptr(a["opacity_logits"]), _ptr(a["sh_dc"]), _ptr(a["sh_rest"]),
                         _ptr(self.deg, _u8p), _ptr(a["mask_logits"]),
                         _ptr(a["sh_mask_logits"]), deg_max)


def sh_basis(dirs):
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    n = dirs.shape[0]
    Y = np.zeros((n, 16))
    dY = np.zeros((n, 16, 3))
    lib().orc_sh_basis(n, _ptr(dirs), _ptr(Y), _ptr(dY))
    return Y, dY


def _alloc_splats(n):
    return dict(mean2d=np.zeros((n, 2)), depth=np.zeros(n), conic=np.zeros((n, 3)),
                opacity=np.zeros(n), rgb=np.zeros((n, 3)), radius=np.zeros(n, np.int32),
                rect=np.zeros((n, 4), np.int32), m_all=np.full(n, np.inf),
                m_edge=np.full(n, np.inf))


def _splats_struct(s):
    return _Splats(_ptr(s["mean2d"]), _ptr(s["depth"]), _ptr(s["conic"]), _ptr(s["opacity"]),
                   _ptr(s["rgb"]), _ptr(s["radius"], _i32p), _ptr(s["rect"], _i32p),
                   _ptr(s.get("m_all")), _ptr(s.get("m_edge")))


def preprocess(scene, cam, st: Settings):
    """Per-Gaussian projection of one view (Eq. 1 with masks and SH colour)."""
    sc = _Scene(scene)
    out = _alloc_splats(sc.n)
    lib().orc_preprocess(C.byref(sc.c), _ptr(cam_vec(cam, st.low_pass)), _ptr(cfg_vec(st)),
                         C.byref(_splats_struct(out)))
    return out


def splats_from(mean2d, depth, conic, opacity, rgb, radius, rect):
    """Per-Gaussian records given from outside (e.g. float32 values), promoted to float64."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    n = np.asarray(radius).shape[0]
    return dict(mean2d=f(mean2d).reshape(n, 2), depth=f(depth).reshape(n),
                conic=f(conic).reshape(n, 3), opacity=f(opacity).reshape(n),
                rgb=f(rgb).reshape(n, 3), radius=i(radius).reshape(n), rect=i(rect).reshape(n, 4),
                m_all=None, m_edge=None)


def keys(radius, rect, depth, W, H, tile, tile_offset=0, value_offset=0, cull=None):
    """Key emission, stable sort and tile ranges of one view. ``cull`` (float32 [n,8]: mean2d
    x, y, conic a, b, c, threshold tau, b / c, b / a) applies the float32 tile cull test of the
    key definition; without it every tile of each rect gets a key."""
    radius = np.ascontiguousarray(radius, np.int32)
    rect = np.ascontiguousarray(rect, np.int32)
    depth = np.ascontiguousarray(depth, np.float64)
    cull = None if cull is None else np.ascontiguousarray(cull, np.float32)
    n = radius.shape[0]
    L = lib()
    K = L.orc_count_keys(n, _ptr(radius, _i32p), _ptr(rect, _i32p), _ptr(cull, _f32p), W, H, tile)
    gx, gy = (W + tile - 1) // tile, (H + tile - 1) // tile
    k = np.zeros(max(K, 1), np.uint64)
    v = np.zeros(max(K, 1), np.uint32)
    r = np.zeros((gx * gy, 2), np.uint32)
    L.orc_keys(n, _ptr(radius, _i32p), _ptr(rect, _i32p), _ptr(depth), _ptr(cull, _f32p), W, H,
               tile, tile_offset, value_offset, _ptr(k, _u64p), _ptr(v, _u32p), _ptr(r, _u32p))
    return k[:K], v[:K], r


def _mask(tile_mask):
    return None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)


def _lists(lists):
    if lists is None:
        return C.cast(None, _u32p), C.cast(None, _u32p), None
    vals = np.ascontiguousarray(lists[0], dtype=np.uint32)
    ranges = np.ascontiguousarray(lists[1], dtype=np.uint32)
    return _ptr(vals, _u32p), _ptr(ranges, _u32p), (vals, ranges)


def blend(splats, W, H, tile=16, bg=(0.0, 0.0, 0.0), brute=False, nthreads=1,
          margins=False, depth_margin=False, tile_mask=None, lists=None):
    """Front-to-back blending of one view (Eq. 2). Returns image [3,H,W], T_final, last
    (1-based position in the tile list of the last contributor, 0 if none), n_contrib,
    n_examined, n_eval (fragments whose rect holds the pixel, up to the stop) and, if
    requested, the per-pixel decision margin. ``tile_mask`` (one byte per
    tile, row-major) restricts the work to the tiles marked 1; other pixels stay 0. ``lists``
    = (values, ranges) from ``keys`` of the same records skips building the tile lists."""
    n = splats["radius"].shape[0]
    out = dict(image=np.zeros((3, H, W)), T_final=np.zeros((H, W)),
               last=np.zeros((H, W), np.int32), n_contrib=np.zeros((H, W), np.int32),
               n_examined=np.zeros((H, W), np.int32), n_eval=np.zeros((H, W), np.int32))
    if margins:
        out["margin"] = np.zeros((H, W))
    bgv = np.asarray(bg, dtype=np.float64)
    tm = _mask(tile_mask)
    lv, lr, _keep = _lists(lists)
    lib().orc_blend(n, C.byref(_splats_struct(splats)), W, H, tile, _ptr(bgv), int(brute),
                    nthreads, int(depth_margin), _ptr(tm, _u8p), lv, lr, _ptr(out["image"]),
                    _ptr(out["T_final"]),
                    _ptr(out["last"], _i32p), _ptr(out["n_contrib"], _i32p),
                    _ptr(out["n_examined"], _i32p), _ptr(out["n_eval"], _i32p),
                    _ptr(out.get("margin")))
    return out


def blend_backward(splats, W, H, dL_dimg, tile=16, bg=(0.0, 0.0, 0.0), nthreads=1,
                   tile_mask=None, lists=None):
    """dL/d(mean2d[2], conic[3], opacity, rgb[3]) per Gaussian, [n,9]."""
    n = splats["radius"].shape[0]
    g9 = np.zeros((n, 9))
    d = np.ascontiguousarray(dL_dimg, dtype=np.float64)
    bgv = np.asarray(bg, dtype=np.float64)
    tm = _mask(tile_mask)
    lv, lr, _keep = _lists(lists)
    lib().orc_blend_backward(n, C.byref(_splats_struct(splats)), W, H, tile, _ptr(bgv), _ptr(d),
                             nthreads, _ptr(tm, _u8p), lv, lr, _ptr(g9))
    return g9


GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest",
             "mask_logits", "sh_mask_logits")


def zero_grads(scene):
    return {k: (None if scene.get(k) is None else np.zeros(np.shape(scene[k])))
            for k in GRAD_KEYS}


def preprocess_backward(scene, cam, st: Settings, g9, grads, stats=None):
    """Adds this view's parameter gradients into ``grads`` and its statistics into ``stats``
    (dict with accum float64 [n], count int32 [n], max_radius int32 [n])."""
    sc = _Scene(scene)
    g9 = np.ascontiguousarray(g9, dtype=np.float64)
    G = _Grads(*[_ptr(grads.get(k)) for k in GRAD_KEYS])
    s = stats or {}
    lib().orc_preprocess_backward(C.byref(sc.c), _ptr(cam_vec(cam, st.low_pass)),
                                  _ptr(cfg_vec(st)), _ptr(g9), C.byref(G),
                                  _ptr(s.get("accum")), _ptr(s.get("count"), _i32p),
                                  _ptr(s.get("max_radius"), _i32p))
    return grads


def render(scene, cam, st: Settings, brute=False, nthreads=1, margins=False):
    """Full forward of one view: preprocess, then blend."""
    sp = preprocess(scene, cam, st)
    out = blend(sp, cam.width, cam.height, st.tile, st.bg, brute=brute, nthreads=nthreads,
                margins=margins, depth_margin=margins)
    out["splats"] = sp
    return out


def hits(splats, W, H, tile=16, brute=False, nthreads=1, tile_mask=None, lists=None):
    """Ray hits of one view for Eq. significance-score: per Gaussian, the number of pixels
    whose blend (Eq. 2) blends it (alpha >= 1/255, before the pixel's stop). int64 [n]."""
    n = splats["radius"].shape[0]
    out = np.zeros(max(n, 1), np.int64)
    tm = _mask(tile_mask)
    lv, lr, _keep = _lists(lists)
    lib().orc_hits(n, C.byref(_splats_struct(splats)), W, H, tile, int(brute), nthreads,
                   _ptr(tm, _u8p), lv, lr, out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out[:n]


def volume_mask(scene, st: Settings):
    """The hard volume mask M of each Gaussian: float32(mask logit) > float32(logit(eps))."""
    n = np.shape(scene["means"])[0]
    m = scene.get("mask_logits")
    if m is None:
        return np.ones(n)
    tau = np.float32(np.log(st.eps_mask / (1.0 - st.eps_mask)))
    return (np.asarray(m, np.float32) > tau).astype(np.float64)


def significance(scene, st: Settings, hit_count, quantile=0.9):
    """Significance score of Eq. significance-score, GS_j = hits_j * alpha_j * gamma(Sigma_j):
    hits_j from ``hits`` summed over the views, alpha_j the Gaussian's opacity o'_j = M
    sigmoid(o_j) and gamma its volume s_x s_y s_z (masked scales M exp(l)) divided by the
    volume at rank floor(quantile (n - 1)) of all n volumes sorted ascending, capped at 1 (1
    where that volume is 0). Float64."""
    n = np.shape(scene["means"])[0]
    M = volume_mask(scene, st)
    o = np.asarray(scene["opacity_logits"], np.float64).reshape(n)
    opac = M / (1.0 + np.exp(-o))
    ls = np.asarray(scene["log_scales"], np.float64).reshape(n, 3)
    vol = M * np.exp(ls[:, 0]) * np.exp(ls[:, 1]) * np.exp(ls[:, 2])
    if n == 0:
        return np.zeros(0)
    vq = np.sort(vol)[int(np.floor(quantile * (n - 1)))]
    gamma = np.minimum(vol / vq, 1.0) if vq > 0 else np.ones(n)
    return np.asarray(hit_count, np.float64) * opac * gamma


def prune_select(scores, fraction):
    """The Gaussians a pruning round removes: the floor(fraction n) lowest scores, equal
    scores by lower index first. bool [n]."""
    scores = np.asarray(scores)
    n = scores.shape[0]
    k = int(np.floor(fraction * n))
    order = np.lexsort((np.arange(n), scores))
    out = np.zeros(n, bool)
    out[order[:k]] = True
    return out


# ---- compaction (Sec. "Pruning with Volume Masking", Eq. significance-score) ------------------

SCENE_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest", "mask_logits",
              "sh_mask_logits", "sh_degree")


def compact(scene, st: Settings, remove=None, masked=True):
    """The scene without the Gaussians a pruning step removes: those with remove[j] set (e.g.
    the significance selection) and, when masked, those whose volume mask M_j is 0 (the
    paper removes masked Gaussians at densification steps). The kept ones stay in order.
    Returns (scene, kept_index) with kept_index[new] = old index."""
    n = np.shape(scene["means"])[0]
    keep = np.ones(n, bool)
    if remove is not None:
        keep &= ~np.asarray(remove, bool)
    if masked and scene.get("mask_logits") is not None:
        keep &= volume_mask(scene, st) > 0.0
    idx = np.flatnonzero(keep)
    out = dict(scene)
    for k in SCENE_KEYS:
        if scene.get(k) is not None:
            out[k] = np.asarray(scene[k])[idx]
    return out, idx


# ---- mask losses of Eq. loss3dgs --------------------------------------------------------------
#
# The training loss adds lambda_m L_m + lambda_sh L_sh (Eq. loss3dgs, lambda_m = lambda_sh = 0.05,
# Sec. "Implementation details"); the paper defers both definitions to the cited works and fixes
# one property: the masking loss of each SH band is weighted by the band's number of
# coefficients (Sec. "Spherical Harmonic (SH) Masking"). Reading used here:
#   L_m  = (1/N) sum_n sigmoid(m_n)                        (mean soft volume mask)
#   L_sh = (1/N) sum_n sum_{l=1..3} w_l sigmoid(m_n^l),    w_l = (2l + 1) / 15
# where 2l + 1 is the number of coefficients of band l per colour channel and 15 their total
# over bands 1..3, so the weights sum to 1 and both losses lie in (0, 1). Every Gaussian and
# every band counts, visible or not. The gradients are the plain derivatives of these soft
# masks (no straight-through step is involved).

MASK_LAMBDA = 0.05
SH_MASK_LAMBDA = 0.05


def sh_band_weights():
    """w_l for l = 1, 2, 3: the share of band l among the 15 rest coefficients per channel."""
    counts = np.array([2 * l + 1 for l in (1, 2, 3)], np.float64)
    return counts / counts.sum()


def mask_loss(scene, lam_m=MASK_LAMBDA, lam_sh=SH_MASK_LAMBDA):
    """lambda_m L_m + lambda_sh L_sh (reading above) and its gradients with respect to the
    mask logits: (loss, {"mask_logits": [N], "sh_mask_logits": [N,3]}); an absent logit
    array contributes nothing and gets no gradient."""
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    loss = 0.0
    grads = {"mask_logits": None, "sh_mask_logits": None}
    m = scene.get("mask_logits")
    if m is not None:
        m = np.asarray(m, np.float64)
        n = m.shape[0]
        s = sig(m)
        loss += lam_m * s.sum() / max(n, 1)
        grads["mask_logits"] = lam_m * s * (1.0 - s) / max(n, 1)
    b = scene.get("sh_mask_logits")
    if b is not None:
        b = np.asarray(b, np.float64).reshape(-1, 3)
        n = b.shape[0]
        s = sig(b)
        w = sh_band_weights()
        loss += lam_sh * (s * w).sum() / max(n, 1)
        grads["sh_mask_logits"] = lam_sh * w * s * (1.0 - s) / max(n, 1)
    return loss, grads


# ---- densification by clone and split (3DGS, which the paper keeps) ----------------------------
#
# The paper densifies as 3DGS does (Sec. "Implementation details": standard densification every
# 100 iterations until 15K, and again from 20K to 20.5K) from the 2D-mean gradient magnitudes
# (Sec. "Preliminaries"); it states no rule of its own. Reading used here, 3DGS's clone and split
# driven by the statistics the preprocess backward accumulates (the per-view norms of dL/d mean2d
# in pixel units summed over the views where the Gaussian is visible, and the visibility count):
#   avg_n   = accum_n / count_n  (float32 division; 0 where count_n = 0)
#   chosen  = avg_n >= tau_g     (float32)
#   large   = max_k l_nk > float32(log(scale_threshold))   (log-scales, float32; the threshold is
#             3DGS's percent_dense x scene extent, compared in the log domain so that no exp
#             rounding can flip the decision)
#   clone   = chosen and not large: an identical copy is added;
#   split   = chosen and large: the Gaussian is replaced by 2 children with means
#             mu + R(q / |q|) (exp(l) * z_c) for caller-drawn standard normals z_c = normals[n, c]
#             and log-scales l - log(1.6) (3DGS divides the scales by 0.8 N, N = 2); every other
#             parameter (mask logits included) is copied.
# New order: the Gaussians not split, in order; then the clones, in order; then the first children
# of the split Gaussians, in order; then their second children (3DGS appends the clones, then the
# children as N stacked copies of the selection, then drops the split originals).

SPLIT_CHILDREN = 2
SPLIT_SCALE_DIVISOR = 0.8 * SPLIT_CHILDREN


def densify(scene, accum, count, grad_threshold, scale_threshold, normals):
    """Clone and split (reading above). normals: float [n, 2, 3] standard normals (only the rows
    of split Gaussians are read). Returns (scene, src, n_clone, n_split) with src[new] = the old
    index each new row comes from."""
    n = np.shape(scene["means"])[0]
    acc = np.asarray(accum, np.float32)
    cnt = np.asarray(count, np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        avg = np.where(cnt > 0, acc / cnt.astype(np.float32), np.float32(0.0)).astype(np.float32)
    chosen = (cnt > 0) & (avg >= np.float32(grad_threshold))
    ls = np.asarray(scene["log_scales"], np.float32)
    large = ls.max(axis=1) > np.float32(np.log(np.float64(scale_threshold)))
    clone = chosen & ~large
    split = chosen & large
    keep_idx = np.flatnonzero(~split)
    clone_idx = np.flatnonzero(clone)
    split_idx = np.flatnonzero(split)
    src = np.concatenate([keep_idx, clone_idx, split_idx, split_idx]).astype(np.int64)
    out = dict(scene)
    for k in SCENE_KEYS:
        if scene.get(k) is not None:
            out[k] = np.asarray(scene[k])[src].copy()
    # the children's means and log-scales
    z = np.asarray(normals, np.float64).reshape(n, SPLIT_CHILDREN, 3)
    q = np.asarray(scene["quats"], np.float64)[split_idx]
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    R = np.stack([_rotation(qq) for qq in q]) if split_idx.size else np.zeros((0, 3, 3))
    s = np.exp(np.asarray(scene["log_scales"], np.float64)[split_idx])
    mu = np.asarray(scene["means"], np.float64)[split_idx]
    base = keep_idx.size + clone_idx.size
    means = np.asarray(out["means"], np.float64)
    log_scales = np.asarray(out["log_scales"], np.float64)
    for c in range(SPLIT_CHILDREN):
        rows = slice(base + c * split_idx.size, base + (c + 1) * split_idx.size)
        means[rows] = mu + np.einsum("nij,nj->ni", R, s * z[split_idx, c])
        log_scales[rows] = np.log(s / SPLIT_SCALE_DIVISOR)
    out["means"], out["log_scales"] = means, log_scales
    return out, src, int(clone_idx.size), int(split_idx.size)


def _rotation(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ---- FP16 storage (Sec. "Experiments", setup: parameters kept as 16-bit halves after training) --

def to_half(scene):
    """Every float parameter rounded to the nearest IEEE binary16 (ties to even, numpy's
    conversion), widened back exactly; the render of FP16 storage is the render of this."""
    out = dict(scene)
    with np.errstate(over="ignore"):   # beyond the half range: +-inf, by definition
        for k in SCENE_KEYS:
            if k != "sh_degree" and scene.get(k) is not None:
                out[k] = np.asarray(scene[k], np.float32).astype(np.float16).astype(np.float32)
    return out


def new_stats(n):
    return dict(accum=np.zeros(n), count=np.zeros(n, np.int32),
                max_radius=np.zeros(n, np.int32))


def grad(scene, cams, st: Settings, dL_dimgs, nthreads=1):
    """Gradients of L with respect to every input, given dL/dimage per view, plus the
    densification statistics; returns (grads, stats, per-view screen-space grads)."""
    n = np.shape(scene["means"])[0]
    grads = zero_grads(scene)
    stats = new_stats(n)
    g9s = []
    for cam, d in zip(cams, dL_dimgs):
        sp = preprocess(scene, cam, st)
        g9 = blend_backward(sp, cam.width, cam.height, d, st.tile, st.bg, nthreads)
        preprocess_backward(scene, cam, st, g9, grads, stats)
        g9s.append(g9)
    return grads, stats, g9s


def l1(images, targets):
    """Mean over views of the mean over 3HW of |C - target|, and dL/dC per view."""
    V = len(images)
    loss = 0.0
    gs = []
    L = lib()
    for img, tgt in zip(images, targets):
        img = np.ascontiguousarray(img, np.float64)
        tgt = np.ascontiguousarray(tgt, np.float64)
        g = np.zeros_like(img)
        loss += L.orc_l1(img.size, _ptr(img), _ptr(tgt), 1.0 / (img.size * V), _ptr(g))
        gs.append(g)
    return loss, gs


# ---- D-SSIM term of the training loss (Eq. loss3dgs) ----------------------------------------
#
# The paper keeps the 3DGS loss, (1 - lambda) L1 + lambda D-SSIM, and speeds up its SSIM with
# separable 1D passes (Sec. "Accelerated training"); it does not restate SSIM. This is the SSIM
# of Wang et al. with the 3DGS settings: an 11 x 11 Gaussian window of sigma 1.5 normalised to
# sum 1, zero outside the image (output of the image's size), C1 = 0.01^2, C2 = 0.03^2 (dynamic
# range 1), per channel; SSIM = mean of the SSIM map over 3HW, D-SSIM = 1 - SSIM. The oracle
# sums over the 2D window directly, not as two 1D passes.

SSIM_WINDOW = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_LAMBDA = 0.2


def ssim_window():
    """The 2D window w[i, j] proportional to exp(-((i - 5)^2 + (j - 5)^2) / (2 sigma^2)), summing to 1."""
    r = SSIM_WINDOW // 2
    k = np.arange(SSIM_WINDOW, dtype=np.float64) - r
    w = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2.0 * SSIM_SIGMA ** 2))
    return w / w.sum()


def _window_sum(a, w):
    """out[.., y, x] = sum_ij w[i, j] a[.., y + i - r, x + j - r], a taken as 0 outside the image."""
    r = w.shape[0] // 2
    H, W = a.shape[-2:]
    p = np.zeros(a.shape[:-2] + (H + 2 * r, W + 2 * r))
    p[..., r:r + H, r:r + W] = a
    out = np.zeros(a.shape, np.float64)
    for i in range(w.shape[0]):
        for j in range(w.shape[1]):
            out += w[i, j] * p[..., i:i + H, j:j + W]
    return out


def _window_sum_adjoint(f, w):
    """The adjoint of _window_sum: a[.., y + i - r, x + j - r] += w[i, j] f[.., y, x], kept inside the image."""
    r = w.shape[0] // 2
    H, W = f.shape[-2:]
    p = np.zeros(f.shape[:-2] + (H + 2 * r, W + 2 * r))
    for i in range(w.shape[0]):
        for j in range(w.shape[1]):
            p[..., i:i + H, j:j + W] += w[i, j] * f
    return p[..., r:r + H, r:r + W]


def ssim_maps(x, y):
    """SSIM map of two images [.., H, W] and the local statistics it is made of: means mu_x,
    mu_y, variances, covariance under the window, and the terms A1 = 2 mu_x mu_y + C1,
    A2 = 2 sigma_xy + C2, B1 = mu_x^2 + mu_y^2 + C1, B2 = sigma_x^2 + sigma_y^2 + C2, S = A1 A2 / (B1 B2)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = ssim_window()
    mx, my = _window_sum(x, w), _window_sum(y, w)
    sxx = _window_sum(x * x, w) - mx * mx
    syy = _window_sum(y * y, w) - my * my
    sxy = _window_sum(x * y, w) - mx * my
    A1 = 2.0 * mx * my + SSIM_C1
    A2 = 2.0 * sxy + SSIM_C2
    B1 = mx * mx + my * my + SSIM_C1
    B2 = sxx + syy + SSIM_C2
    S = A1 * A2 / (B1 * B2)
    return S, dict(mu_x=mx, mu_y=my, var_x=sxx, var_y=syy, cov=sxy, A1=A1, A2=A2, B1=B1, B2=B2)


def l1_dssim(images, targets, lam=SSIM_LAMBDA):
    """Eq. loss3dgs without the mask terms, over V views: L = mean over views of
    (1 - lam) mean_3HW |C - t| + lam (1 - mean_3HW SSIM(C, t)), and dL/dC per view.
    The SSIM part of the gradient is the exact chain rule through the window sums:
    sigma_x^2 = E[x^2] - mu_x^2 and sigma_xy = E[xy] - mu_x mu_y, each E[.] a window sum, so
    dL/dx(q) = sum_p w(q - p) dL/dS(p) (dS/dmu_x(p) + 2 x(q) dS/dE[x^2](p) + y(q) dS/dE[xy](p))."""
    V = len(images)
    w = ssim_window()
    loss = 0.0
    gs = []
    for img, tgt in zip(images, targets):
        x = np.asarray(img, np.float64)
        y = np.asarray(tgt, np.float64)
        n = x.size
        S, m = ssim_maps(x, y)
        loss += ((1.0 - lam) * np.abs(x - y).sum() / n + lam * (1.0 - S.sum() / n)) / V
        dS = -lam / (n * V)                                    # dL/dS at every pixel
        B1B2 = m["B1"] * m["B2"]
        dS_dmx = 2.0 * m["mu_y"] * m["A2"] / B1B2 - 2.0 * m["mu_x"] * S / m["B1"]
        dS_dvx = -S / m["B2"]                                  # holding mu_x, sigma_xy
        dS_dcov = 2.0 * m["A1"] / B1B2
        # raw moments: d/dmu_x picks up -2 mu_x from sigma_x^2 and -mu_y from sigma_xy
        d_m1 = dS * (dS_dmx - 2.0 * m["mu_x"] * dS_dvx - m["mu_y"] * dS_dcov)
        d_m2 = dS * dS_dvx
        d_mxy = dS * dS_dcov
        g = (_window_sum_adjoint(d_m1, w) + 2.0 * x * _window_sum_adjoint(d_m2, w)
             + y * _window_sum_adjoint(d_mxy, w))
        g += (1.0 - lam) * np.sign(x - y) / (n * V)
        gs.append(g)
    return loss, gs
