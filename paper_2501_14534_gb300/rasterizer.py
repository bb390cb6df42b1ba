"""Torch-facing wrappers of libtgs: device tensors in, device tensors out.

This module only marshals arguments (tensor pointers, camera structs, the current stream)
into the C ABI of include/tgs.h; all arithmetic runs in the library's kernels. PyTorch is
used for device memory and streams.

``RasterizeViews`` is a ``torch.autograd.Function`` over V views. Its forward keeps, per
view, only the pixel state the backward needs (final transmittance and the position of the
last contributor); the per-view Gaussian lists are rebuilt in the backward (per-view
checkpointing), except for the last view rendered, whose binning the library keeps.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import _binding as B

SPLAT_WORDS = 16   # words per splat record (include/tgs.h)
PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest",
              "mask_logits", "sh_mask_logits")


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_tensor(t, name, dtype=torch.float32, host=False):
    if t is None:
        return
    if t.is_cuda == host or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {'host' if host else 'CUDA'} {dtype} tensor")


@dataclasses.dataclass
class Gaussians:
    """Gaussian parameters as CUDA tensors (layout of include/tgs.h)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh_dc: torch.Tensor
    sh_rest: torch.Tensor | None = None
    mask_logits: torch.Tensor | None = None
    sh_mask_logits: torch.Tensor | None = None
    sh_degree: torch.Tensor | None = None       # uint8 [N]
    sh_degree_max: int | None = None

    @property
    def n(self):
        return self.means.shape[0]

    @property
    def half(self):
        """FP16 storage: every parameter array holds float16 (render path only)."""
        return self.means.dtype == torch.float16

    def struct(self, host=False):
        """The tgs_gaussians of these tensors (device tensors; host=True: host tensors, for
        tgs_train_step_batched_host)."""
        dt = torch.float16 if self.half else torch.float32
        for k in PARAM_KEYS:
            _check_tensor(getattr(self, k), k, dt, host)
        _check_tensor(self.sh_degree, "sh_degree", torch.uint8, host)
        deg = self.sh_degree_max
        if deg is None:
            deg = 3 if self.sh_rest is not None else 0
        return B.tgs_gaussians(self.n, deg, B.TGS_PARAM_F16 if self.half else B.TGS_PARAM_F32,
                               _p(self.means), _p(self.log_scales),
                               _p(self.quats), _p(self.opacity_logits), _p(self.sh_dc),
                               _p(self.sh_rest), _p(self.sh_degree), _p(self.mask_logits),
                               _p(self.sh_mask_logits))

    @staticmethod
    def from_numpy(scene, device="cuda"):
        def t(k, dtype=torch.float32):
            v = scene.get(k)
            if v is None:
                return None
            return torch.from_numpy(np.ascontiguousarray(v)).to(device=device, dtype=dtype)
        return Gaussians(t("means"), t("log_scales"), t("quats"), t("opacity_logits"),
                         t("sh_dc"), t("sh_rest"), t("mask_logits"), t("sh_mask_logits"),
                         t("sh_degree", torch.uint8), scene.get("deg_max"))

    def params(self):
        return {k: getattr(self, k) for k in PARAM_KEYS if getattr(self, k) is not None}


def camera_struct(cam, low_pass=0.0):
    c = B.tgs_camera()
    vm = np.asarray(cam.viewmat, dtype=np.float32).reshape(-1)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    cp = np.asarray(cam.campos, dtype=np.float32)
    for i in range(3):
        c.campos[i] = float(cp[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.low_pass = float(low_pass)
    return c


def cameras_array(cams):
    arr = (B.tgs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = c if isinstance(c, B.tgs_camera) else camera_struct(c)
    return arr


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Rasterizer:
    """One libtgs context (its settings and its scratch arena) on the current device."""

    def __init__(self, tile=16, ppt=1, support=B.TGS_SUPPORT_BOX3, low_pass=0.3, eps_mask=0.05,
                 eps_sh=0.1, near=0.2, bg=(0.0, 0.0, 0.0), key_capacity=0, ssim_lambda=0.2,
                 lambda_mask=0.05, lambda_sh_mask=0.05, batch=1):
        cfg = B.tgs_config()
        B.lib.tgs_default_config(C.byref(cfg))
        cfg.ssim_lambda = ssim_lambda
        cfg.lambda_mask, cfg.lambda_sh_mask = lambda_mask, lambda_sh_mask
        cfg.batch = batch
        cfg.tile, cfg.ppt, cfg.support = tile, ppt, support
        cfg.low_pass, cfg.eps_mask, cfg.eps_sh, cfg.near_plane = low_pass, eps_mask, eps_sh, near
        for i in range(3):
            cfg.bg[i] = bg[i]
        cfg.key_capacity = key_capacity
        h = C.c_void_p()
        B.check(B.lib.tgs_create(C.byref(h), C.byref(cfg)), "tgs_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and B is not None and B.lib is not None:
            B.lib.tgs_destroy(h)
            self._h = None

    @property
    def config(self):
        cfg = B.tgs_config()
        B.check(B.lib.tgs_get_config(self._h, C.byref(cfg)), "tgs_get_config")
        return cfg

    def set(self, **kw):
        cfg = self.config
        for k, v in kw.items():
            if k == "bg":
                for i in range(3):
                    cfg.bg[i] = v[i]
            else:
                setattr(cfg, k, v)
        B.check(B.lib.tgs_set_config(self._h, C.byref(cfg)), "tgs_set_config")

    def poll(self):
        B.check(B.lib.tgs_poll_status(self._h, _stream()), "device status")

    # ---- plain path ----------------------------------------------------------------------

    def _alloc_views(self, cams, n, want_state=True, want_examined=False, want_radii=False,
                     want_counts=False):
        outs = []
        for c in cams:
            H, W = c.height, c.width
            d = dict(image=torch.empty((3, H, W), device="cuda"))
            if want_state:
                d["T_final"] = torch.empty((H, W), device="cuda")
                d["last"] = torch.empty((H, W), device="cuda", dtype=torch.int32)
            if want_examined:
                d["n_examined"] = torch.empty((H, W), device="cuda", dtype=torch.int32)
            if want_radii:
                d["radii"] = torch.empty((n,), device="cuda", dtype=torch.int32)
            if want_counts:
                d["n_contrib"] = torch.empty((H, W), device="cuda", dtype=torch.int32)
                d["n_eval"] = torch.empty((H, W), device="cuda", dtype=torch.int32)
            outs.append(d)
        return outs

    @staticmethod
    def _out_structs(outs):
        arr = (B.tgs_view_out * len(outs))()
        for i, d in enumerate(outs):
            arr[i] = B.tgs_view_out(_p(d.get("image")), _p(d.get("T_final")), _p(d.get("last")),
                                    _p(d.get("n_examined")), _p(d.get("radii")),
                                    _p(d.get("n_contrib")), _p(d.get("n_eval")))
        return arr

    def forward(self, g: Gaussians, cams, want_state=True, want_examined=False,
                want_radii=False, want_counts=False, outs=None):
        outs = outs or self._alloc_views(cams, g.n, want_state, want_examined, want_radii,
                                         want_counts)
        B.check(B.lib.tgs_forward(self._h, C.byref(g.struct()), cameras_array(cams), len(cams),
                                  self._out_structs(outs), 0, _stream()), "tgs_forward")
        return outs

    @staticmethod
    def alloc_grads(g: Gaussians, no_sh_rest=False):
        d = {}
        for k, v in g.params().items():
            if k == "sh_rest" and no_sh_rest:
                continue
            d[k] = torch.zeros_like(v)
        return d

    @staticmethod
    def alloc_stats(n, hits=False):
        """Densification statistics; with hits also the ray-hit counter of the significance
        score (Eq. significance-score), which the batched step then fills as well."""
        st = dict(grad_norm_accum=torch.zeros(n, device="cuda"),
                  vis_count=torch.zeros(n, device="cuda", dtype=torch.int32),
                  max_radius=torch.zeros(n, device="cuda", dtype=torch.int32))
        if hits:
            st["hit_count"] = torch.zeros(n, device="cuda", dtype=torch.int32)
        return st

    @staticmethod
    def _grad_struct(grads):
        grads = grads or {}
        return B.tgs_grads(*[_p(grads.get(k)) for k in PARAM_KEYS])

    @staticmethod
    def _stats_struct(stats):
        stats = stats or {}
        return B.tgs_stats(_p(stats.get("grad_norm_accum")), _p(stats.get("vis_count")),
                           _p(stats.get("max_radius")), _p(stats.get("hit_count")))

    def backward(self, g: Gaussians, cams, outs, dL_dimages, grads=None, stats=None,
                 accumulate=False, no_sh_rest=False, mask_loss=False):
        if grads is None:
            grads = self.alloc_grads(g, no_sh_rest)
        if stats is None:
            stats = self.alloc_stats(g.n)
        flags = ((B.TGS_ACCUMULATE if accumulate else 0) | (B.TGS_NO_SH_REST_GRAD if no_sh_rest else 0) |
                 (B.TGS_MASK_LOSS if mask_loss else 0))
        dl = [d.contiguous() for d in dL_dimages]
        B.check(B.lib.tgs_backward(self._h, C.byref(g.struct()), cameras_array(cams), len(cams),
                                   self._out_structs(outs), _ptr_array(dl),
                                   C.byref(self._grad_struct(grads)),
                                   C.byref(self._stats_struct(stats)), flags, _stream()),
                "tgs_backward")
        return grads, stats

    @staticmethod
    def l1_loss(image, target, scale, loss_accum, grad):
        B.check(B.lib.tgs_l1_loss(_p(image), _p(target), image.numel(), float(scale),
                                  _p(loss_accum), _p(grad), _stream()), "tgs_l1_loss")

    def l1_dssim_loss(self, images, targets, lam=0.2, loss=None, grads=None):
        """Eq. loss3dgs without the mask terms over views of any sizes: adds to loss (device
        float [1], zeros if None) the mean over views of (1 - lam) L1 + lam (1 - SSIM) and
        returns (loss, grads) with grads[v] = dL/d images[v]."""
        V = len(images)
        if loss is None:
            loss = torch.zeros(1, device="cuda", dtype=torch.float32)
        if grads is None:
            grads = [torch.empty_like(x) for x in images]
        cams = (B.tgs_camera * V)()
        for v, x in enumerate(images):
            assert x.dtype == torch.float32 and x.is_contiguous() and x.dim() == 3 and x.shape[0] == 3
            assert targets[v].shape == x.shape and targets[v].is_contiguous() and grads[v].shape == x.shape
            cams[v].width, cams[v].height = x.shape[2], x.shape[1]
        B.check(B.lib.tgs_l1_dssim_loss(self._h, cams, V, _ptr_array(images), _ptr_array(targets),
                                        float(lam), _p(loss), _ptr_array(grads), _stream()),
                "tgs_l1_dssim_loss")
        return loss, grads

    def mask_loss(self, g: Gaussians, loss=None, grads=None):
        """Adds lambda_m L_m + lambda_sh L_sh of Eq. loss3dgs to loss (device float [1], zeros if
        None) and their gradients to grads["mask_logits"] / grads["sh_mask_logits"] when given;
        returns loss (tgs_mask_loss)."""
        if loss is None:
            loss = torch.zeros(1, device="cuda", dtype=torch.float32)
        B.check(B.lib.tgs_mask_loss(self._h, C.byref(g.struct()), _p(loss),
                                    C.byref(self._grad_struct(grads)) if grads else None, _stream()),
                "tgs_mask_loss")
        return loss

    # ---- individual steps -----------------------------------------------------------------

    def preprocess(self, g: Gaussians, cams):
        V = len(cams)
        splats = torch.empty((V * g.n, SPLAT_WORDS), device="cuda")
        radii = torch.empty((V * g.n,), device="cuda", dtype=torch.int32)
        B.check(B.lib.tgs_preprocess(self._h, C.byref(g.struct()), cameras_array(cams), V,
                                     _p(splats), _p(radii), _stream()), "tgs_preprocess")
        return splats, radii

    def num_tiles(self, cams):
        return int(B.lib.tgs_num_tiles(self._h, cameras_array(cams), len(cams)))

    def bin(self, splats, radii, n, cams, capacity=None, want_keys=True):
        """Returns (sorted record ids, sorted 64-bit keys as int64, ranges [tiles,2], K)."""
        V = len(cams)
        T = self.num_tiles(cams)
        ranges = torch.empty((T, 2), device="cuda", dtype=torch.int32)
        K = C.c_int64(0)
        cap = capacity
        if cap is None:
            # first pass only counts
            dummy = torch.empty((1,), device="cuda", dtype=torch.int32)
            st = B.lib.tgs_bin(self._h, _p(splats), _p(radii), n, cameras_array(cams), V,
                               _p(dummy), None, _p(ranges), 0, C.byref(K), _stream())
            if st not in (B.TGS_OK, B.TGS_ERR_CAPACITY):
                B.check(st, "tgs_bin")
            cap = max(int(K.value), 1)
        ids = torch.empty((cap,), device="cuda", dtype=torch.int32)
        keys = torch.empty((cap,), device="cuda", dtype=torch.int64) if want_keys else None
        B.check(B.lib.tgs_bin(self._h, _p(splats), _p(radii), n, cameras_array(cams), V, _p(ids),
                              _p(keys), _p(ranges), cap, C.byref(K), _stream()), "tgs_bin")
        k = int(K.value)
        return ids[:k], (keys[:k] if keys is not None else None), ranges, k

    def blend_forward(self, splats, ids, ranges, cams, want_examined=True, want_counts=True):
        outs = self._alloc_views(cams, 0, True, want_examined, want_counts=want_counts)
        B.check(B.lib.tgs_blend_forward(self._h, _p(splats), _p(ids), _p(ranges),
                                        cameras_array(cams), len(cams), self._out_structs(outs),
                                        _stream()), "tgs_blend_forward")
        return outs

    def blend_backward(self, splats, ids, ranges, cams, outs, dL_dimages):
        sg = torch.zeros((splats.shape[0], 12), device="cuda")
        dl = [d.contiguous() for d in dL_dimages]
        B.check(B.lib.tgs_blend_backward(self._h, _p(splats), _p(ids), _p(ranges),
                                         cameras_array(cams), len(cams), self._out_structs(outs),
                                         _ptr_array(dl), _p(sg), _stream()), "tgs_blend_backward")
        return sg

    def preprocess_backward(self, g: Gaussians, cams, splat_grads, radii, grads=None, stats=None,
                            accumulate=False, no_sh_rest=False):
        if grads is None:
            grads = self.alloc_grads(g, no_sh_rest)
        if stats is None:
            stats = self.alloc_stats(g.n)
        flags = (B.TGS_ACCUMULATE if accumulate else 0) | (B.TGS_NO_SH_REST_GRAD if no_sh_rest else 0)
        B.check(B.lib.tgs_preprocess_backward(self._h, C.byref(g.struct()), cameras_array(cams),
                                              len(cams), _p(splat_grads), _p(radii),
                                              C.byref(self._grad_struct(grads)),
                                              C.byref(self._stats_struct(stats)), flags,
                                              _stream()), "tgs_preprocess_backward")
        return grads, stats

    # ---- batched path ----------------------------------------------------------------------

    def plan(self, g: Gaussians, cams, headroom=1.25):
        K = C.c_int64(0)
        B.check(B.lib.tgs_plan(self._h, C.byref(g.struct()), cameras_array(cams), len(cams),
                               float(headroom), C.byref(K)), "tgs_plan")
        return int(K.value)

    def train_step_batched(self, g: Gaussians, cams, targets, grads, stats=None, loss=None,
                           images=None, graph=False, accumulate=False, no_sh_rest=False,
                           cams_struct=None, fused=True, dssim=False, mask_loss=False):
        flags = ((B.TGS_USE_GRAPH if graph else 0) | (B.TGS_ACCUMULATE if accumulate else 0) |
                 (B.TGS_NO_SH_REST_GRAD if no_sh_rest else 0) | (0 if fused else B.TGS_UNFUSED) |
                 (B.TGS_LOSS_DSSIM if dssim else 0) | (B.TGS_MASK_LOSS if mask_loss else 0))
        camarr = cams_struct if cams_struct is not None else cameras_array(cams)
        B.check(B.lib.tgs_train_step_batched(
            self._h, C.byref(g.struct()), camarr, len(camarr), _ptr_array(targets),
            _ptr_array(images) if images is not None else None, C.byref(self._grad_struct(grads)),
            C.byref(self._stats_struct(stats)), _p(loss), flags, _stream()),
            "tgs_train_step_batched")

    def train_step_batched_host(self, g_host: Gaussians, cams, targets_host, grads, stats=None, loss_host=None,
                                graph=False, cams_struct=None):
        """The batched step from host tensors (pinned for asynchronous copies): the library
        copies the parameters and targets to the device, runs the step and copies the loss
        into loss_host (a host float tensor [1]); see tgs_train_step_batched_host."""
        flags = B.TGS_USE_GRAPH if graph else 0
        for i, t in enumerate(targets_host):
            _check_tensor(t, f"targets_host[{i}]", host=True)
        if loss_host is not None:
            _check_tensor(loss_host, "loss_host", host=True)
        camarr = cams_struct if cams_struct is not None else cameras_array(cams)
        B.check(B.lib.tgs_train_step_batched_host(
            self._h, C.byref(g_host.struct(host=True)), camarr, len(camarr), _ptr_array(targets_host),
            C.byref(self._grad_struct(grads)), C.byref(self._stats_struct(stats)), _p(loss_host), flags,
            _stream()), "tgs_train_step_batched_host")

    def render_batched(self, g: Gaussians, cams, outs=None, want_state=False, graph=False, cams_struct=None):
        """Forward-only render of the views through the batched machinery (tgs_render_batched):
        no host synchronisation once the key capacity is planned (plan)."""
        outs = outs or self._alloc_views(cams, g.n, want_state)
        for d in outs:
            assert "radii" not in d
        camarr = cams_struct if cams_struct is not None else cameras_array(cams)
        B.check(B.lib.tgs_render_batched(self._h, C.byref(g.struct()), camarr, len(camarr), self._out_structs(outs),
                                         B.TGS_USE_GRAPH if graph else 0, _stream()), "tgs_render_batched")
        return outs

    # ---- FP16 storage ----

    @staticmethod
    def to_half(g: Gaussians):
        """The Gaussians with every parameter rounded to IEEE half (ties to even), for
        rendering from FP16 storage."""
        out = {k: torch.empty(v.shape, device="cuda", dtype=torch.float16) for k, v in g.params().items()}
        hp = B.tgs_half_params(*[_p(out.get(k)) for k in PARAM_KEYS])
        B.check(B.lib.tgs_params_to_half(C.byref(g.struct()), C.byref(hp), _stream()), "tgs_params_to_half")
        return Gaussians(**out, sh_degree=g.sh_degree, sh_degree_max=g.sh_degree_max)

    # ---- compaction ----

    def compact(self, g: Gaussians, remove=None, masked=True, want_index=True):
        """The Gaussians that stay after a pruning step, in order: without those marked in
        remove (uint8 or bool [n] on the device, e.g. prune_select's output) and, if masked,
        without those whose volume mask is 0. Returns (Gaussians, kept_index or None)."""
        if remove is not None:
            assert remove.is_cuda and remove.numel() == g.n and remove.dtype in (torch.uint8, torch.bool)
            remove = remove.to(torch.uint8).contiguous()
        out = {k: torch.empty_like(v) for k, v in g.params().items()}
        deg = torch.empty_like(g.sh_degree) if g.sh_degree is not None else None
        idx = torch.empty(g.n, device="cuda", dtype=torch.int32) if want_index else None
        n_kept = C.c_int64(0)
        B.check(B.lib.tgs_compact(self._h, C.byref(g.struct()), _p(remove),
                                  B.TGS_COMPACT_MASKED if masked else 0, C.byref(self._grad_struct(out)),
                                  _p(deg), _p(idx), C.byref(n_kept), _stream()), "tgs_compact")
        k = int(n_kept.value)
        kept = Gaussians(**{name: t[:k] for name, t in out.items()},
                         sh_degree=deg[:k] if deg is not None else None, sh_degree_max=g.sh_degree_max)
        return kept, (idx[:k] if idx is not None else None)

    # ---- densification ----

    def densify(self, g: Gaussians, stats, normals, grad_threshold, scale_threshold):
        """Clone and split from the statistics of the preprocess backward (tgs_densify; 3DGS's
        rule). normals: CUDA float32 [n,2,3] standard normal draws. Returns (Gaussians, src_index,
        n_clone, n_split) with src_index[new] = the old index of each row."""
        assert normals.is_cuda and normals.dtype == torch.float32 and normals.is_contiguous()
        assert normals.numel() == 6 * g.n
        cap = 2 * g.n
        out = {k: torch.empty((cap,) + tuple(v.shape[1:]), device="cuda", dtype=v.dtype)
               for k, v in g.params().items()}
        deg = torch.empty(cap, device="cuda", dtype=torch.uint8) if g.sh_degree is not None else None
        src = torch.empty(cap, device="cuda", dtype=torch.int32)
        n_out, n_clone, n_split = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        B.check(B.lib.tgs_densify(self._h, C.byref(g.struct()), C.byref(self._stats_struct(stats)), _p(normals),
                                  float(grad_threshold), float(scale_threshold), C.byref(self._grad_struct(out)),
                                  _p(deg), _p(src), cap, C.byref(n_out), C.byref(n_clone), C.byref(n_split),
                                  _stream()), "tgs_densify")
        k = int(n_out.value)
        new = Gaussians(**{name: t[:k] for name, t in out.items()},
                        sh_degree=deg[:k] if deg is not None else None, sh_degree_max=g.sh_degree_max)
        return new, src[:k], int(n_clone.value), int(n_split.value)

    # ---- significance pruning (Eq. significance-score) ----

    def count_hits(self, g: Gaussians, cams, hit_count=None):
        """Adds each Gaussian's ray hits over these views to hit_count (int32 [n], zeros if
        None) and returns it: the pixels whose blend blends it."""
        if hit_count is None:
            hit_count = torch.zeros(g.n, device="cuda", dtype=torch.int32)
        assert hit_count.dtype == torch.int32 and hit_count.is_cuda and hit_count.numel() == g.n
        camarr = cameras_array(cams)
        B.check(B.lib.tgs_count_hits(self._h, C.byref(g.struct()), camarr, len(camarr), _p(hit_count),
                                     _stream()), "tgs_count_hits")
        return hit_count

    def significance(self, g: Gaussians, hit_count, quantile=0.9):
        """Significance score of each Gaussian (float32 [n]) from its ray hits, opacity and
        volume; quantile picks the reference volume (the paper's choice: 0.9)."""
        scores = torch.empty(g.n, device="cuda", dtype=torch.float32)
        B.check(B.lib.tgs_significance(self._h, C.byref(g.struct()), _p(hit_count), float(quantile),
                                       _p(scores), _stream()), "tgs_significance")
        return scores

    @staticmethod
    def pruning_fractions(rounds=6, first=0.6, decay=0.7):
        """Fraction of the Gaussians each significance pruning round removes (tgs_prune_schedule;
        Sec. "Implementation details": 6 rounds, 60 % first, decay 0.7)."""
        out = (C.c_double * max(rounds, 1))()
        B.check(B.lib.tgs_prune_schedule(int(rounds), float(first), float(decay), out), "tgs_prune_schedule")
        return [float(out[k]) for k in range(rounds)]

    def prune_select(self, scores, fraction):
        """bool [n]: the floor(fraction n) lowest scores (equal scores: lower index first)."""
        scores = scores.contiguous()
        out = torch.empty(scores.numel(), device="cuda", dtype=torch.uint8)
        B.check(B.lib.tgs_prune_select(self._h, _p(scores), scores.numel(), float(fraction), _p(out),
                                       _stream()), "tgs_prune_select")
        return out.bool()

    def set_profiling(self, on=True):
        B.check(B.lib.tgs_set_profiling(self._h, int(on)), "tgs_set_profiling")

    def stage_times(self):
        """{stage name: milliseconds} of the most recent batched step (profiling on)."""
        ms = (C.c_float * B.TGS_MAX_STAGES)()
        n = C.c_int32(0)
        B.check(B.lib.tgs_stage_times(self._h, ms, B.TGS_MAX_STAGES, C.byref(n)), "tgs_stage_times")
        return {B.lib.tgs_stage_name(self._h, i).decode(): float(ms[i]) for i in range(n.value)}

    def kernels_per_step(self):
        return int(B.lib.tgs_kernels_per_step(self._h))

    def arena_bytes(self):
        """Device bytes of this context's scratch arena."""
        return int(B.lib.tgs_arena_bytes(self._h))

    @staticmethod
    def measure_peaks():
        """FP32 FMA (scalar and packed) and SFU (ex2, rcp) rates of the current GPU, per second
        (tgs_measure_peaks)."""
        p = B.tgs_peaks()
        B.check(B.lib.tgs_measure_peaks(C.byref(p), _stream()), "tgs_measure_peaks")
        return {k: getattr(p, k) for k, _ in p._fields_}

    def autotune(self, g: Gaussians, cams, targets, cache_path=None):
        B.check(B.lib.tgs_autotune(self._h, C.byref(g.struct()), cameras_array(cams), len(cams),
                                   _ptr_array(targets),
                                   None if cache_path is None else cache_path.encode(),
                                   _stream()), "tgs_autotune")
        cfg = self.config
        return dict(tile=cfg.tile, ppt=cfg.ppt, batch=cfg.batch, key_capacity=cfg.key_capacity)


class RasterizeViews(torch.autograd.Function):
    """images = RasterizeViews.apply(rasterizer, gaussians, cams, *params).

    ``params`` are the differentiable tensors of ``gaussians`` in PARAM_KEYS order (None
    entries skipped). Returns one [3,H,W] image per view."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, g: Gaussians, cams, *params):
        outs = rast.forward(g, cams, want_state=True)
        ctx.rast, ctx.g, ctx.cams = rast, g, cams
        ctx.keys = [k for k in PARAM_KEYS if getattr(g, k) is not None]
        # per-view checkpoint: T_final and last only
        ctx.state = [dict(T_final=o["T_final"], last=o["last"]) for o in outs]
        return tuple(o["image"] for o in outs)

    @staticmethod
    def backward(ctx, *dL):
        outs = [dict(image=None, **s) for s in ctx.state]
        dL = [torch.zeros_like(o["T_final"]).expand(3, -1, -1).contiguous() if d is None else d
              for d, o in zip(dL, outs)]
        grads, stats = ctx.rast.backward(ctx.g, ctx.cams, outs, dL)
        ctx.stats = stats
        return (None, None, None) + tuple(grads.get(k) for k in ctx.keys)


def rasterize(rast: Rasterizer, g: Gaussians, cams):
    """Differentiable rendering of V views; gradients flow into ``g``'s tensors."""
    params = [getattr(g, k) for k in PARAM_KEYS if getattr(g, k) is not None]
    return RasterizeViews.apply(rast, g, cams, *params)
