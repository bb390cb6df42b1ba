"""Seeded synthetic scenes, cameras and target images.

This module only draws random numbers and builds camera poses. It contains none of the
rasterizer's arithmetic (no projection, no covariance, no spherical harmonics, no blending),
so the CPU oracle and the CUDA path can both be fed from it without sharing any of the
method's code.

Every array is produced in float64 by ``numpy.random.default_rng(seed)`` and rounded to
float32 once; the float32 bytes are what both sides receive.

Scene layout (structure of arrays, float32, C-contiguous):
  means [N,3], log_scales [N,3], quats [N,4] (w, x, y, z), opacity_logits [N],
  sh_dc [N,3], sh_rest [N,15,3] (bands 1..3, coefficient-major, channel-minor),
  mask_logits [N] or None, sh_mask_logits [N,3] or None, sh_degree uint8 [N] or None.

Cameras are pinhole, OpenCV axes (x right, y down, z forward), world->camera 4x4 row-major.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray  # [4,4] float32, world -> camera, row-major
    campos: np.ndarray   # [3] float32, camera centre in world space
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def look_at_camera(pos, width, height, focal=None, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """Pinhole camera at ``pos`` looking at ``target``; principal point at the image centre.

    ``focal`` defaults to 0.866 * width (a 60 degree horizontal field of view)."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])          # rows: camera axes in world coordinates
    vm = np.eye(4)
    vm[:3, :3] = rot
    vm[:3, 3] = -rot @ pos
    f = 0.866 * width if focal is None else float(focal)
    # Camera intrinsics are stored as float32 values; the Python floats below are exactly
    # those float32 values so both sides read identical numbers.
    f32 = float(np.float32(f))
    return Camera(viewmat=_f32(vm), campos=_f32(pos), fx=f32, fy=f32,
                  cx=float(np.float32(width / 2.0)), cy=float(np.float32(height / 2.0)),
                  width=int(width), height=int(height))


def ring_cameras(n_views, sizes, radius=4.0, height=0.5, phase=0.0):
    """``n_views`` cameras evenly spaced on a horizontal ring, looking at the origin.

    ``sizes`` is a list of (width, height), one per view."""
    cams = []
    for v in range(n_views):
        a = phase + 2.0 * math.pi * v / n_views
        w, h = sizes[v]
        cams.append(look_at_camera((radius * math.cos(a), radius * math.sin(a), height), w, h))
    return cams


def hemisphere_cameras(n_views, width, height, radius=4.0, seed=0, max_elev_deg=75.0):
    """Random cameras on the upper hemisphere (elevation below ``max_elev_deg``)."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n_views):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(0.0, max_elev_deg))
        pos = (radius * math.cos(el) * math.cos(az), radius * math.cos(el) * math.sin(az),
               radius * math.sin(el))
        cams.append(look_at_camera(pos, width, height))
    return cams


def _random_unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def uniform_scene(n, seed, log_scale=(-3.0, 0.5), extent=1.0, sh_rest_std=0.1):
    """Gaussians with means uniform in [-extent, extent]^3 and no masks."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, size=(n, 3))
    log_scales = rng.normal(log_scale[0], log_scale[1], size=(n, 3))
    quats = _random_unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, size=n)
    sh_dc = rng.uniform(0.0, 1.0, size=(n, 3))
    sh_rest = rng.normal(0.0, sh_rest_std, size=(n, 15, 3))
    return dict(means=_f32(means), log_scales=_f32(log_scales), quats=_f32(quats),
                opacity_logits=_f32(opacity), sh_dc=_f32(sh_dc), sh_rest=_f32(sh_rest),
                mask_logits=None, sh_mask_logits=None, sh_degree=None)


def blob_scene(n, n_blobs, seed, log_scale=(-4.0, 0.5), shell_fraction=0.1,
               shell_radius=(6.0, 8.0), masks=True, per_gaussian_degree=False,
               sh_rest_std=0.1):
    """Mixture of ``n_blobs`` anisotropic 3D blobs plus a uniform spherical background shell.

    Blob centres are uniform in [-1,1]^3, per-axis standard deviations uniform in
    [0.05, 0.3], each blob with a random orientation; blobs have equal weight. The shell
    holds ``shell_fraction`` of the Gaussians at radius uniform in ``shell_radius``."""
    rng = np.random.default_rng(seed)
    n_shell = int(round(shell_fraction * n))
    n_blob = n - n_shell
    centres = rng.uniform(-1.0, 1.0, size=(n_blobs, 3))
    sigmas = rng.uniform(0.05, 0.3, size=(n_blobs, 3))
    rots = np.stack([np.linalg.qr(rng.normal(size=(3, 3)))[0] for _ in range(n_blobs)])
    which = rng.integers(0, n_blobs, size=n_blob)
    local = rng.normal(size=(n_blob, 3)) * sigmas[which]
    blob_pts = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    d = rng.normal(size=(n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shell_pts = d * rng.uniform(shell_radius[0], shell_radius[1], size=(n_shell, 1))
    means = np.concatenate([blob_pts, shell_pts])
    perm = rng.permutation(n)
    means = means[perm]
    log_scales = rng.normal(log_scale[0], log_scale[1], size=(n, 3))
    quats = _random_unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, size=n)
    sh_dc = rng.uniform(0.0, 1.0, size=(n, 3))
    sh_rest = rng.normal(0.0, sh_rest_std, size=(n, 15, 3))
    out = dict(means=_f32(means), log_scales=_f32(log_scales), quats=_f32(quats),
               opacity_logits=_f32(opacity), sh_dc=_f32(sh_dc), sh_rest=None,
               mask_logits=None, sh_mask_logits=None, sh_degree=None)
    if per_gaussian_degree:
        deg = rng.integers(0, 4, size=n)
        # coefficient k belongs to band 1 for k<3, band 2 for k<8, band 3 otherwise
        band_of_coeff = np.array([1] * 3 + [2] * 5 + [3] * 7)
        keep = band_of_coeff[None, :] <= deg[:, None]
        sh_rest = sh_rest * keep[:, :, None]
        out["sh_degree"] = np.ascontiguousarray(deg.astype(np.uint8))
    out["sh_rest"] = _f32(sh_rest)
    if masks:
        out["mask_logits"] = _f32(rng.normal(2.0, 1.0, size=n))
        out["sh_mask_logits"] = _f32(rng.normal(2.0, 1.0, size=(n, 3)))
    return out


def target_images(seed, sizes):
    """One seeded target image per (width, height), float32 [3,H,W] uniform in [0,1)."""
    rng = np.random.default_rng(seed)
    return [_f32(rng.uniform(0.0, 1.0, size=(3, h, w))) for (w, h) in sizes]


# --------------------------------------------------------------------------------------
# The five workloads. seed = 1000 * config + 1.
# --------------------------------------------------------------------------------------

C3_SIZES = [(320, 208)] * 4 + [(640, 416)] * 6 + [(1280, 832)] * 6


def workload(config, n=None, n_views=None):
    """Scene, cameras, targets and settings of one workload.

    ``n`` and ``n_views`` shrink a workload (same recipe, fewer Gaussians or views) for tests.
    Returns a dict with keys scene, cams, targets, eps_mask, eps_sh, tile, name."""
    seed = 1000 * config + 1
    if config == 1:
        n = 10_000 if n is None else n
        scene = uniform_scene(n, seed)
        cams = [look_at_camera((0.0, -4.0, 0.0), 128, 128, focal=150.0)]
        eps = (0.05, 0.1)
        name = f"plain fwd+bwd, {n} Gaussians uniform in [-1,1]^3, 128x128, f=150, SH3, L1"
    elif config == 2:
        n = 1_000_000 if n is None else n
        scene = blob_scene(n, 64, seed)
        v = 16 if n_views is None else n_views
        cams = ring_cameras(v, [(1280, 832)] * v)
        eps = (0.5, 0.5)
        name = (f"Trick-GS-masked fwd+bwd, {n} Gaussians (64 blobs + 10% shell), "
                f"{v} ring views 1280x832, SH3, masks eps=0.5, L1")
    elif config == 3:
        n = 500_000 if n is None else n
        scene = blob_scene(n, 64, seed)
        sizes = C3_SIZES if n_views is None else C3_SIZES[:: max(1, 16 // n_views)][:n_views]
        cams = ring_cameras(len(sizes), sizes)
        eps = (0.5, 0.5)
        name = f"batched progressive-resolution step, {n} Gaussians, {len(sizes)} mixed views"
    elif config == 4:
        n = 300_000 if n is None else n
        scene = blob_scene(n, 64, seed, masks=False, per_gaussian_degree=True)
        v = 100 if n_views is None else n_views
        cams = hemisphere_cameras(v, 1920, 1080, seed=seed + 7)
        eps = (0.05, 0.1)
        name = f"render-only, {n} Gaussians, per-Gaussian SH degree, 1920x1080, {v} poses"
    elif config == 5:
        n = 3_000_000 if n is None else n
        scene = blob_scene(n, 256, seed, log_scale=(-4.0, 0.7))
        v = 8 if n_views is None else n_views
        cams = ring_cameras(v, [(1600, 1064)] * v)
        eps = (0.5, 0.5)
        name = f"large-scene batched fwd+bwd, {n} Gaussians (256 blobs), {v} views 1600x1064"
    else:
        raise ValueError(f"unknown workload {config}")
    targets = target_images(seed + 500, [(c.width, c.height) for c in cams])
    return dict(scene=scene, cams=cams, targets=targets, eps_mask=eps[0], eps_sh=eps[1],
                tile=16, name=name, seed=seed)
