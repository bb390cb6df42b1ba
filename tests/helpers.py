"""Helpers shared by the GPU parity tests: conversions between the library's splat records
and the oracle's per-Gaussian arrays, and the comparison rules.

Comparison rules (tolerances of the parity tests):
  - keys, values, ranges, radii and rects: bit-exact, except a radius or rect that the FP64
    oracle puts within 1e-5 relative of an integer boundary (counted);
  - images: max |gpu - oracle| <= 1e-4 over pixels whose every blend decision is clear of its
    threshold by more than the float32 uncertainty (the oracle's per-pixel margin >= 1);
  - gradients: per tensor ||g - g*|| / ||g*|| <= 1e-3, and per element
    |g - g*| <= 1e-3 |g*| + 1e-3 max |g*| (check_grad).
"""
import numpy as np

import oracle

IMAGE_ATOL = 1e-4
GRAD_RTOL = 1e-3


def splats_to_oracle(rec, radii):
    """Library splat records [n,12] float32 (numpy) -> oracle per-Gaussian arrays."""
    rec = np.asarray(rec, dtype=np.float32)
    bits = rec.view(np.uint32)
    rx, ry = bits[:, 9], bits[:, 10]
    rect = np.stack([rx & 0xFFFF, rx >> 16, ry & 0xFFFF, ry >> 16], axis=1).astype(np.int32)
    radii = np.asarray(radii, dtype=np.int32)
    vis = radii > 0
    z = lambda a: np.where(vis.reshape((-1,) + (1,) * (a.ndim - 1)), a, 0)
    return oracle.splats_from(z(rec[:, 0:2]), z(rec[:, 11]), z(rec[:, 2:5]), z(rec[:, 5]),
                              z(rec[:, 6:9]), radii, np.where(vis[:, None], rect, 0))


def cull_data(rec):
    """Float32 cull data of library splat records: mean2d, conic a, b, c, tau, b/c, b/a."""
    rec = np.asarray(rec, dtype=np.float32)
    return np.ascontiguousarray(rec[:, [0, 1, 2, 3, 4, 12, 13, 14]])


def gpu_lists(rec, radii, W, H, tile):
    """The key oracle's tile lists (values, ranges) of library records, culled as the library
    culls them."""
    gs = splats_to_oracle(rec, radii)
    _, v, r = oracle.keys(gs["radius"], gs["rect"], np.asarray(rec, np.float32)[:, 11], W, H, tile,
                          cull=cull_data(rec))
    return v, r


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def image_compare(gpu, ref, margin):
    """Returns (max abs diff over clear pixels, fraction of pixels excluded)."""
    clear = margin >= 1.0
    diff = np.abs(np.asarray(gpu, np.float64) - ref).max(axis=0)
    m = float(diff[clear].max()) if clear.any() else 0.0
    return m, 1.0 - clear.mean()


def mismatch_fraction(gpu, ref):
    """Fraction of all pixels (margin cases included) where some channel differs by more than
    IMAGE_ATOL: the pixels where a decision actually fell the other way."""
    diff = np.abs(np.asarray(gpu, np.float64) - ref).max(axis=0)
    return float((diff > IMAGE_ATOL).mean())


def elem_err(a, b, rtol=GRAD_RTOL, stol=GRAD_RTOL):
    """Largest |a - b| / (rtol |b| + stol max|b|) over the elements (<= 1 passes); b is the
    reference. An all-zero reference requires an all-zero a."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = float(np.abs(b).max()) if b.size else 0.0
    if scale == 0.0:
        return 0.0 if not np.any(a) else float("inf")
    return float((np.abs(a - b) / (rtol * np.abs(b) + stol * scale)).max())


def check_grad(got, ref, name, rel=GRAD_RTOL, elem=GRAD_RTOL):
    """Per-tensor relative L2 error <= rel and per-element |g - g*| <= elem |g*| + elem max|g*|."""
    e = rel_err(got, ref)
    r = elem_err(got, ref, elem, elem)
    assert e <= rel and r <= 1.0, (name, "rel", e, "elem", r)
    return e, r


def zero_margin_pixels(dl, margin):
    """dL/dimage with the pixels whose blend decisions are within the float32 uncertainty set
    to 0: every gradient term of a pixel is proportional to its dL/dC, so such a pixel then
    contributes nothing on either side, whichever way its decisions fall."""
    dl = np.array(dl, copy=True)
    dl[:, np.asarray(margin) < 1.0] = 0.0
    return dl
