"""FP64 CPU oracle of GLR demosaicing for multispectral filter arrays (MSFA).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the library never imports it.

The MSFA model of Section 3 is y = sum_b A_b x_b (Eq. 8) with masks that do
not overlap (Eq. 9: A_b * A_c = 0 for b != c), so the
GAP normaliser R = sum_b A_b^2 is 1 wherever a band is sampled.  One
iteration denoises the whole multispectral image with GLR, patches spanning
all bands (C = bands, d = bands P^2; multi-channel matching as in the paper's
MSFA experiments), then projects back onto y = Phi x.  A batch holds images of
different sizes; each is reconstructed on its own (the batch only groups the
work).

Readings: F1  per-image key count N = min(8192, 1024 (side / 256)^2) (the
workload description's rule); F2  noiseless snapshots (the workload is silent
on noise); F3  sigma_w schedule geometric 0.1 -> 0.02 (not given in the paper);
F4  the start is bilinear interpolation of each band (normalised convolution with
a tent of half-width sqrt(bands)): the paper gives none, and from the zero-filled
Phi^T y every patch carries the mosaic pattern, which the low-rank step keeps.
"""
from __future__ import annotations

import numpy as np

from . import glr_oracle as G


def mosaic_init(y: np.ndarray, masks: np.ndarray, s: int) -> np.ndarray:
    """Reading F4: per band, normalised convolution of the samples with the tent
    w(dr, dc) = (1 - |dr|/s)(1 - |dc|/s), |dr|, |dc| < s, over the pixels inside
    the image (bilinear interpolation for a mosaic of period s); 0 without samples."""
    y = np.asarray(y, dtype=np.float64)
    A = np.asarray(masks, dtype=np.float64)
    T, H, W = A.shape
    num = np.zeros((T, H, W))
    den = np.zeros((T, H, W))
    for dr in range(-(s - 1), s):
        for dc in range(-(s - 1), s):
            w = (1.0 - abs(dr) / s) * (1.0 - abs(dc) / s)
            # output p = (r, c) takes the sample at q = (r + dr, c + dc) when q is inside
            r0, r1 = max(0, -dr), min(H, H - dr)
            c0, c1 = max(0, -dc), min(W, W - dc)
            q = (slice(r0 + dr, r1 + dr), slice(c0 + dc, c1 + dc))
            num[:, r0:r1, c0:c1] += w * A[:, q[0], q[1]] * y[None, q[0], q[1]]
            den[:, r0:r1, c0:c1] += w * A[:, q[0], q[1]]
    out = np.zeros((T, H, W))
    m = den > 0
    out[m] = num[m] / den[m]
    return out


def msfa_reconstruct(y, masks, P, N, K, sigmas, c, th, eps=1e-16, callback=None, s=None):
    """GAP + GLR for one mosaic snapshot y [H][W] with masks [bands][H][W]; returns x [bands][H][W].
    The start is mosaic_init with s = sqrt(bands) (reading F4)."""
    if s is None:
        s = int(round(np.sqrt(np.asarray(masks).shape[0])))
    x = mosaic_init(y, masks, s)
    for it, sw in enumerate(sigmas):
        v, _ = G.glr_denoise(x[None], P, N, K, sw, c, th, eps)
        x, _ = G.gap_project(y, masks, v[0])
        if callback is not None:
            callback(it, x)
    return x


def msfa_reconstruct_batch(images, P, K, sigmas, c, th, eps=1e-16):
    """Every image of an uneven batch (objects with .y, .masks, .N) reconstructed independently."""
    return [msfa_reconstruct(im.y, im.masks, P, im.N, K, sigmas, c, th, eps) for im in images]
