"""Degenerate and extreme cases through the C ABI, against the oracle.

K = every position, N = K = 1, images with no valid key rows (n_found = 0),
one-column groups, the smallest FFT, and the largest window.  Collected after
the parity files; each case is small.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from oracle import mri_oracle as MO  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_match_k_equals_every_position(mode):
    """10 x 11 image, P = 8: 12 positions, K = 12: every position, sorted by distance."""
    x = synth.textured_frames(synth.rng_for("kall"), 1, 10, 11)[None]
    keys = np.array([[0, 5, 11]], np.int32)
    idx, dist = glr.match_topk(cuda(x), 8, cuda(keys, torch.int32), cuda(np.array([3], np.int32), torch.int32), 12, mode)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy()[0], dist.cpu().numpy()[0]
    Q = O.patch_matrix(x[0], 8)
    for i, k in enumerate(keys[0]):
        assert sorted(idx[i].tolist()) == list(range(12))
        d = O.all_distances(x[0], 8, int(k), Q)
        np.testing.assert_allclose(dist[i], np.sort(d), rtol=2e-5, atol=2e-6)


@pytest.mark.parametrize("mode", ["fp32", "bf16", "edge"])
def test_single_key_single_match(mode):
    x = synth.quantize8(synth.textured_frames(synth.rng_for("one-one"), 1, 40, 40))[None]
    keys = np.array([[123]], np.int32)
    idx, dist = glr.match_topk(cuda(x), 8, cuda(keys, torch.int32), cuda(np.array([1], np.int32), torch.int32), 1, mode)
    torch.cuda.synchronize()
    if mode == "edge":
        h = O.edge_heatmap(x[0], 8, 123, 0.1)
        assert float(dist.cpu()[0, 0, 0]) == h.max()
    else:
        assert int(idx.cpu()[0, 0, 0]) == 123 and float(dist.cpu()[0, 0, 0]) == 0.0


def test_image_without_keys_is_left_unchanged():
    """n_found = 0 for one image: no groups, aggregation returns the input there."""
    x = synth.textured_frames(synth.rng_for("nf0"), 2, 30, 30)[:, None]
    P, N, K = 6, 10, 4
    keys = np.tile(np.arange(N, dtype=np.int32) * 11, (2, 1))
    nf = cuda(np.array([10, 0], np.int32), torch.int32)
    xt = cuda(x)
    idx, _ = glr.match_topk(xt, P, cuda(keys, torch.int32), nf, K)
    groups, rank = glr.lowrank_groups(xt, P, idx, nf, 0.1, 2 * math.sqrt(K))
    v = glr.aggregate(groups, idx, nf, xt, P)
    torch.cuda.synchronize()
    assert torch.equal(v[1], xt[1])
    assert not torch.equal(v[0], xt[0])


@pytest.mark.parametrize("complex_", [False, True])
def test_one_column_groups(complex_):
    """K = 1: the group is a single column; WNNM shrinks its norm by the closed form."""
    if complex_:
        x = synth.complex_phantom(synth.rng_for("k1c"), 20, 20)[None]
    else:
        x = synth.textured_frames(synth.rng_for("k1"), 1, 20, 20)[None]
    P, sw = 6, 0.3
    idx = np.array([[[7], [40], [100]]], np.int32)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(np.array([3], np.int32), torch.int32),
                                      sw, 2.0, complex_=complex_)
    torch.cuda.synchronize()
    Y = O.gather_groups(x[0], P, idx[0])
    for i in range(3):
        s = np.linalg.norm(Y[i])
        sh = math.sqrt(max(s * s - sw * sw, 0.0))
        sp = max(s - 2.0 * sw * sw / (sh + 1e-8), 0.0)
        np.testing.assert_allclose(groups.cpu().numpy()[0, i], Y[i] * (sp / s), rtol=1e-5, atol=1e-6)


def test_smallest_fft():
    z = np.array([[[1.0, -2.0], [0.5, 3.0]], [[0.0, 1.0], [2.0, -1.0]]], np.float32)[None]
    out = glr.fft2(cuda(z))
    torch.cuda.synchronize()
    want = MO.fft2c(z[0, 0].astype(np.float64) + 1j * z[0, 1])
    got = out.cpu().numpy()[0]
    np.testing.assert_allclose(got[0] + 1j * got[1], want, atol=1e-6)


def test_window_covering_the_grid_is_global_matching():
    x = synth.textured_frames(synth.rng_for("wg"), 1, 40, 40)[None]  # 33 x 33 positions, w = 16 covers them
    keys = np.array([[0, 500, 1088]], np.int32)
    nf = cuda(np.array([3], np.int32), torch.int32)
    gi, gd = glr.match_topk(cuda(x), 8, cuda(keys, torch.int32), nf, 10, "fp32")
    wi, wd = glr.match_topk(cuda(x), 8, cuda(keys, torch.int32), nf, 10, "window", window=16)
    torch.cuda.synchronize()
    np.testing.assert_allclose(wd.cpu().numpy(), gd.cpu().numpy(), rtol=2e-5, atol=2e-6)
