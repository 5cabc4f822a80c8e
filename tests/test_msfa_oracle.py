"""Pins of the MSFA oracle and its inputs (CPU only)."""
import numpy as np
import pytest

from oracle import glr_oracle as G
from oracle import msfa_oracle as FO
from paper_2301_03047_gb300 import synth


def test_mosaic_masks_are_orthogonal_and_cover():
    m = synth.mosaic_masks(10, 13, 16)
    assert np.all(m.sum(0) == 1)  # every pixel sees exactly one band (Eq. 9: A_b A_c = 0)
    for b in range(16):
        rr, cc = np.nonzero(m[b])
        assert np.all(4 * (rr % 4) + (cc % 4) == b)
    assert np.all(G.gap_normaliser(m) == 1)


def test_key_count_rule():
    cfg = synth.MSFA_LARGE
    assert [cfg.N_of(s) for s in (256, 384, 512, 768, 1024)] == [1024, 2304, 4096, 8192, 8192]
    assert len(cfg.sides) == 32 and set(cfg.sides) <= {256, 384, 512, 768, 1024}


def test_projection_keeps_the_snapshot():
    """After every iteration Phi x = y exactly (orthogonal masks, R = 1)."""
    im = synth.msfa_problem(synth.MSFA_SMALL)[0]
    cfg = synth.MSFA_SMALL
    seen = []
    FO.msfa_reconstruct(im.y, im.masks, cfg.P, 24, 8, [0.3], cfg.c_wnnm, cfg.edge_th,
                        callback=lambda it, x: seen.append((im.masks * x).sum(0)))
    assert np.allclose(seen[0], im.y, atol=1e-12)


def test_multichannel_distance_is_the_sum_over_bands():
    rng = synth.rng_for("mc")
    x = rng.random((3, 12, 12))
    keys = np.array([5, 40], np.int32)
    idx, dist = G.match_topk(x, 4, keys, 6)
    for i, k in enumerate(keys):
        r0, c0 = divmod(int(k), 9)
        for j in range(6):
            r, c = divmod(int(idx[i, j]), 9)
            want = sum(((x[b, r:r + 4, c:c + 4] - x[b, r0:r0 + 4, c0:c0 + 4]) ** 2).sum() for b in range(3))
            assert np.isclose(dist[i, j], want)


@pytest.mark.slow
def test_glr_improves_on_the_mosaic_start():
    cfg = synth.MSFA_SMALL
    im = synth.msfa_problem(cfg)[2]
    x0 = FO.mosaic_init(im.y, im.masks, 4)
    x = FO.msfa_reconstruct(im.y, im.masks, cfg.P, im.N, cfg.K, [0.1, 0.05, 0.03, 0.02], cfg.c_wnnm, cfg.edge_th)
    assert G.psnr(x, im.truth) > G.psnr(x0, im.truth) + 0.1
    assert G.psnr(x0, im.truth) > G.psnr(G.gap_init(im.y, im.masks), im.truth) + 10.0


def test_mosaic_init_closed_forms():
    cfg = synth.MSFA_SMALL
    m = synth.mosaic_masks(16, 20, 16)
    # a constant scene is reproduced exactly (weights normalised)
    y = (m * 0.7).sum(0)
    assert np.allclose(FO.mosaic_init(y, m, 4), 0.7)
    # a band that is linear in the column index is reproduced exactly away from the border
    # (bilinear interpolation of a linear function between samples 4 apart)
    cube = np.zeros((16, 16, 20))
    cube[:] = np.arange(20)[None, None, :] * 0.01
    y = (m * cube).sum(0)
    x0 = FO.mosaic_init(y, m, 4)
    assert np.allclose(x0[:, 4:12, 4:16], cube[:, 4:12, 4:16])
    # samples of a band are s apart, so at a sampled pixel the tent weights every other
    # sample of that band by 0: the start reproduces the snapshot exactly
    rng = synth.rng_for("mi")
    cube = rng.random((16, 16, 20))
    y = (m * cube).sum(0)
    x0 = FO.mosaic_init(y, m, 4)
    assert np.allclose((m * x0).sum(0), y)
