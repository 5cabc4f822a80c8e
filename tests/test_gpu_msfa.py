"""MSFA demosaicing path (multi-channel patches, uneven image batches) against the FP64 oracle.

* glr_mosaic_init: the bilinear start within 1e-6 (FP32 sums of at most 49 terms).
* multi-channel FP32 matching (16 bands, 6 x 6 patches, d = 576: the key tile is
  streamed through shared memory in channel chunks): ids bit-exact where the
  oracle's distances are separated, distances within 2e-5 relative.
* one GAP + GLR iteration of every size class of an uneven batch, teacher-forced
  against the oracle; CUDA-graph replay of the whole batch iteration equal to
  eager execution.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from oracle import msfa_oracle as FO  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402

TAU_SEP = 1e-4


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("shared", [True, False])
def test_mosaic_init_matches_oracle(shared):
    rng = synth.rng_for("mi-gpu")
    G, T, H, W = 2, 16, 37, 45
    m = synth.mosaic_masks(H, W, T)
    masks = m if shared else np.stack([m, np.roll(m, 1, axis=0)])
    y = rng.random((G, H, W)).astype(np.float32)
    x0 = glr.mosaic_init(cuda(y), cuda(masks), 4)
    torch.cuda.synchronize()
    for g in range(G):
        want = FO.mosaic_init(y[g], masks if shared else masks[g], 4)
        np.testing.assert_allclose(x0.cpu().numpy()[g], want, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("case", [("f1", 16, 30, 40, 6, 20, 16), ("f2", 4, 33, 29, 6, 25, 12), ("f3", 16, 24, 70, 5, 12, 8)])
def test_match_fp32_multichannel_parity(case):
    tag, C, H, W, P, N, K = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, C, H, W)[None]
    npos = (H - P + 1) * (W - P + 1)
    keys = rng.choice(npos, size=(1, N), replace=False).astype(np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([N], np.int32), torch.int32), K, "fp32")
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy()[0], dist.cpu().numpy()[0]
    Q = O.patch_matrix(x[0], P)
    for i in range(N):
        d_all = O.all_distances(x[0], P, keys[0, i], Q)
        order = np.lexsort((np.arange(len(d_all)), d_all))
        ds = d_all[order]
        np.testing.assert_allclose(dist[i], d_all[idx[i]], rtol=2e-5, atol=2e-6)
        for j in range(K):
            sep = min(ds[j + 1] - ds[j] if j + 1 < len(ds) else np.inf, ds[j] - ds[j - 1] if j > 0 else np.inf)
            if sep > TAU_SEP * (1 + ds[j]):
                assert idx[i, j] == order[j], (i, j)
        assert np.all(d_all[idx[i]] <= ds[K - 1] + TAU_SEP * (1 + ds[K - 1]))


def test_batch_iteration_tracks_oracle_teacher_forced():
    cfg = synth.MSFA_SMALL
    imgs = synth.msfa_problem(cfg)
    rec = glr.MsfaBatchReconstructor([im.y.shape[0] for im in imgs], [im.N for im in imgs], cfg.bands, cfg.P,
                                     cfg.K, mode="fp32")
    masks = {im.y.shape[0]: cuda(im.masks) for im in imgs}
    rec.start([cuda(im.y) for im in imgs], masks)
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        np.testing.assert_allclose(rec.images()[i].cpu().numpy(), FO.mosaic_init(im.y, im.masks, 4), rtol=1e-5, atol=1e-6)
    for sw in cfg.sigma_schedule():
        for c in rec.classes:  # quantise the state so both sides take the same edge decisions
            c["x"].copy_(torch.round(c["x"] * 256.0) / 256.0)
        xs = [t.cpu().numpy().astype(np.float64) for t in rec.images()]
        rec.step(sw, cfg.c_wnnm)
        torch.cuda.synchronize()
        for c in rec.classes:
            for j, i in enumerate(c["ids"]):
                v_or, _ = O.glr_denoise(xs[i][None], cfg.P, imgs[i].N, cfg.K, sw, cfg.c_wnnm, cfg.edge_th, eps=1e-8)
                err = np.abs(c["v"][j].cpu().numpy() - v_or[0])
                assert np.sqrt(np.mean(err ** 2)) < 2e-4 and err.max() < 2e-3, (i, err.max())
                x_or, _ = O.gap_project(imgs[i].y, imgs[i].masks, c["v"][j].cpu().numpy())
                np.testing.assert_allclose(c["x"][j].cpu().numpy(), x_or, rtol=1e-5, atol=1e-6)


def test_batch_graph_replay_matches_eager():
    cfg = synth.MSFA_SMALL
    imgs = synth.msfa_problem(cfg)
    sides = [im.y.shape[0] for im in imgs]
    masks = {im.y.shape[0]: cuda(im.masks) for im in imgs}
    a = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode="fp32")
    b = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode="fp32")
    a.start([cuda(im.y) for im in imgs], masks)
    b.start([cuda(im.y) for im in imgs], masks)
    sig = cfg.sigma_schedule()
    b.capture(sig, cfg.c_wnnm)
    for sw in sig:
        a.step(sw, cfg.c_wnnm)
        b.step_graph(sw)
    torch.cuda.synchronize()
    for xa, xb in zip(a.images(), b.images()):
        np.testing.assert_allclose(xb.cpu().numpy(), xa.cpu().numpy(), rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("case", [("w1", 16, 40, 70, 6, 30, 32, 0), ("w2", 4, 50, 60, 6, 40, 16, 2),
                                  ("w3", 3, 36, 300, 5, 130, 24, 0), ("w4", 16, 24, 24, 4, 20, 8, 3)])
def test_match_bf16_wide_recall(case):
    """d = 576, 144, 75, 256: the tensor-core path streams 64-column chunks of keys and positions."""
    tag, C, H, W, P, N, K, splits = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, C, H, W)[None]
    npos = (H - P + 1) * (W - P + 1)
    keys = rng.choice(npos, size=(1, N), replace=False).astype(np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([N], np.int32), torch.int32), K,
                               "bf16", splits=splits)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy()[0], dist.cpu().numpy()[0]
    Q = O.patch_matrix(x[0], P)
    hits = 0
    for i in range(N):
        d_all = O.all_distances(x[0], P, keys[0, i], Q)
        np.testing.assert_allclose(dist[i], d_all[idx[i]], rtol=2e-5, atol=2e-6)
        assert np.all(np.diff(dist[i]) >= -1e-4)
        order = np.lexsort((np.arange(len(d_all)), d_all))[:K]
        hits += len(set(order.tolist()) & set(idx[i].tolist()))
    assert hits / (N * K) >= 0.99, hits / (N * K)


def test_batch_bf16_matches_fp32_form():
    """The chosen (BF16 + exact re-rank) form of a batch iteration agrees with the FP32 form."""
    cfg = synth.MSFA_SMALL
    imgs = synth.msfa_problem(cfg)
    sides = [im.y.shape[0] for im in imgs]
    masks = {im.y.shape[0]: cuda(im.masks) for im in imgs}
    outs = []
    for mode in ("bf16", "fp32"):
        r = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode=mode)
        r.start([cuda(im.y) for im in imgs], masks)
        for sw in cfg.sigma_schedule():
            r.step(sw, cfg.c_wnnm)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in r.images()])
    for a, b, im in zip(outs[0], outs[1], imgs):
        assert abs(O.psnr(a, im.truth) - O.psnr(b, im.truth)) < 0.05


def test_persistent_batch_matching_equals_class_path():
    """The whole batch's matching as one persistent launch (glr_match_topk_batch) gives the same
    matches as one launch per size class, so a full BF16 run of the schedule is identical bit for
    bit; CUDA-graph replay of the persistent form equals its eager run."""
    cfg = synth.MSFA_SMALL
    imgs = synth.msfa_problem(cfg)
    sides = [im.y.shape[0] for im in imgs]
    masks = {im.y.shape[0]: cuda(im.masks) for im in imgs}
    ys = [cuda(im.y) for im in imgs]
    sig = cfg.sigma_schedule()
    a = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode="bf16")
    b = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode="bf16", persistent=True)
    c = glr.MsfaBatchReconstructor(sides, [im.N for im in imgs], cfg.bands, cfg.P, cfg.K, mode="bf16", persistent=True)
    for r in (a, b, c):
        r.start(ys, masks)
    c.capture(sig, cfg.c_wnnm)
    for sw in sig:
        a.step(sw, cfg.c_wnnm)
        b.step(sw, cfg.c_wnnm)
        c.step_graph(sw)
    torch.cuda.synchronize()
    for xa, xb, xc in zip(a.images(), b.images(), c.images()):
        assert torch.equal(xa, xb)
        assert torch.equal(xb, xc)
