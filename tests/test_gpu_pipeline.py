"""End-to-end GLR iterations on the GPU: CUDA-graph replay, the autotuner, and the
whole reconstruction against the oracle step by step (teacher forcing)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def _problem(T=4, H=96, W=100, N=80, K=24):
    cfg = synth.scaled(synth.SCI_SMALL, T=T, H=H, W=W, N=N, K=K, iters=3)
    prob = synth.sci_problem(cfg)
    return cfg, prob, torch.from_numpy(prob.y).cuda(), torch.from_numpy(prob.masks).cuda()


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_graph_replay_matches_eager(mode):
    cfg, prob, y, m = _problem()
    sig = cfg.sigma_schedule()
    a = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=mode)
    b = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode=mode)
    a.start(y, m)
    b.start(y, m)
    b.capture(sig, cfg.c_wnnm)
    for s in sig:
        a.step(s, cfg.c_wnnm)
        b.step_graph(s)
    torch.cuda.synchronize()
    # every step is order-independent (the aggregation sums in fixed point), so the replayed
    # graph and the eager launches give the same bits
    assert torch.equal(b.x, a.x)


@pytest.mark.parametrize("mode", ["bf16", "learned"])
def test_frames_per_call_equals_all_frames_at_once(mode):
    """The denoiser run on 3 frames per call (the large-frame form: workspaces sized for 3, the
    last call ragged) gives the same bits as one call over all frames: frames are independent
    and every step is order-independent.  Also under CUDA-graph replay."""
    cfg, prob, y, m = _problem(T=7)
    sig = cfg.sigma_schedule()
    kw = dict(mode=mode)
    if mode == "learned":
        kw["encoder"] = glr.Encoder(seed=4).params
    a = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, **kw)
    b = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, frames_per_call=3, **kw)
    c = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, frames_per_call=3, **kw)
    for r in (a, b, c):
        r.start(y, m)
    c.capture(sig, cfg.c_wnnm)
    for s in sig:
        a.step(s, cfg.c_wnnm)
        b.step(s, cfg.c_wnnm)
        c.step_graph(s)
    torch.cuda.synchronize()
    assert torch.equal(b.x, a.x)
    assert torch.equal(c.x, a.x)


def test_autotune_picks_a_working_schedule():
    cfg, prob, y, m = _problem(T=2, H=128, W=128, N=200, K=32)
    x = glr.gap_step(y[None], m, None).view(cfg.T, 1, cfg.H, cfg.W).contiguous()
    keys, nf, _ = glr.select_keys(x, cfg.P, cfg.N)
    cands = [(48, 1, 0, 4, 1), (48, 2, 192, 2, -1), (64, 1, 320, 4, 1), (48, 2, 0, 2, 1)]
    best = glr.autotune_match(x, cfg.P, keys, nf, cfg.K, "bf16", candidates=cands)
    assert best in cands
    ref, _ = glr.match_topk(x, cfg.P, keys, nf, cfg.K, "fp32")
    got, _ = glr.match_topk(x, cfg.P, keys, nf, cfg.K, "bf16", k_over=best[0], splits=best[1], cap=best[2],
                            epi_batch=best[3], bound_pass=best[4])
    a, b = ref.cpu().numpy(), got.cpu().numpy()
    same = np.mean([len(set(a[f, k]) & set(b[f, k])) / cfg.K for f in range(cfg.T) for k in range(cfg.N)])
    assert same >= 0.99


def test_reconstruction_tracks_oracle_teacher_forced():
    """Three GAP iterations: each GPU step is fed the GPU state, and the oracle's step on the
    same state must agree (keys bit-exact for 8-bit-quantised states, denoised frames close)."""
    cfg, prob, y, m = _problem(T=2, H=64, W=72, N=60, K=16)
    rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="fp32")
    rec.start(y, m)
    for s in cfg.sigma_schedule():
        # quantise the state so that both sides take the same edge decisions
        q = torch.round(rec.x * 256.0) / 256.0
        rec.x.copy_(q)
        xs = rec.x.cpu().numpy()[0][:, None].astype(np.float64)
        rec.step(s, cfg.c_wnnm)
        v_gpu = rec.v.cpu().numpy()[0]
        v_or, _ = O.glr_denoise(xs, cfg.P, cfg.N, cfg.K, s, cfg.c_wnnm, cfg.edge_th, eps=1e-8)
        err = np.abs(v_gpu - v_or[:, 0])
        assert np.sqrt(np.mean(err ** 2)) < 2e-4 and err.max() < 2e-3
        x_or, _ = O.gap_project(prob.y, prob.masks, v_gpu)
        np.testing.assert_allclose(rec.x.cpu().numpy()[0], x_or, rtol=1e-4, atol=1e-5)


def test_config1_free_running_against_oracle():
    """The whole plain FP32 reconstruction of the small video workload (8 frames of 128 x 128,
    N = 200 keys, K = 40, 3 GAP iterations), free running on both sides from the same
    snapshot: the GPU result must stay within 50 dB PSNR of the FP64 oracle's (a key picked
    differently on a near-tied corner response changes a few patches, not the image)."""
    cfg = synth.SCI_SMALL
    prob = synth.sci_problem(cfg)
    rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="fp32")
    rec.start(torch.from_numpy(prob.y).cuda(), torch.from_numpy(prob.masks).cuda())
    for s in cfg.sigma_schedule():
        rec.step(s, cfg.c_wnnm)
    torch.cuda.synchronize()
    x_gpu = rec.x.cpu().numpy()[0]
    x_or = O.glr_reconstruct(prob.y, prob.masks, cfg.P, cfg.N, cfg.K, cfg.sigma_schedule(), cfg.c_wnnm,
                             cfg.edge_th, eps=1e-8)
    agree = O.psnr(x_gpu, x_or)
    assert agree >= 50.0, agree
    # and both reconstruct the scene equally well
    assert abs(O.psnr_framewise(x_gpu, prob.truth) - O.psnr_framewise(x_or, prob.truth)) < 0.05
