"""Corner + uniform key mixes and ADMM for video SCI through the C ABI, against the oracle.

* glr_select_keys_mixed: bit-exact (8-bit-quantised inputs make the edge maps
  exact; everything after them is integer).
* glr_admm_sci_step: u, x', w within 1e-5 relative / 1e-6 absolute.
* one ADMM reconstruction step teacher-forced against the oracle's denoiser and step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("nu", [0, 1, 7, 20, 40])
@pytest.mark.parametrize("case", [("mx1", 2, 1, 64, 72, 8, 40), ("mx2", 1, 3, 40, 50, 5, 40)])
def test_select_mixed_bit_exact(case, nu):
    tag, F, C, H, W, P, N = case
    x = synth.quantize8(synth.textured_frames(synth.rng_for(tag), F * C, H, W)).reshape(F, C, H, W)
    keys, nf, nc = glr.select_keys(cuda(x), P, N, 0.1, n_uniform=nu)
    torch.cuda.synchronize()
    for f in range(F):
        want, nco = O.select_keys(x[f], P, N, 0.1, n_uniform=nu)
        np.testing.assert_array_equal(keys.cpu().numpy()[f], want)
        assert int(nc[f]) == nco and int(nf[f]) == N


def test_admm_sci_step_matches_oracle():
    rng = synth.rng_for("admm-gpu")
    G, T, H, W = 2, 5, 33, 40
    A = (rng.random((T, H, W)) < 0.5).astype(np.float32)
    y = rng.random((G, H, W)).astype(np.float32)
    z, x, u = (rng.random((G, T, H, W)).astype(np.float32) for _ in range(3))
    ut = cuda(u)
    xo, wo = glr.admm_sci_step(cuda(y), cuda(A), cuda(z), cuda(x), ut, 0.3)
    torch.cuda.synchronize()
    for g in range(G):
        xn, un, wn = O.admm_sci_step(y[g], A, z[g], x[g], u[g], 0.3)
        np.testing.assert_allclose(ut.cpu().numpy()[g], un, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(xo.cpu().numpy()[g], xn, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(wo.cpu().numpy()[g], wn, rtol=1e-5, atol=1e-6)


def test_admm_reconstruction_step_tracks_oracle():
    cfg = synth.scaled(synth.SCI_SMALL, T=2, H=64, W=72, N=60, K=16)
    prob = synth.sci_problem(cfg)
    rec = glr.SciReconstructor(cfg.T, cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="fp32", admm_rho=0.5, n_uniform=10)
    rec.start(cuda(prob.y), cuda(prob.masks))
    for s in cfg.sigma_schedule():
        rec.w.copy_(torch.round(rec.w * 256.0) / 256.0)  # same edge decisions on both sides
        w = rec.w.cpu().numpy()[0].astype(np.float64)
        x_prev, u_prev = rec.x.cpu().numpy()[0], rec.u.cpu().numpy()[0]
        rec.step(s, cfg.c_wnnm)
        torch.cuda.synchronize()
        z_gpu = rec.v.cpu().numpy()[0]
        # the oracle's denoiser with the same key mix
        outs = []
        for t in range(cfg.T):
            xt = w[t][None]
            Q = O.patch_matrix(xt, cfg.P)
            keys, _ = O.select_keys(xt, cfg.P, cfg.N, cfg.edge_th, n_uniform=10)
            idx, _ = O.match_topk(xt, cfg.P, keys, cfg.K, Q)
            xh, _ = O.lowrank_groups(O.gather_groups(xt, cfg.P, idx, Q), s, cfg.c_wnnm, eps=1e-8)
            outs.append(O.aggregate(xh, idx, xt, cfg.P)[0])
        z_or = np.stack(outs)
        err = np.abs(z_gpu - z_or)
        assert np.sqrt(np.mean(err ** 2)) < 2e-4 and err.max() < 2e-3
        xn, un, wn = O.admm_sci_step(prob.y, prob.masks, z_gpu, x_prev, u_prev, 0.5)
        np.testing.assert_allclose(rec.x.cpu().numpy()[0], xn, rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(rec.w.cpu().numpy()[0], wn, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("case", [("w1", 2, 1, 50, 60, 8, 30, 16, 20), ("w2", 1, 3, 40, 44, 5, 25, 12, 6),
                                  ("w3", 1, 1, 30, 30, 6, 20, 9, 1)])
def test_window_matching_parity(case):
    tag, F, C, H, W, P, N, K, w = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, F * C, H, W).reshape(F, C, H, W)
    npos = (H - P + 1) * (W - P + 1)
    keys = np.stack([rng.choice(npos, size=N, replace=False) for _ in range(F)]).astype(np.int32)
    keys[:, 0] = 0  # a corner key: its window is shifted inside the grid
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.full(F, N, np.int32), torch.int32), K,
                               "window", window=w)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    for f in range(F):
        oi, od = O.window_match_topk(x[f], P, keys[f], K, w)
        np.testing.assert_allclose(dist[f], od, rtol=2e-5, atol=2e-6)
        for i in range(N):
            for j in range(K):
                sep = min(od[i, j + 1] - od[i, j] if j + 1 < K else np.inf, od[i, j] - od[i, j - 1] if j > 0 else np.inf)
                if sep > 1e-4:
                    assert idx[f, i, j] == oi[i, j], (f, i, j)
