"""MRI (ADMM) path through the C ABI against the FP64 oracle.

* glr_fft2: the orthonormal unshifted DFT within 2e-6 of the largest output
  magnitude (FP32 radix-2 error grows like log2(n) * 2^-24).
* glr_admm_step: u, x', w and the FP64 residual against the oracle's
  data-consistency update on the same inputs.
* glr_lowrank_groups_complex: complex WNNM of teacher-forced groups within the
  real path's bar (RMS 2e-4 ||Y||_F / sqrt(dK), max 1e-3 max|Y|, rank within 1).
* the real paths for d > 64 or K > 64 under the same bar: the shared-memory
  one-sided Jacobi and, for tall groups (d >= 2K, K <= 32), the Gram matrix with
  a two-sided Jacobi eigensolver.
* BF16 tensor-core matching of complex 6 x 6 patches (d = 72, values spill
  into the second operand tile): raw scores vs the host BF16 computation, and
  recall after the exact re-rank.
* one MRI reconstruction step teacher-forced against the oracle, and CUDA-graph
  replay equal to eager execution.
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


def cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def planes(z):
    return np.stack([z.real, z.imag]).astype(np.float32)


@pytest.mark.parametrize("HW", [(8, 16), (64, 128), (1024, 1024), (2, 4096)])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2_matches_oracle(HW, inverse):
    H, W = HW
    rng = synth.rng_for("fft-gpu", H * 7 + W)
    n = 2 if H * W <= 8192 else 1
    z = cplx(rng, n, H, W)
    xin = np.stack([planes(z[i]) for i in range(n)])
    out = glr.fft2(cuda(xin), inverse=inverse)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for i in range(n):
        zi = xin[i, 0].astype(np.float64) + 1j * xin[i, 1]
        want = MO.ifft2c(zi) if inverse else MO.fft2c(zi)
        g = got[i, 0] + 1j * got[i, 1]
        assert np.abs(g - want).max() <= 2e-6 * np.abs(want).max() * math.log2(max(H, W)), np.abs(g - want).max()


def test_fft2_in_place_and_round_trip():
    rng = synth.rng_for("fft-rt")
    z = planes(cplx(rng, 32, 64))[None]
    t = cuda(z)
    glr.fft2(t, out=t)
    glr.fft2(t, inverse=True, out=t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t.cpu().numpy(), z, atol=5e-6 * np.abs(z).max())


@pytest.mark.parametrize("HW", [(16, 32), (256, 128)])
def test_admm_step_matches_oracle(HW):
    H, W = HW
    rng = synth.rng_for("admm", H)
    n, rho = 2, 0.7
    mask = (rng.random((n, H, W)) < 0.3).astype(np.float32)
    y = np.stack([planes(mask[i] * cplx(rng, H, W)) for i in range(n)])
    z = np.stack([planes(cplx(rng, H, W)) for _ in range(n)])
    x = np.stack([planes(cplx(rng, H, W)) for _ in range(n)])
    u = np.stack([planes(cplx(rng, H, W)) for _ in range(n)])
    ut = cuda(u)
    xo, wo, res = glr.admm_step(cuda(y), cuda(mask), cuda(z), cuda(x), ut, rho)
    torch.cuda.synchronize()
    c = lambda p: p[0].astype(np.float64) + 1j * p[1]
    for i in range(n):
        u_new = c(u[i]) + c(x[i]) - c(z[i])
        x_new = MO.admm_dc(c(y[i]), mask[i], c(z[i]) - u_new, rho)
        scale = np.abs(x_new).max()
        np.testing.assert_allclose(ut.cpu().numpy()[i], planes(u_new), atol=1e-5 * np.abs(u_new).max())
        got = xo.cpu().numpy()[i]
        assert np.abs(c(got) - x_new).max() <= 2e-5 * scale
        assert np.abs(c(wo.cpu().numpy()[i]) - (x_new + u_new)).max() <= 2e-5 * np.abs(x_new + u_new).max()
        want_res = MO.dc_residual(x_new, c(y[i]), mask[i])
        assert abs(float(res[i]) - want_res) <= 1e-5 * want_res


def test_admm_step_rejects_bad_aliasing_and_sizes():
    z = torch.zeros((1, 2, 16, 16), device="cuda")
    m = torch.ones((1, 16, 16), device="cuda")
    with pytest.raises(glr.GlrError):
        glr.admm_step(z, m, z.clone(), z.clone(), z.clone(), 0.5, w_out=None, x_out=z)  # x_out aliases y
    bad = torch.zeros((1, 2, 12, 16), device="cuda")
    with pytest.raises(glr.GlrError):
        glr.fft2(bad)
    with pytest.raises(glr.GlrError):
        glr.admm_step(z, m, z.clone(), z.clone(), z.clone(), 0.0)


def resolvable_rank(Yg, sw, cw, fn):
    """Oracle rank over the components an FP32 SVD resolves (s_i above max(rows, K) 2^-24 s_1)."""
    _, _, s, s_new = fn(Yg, sw, cw, 1e-8)
    tol = max(Yg.shape) * 2.0 ** -24 * s[0]
    return int(np.count_nonzero((s_new > 0) & (s > tol)))


def sv_entry_errors(Mg, Mo, s, s_new, sw, K):
    """(worst singular-value error, worst entry error), both over s_1: the singular values of the
    returned group Mg (FP64 SVD) against the oracle's shrunk values where the shrinkage is well
    conditioned (s_hat >= s / 2), and the entries of Mg against the oracle's estimate Mo."""
    sg = np.linalg.svd(Mg, compute_uv=False)
    s_hat = np.sqrt(np.maximum(s * s - K * sw * sw, 0.0))
    good = (s_new > 0) & (s_hat >= 0.5 * s)
    n = min(len(sg), len(s_new))
    ds = np.abs(sg[:n] - s_new[:n])[good[:n]]
    return (float(ds.max()) if ds.size else 0.0) / s[0], float(np.abs(Mg - Mo).max()) / s[0]


def complex_image(tag, H, W):
    return synth.complex_phantom(synth.rng_for(tag), H, W)


@pytest.mark.parametrize("case", [("c1", 40, 44, 6, 30, 48, 0.05), ("c2", 30, 30, 6, 20, 23, 0.2),
                                  ("c3", 30, 30, 6, 10, 48, 0.0), ("c4", 28, 30, 4, 25, 64, 0.02),
                                  ("c5", 36, 36, 6, 12, 96, 0.03)])
def test_lowrank_complex_parity(case):
    tag, H, W, P, N, K, sw = case
    x = complex_image(tag, H, W)[None]
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(1, N, K)).astype(np.int32)
    cw = 2 * math.sqrt(K)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(np.array([N], np.int32), torch.int32),
                                      sw, cw, complex_=True)
    torch.cuda.synchronize()
    g = groups.cpu().numpy()[0]
    rk = rank.cpu().numpy()[0]
    Y = O.gather_groups(x[0], P, idx[0])
    Xo, _ = MO.lowrank_groups_complex(Y, sw, cw, eps=1e-8)
    ro = [resolvable_rank(MO.group_to_complex(Y[i]), sw, cw, MO.wnnm_complex) for i in range(N)]
    d = 2 * P * P
    worst = [0.0, 0.0]
    for i in range(N):
        scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
        err = g[i] - Xo[i]
        assert np.sqrt(np.mean(err ** 2)) <= 2e-4 * max(scale, 1e-3), i
        assert np.abs(err).max() <= 1e-3 * max(np.abs(Y[i]).max(), 1e-3), i
        assert abs(int(rk[i]) - int(ro[i])) <= 1
        _, _, sv, s_new = MO.wnnm_complex(MO.group_to_complex(Y[i]), sw, cw, 1e-8)
        e = sv_entry_errors(MO.group_to_complex(g[i].astype(np.float64)), MO.group_to_complex(Xo[i]), sv, s_new, sw, K)
        worst = [max(worst[0], e[0]), max(worst[1], e[1])]
    print(f"complex {tag}: worst singular-value error {worst[0]:.2e} s_1, worst entry error {worst[1]:.2e} s_1")
    assert max(worst) <= 1e-5, worst  # the survey's bar (measured worst 6.7e-6, Gram path entries)


@pytest.mark.parametrize("case", [("w1", 1, 4, 30, 32, 6, 20, 32, 0.1), ("w2", 1, 1, 30, 30, 8, 12, 96, 0.05),
                                  ("w3", 1, 16, 24, 24, 6, 8, 32, 0.2), ("w4", 1, 2, 24, 24, 6, 8, 17, 0.0),
                                  ("w5", 1, 16, 24, 24, 6, 8, 32, 0.0), ("w6", 1, 16, 30, 30, 6, 12, 32, 0.02),
                                  ("w7", 1, 3, 30, 30, 6, 12, 40, 0.05)])
def test_lowrank_wide_real_parity(case):
    tag, F, C, H, W, P, N, K, sw = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, F * C, H, W).reshape(F, C, H, W)
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    cw = 2 * math.sqrt(K)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(np.full(F, N, np.int32), torch.int32),
                                      sw, cw)
    torch.cuda.synchronize()
    g = groups.cpu().numpy()[0]
    rk = rank.cpu().numpy()[0]
    Y = O.gather_groups(x[0], P, idx[0])
    Xo, _ = O.lowrank_groups(Y, sw, cw, eps=1e-8)
    d = C * P * P
    worst = [0.0, 0.0]
    for i in range(N):
        scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
        err = g[i] - Xo[i]
        assert np.sqrt(np.mean(err ** 2)) <= 2e-4 * max(scale, 1e-3), i
        assert np.abs(err).max() <= 1e-3 * max(np.abs(Y[i]).max(), 1e-3), i
        # rank: components the FP32 path cannot resolve may be counted or not.  The
        # one-sided Jacobi resolves s_i down to max(d, K) 2^-24 s_1; the Gram path
        # (tall groups) works on s_i^2 and resolves down to sqrt(max(d, K) 2^-24) s_1.
        _, _, sv, s_new = O.wnnm(Y[i].T, sw, cw, 1e-8)
        tol_hi = math.sqrt(max(d, K) * 2.0 ** -24) * sv[0]
        lo = int(np.count_nonzero((s_new > 0) & (sv > tol_hi)))
        hi = int(np.count_nonzero(s_new > 0))
        assert lo - 1 <= int(rk[i]) <= hi + 1, (i, int(rk[i]), lo, hi)
        e = sv_entry_errors(g[i].T.astype(np.float64), Xo[i].T, sv, s_new, sw, K)
        worst = [max(worst[0], e[0]), max(worst[1], e[1])]
    print(f"wide {tag} (d {d}, K {K}): worst singular-value error {worst[0]:.2e} s_1, worst entry error {worst[1]:.2e} s_1")
    assert max(worst) <= 1e-5, worst  # the survey's bar (measured worst 6.7e-6, Gram path entries)


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("case", [("m1", 2, 6, 40, 300, 100), ("m2", 2, 5, 30, 40, 20)])
def test_tc_raw_scores_two_channels(case):
    """d = 72 (2 x 6 x 6) and d = 50: patch values beyond 64 sit in the 16-column tile."""
    tag, C, P, H, W, N = case
    rng = synth.rng_for(tag)
    x = complex_image(tag, H, W)[None]
    npos = (H - P + 1) * (W - P + 1)
    keys = rng.choice(npos, size=(1, N), replace=False).astype(np.int32)
    sc = glr.debug_match_scores(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([N], np.int32), torch.int32), 8)
    torch.cuda.synchronize()
    sc = sc.cpu().numpy()
    ncol = min(256, npos)
    mu = np.float32(np.float64(x[0]).mean())
    Q = bf16(O.patch_matrix((x[0] - mu).astype(np.float32), P))
    for i in range(N):
        p = Q[keys[0, i]]
        want = ((Q[:ncol] - p) ** 2).sum(1)
        scale = (p * p).sum() + (Q[:ncol] ** 2).sum(1)
        err = np.abs(sc[0, i, :ncol] - want)
        assert np.all(err <= 2e-6 * scale + 1e-6), (i, err.max())


@pytest.mark.parametrize("splits", [0, 2])
def test_match_bf16_complex_recall(splits):
    H, W, P, N, K = 60, 200, 6, 80, 48
    x = complex_image("mr", H, W)[None]
    rng = synth.rng_for("mrk")
    npos = (H - P + 1) * (W - P + 1)
    keys = rng.choice(npos, size=(1, N), replace=False).astype(np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([N], np.int32), torch.int32), K,
                               "bf16", splits=splits)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    Q = O.patch_matrix(x[0], P)
    hits = 0
    for i in range(N):
        d_all = O.all_distances(x[0], P, keys[0, i], Q)
        np.testing.assert_allclose(dist[0, i], d_all[idx[0, i]], rtol=2e-5, atol=2e-6)
        order = np.lexsort((np.arange(len(d_all)), d_all))[:K]
        hits += len(set(order.tolist()) & set(idx[0, i].tolist()))
    assert hits / (N * K) >= 0.99


def _mri(H=64, W=64, N=60, K=16, iters=2):
    cfg = synth.mri_scaled(synth.MRI_SMALL, H=H, W=W, N=N, K=K, iters=iters, centre_lines=8)
    p = synth.mri_problem(cfg)
    return cfg, p


def test_mri_step_tracks_oracle_teacher_forced():
    cfg, p = _mri()
    rec = glr.MriReconstructor(cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="fp32", rho=cfg.rho)
    rec.start(cuda(p.y), cuda(p.mask))
    y = MO.planes_to_complex(p.y)
    x0 = rec.x.cpu().numpy()[0]
    np.testing.assert_allclose(MO.planes_to_complex(x0), MO.ifft2c(y), atol=2e-5 * np.abs(y).max())
    for s in cfg.sigma_schedule():
        # quantise the denoiser input so both sides take the same edge decisions
        rec.w.copy_(torch.round(rec.w * 256.0) / 256.0)
        w = rec.w.cpu().numpy()[0].astype(np.float64)
        x_prev = MO.planes_to_complex(rec.x.cpu().numpy()[0])
        u_prev = MO.planes_to_complex(rec.u.cpu().numpy()[0])
        rec.step(s, cfg.c_wnnm)
        torch.cuda.synchronize()
        z_gpu = rec.z.cpu().numpy()[0]
        z_or, _ = MO.mri_denoise(w, cfg.P, cfg.N, cfg.K, s, cfg.c_wnnm, cfg.edge_th, eps=1e-8)
        err = np.abs(z_gpu - z_or)
        assert np.sqrt(np.mean(err ** 2)) < 2e-4 and err.max() < 2e-3
        zc = MO.planes_to_complex(z_gpu)
        u_new = u_prev + x_prev - zc
        x_new = MO.admm_dc(y, p.mask, zc - u_new, cfg.rho)
        assert np.abs(MO.planes_to_complex(rec.x.cpu().numpy()[0]) - x_new).max() < 1e-4
        assert abs(float(rec.residual[0]) - MO.dc_residual(x_new, y, p.mask)) <= 1e-4 * MO.dc_residual(x_new, y, p.mask)


def test_mri_graph_replay_matches_eager():
    cfg, p = _mri(H=64, W=128, N=80, K=24, iters=3)
    a = glr.MriReconstructor(cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="bf16", rho=cfg.rho)
    b = glr.MriReconstructor(cfg.H, cfg.W, cfg.P, cfg.N, cfg.K, mode="bf16", rho=cfg.rho)
    sig = cfg.sigma_schedule()
    a.start(cuda(p.y), cuda(p.mask))
    b.start(cuda(p.y), cuda(p.mask))
    b.capture(sig, cfg.c_wnnm)
    for s in sig:
        a.step(s, cfg.c_wnnm)
        b.step_graph(s)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.x.cpu().numpy(), a.x.cpu().numpy(), rtol=1e-4, atol=1e-4)


def _fallback_run(x, P, idx, nf, sw, cw, complex_):
    im = glr.images(x.shape[0], x.shape[1], x.shape[2], x.shape[3], P)
    N, K = idx.shape[1], idx.shape[2]
    ws = glr.workspace(glr.L.GLR_OP_LOWRANK, im, N, K)
    old = glr.debug_wnnm_sweep_cap(1)
    try:
        groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(nf, torch.int32), sw, cw, ws=ws,
                                          complex_=complex_)
        torch.cuda.synchronize()
        _, cnt = glr.poll_status(ws)
    finally:
        glr.debug_wnnm_sweep_cap(old)
    return groups.cpu().numpy(), rank.cpu().numpy(), cnt


@pytest.mark.parametrize("case", [("fbw1", 16, 24, 26, 6, 8, 32, 0.05),   # tall groups: the Gram path (d 576, K 32)
                                  ("fbw2", 3, 24, 26, 6, 8, 40, 0.1),    # shared-memory path (d 108, K 40)
                                  ("fbw3", 2, 24, 24, 8, 6, 90, 0.02)])  # shared-memory path, K 90 (FP64 size 96)
def test_lowrank_fp64_fallback_wide_real(case):
    """A sweep cap of 1 sends the groups the FP32 Gram / shared-memory Jacobi cannot finish in one
    sweep to the FP64 fallback; its X^ is the oracle's to FP32 output rounding (the bar of the
    register path's fallback test)."""
    tag, C, H, W, P, N, K, sw = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, C, H, W).reshape(1, C, H, W)
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(1, N, K)).astype(np.int32)
    cw = 2 * math.sqrt(K)
    g, rk, cnt = _fallback_run(x, P, idx, np.array([N], np.int32), sw, cw, False)
    assert cnt[1] > 0
    Y = O.gather_groups(x[0], P, idx[0])
    Xo, ro = O.lowrank_groups(Y, sw, cw, eps=1e-8)
    d = C * P * P
    for i in range(N):
        scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
        err = g[0, i] - Xo[i]
        assert np.sqrt(np.mean(err**2)) <= 4e-6 * max(scale, 1e-3), i
        assert np.abs(err).max() <= 2e-5 * max(np.abs(Y[i]).max(), 1e-3), i
        assert abs(int(rk[0, i]) - int(ro[i])) <= 1


@pytest.mark.parametrize("case", [("fbc1", 30, 30, 6, 10, 24, 0.05),   # complex register path (FP64 size 48)
                                  ("fbc2", 30, 32, 6, 8, 48, 0.02),    # complex register path, K 48 (FP64 size 96)
                                  ("fbc3", 30, 30, 8, 6, 16, 0.05)])   # complex shared-memory path (d 128)
def test_lowrank_fp64_fallback_complex(case):
    """Complex groups at the sweep cap go to the FP64 fallback as the real 2m x 2K matrix
    [[A, -B], [B, A]]; its result is the oracle's complex WNNM to FP32 output rounding."""
    tag, H, W, P, N, K, sw = case
    x = complex_image(tag, H, W)[None]
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(1, N, K)).astype(np.int32)
    cw = 2 * math.sqrt(K)
    g, rk, cnt = _fallback_run(x, P, idx, np.array([N], np.int32), sw, cw, True)
    assert cnt[1] > 0
    Y = O.gather_groups(x[0], P, idx[0])
    Xo, ro = MO.lowrank_groups_complex(Y, sw, cw, eps=1e-8)
    d = 2 * P * P
    for i in range(N):
        scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
        err = g[0, i] - Xo[i]
        assert np.sqrt(np.mean(err**2)) <= 4e-6 * max(scale, 1e-3), i
        assert np.abs(err).max() <= 2e-5 * max(np.abs(Y[i]).max(), 1e-3), i
        assert abs(int(rk[0, i]) - int(ro[i])) <= 1
