"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step.

Every test feeds both sides the same seeded input (teacher forcing) and
compares element by element:
  * key selection: bit-exact (integer arithmetic after the edge maps; inputs
    are 8-bit quantised so the FP32 Sobel sums are exact);
  * matching: indices bit-exact wherever the oracle's distances are separated
    by more than TAU_SEP, otherwise the GPU set must be a valid top-K within
    TAU_SEP; distances within 2e-5 relative;
  * low-rank step: X^ within 2e-4 * ||Y||_F / sqrt(dK) RMS and 1e-3 max
    (FP32 one-sided Jacobi vs FP64 LAPACK);
  * aggregation and GAP: within 1e-5 relative / 1e-6 absolute.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402

TAU_SEP = 1e-4


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def scene(tag, F, H, W, quant=True, C=1):
    rng = synth.rng_for(tag)
    fr = synth.textured_frames(rng, F * C, H, W).reshape(F, C, H, W)
    return synth.quantize8(fr) if quant else fr


# ---------------------------------------------------------------------------
# GAP projection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("accelerate", [False, True])
@pytest.mark.parametrize("HW", [(37, 53), (64, 64)])
def test_gap_step_matches_oracle(accelerate, HW):
    H, W = HW
    rng = synth.rng_for("gap-gpu", H)
    T = 5
    A = (rng.random((T, H, W)) < 0.5).astype(np.float32)
    A[:, 0, :3] = 0.0
    y = rng.random((1, H, W)).astype(np.float32)
    v = rng.random((1, T, H, W)).astype(np.float32)
    yacc = rng.random((1, H, W)).astype(np.float32)
    ya = cuda(yacc)
    x = glr.gap_step(cuda(y), cuda(A), cuda(v), accelerate=accelerate, y_acc=ya if accelerate else None)
    torch.cuda.synchronize()
    xo, yo = O.gap_project(y[0], A, v[0], yacc[0] if accelerate else None)
    np.testing.assert_allclose(x.cpu().numpy()[0], xo, rtol=1e-5, atol=1e-6)
    if accelerate:
        np.testing.assert_allclose(ya.cpu().numpy()[0], yo, rtol=1e-5, atol=1e-6)
    x0 = glr.gap_step(cuda(y), cuda(A), None)
    np.testing.assert_allclose(x0.cpu().numpy()[0], O.gap_init(y[0], A), rtol=1e-6, atol=1e-7)


def test_gap_step_per_group_masks_and_alias():
    rng = synth.rng_for("gap-groups")
    G, T, H, W = 3, 4, 16, 20
    A = rng.random((G, T, H, W)).astype(np.float32)
    y = rng.random((G, H, W)).astype(np.float32)
    v = rng.random((G, T, H, W)).astype(np.float32)
    vt = cuda(v)
    glr.gap_step(cuda(y), cuda(A), vt, out=vt)  # in place
    torch.cuda.synchronize()
    for g in range(G):
        xo, _ = O.gap_project(y[g], A[g], v[g])
        np.testing.assert_allclose(vt.cpu().numpy()[g], xo, rtol=1e-5, atol=1e-6)


# ---------------------------------------------------------------------------
# Key selection (bit-exact)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize(
    "case",
    [
        ("scene", 3, 1, 96, 130, 8, 200),  # several Harris tiles, ragged edge
        ("scene-many", 2, 1, 64, 64, 8, 1200),  # N above the number of corners -> grid fill
        ("scene-P5", 2, 1, 70, 45, 5, 60),
        ("msfa", 2, 3, 48, 40, 6, 80),  # multi-channel edge maps OR-ed over channels
    ],
)
def test_select_keys_bit_exact(case):
    tag, F, C, H, W, P, N = case
    x = scene(tag, F, H, W, C=C)
    keys, nf, nc = glr.select_keys(cuda(x), P, N, 0.1)
    torch.cuda.synchronize()
    keys, nf, nc = keys.cpu().numpy(), nf.cpu().numpy(), nc.cpu().numpy()
    for f in range(F):
        ok, onc = O.select_keys(x[f], P, N, 0.1)
        assert nf[f] == N
        assert nc[f] == onc
        np.testing.assert_array_equal(keys[f], ok)


def test_select_keys_flat_and_rectangles():
    H, W, P = 40, 44, 8
    flat = np.full((1, 1, H, W), 0.25, np.float32)
    rect = np.zeros((1, 1, H, W), np.float32)
    rect[0, 0, 1:12, 1:12] = 1.0  # corners that clamp onto the same patches
    rect[0, 0, 20:39, 25:43] = 0.5
    for x, N in ((flat, 17), (rect, 30), (rect, 3)):
        keys, nf, nc = glr.select_keys(cuda(x), P, N, 0.1)
        ok, onc = O.select_keys(x[0], P, N, 0.1)
        assert int(nc.cpu()[0]) == onc
        np.testing.assert_array_equal(keys.cpu().numpy()[0], ok)


def test_select_keys_single_position():
    """Degenerate size: the image is exactly one patch (Hq = Wq = 1)."""
    x = scene("one", 1, 8, 8)
    keys, nf, nc = glr.select_keys(cuda(x), 8, 1, 0.1)
    assert keys.cpu().numpy().tolist() == [[0]]


# ---------------------------------------------------------------------------
# Matching
# ---------------------------------------------------------------------------
def check_topk(x, P, keys, K, idx_gpu, dist_gpu, n_found=None, tau=TAU_SEP):
    F = x.shape[0]
    nbad_sep = 0
    for f in range(F):
        Q = O.patch_matrix(x[f], P)
        nf = keys.shape[1] if n_found is None else n_found[f]
        for i in range(nf):
            d_all = O.all_distances(x[f], P, keys[f, i], Q)
            order = np.lexsort((np.arange(len(d_all)), d_all))
            ds = d_all[order]
            g_idx = idx_gpu[f, i]
            # distances reported are the exact ones of the reported ids
            np.testing.assert_allclose(dist_gpu[f, i], d_all[g_idx], rtol=2e-5, atol=2e-6)
            # ranks: GPU distances are a valid sorted top-K within tau
            assert np.all(np.diff(dist_gpu[f, i]) >= -tau)
            assert np.all(d_all[g_idx] <= ds[K - 1] + tau)
            assert len(set(g_idx.tolist())) == K
            # bit-exact where separated
            for j in range(K):
                lo = ds[j] - ds[j - 1] if j > 0 else np.inf
                hi = ds[j + 1] - ds[j] if j + 1 < len(ds) else np.inf
                if lo > tau and hi > tau:
                    if g_idx[j] != order[j]:
                        nbad_sep += 1
    assert nbad_sep == 0


@pytest.mark.parametrize(
    "case",
    [
        ("m1", 2, 1, 60, 150, 8, 130, 40),  # 2 key tiles (ragged), 2 column tiles per row (ragged)
        ("m2", 1, 1, 37, 41, 4, 50, 9),
        ("m3", 2, 2, 30, 33, 5, 20, 12),  # multi-channel
        ("m4", 1, 1, 24, 26, 3, 300, 128),  # K at its maximum
    ],
)
@pytest.mark.parametrize("splits", [0, 3])
def test_match_fp32_parity(case, splits):
    tag, F, C, H, W, P, N, K = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "keys")
    npos = (H - P + 1) * (W - P + 1)
    keys = np.stack([rng.choice(npos, size=N, replace=False) for _ in range(F)]).astype(np.int32)
    nf = np.full(F, N, np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(nf, torch.int32), K, "fp32", splits=splits)
    torch.cuda.synchronize()
    check_topk(x, P, keys, K, idx.cpu().numpy(), dist.cpu().numpy())


def test_match_planted_copies_and_constant():
    H, W, P, K = 40, 50, 8, 6
    rng = synth.rng_for("planted-gpu")
    x = rng.random((2, 1, H, W)).astype(np.float32)
    Wq = W - P + 1
    src = (5, 7)
    spots = [(20, 3), (0, 30), (31, 40)]
    for r, c in spots:
        x[0, 0, r : r + P, c : c + P] = x[0, 0, src[0] : src[0] + P, src[1] : src[1] + P]
    x[1] = 0.5  # constant image: every distance is 0, ties by id
    keys = np.array([[src[0] * Wq + src[1]], [77]], np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([1, 1], np.int32), torch.int32), K)
    idx = idx.cpu().numpy()
    want = sorted([src[0] * Wq + src[1]] + [r * Wq + c for r, c in spots])
    assert idx[0, 0, :4].tolist() == want
    assert np.all(dist.cpu().numpy()[0, 0, :4] == 0)
    assert idx[1, 0].tolist() == list(range(K))


def test_match_n_found_masks_rows():
    x = scene("nf", 2, 30, 30, quant=False)
    P, N, K = 6, 20, 5
    keys = np.tile(np.arange(N, dtype=np.int32) * 7, (2, 1))
    nf = np.array([20, 9], np.int32)
    idx = torch.full((2, N, K), -7, dtype=torch.int32, device="cuda")
    glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(nf, torch.int32), K, idx=idx)
    idx = idx.cpu().numpy()
    assert np.all(idx[1, 9:] == -7) and np.all(idx[1, :9] >= 0) and np.all(idx[0] >= 0)


# ---------------------------------------------------------------------------
# Low-rank step (teacher-forced idx)
# ---------------------------------------------------------------------------
def resolvable_rank(Yg, sw, cw):
    """Oracle rank counted over the components an FP32 SVD resolves: s_i above the
    numerical-rank tolerance max(rows, K) 2^-24 s_1 (reading A15: FP32 arithmetic)."""
    _, _, s, s_new = O.wnnm(Yg, sw, cw, eps=1e-8)
    tol = max(Yg.shape) * 2.0 ** -24 * s[0]
    return int(np.count_nonzero((s_new > 0) & (s > tol)))


@pytest.mark.parametrize("case", [("l1", 2, 1, 40, 44, 8, 30, 40, 0.3), ("l2", 1, 1, 30, 30, 8, 20, 64, 0.1),
                                  ("l3", 1, 1, 25, 27, 4, 15, 7, 0.05), ("l4", 1, 1, 30, 30, 8, 10, 64, 0.0),
                                  ("l5", 1, 1, 30, 30, 4, 10, 40, 0.0)])
def test_lowrank_parity(case):
    tag, F, C, H, W, P, N, K, sw = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    nf = np.full(F, N, np.int32)
    cw = 2 * math.sqrt(K)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(nf, torch.int32), sw, cw)
    torch.cuda.synchronize()
    g = groups.cpu().numpy()
    rk = rank.cpu().numpy()
    d = C * P * P
    for f in range(F):
        Y = O.gather_groups(x[f], P, idx[f])
        Xo, _ = O.lowrank_groups(Y, sw, cw, eps=1e-8)
        ro = [resolvable_rank(Y[i].T, sw, cw) for i in range(N)]
        for i in range(N):
            scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
            err = g[f, i] - Xo[i]
            assert np.sqrt(np.mean(err**2)) <= 2e-4 * max(scale, 1e-3), (f, i)
            assert np.abs(err).max() <= 1e-3 * max(np.abs(Y[i]).max(), 1e-3)
            assert abs(int(rk[f, i]) - int(ro[i])) <= 1


@pytest.mark.parametrize("case", [("f1", 2, 1, 40, 44, 8, 30, 40, 0.3), ("f2", 1, 1, 30, 30, 8, 20, 64, 0.1),
                                  ("f3", 1, 1, 25, 27, 4, 15, 7, 0.05), ("f4", 1, 1, 30, 30, 8, 10, 64, 0.0)])
def test_lowrank_fp64_fallback(case):
    """A sweep cap of 1 sends the groups the FP32 Jacobi cannot finish in one sweep to the FP64
    fallback (Gram matrix + two-sided Jacobi); its X^ is the oracle's to FP32 output rounding and
    its rank the oracle's over the components an FP64 Gram matrix resolves."""
    tag, F, C, H, W, P, N, K, sw = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    nf = np.full(F, N, np.int32)
    cw = 2 * math.sqrt(K)
    im = glr.images(F, C, H, W, P)
    ws = glr.workspace(glr.L.GLR_OP_LOWRANK, im, N, K)
    old = glr.debug_wnnm_sweep_cap(1)
    try:
        groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(nf, torch.int32), sw, cw, ws=ws)
        torch.cuda.synchronize()
        _, cnt = glr.poll_status(ws)
    finally:
        glr.debug_wnnm_sweep_cap(old)
    assert cnt[1] > 0  # groups sent to the fallback
    g = groups.cpu().numpy()
    rk = rank.cpu().numpy()
    d = C * P * P
    for f in range(F):
        Y = O.gather_groups(x[f], P, idx[f])
        Xo, _ = O.lowrank_groups(Y, sw, cw, eps=1e-8)
        for i in range(N):
            # FP64 arithmetic, FP32 output: 50x tighter than the FP32 Jacobi's bar
            scale = np.linalg.norm(Y[i]) / math.sqrt(d * K)
            err = g[f, i] - Xo[i]
            assert np.sqrt(np.mean(err**2)) <= 4e-6 * max(scale, 1e-3), (f, i)
            assert np.abs(err).max() <= 2e-5 * max(np.abs(Y[i]).max(), 1e-3)
            _, _, sv, s_new = O.wnnm(Y[i].T, sw, cw, eps=1e-8)
            tol = math.sqrt(2 * max(d, K) * 2.0 ** -52) * sv[0]
            ro = int(np.count_nonzero((s_new > 0) & (sv > tol)))
            assert abs(int(rk[f, i]) - ro) <= 1, (f, i, int(rk[f, i]), ro)


def test_lowrank_noiseless_low_rank_recovery():
    """Groups of exactly rank 2 are returned unchanged (up to FP32) for a tiny sigma_w."""
    H, W, P, K = 20, 20, 8, 32
    rr = np.arange(H)[:, None] / H
    cc = np.arange(W)[None, :] / W
    x = (0.3 + 0.2 * rr + 0.1 * cc + 0.05 * rr * cc).astype(np.float32)[None, None]
    rng = synth.rng_for("lr-rec")
    idx = rng.integers(0, (H - P + 1) ** 2, size=(1, 5, K)).astype(np.int32)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(np.array([5], np.int32), torch.int32), 1e-5, 2 * math.sqrt(K))
    Y = O.gather_groups(x[0], P, idx[0])
    g = groups.cpu().numpy()[0]
    assert np.linalg.norm(g - Y) / np.linalg.norm(Y) < 1e-5


# ---------------------------------------------------------------------------
# Aggregation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", [("a1", 2, 1, 33, 47, 8, 25, 10), ("a2", 1, 3, 20, 21, 4, 12, 6),
                                  # K > 128 (rows past the preloaded ones), one warp per row (d > 128),
                                  # a patch side without a compiled specialisation
                                  ("a3", 1, 1, 40, 44, 6, 9, 160), ("a4", 1, 4, 30, 30, 6, 7, 20),
                                  ("a5", 1, 2, 25, 27, 5, 8, 10)])
def test_aggregate_parity(case):
    tag, F, C, H, W, P, N, K = case
    rng = synth.rng_for(tag)
    x = rng.random((F, C, H, W)).astype(np.float32)
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    g = rng.random((F, N, K, C * P * P)).astype(np.float32)
    nf = np.full(F, N, np.int32)
    v = glr.aggregate(cuda(g), cuda(idx, torch.int32), cuda(nf, torch.int32), cuda(x), P)
    torch.cuda.synchronize()
    for f in range(F):
        vo = O.aggregate(g[f], idx[f], x[f], P)
        np.testing.assert_allclose(v.cpu().numpy()[f], vo, rtol=1e-5, atol=1e-6)


# ---------------------------------------------------------------------------
# Device status, workspace errors
# ---------------------------------------------------------------------------
def test_nonfinite_input_is_flagged():
    x = scene("nan", 1, 24, 24, quant=False)
    x[0, 0, 3, 3] = np.nan
    idx = np.zeros((1, 2, 8), np.int32)
    ws = glr.workspace(glr.L.GLR_OP_LOWRANK, glr.images(1, 1, 24, 24, 8))
    glr.lowrank_groups(cuda(x), 8, cuda(idx, torch.int32), cuda(np.array([2], np.int32), torch.int32), 0.1, 4.0, ws=ws)
    bits, cnt = glr.poll_status(ws)
    assert bits & glr.L.GLR_DEV_NONFINITE


def test_workspace_too_small():
    x = cuda(scene("ws", 1, 32, 32))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(glr.GlrError) as e:
        glr.select_keys(x, 8, 10, ws=ws)
    assert e.value.code == glr.L.GLR_ENOMEM


# ---------------------------------------------------------------------------
# Fused grouping + WNNM + aggregation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", [("fz1", 2, 1, 60, 70, 8, 50, 40, 0.2), ("fz2", 1, 3, 33, 40, 4, 30, 24, 0.05),
                                  ("fz3", 1, 1, 40, 40, 8, 20, 64, 0.0)])
def test_fused_lowrank_aggregate_equals_separate_steps_bitwise(case):
    tag, F, C, H, W, P, N, K, sw = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    nf = np.full(F, N, np.int32)
    nf[0] = N - 3  # rows beyond n_found take no part
    cw = 2 * math.sqrt(K)
    xt, it, nt = cuda(x), cuda(idx, torch.int32), cuda(nf, torch.int32)
    groups, rank = glr.lowrank_groups(xt, P, it, nt, sw, cw)
    want = glr.aggregate(groups, it, nt, xt, P)
    rk = torch.empty_like(rank)
    got = glr.lowrank_aggregate(xt, P, it, nt, sw, cw, rank=rk)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    assert torch.equal(rk[0, :N - 3], rank[0, :N - 3])


@pytest.mark.parametrize("case", [("fo1", 2, 1, 60, 70, 8, 50, 40, 0.2), ("fo2", 1, 3, 33, 40, 4, 30, 24, 0.05)])
def test_fused_lowrank_aggregate_matches_oracle(case):
    """The fused pass against the oracle's own steps (gather, WNNM, aggregate) on the same idx:
    a fault shared by the fused and the separate kernels would not show in the bitwise test
    above.  Each output pixel averages WNNM estimates, so it stays within the low-rank bar."""
    tag, F, C, H, W, P, N, K, sw = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    nf = np.full(F, N, np.int32)
    nf[-1] = N - 5
    cw = 2 * math.sqrt(K)
    got = glr.lowrank_aggregate(cuda(x), P, cuda(idx, torch.int32), cuda(nf, torch.int32), sw, cw)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    for f in range(F):
        Y = O.gather_groups(x[f], P, idx[f, : nf[f]])
        Xo, _ = O.lowrank_groups(Y, sw, cw, eps=1e-8)
        vo = O.aggregate(Xo, idx[f, : nf[f]], x[f], P)
        err = got[f] - vo
        assert np.sqrt(np.mean(err**2)) <= 2e-4 * max(np.sqrt(np.mean(x[f] ** 2)), 1e-3)
        assert np.abs(err).max() <= 1e-3 * max(np.abs(x[f]).max(), 1e-3)


@pytest.mark.parametrize("case", [("s1", 2, 1, 40, 44, 8, 30, 40, 0.3), ("s2", 1, 1, 30, 30, 8, 20, 64, 0.1),
                                  ("s3", 1, 1, 25, 27, 4, 15, 7, 0.05), ("s4", 1, 1, 30, 30, 8, 10, 64, 0.0),
                                  ("s5", 1, 1, 30, 30, 4, 10, 40, 0.0)])
def test_lowrank_singular_values_and_estimate_tight_bar(case):
    """The FP32 one-sided Jacobi at the bar it meets.  It stops when every normalised inner
    product is below tol = 1e-5, so each computed singular value is within about tol s_1 of the
    exact one, and FP32 rounding of d-long sums adds ~d 2^-24 s_1; the shrinkage
    s' = s - C sw^2 / sqrt(s^2 - K sw^2) amplifies an error in s by 1 + C sw^2 s / s_hat^3, at most
    about 2.5 where s_hat >= s / 2.  Bar (the survey's 1e-5): the singular values of the
    returned X^ (by an FP64 SVD) within 1e-5 s_1 of the oracle's s' wherever s_hat >= s / 2 and
    s' > 0, and every entry of X^ within 1e-5 s_1 of the oracle's.  Measured worst over these
    cases: 3.7e-6 s_1 (singular values) and 1.9e-6 s_1 (entries), both at sigma_w = 0, K = 64."""
    tag, F, C, H, W, P, N, K, sw = case
    x = scene(tag, F, H, W, quant=False, C=C)
    rng = synth.rng_for(tag + "idx")
    npos = (H - P + 1) * (W - P + 1)
    idx = rng.integers(0, npos, size=(F, N, K)).astype(np.int32)
    nf = np.full(F, N, np.int32)
    cw = 2 * math.sqrt(K)
    groups, _ = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(nf, torch.int32), sw, cw)
    torch.cuda.synchronize()
    g = groups.cpu().numpy().astype(np.float64)
    worst_s = worst_x = 0.0
    for f in range(F):
        Y = O.gather_groups(x[f], P, idx[f])
        for i in range(N):
            Xo, _, s, s_new = O.wnnm(Y[i].T, sw, cw, eps=1e-8)
            s1 = s[0]
            sg = np.linalg.svd(g[f, i].T, compute_uv=False)
            s_hat = np.sqrt(np.maximum(s * s - K * sw * sw, 0.0))
            good = (s_new > 0) & (s_hat >= 0.5 * s)
            n = min(len(sg), len(s_new))
            ds = np.abs(sg[:n] - s_new[:n])[good[:n]]
            worst_s = max(worst_s, float(ds.max() / s1) if ds.size else 0.0)
            worst_x = max(worst_x, float(np.abs(g[f, i].T - Xo).max() / s1))
    print(f"worst singular-value error {worst_s:.2e} s_1, worst entry error {worst_x:.2e} s_1")
    assert worst_s <= 1e-5, worst_s
    assert worst_x <= 1e-5, worst_x


@pytest.mark.parametrize("kind", ["one", "spread", "two"])
def test_lowrank_rank1_certificate(kind):
    """Groups of near copies of one 8 x 8 pattern plus noise at sigma_w = 0.1, where
    s_crit^2 = sw^2 (K + sqrt(K^2 + 4 C^2)) / 2 = 0.678.
    one: noise std 0.01, residual energy ~63 x 64 x 1e-4 = 0.40 below s_crit^2, so the energy
    bound settles every group (status counter 7) without sweeps.
    spread: noise std 0.02, residual energy ~1.6 above s_crit^2, but spread over 63 components:
    ||R^T R||_F ~ sqrt(2 x 63) x 64 x 4e-4 = 0.29 is below it, so the Gram bound settles every
    group (counter 9) without sweeps.
    two: two patterns per group, s_2 far above s_crit: no group is certified, the sweeps run.
    In every case X^ must equal the oracle's within 1e-5 s_1 and the rank the oracle's."""
    rng = np.random.default_rng(21)
    H = W = 8 * 12
    pa = rng.random((8, 8))
    pb = rng.random((8, 8))
    base = np.tile(pa, (12, 12))
    if kind == "two":
        base[:, 48:] = np.tile(pb, (12, 6))
    noise = 0.02 if kind == "spread" else 0.01
    x = (base + noise * rng.standard_normal((H, W))).astype(np.float32)[None, None]
    P, K, N = 8, 64, 40
    Wq = W - P + 1
    grid = [r * Wq + c for r in range(0, 89, 8) for c in range(0, 89, 8)]  # 12 x 12 aligned positions
    idx = np.stack([rng.choice(grid, size=K, replace=False) for _ in range(N)]).astype(np.int32)[None]
    sw, cw = 0.1, 2 * math.sqrt(K)
    im = glr.images(1, 1, H, W, P)
    ws = glr.workspace(glr.L.GLR_OP_LOWRANK, im, N, K)
    groups, rank = glr.lowrank_groups(cuda(x), P, cuda(idx, torch.int32), cuda(np.array([N], np.int32), torch.int32),
                                      sw, cw, ws=ws)
    torch.cuda.synchronize()
    _, cnt = glr.poll_status(ws)
    g = groups.cpu().numpy()[0].astype(np.float64)
    rk = rank.cpu().numpy()[0]
    Y = O.gather_groups(x[0], P, idx[0])
    scrit2 = sw * sw * (K + math.sqrt(K * K + 4 * cw * cw)) / 2
    for i in range(N):
        Xo, ro, s, _ = O.wnnm(Y[i].T, sw, cw, eps=1e-8)
        assert np.abs(g[i].T - Xo).max() <= 1e-5 * s[0], i
        assert int(rk[i]) == ro, (i, int(rk[i]), ro)
        if kind == "spread":  # the case is what it claims: energy above s_crit^2, Gram bound below
            s2 = s[1:] ** 2
            assert s2.sum() > scrit2 and math.sqrt((s2 ** 2).sum()) < scrit2
    if kind == "two":
        assert cnt[7] < N and cnt[2] > 0  # the mixed groups needed sweeps
    elif kind == "one":
        assert cnt[7] == N and cnt[9] == 0 and cnt[2] == 0, cnt  # the energy bound settled every group
    else:
        assert cnt[7] == N and cnt[9] == N and cnt[10] == N and cnt[2] == 0, cnt  # the Gram bound did
