"""Tensor-core matching with and without the minima scan.

The minima scan records, per key, the minimum BF16 score of every half tile
(128 positions); the K'-th smallest of those minima bounds the K'-th smallest
score of the key, and the candidate scan starts from that bound.  The bound
only removes candidates that cannot be among the K' smallest scores, so the
matches must not change: the reported distances are equal element by element
with the scan on and off, and the ids agree except among exactly tied
distances.  Cases: one and several position splits, a ragged last position
tile, several images, the chunked operand rows of wide patches (d > 74), and
the learned and heat-map proposals.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def run(x, P, keys, nf, K, mode, bound_pass, **kw):
    idx, dist = glr.match_topk(x, P, keys, nf, K, mode, bound_pass=bound_pass, **kw)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


def same_matches(a, b):
    (ia, da), (ib, db) = a, b
    np.testing.assert_array_equal(da, db)
    # ids: equal as sets within every run of equal distances
    for f in range(ia.shape[0]):
        for k in range(ia.shape[1]):
            if not np.array_equal(ia[f, k], ib[f, k]):
                for v in np.unique(da[f, k]):
                    sel = da[f, k] == v
                    assert set(ia[f, k][sel]) == set(ib[f, k][sel]), (f, k, v)


def frames(tag, F, C, H, W):
    rng = synth.rng_for(tag)
    x = np.stack([synth.textured_frames(rng, F, H, W) for _ in range(C)], axis=1).astype(np.float32)
    return torch.from_numpy(x).cuda()


@pytest.mark.parametrize("splits", [1, 2, 3])
def test_bound_pass_keeps_matches_narrow(splits):
    x = frames("bp_narrow", 2, 1, 200, 230)  # 193 x 223 positions: ragged last tile
    P, N, K = 8, 300, 40
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    on = run(x, P, keys, nf, K, "bf16", 1, splits=splits)
    off = run(x, P, keys, nf, K, "bf16", -1, splits=splits)
    same_matches(on, off)


def test_bound_pass_keeps_matches_two_channels():
    x = frames("bp_c2", 1, 2, 150, 170)
    P, N, K = 6, 256, 48
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    same_matches(run(x, P, keys, nf, K, "bf16", 1, k_over=64), run(x, P, keys, nf, K, "bf16", -1, k_over=64))


def test_bound_pass_keeps_matches_wide():
    x = frames("bp_wide", 2, 16, 96, 104)  # d = 16 x 36 = 576: chunked operand rows
    P, N, K = 6, 128, 32
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    same_matches(run(x, P, keys, nf, K, "bf16", 1), run(x, P, keys, nf, K, "bf16", -1))


def test_bound_pass_keeps_matches_edge_heatmap():
    x = frames("bp_edge", 1, 1, 140, 150)
    P, N, K = 8, 200, 32
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    same_matches(run(x, P, keys, nf, K, "edge", 1, edge_th=0.05), run(x, P, keys, nf, K, "edge", -1, edge_th=0.05))


def test_bound_pass_keeps_matches_learned():
    x = frames("bp_learned", 1, 1, 300, 300)  # K' = 256 needs at least 128 position tiles
    P, N, K = 8, 128, 32
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    enc = glr.Encoder(seed=3)
    kw = dict(encoder=enc.params)
    same_matches(run(x, P, keys, nf, K, "learned", 1, **kw), run(x, P, keys, nf, K, "learned", -1, **kw))


def test_stream_final_selection_and_rerank_selection_agree():
    """With few streams the re-rank takes the unreduced buffers and selects the K' best itself;
    with many (8 splits, capacity 512) every stream ends with its own exact K' selection.  The
    key's K' best (score, id) pairs are the same either way, so are the matches."""
    x = frames("bp_finish", 1, 1, 220, 240)
    P, N, K = 8, 256, 48
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    few = run(x, P, keys, nf, K, "bf16", 1, splits=1)
    many = run(x, P, keys, nf, K, "bf16", 1, splits=8, cap=512)
    same_matches(few, many)


@pytest.mark.parametrize("bound_pass", [-1, 1])
def test_stream_compactions_against_the_oracle(bound_pass):
    """A stream capacity of K' + 16 (the next multiple of 32) with three position splits makes the streams compact
    many times; keys on a flat half of the image tie exactly (every BF16 score and every exact
    distance there is equal), so compaction has to fall back from its sampled pivot to the exact
    radix select and keep the smaller ids.  Against the FP64 oracle: flat keys return exactly the
    oracle's K smallest ids among the tied positions, textured keys pass the BF16 separation
    check of the tensor-core tests."""
    from oracle import glr_oracle as O
    from test_gpu_tc import check_bf16_topk

    rng = synth.rng_for("compact")
    H, W, P, K, Kp = 100, 120, 8, 32, 48
    x = synth.textured_frames(rng, 1, H, W)[:, None].astype(np.float32)
    x[0, 0, : H // 2] = 0.5
    Wq = W - P + 1
    flat = [r * Wq + c for r in (3, 10, 20, 30) for c in (5, 50, 100)]
    textured = [r * Wq + c for r in (60, 70, 80, 90) for c in (7, 44, 81, 110)]
    keys = np.array([flat + textured], np.int32)
    N = keys.shape[1]
    kt = torch.from_numpy(keys).cuda()
    nf = torch.tensor([N], dtype=torch.int32, device="cuda")
    xt = torch.from_numpy(x).cuda()
    im = glr.images_of(xt, P)
    opts = glr.match_opts("bf16", k_over=Kp, splits=3, cap=Kp + 16, bound_pass=bound_pass)
    ws = glr.workspace(glr.L.GLR_OP_MATCH, im, N, K, opts)
    idx, dist = glr.match_topk(xt, P, kt, nf, K, "bf16", k_over=Kp, splits=3, cap=Kp + 16, bound_pass=bound_pass,
                               ws=ws)
    torch.cuda.synchronize()
    _, cnt = glr.poll_status(ws)
    assert cnt[5] > 0  # compactions happened
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    Q = O.patch_matrix(x[0], P)
    for i in range(len(flat)):
        d_all = O.all_distances(x[0], P, keys[0, i], Q)
        order = np.lexsort((np.arange(len(d_all)), d_all))
        assert d_all[order[K - 1]] == 0.0
        assert idx[0, i].tolist() == order[:K].tolist(), i
        assert np.all(dist[0, i] == 0.0)
    # every textured key is checked (exact ids where the BF16 bound separates, else distances
    # within the bound); the bound separates 9 of these 16 keys, computed from the oracle alone
    covered = check_bf16_topk(x, P, keys[:, len(flat):], K, Kp, idx[:, len(flat):], dist[:, len(flat):])
    assert covered >= 0.5, covered


def test_forced_wait_expiry_reports_timeout_and_recovers():
    """The scorer's pipeline waits given a 1 ns limit: the first wait that is not already
    satisfied expires, the call records GLR_DEV_TIMEOUT and glr_poll_status returns
    GLR_ETIMEDOUT; the CTAs still drain the copies and MMAs they issued.  With the default
    limit restored, the next call on the same workspace returns the same matches as a call on
    a fresh workspace."""
    import ctypes

    x = frames("timeout", 1, 1, 90, 100)
    P, N, K = 8, 128, 16
    keys, nf, _ = glr.select_keys(x, P, N, 0.05)
    im = glr.images_of(x, P)
    opts = glr.match_opts("bf16")
    ws = glr.workspace(glr.L.GLR_OP_MATCH, im, N, K, opts)
    lib = glr.L.load()
    old = glr.debug_match_wait_ns(1)
    try:
        glr.match_topk(x, P, keys, nf, K, "bf16", ws=ws)
        torch.cuda.synchronize()
    finally:
        glr.debug_match_wait_ns(old)
    bits = ctypes.c_uint32(0)
    code = lib.glr_poll_status(glr._ws(ws)[0], ctypes.byref(bits), None, 1, torch.cuda.current_stream().cuda_stream)
    assert code == glr.L.GLR_ETIMEDOUT and bits.value & glr.L.GLR_DEV_TIMEOUT
    again = run(x, P, keys, nf, K, "bf16", 0, ws=ws)
    code = lib.glr_poll_status(glr._ws(ws)[0], ctypes.byref(bits), None, 0, torch.cuda.current_stream().cuda_stream)
    assert code == glr.L.GLR_OK and bits.value == 0
    fresh = run(x, P, keys, nf, K, "bf16", 0)
    np.testing.assert_array_equal(again[0], fresh[0])
    np.testing.assert_array_equal(again[1], fresh[1])
