"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
worked by hand, invariants, special cases that reduce to a textbook result,
an independent library algorithm (k-d tree nearest neighbours), and brute
force on tiny inputs.  A dropped term, a flipped sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import glr_oracle as O
from paper_2301_03047_gb300 import synth

# ---------------------------------------------------------------------------
# Eq. 2 / Eq. 3: Sobel and binary edge maps
# ---------------------------------------------------------------------------


def test_sobel_ramp_closed_form():
    """A ramp x = a*c + b*r gives g_h = 8a, g_v = 8b inside; 4a / 4b on replicated borders."""
    a, b = 0.0625, -0.03125
    H, W = 9, 11
    r = np.arange(H)[:, None]
    c = np.arange(W)[None, :]
    img = a * c + b * r
    gh, gv = O.sobel(img)
    assert np.allclose(gh[:, 1:-1], 8 * a) and np.allclose(gh[:, 0], 4 * a) and np.allclose(gh[:, -1], 4 * a)
    assert np.allclose(gv[1:-1, :], 8 * b) and np.allclose(gv[0, :], 4 * b) and np.allclose(gv[-1, :], 4 * b)


def test_edge_maps_signs_reading_a1():
    """A rising step in x lights only h+, a falling one only h-, and likewise for v (reading A1)."""
    img = np.zeros((6, 8))
    img[:, 4:] = 1.0  # rising left->right
    m = O.edge_maps(img, 0.1)
    assert m["h+"][:, 3:5].all() and m["h+"].sum() == 12
    assert m["h-"].sum() == 0 and m["v+"].sum() == 0 and m["v-"].sum() == 0
    m2 = O.edge_maps(1.0 - img, 0.1)
    assert m2["h-"].sum() == 12 and m2["h+"].sum() == 0
    m3 = O.edge_maps(img.T.copy(), 0.1)  # rising top->bottom
    assert m3["v+"].sum() == 12 and m3["v-"].sum() == 0 and m3["h+"].sum() == 0


def test_threshold_is_strict():
    """Eq. 3: T(z) = 1 only for z > th; z == th gives 0."""
    z = np.array([0.09, 0.1, 0.11])
    assert list(O.threshold(z, 0.1)) == [0, 0, 1]


def test_golden_edge_fixture():
    """Hand-worked Sobel / edge maps of a 5x5 image (tests/golden/edges_5x5.txt)."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "edges_5x5.txt")
    blocks = {}
    cur = None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.endswith(":"):
            cur = line[:-1]
            blocks[cur] = []
        else:
            blocks[cur].append([float(t) for t in line.split()])
    img = np.array(blocks["image"])
    gh, gv = O.sobel(img)
    assert np.array_equal(gh, np.array(blocks["g_h"]))
    assert np.array_equal(gv, np.array(blocks["g_v"]))
    m = O.edge_maps(img, blocks["th"][0][0])
    for k in ("h+", "h-", "v+", "v-"):
        assert np.array_equal(m[k], np.array(blocks[k], dtype=np.uint8)), k
    assert np.array_equal(O.edge_sum(img[None], blocks["th"][0][0]), np.array(blocks["S"], dtype=np.int64))


def test_edge_sum_or_over_channels():
    img = np.zeros((2, 6, 8))
    img[0, :, 4:] = 1.0
    img[1, :, 4:] = 1.0
    s2 = O.edge_sum(img, 0.1)
    s1 = O.edge_sum(img[:1], 0.1)
    assert np.array_equal(s1, s2)


# ---------------------------------------------------------------------------
# Corner detection (reading A3)
# ---------------------------------------------------------------------------


def test_harris_flat_and_straight_edge():
    """Flat maps give R = 0; a straight full-height edge gives R <= 0 everywhere (no corner)."""
    assert np.all(O.corner_response(np.zeros((12, 12), dtype=np.int64)) == 0)
    S = np.zeros((16, 16), dtype=np.int64)
    S[:, 7:9] = 2
    R = O.corner_response(S)
    assert R.max() <= 0 and R.min() < 0


def test_harris_rectangle_corners():
    """The four strongest NMS corners of a filled rectangle are its four corner pixels."""
    img = np.zeros((40, 40))
    img[10:30, 12:28] = 1.0
    S = O.edge_sum(img[None], 0.1)
    R = O.corner_response(S)
    keep = O.nms3(R)
    rr, cc = np.nonzero(keep)
    order = np.lexsort((rr * 40 + cc, -R[rr, cc]))[:4]
    got = sorted((int(rr[i]), int(cc[i])) for i in order)
    assert got == [(10, 12), (10, 27), (29, 12), (29, 27)]


def test_nms_plateau_tie_break():
    """A plateau keeps only its lowest-index pixel; strict maxima survive; R <= 0 never does."""
    R = np.zeros((5, 6), dtype=np.int64)
    R[1, 1] = R[1, 2] = R[2, 1] = R[2, 2] = 7  # 2x2 plateau
    R[3, 4] = 9
    R[4, 0] = -3
    keep = O.nms3(R)
    assert set(zip(*np.nonzero(keep))) == {(1, 1), (3, 4)}


def test_select_keys_grid_fill_closed_form():
    """No edges -> all keys come from the row-major grid of stride isqrt(Hq*Wq // N) (A5)."""
    x = np.full((1, 20, 20), 0.3)
    P, N = 4, 10
    keys, nc = O.select_keys(x, P, N, 0.1)
    Hq = Wq = 17
    s = math.isqrt(Hq * Wq // N)
    assert s == 5 and nc == 0
    expect = [gr * Wq + gc for gr in range(0, Hq, s) for gc in range(0, Wq, s)][:N]
    assert list(keys) == expect


def test_select_keys_clamp_and_dedupe():
    """Corners near the border clamp to the same top-left patch; later duplicates are dropped (A4)."""
    img = np.zeros((1, 24, 24))
    img[0, 1:12, 1:12] = 1.0  # corner pixels (1,1),(1,11),(11,1),(11,11)
    P, N = 8, 6
    keys, nc = O.select_keys(img, P, N, 0.1)
    Wq = 24 - P + 1
    # corner (1,1) -> top-left (max(1-4,0), max(1-4,0)) = (0,0); (1,11) -> (0,7); (11,1) -> (7,0); (11,11) -> (7,7)
    corner_tl = {0 * Wq + 0, 0 * Wq + 7, 7 * Wq + 0, 7 * Wq + 7}
    assert set(int(k) for k in keys[:nc]) <= corner_tl | set(range(Wq * Wq))
    assert {0, 7, 7 * Wq, 7 * Wq + 7} <= set(int(k) for k in keys[:nc])
    assert len(set(int(k) for k in keys)) == N
    # Two corners 1 px apart near the origin clamp to the same patch.
    img2 = np.zeros((1, 24, 24))
    img2[0, 2:20, 2:20] = 1.0
    img2[0, 2:4, 2:4] = 0.5
    k2, nc2 = O.select_keys(img2, P, 20, 0.1)
    assert len(set(int(k) for k in k2)) == 20


# ---------------------------------------------------------------------------
# Global matching (Eq. 1 over the whole image)
# ---------------------------------------------------------------------------


def test_topk_ramp_closed_form():
    """On x = a*c every pixel of two patches differs by a*dc, so d = P^2 a^2 dc^2 exactly:
    the ranking is (|dc|, id)."""
    a = 0.25
    H, W, P, K = 12, 14, 3, 20
    img = (a * np.arange(W)[None, :] * np.ones((H, 1)))[None]
    Hq, Wq = H - P + 1, W - P + 1
    key = 4 * Wq + 5
    idx, dist = O.match_topk(img, P, np.array([key]), K)
    ids = np.arange(Hq * Wq)
    dc = np.abs(ids % Wq - 5)
    expect = ids[np.lexsort((ids, dc))][:K]
    assert list(idx[0]) == list(expect)
    assert np.allclose(dist[0], P * P * a * a * dc[expect] ** 2)


def test_topk_planted_copies():
    """Exact copies of the key patch have distance 0 and come first, in id order."""
    rng = synth.rng_for("planted")
    H, W, P = 20, 22, 4
    img = rng.random((1, H, W))
    Wq = W - P + 1
    src = (3, 5)
    for r, c in [(12, 1), (0, 15), (15, 16)]:
        img[0, r : r + P, c : c + P] = img[0, src[0] : src[0] + P, src[1] : src[1] + P]
    key = src[0] * Wq + src[1]
    idx, dist = O.match_topk(img, P, np.array([key]), 6)
    want = sorted([key, 12 * Wq + 1, 0 * Wq + 15, 15 * Wq + 16])
    assert list(idx[0][:4]) == want and np.all(dist[0][:4] == 0) and np.all(dist[0][4:] > 0)


def test_topk_constant_image_ties_by_id():
    img = np.full((1, 10, 10), 0.5)
    idx, dist = O.match_topk(img, 3, np.array([17, 40]), 7)
    assert np.all(dist == 0) and list(idx[0]) == list(range(7)) and list(idx[1]) == list(range(7))


def test_topk_matches_kdtree_where_separated():
    """An independent exact nearest-neighbour search (scipy k-d tree) agrees wherever
    the K-th and (K+1)-th distances are separated."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = synth.rng_for("kdtree")
    img = rng.random((1, 18, 17))
    P, K = 4, 9
    Q = O.patch_matrix(img, P)
    keys = np.array([0, 31, 77, 130, Q.shape[0] - 1])
    idx, dist = O.match_topk(img, P, keys, K)
    tree = spatial.cKDTree(Q)
    for i, k in enumerate(keys):
        dd, ii = tree.query(Q[k], k=K + 1)
        if dd[K] ** 2 - dd[K - 1] ** 2 > 1e-9:
            assert set(ii[:K]) == set(idx[i])
        assert np.allclose(np.sqrt(dist[i]), dd[:K], atol=1e-12)


def test_patch_matrix_layout():
    """Patch vector index = ch*P*P + dr*P + dc at position id r*Wq + c."""
    x = np.arange(2 * 5 * 6, dtype=np.float64).reshape(2, 5, 6)
    P = 2
    Q = O.patch_matrix(x, P)
    Wq = 5
    q = 2 * Wq + 3
    assert Q.shape == (4 * 5, 8)
    assert Q[q, 1 * 4 + 1 * 2 + 0] == x[1, 3, 3] and Q[q, 0 * 4 + 0 * 2 + 1] == x[0, 2, 4]


# ---------------------------------------------------------------------------
# WNNM (Eq. 5, reading A9)
# ---------------------------------------------------------------------------


def test_wnnm_zero_noise_is_identity():
    rng = synth.rng_for("wnnm-id")
    Y = rng.random((16, 8))
    X, r, s, s2 = O.wnnm(Y, 0.0, 2 * math.sqrt(8))
    assert np.allclose(X, Y, atol=1e-12) and r == 8


def test_wnnm_rank_one_closed_form():
    """Y = sigma u v^T: X^ = (s'/sigma) Y with s' = sigma - C sw^2 / (sqrt(sigma^2 - K sw^2) + eps)."""
    rng = synth.rng_for("wnnm-r1")
    d, K = 12, 6
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(K)
    v /= np.linalg.norm(v)
    sigma, sw, C = 3.0, 0.2, 2 * math.sqrt(K)
    X, r, s, s2 = O.wnnm(sigma * np.outer(u, v), sw, C)
    s_new = sigma - C * sw * sw / (math.sqrt(sigma * sigma - K * sw * sw) + 1e-16)
    assert r == 1 and abs(s2[0] - s_new) < 1e-12
    assert np.allclose(X, (s_new / sigma) * sigma * np.outer(u, v), atol=1e-12)


def test_wnnm_two_by_two_singular_values():
    """[[3,0],[4,5]] has Y^T Y = [[25,20],[20,25]] -> singular values sqrt(45), sqrt(5)."""
    _, _, s, _ = O.wnnm(np.array([[3.0, 0.0], [4.0, 5.0]]), 0.0, 1.0)
    assert np.allclose(s, [math.sqrt(45), math.sqrt(5)], atol=1e-13)


def test_wnnm_orthogonal_columns_closed_form():
    """Orthogonal columns of norms s_i: X^ scales column i by s'_i / s_i (a textbook diagonal case)."""
    rng = synth.rng_for("wnnm-orth")
    d, K = 10, 4
    Qm, _ = np.linalg.qr(rng.standard_normal((d, K)))
    s = np.array([5.0, 2.0, 0.9, 0.3])
    Y = Qm * s
    sw, C = 0.25, 2 * math.sqrt(K)
    X, r, _, s2 = O.wnnm(Y, sw, C)
    sh = np.sqrt(np.maximum(s * s - K * sw * sw, 0))
    sp = np.maximum(s - C * sw * sw / (sh + 1e-16), 0)
    assert np.allclose(X, Qm * sp, atol=1e-12) and r == int((sp > 0).sum())
    assert sp[-1] == 0.0  # s^2 < K sw^2 -> sigma_hat = 0 -> the component is removed


def test_wnnm_noise_only_group_vanishes():
    rng = synth.rng_for("wnnm-noise")
    Y = rng.standard_normal((8, 8)) * 1e-3
    X, r, _, _ = O.wnnm(Y, 1.0, 2 * math.sqrt(8))
    assert r == 0 and np.all(X == 0)


def test_wnnm_recovers_noiseless_low_rank():
    rng = synth.rng_for("wnnm-lr")
    Y = rng.standard_normal((64, 3)) @ rng.standard_normal((3, 40))
    X, r, _, _ = O.wnnm(Y, 1e-7, 2 * math.sqrt(40))
    assert r >= 3 and np.linalg.norm(X - Y) / np.linalg.norm(Y) < 1e-9


# ---------------------------------------------------------------------------
# Aggregation (reading A10)
# ---------------------------------------------------------------------------


def test_aggregate_identity_denoiser_returns_input():
    rng = synth.rng_for("agg-id")
    x = rng.random((2, 9, 10))
    P = 3
    Q = O.patch_matrix(x, P)
    idx = rng.integers(0, Q.shape[0], size=(5, 4))
    v = O.aggregate(O.gather_groups(x, P, idx, Q), idx, x, P)
    assert np.allclose(v, x, atol=1e-14)


def test_aggregate_hand_worked_overlap():
    """Two 2x2 patches on a 3x4 image overlapping in one column; hand-computed average."""
    x = np.full((1, 3, 4), 9.0)
    P = 2
    Wq = 3
    idx = np.array([[0 * Wq + 0], [0 * Wq + 1]])  # top-left (0,0) and (0,1)
    g = np.array([[[1.0, 2.0, 3.0, 4.0]], [[10.0, 20.0, 30.0, 40.0]]])  # rows (0,0),(0,1),(1,0),(1,1)
    v = O.aggregate(g, idx, x, P)
    want = np.array([[1.0, (2 + 10) / 2, 20.0, 9.0], [3.0, (4 + 30) / 2, 40.0, 9.0], [9.0, 9.0, 9.0, 9.0]])
    assert np.allclose(v[0], want)


# ---------------------------------------------------------------------------
# GAP projection (Eq. 6 / Eq. 8)
# ---------------------------------------------------------------------------


def test_gap_projection_is_consistent():
    """Phi(x) = y wherever some mask is non-zero; untouched where all masks are zero."""
    rng = synth.rng_for("gap")
    T, H, W = 4, 7, 9
    A = (rng.random((T, H, W)) < 0.5).astype(float)
    A[:, 0, 0] = 0.0
    y = rng.random((H, W))
    v = rng.random((T, H, W))
    x, _ = O.gap_project(y, A, v)
    phi = (A * x).sum(0)
    cov = A.sum(0) > 0
    assert np.allclose(phi[cov], y[cov], atol=1e-13)
    assert np.allclose(x[:, 0, 0], v[:, 0, 0])


def test_gap_fixed_point_and_init():
    rng = synth.rng_for("gap2")
    T, H, W = 3, 5, 6
    A = rng.random((T, H, W))
    v = rng.random((T, H, W))
    y = (A * v).sum(0)
    x, _ = O.gap_project(y, A, v)
    assert np.allclose(x, v, atol=1e-14)
    x0 = O.gap_init(y, A)
    R = (A * A).sum(0)
    assert np.allclose(x0, A * (y / R)[None])
    # one pixel by hand: masks (1, 0, 1), y = 6 -> R = 2 -> x0 = (3, 0, 3)
    A1 = np.array([1.0, 0.0, 1.0]).reshape(3, 1, 1)
    assert np.allclose(O.gap_init(np.array([[6.0]]), A1).ravel(), [3.0, 0.0, 3.0])


def test_gap_accelerated_accumulates_residual():
    rng = synth.rng_for("gap3")
    T, H, W = 2, 3, 3
    A = (rng.random((T, H, W)) < 0.5).astype(float) + 0.5
    v = rng.random((T, H, W))
    y = rng.random((H, W))
    yacc0 = y.copy()
    x, yacc = O.gap_project(y, A, v, yacc0)
    assert np.allclose(yacc, y + (y - (A * v).sum(0)))
    assert np.allclose((A * x).sum(0), yacc)


def test_msfa_orthogonal_masks_give_unit_normaliser():
    """Eq. 9: orthogonal binary masks that tile the plane give R = 1 everywhere."""
    H = W = 8
    A = np.zeros((16, H, W))
    for b in range(16):
        A[b, (b // 4)::4, (b % 4)::4] = 1.0
    assert np.all(O.gap_normaliser(A) == 1.0)
    for i in range(16):
        for j in range(i + 1, 16):
            assert not np.any(A[i] * A[j])


def test_psnr():
    a = np.zeros((2, 4, 4))
    b = np.full((2, 4, 4), 0.1)
    assert abs(O.psnr(a, b) - 20.0) < 1e-12


@pytest.mark.slow
def test_sigma_schedule_reading():
    """Reading A11: from x0 = Phi^T(y/R) a noise level of 0.5 -> 0.1 denoises, 0.08 -> 0.02 barely does."""
    cfg = synth.scaled(synth.SCI_SMALL, T=8, H=64, W=64, N=100)
    prob = synth.sci_problem(cfg)
    res = {}
    for name, sched in (("low", [0.08, 0.04, 0.02]), ("used", [0.5, 0.3, 0.15])):
        x = O.glr_reconstruct(prob.y, prob.masks, cfg.P, cfg.N, cfg.K, sched, cfg.c_wnnm, cfg.edge_th)
        res[name] = O.psnr_framewise(x, prob.truth)
    assert res["used"] > res["low"] + 8.0, res


# ---------------------------------------------------------------------------
# The paper's heat-map score (Eq. 4), reading A18
# ---------------------------------------------------------------------------
def test_edge_heatmap_counts_shared_edge_pixels():
    """H(q) is the number of (map, channel, pixel) edge entries the two patches share:
    brute force over the maps on a tiny two-channel image."""
    rng = synth.rng_for("hm")
    x = synth.quantize8(rng.random((2, 9, 11)))
    P, th = 3, 0.3
    E = O.edge_planes(x, th)
    assert set(np.unique(E)) <= {0.0, 1.0}
    Hq, Wq = 7, 9
    key = 2 * Wq + 5
    h = O.edge_heatmap(x, P, key, th)
    kr, kc = divmod(key, Wq)
    for q in range(Hq * Wq):
        r, c = divmod(q, Wq)
        want = 0
        for m in range(8):
            want += int(np.sum(E[m, r:r + P, c:c + P] * E[m, kr:kr + P, kc:kc + P]))
        assert h[q] == want


def test_edge_heatmap_self_is_maximal_and_copies_tie():
    """H(q) <= H(key) for every q (shared entries cannot exceed the key's own count),
    and a planted copy of the key region ties with the key (then smaller id first)."""
    rng = synth.rng_for("hm2")
    x = synth.quantize8(rng.random((1, 20, 24)))
    x[0, 12:20, 14:22] = x[0, 2:10, 3:11]  # copy including a 1-pixel margin for the Sobel support
    P, th = 6, 0.25
    key = 3 * 19 + 4  # top-left (3, 4); its copy sits at (13, 15)
    h = O.edge_heatmap(x, P, key, th)
    assert h.max() == h[key]
    assert h[13 * 19 + 15] == h[key]
    idx, val = O.edge_match_topk(x, P, np.array([key]), 3, th)
    assert val[0, 0] == h[key] and idx[0, 0] == min(key, 13 * 19 + 15)


def test_edge_heatmap_flat_image_is_zero():
    x = np.full((1, 12, 12), 0.4)
    assert np.all(O.edge_heatmap(x, 4, 10, 0.1) == 0)


# ---------------------------------------------------------------------------
# Corner + uniform keys (A19) and ADMM for SCI (A20)
# ---------------------------------------------------------------------------
def test_select_keys_uniform_mix_closed_form():
    """On a flat image there are no corners: the uniform keys are the grid of stride 9
    (the smallest stride whose grid has at most 9 points on 26 x 26 positions:
    stride 8 gives 4 x 4), which spans the whole image; the rest come from the A5 grid."""
    x = np.full((1, 30, 30), 0.5)
    P, N, nu = 5, 20, 9
    keys, nc = O.select_keys(x, P, N, 0.1, n_uniform=nu)
    Wq = 26
    want = [r * Wq + c for r in (0, 9, 18) for c in (0, 9, 18)]
    assert nc == 0 and list(keys[:nu]) == want and len(set(keys.tolist())) == N


def test_select_keys_uniform_mix_caps_corners():
    x = synth.quantize8(synth.textured_frames(synth.rng_for("mix"), 1, 64, 64))[None][0]
    k0, n0 = O.select_keys(x, 8, 40, 0.1)
    k1, n1 = O.select_keys(x, 8, 40, 0.1, n_uniform=15)
    assert n1 <= 25 and list(k1[:n1]) == list(k0[:n1])  # the same corners, in rank order, capped


def test_admm_sci_step_is_the_minimiser():
    rng = synth.rng_for("admm-sci")
    T, H, W = 4, 9, 11
    A = (rng.random((T, H, W)) < 0.5).astype(float)
    y = rng.random((H, W))
    z, x, u = rng.random((T, H, W)), rng.random((T, H, W)), rng.random((T, H, W))
    for rho in (0.05, 1.0, 5.0):
        xn, un, wn = O.admm_sci_step(y, A, z, x, u, rho)
        assert np.allclose(un, u + x - z) and np.allclose(wn, xn + un)
        w = z - un
        # gradient of ||y - Phi x||^2 / 2 + rho ||x - w||^2 / 2 vanishes
        g = A * ((A * xn).sum(0) - y)[None] + rho * (xn - w)
        assert np.abs(g).max() < 1e-12
    # rho -> 0 gives the GAP projection of w (Phi x = y where R > 0)
    xn, _, _ = O.admm_sci_step(y, A, z, x, u, 1e-12)
    R = (A * A).sum(0)
    assert np.allclose(((A * xn).sum(0) - y)[R > 0], 0, atol=1e-9)


def test_window_matching_is_global_matching_restricted():
    """Reading A21: the window result equals global matching on the window's positions
    (brute force), and a window covering the whole grid gives the global result."""
    rng = synth.rng_for("win")
    x = rng.random((1, 14, 15))
    P, K = 3, 6
    Hq, Wq = 12, 13
    keys = np.array([0, 40, 155], np.int32)
    Q = O.patch_matrix(x, P)
    idx, dist = O.window_match_topk(x, P, keys, K, 2, Q)
    for i, k in enumerate(keys):
        kr, kc = divmod(int(k), Wq)
        r0, c0 = min(max(kr - 2, 0), Hq - 5), min(max(kc - 2, 0), Wq - 5)
        cand = [(r, c) for r in range(r0, r0 + 5) for c in range(c0, c0 + 5)]
        d = sorted((float(((Q[r * Wq + c] - Q[k]) ** 2).sum()), r * Wq + c) for r, c in cand)[:K]
        assert [q for _, q in d] == list(idx[i]) and np.allclose([v for v, _ in d], dist[i])
    xs = rng.random((1, 13, 13))  # an 11 x 11 position grid: w = 5 covers all of it
    Qs = O.patch_matrix(xs, P)
    gi, gd = O.match_topk(xs, P, np.array([37]), K, Qs)
    wi, wd = O.window_match_topk(xs, P, np.array([37]), K, 5, Qs)
    assert np.array_equal(gi, wi) and np.allclose(gd, wd)


# ---------------------------------------------------------------------------
# Eq. 5 glue: lowrank_groups, glr_denoise; Eq. 6 loops: glr_reconstruct(_admm)
# ---------------------------------------------------------------------------
def test_lowrank_groups_shrinks_with_member_count_k():
    """lowrank_groups reads a group [K][d] as the d x K matrix of Eq. 5: the noise term of
    sigma_hat is K sigma_w^2 with K the number of members.  A rank-1 group with K = 3 members
    of d = 5 values, s^2 = 2.4 and sigma_w^2 = 0.6 lies between K sigma_w^2 = 1.8 (kept) and
    d sigma_w^2 = 3.0 (which would remove it), so reading d for K, or a transposed group,
    changes the result.  By hand: sigma_hat = sqrt(0.6), tau = 0.5 * 0.6 / sqrt(0.6) = sqrt(0.6) / 2,
    s = sqrt(2.4) = 2 sqrt(0.6), s' = s - tau = 1.5 sqrt(0.6), X^ = (s'/s) Y = 0.75 Y."""
    a = np.array([1.0, 1.0, 1.0])  # member weights (K = 3)
    b = np.full(5, 0.4)  # patch (d = 5)
    g = np.outer(a, b)[None]  # [N=1][K=3][d=5]
    out, rank = O.lowrank_groups(g, math.sqrt(0.6), 0.5)
    assert out.shape == (1, 3, 5)
    assert rank.tolist() == [1]
    np.testing.assert_allclose(out[0], 0.75 * g[0], rtol=1e-12, atol=1e-14)
    # the same group with 5 members of 3 values: now K sigma_w^2 = 3.0 > s^2 = 2.4, removed
    out2, rank2 = O.lowrank_groups(np.outer(b, a)[None], math.sqrt(0.6), 0.5)
    assert rank2.tolist() == [0] and np.all(out2 == 0)


def test_glr_denoise_without_noise_returns_the_image():
    """sigma_w = 0: WNNM keeps every singular value (tau = 0), so each group comes back
    unchanged and averaging the exact patches returns x wherever a patch covers it and x
    itself elsewhere: the whole pass is the identity (two channels, P = 3)."""
    rng = synth.rng_for("denoise-identity")
    x = rng.random((2, 2, 12, 13))
    v, info = O.glr_denoise(x, 3, 20, 5, 0.0, 4.0, 0.1)
    np.testing.assert_allclose(v, x, rtol=0, atol=1e-12)
    assert all(len(i["keys"]) == 20 for i in info)


def test_glr_denoise_constant_image_closed_form():
    """A constant image c: no corners, so the keys are the reading-A5 grid; every distance is
    0, so every key's K matches are positions 0..K-1 (ties by id); each group is c times a
    d x K matrix of ones with s = c sqrt(dK), and WNNM scales it by s'/s.  Covered pixels
    (rows 0..P-1, columns 0..K+P-2) become c s'/s, the rest keep c."""
    c, P, N, K, sw = 0.5, 3, 10, 4, 0.4
    H = W = 10
    x = np.full((1, 1, H, W), c)
    C_w = 2.0 * math.sqrt(K)
    v, info = O.glr_denoise(x, P, N, K, sw, C_w, 0.1)
    d = P * P
    s = c * math.sqrt(d * K)
    s_hat = math.sqrt(s * s - K * sw * sw)
    s_new = s - C_w * sw * sw / s_hat
    want = np.full((H, W), c)
    want[:P, : K + P - 1] = c * s_new / s
    np.testing.assert_allclose(v[0, 0], want, rtol=1e-12)
    assert info[0]["n_corner"] == 0
    assert np.all(info[0]["idx"] == np.arange(K))


def test_glr_reconstruct_full_mask_is_the_projection():
    """One frame behind a mask of 2 everywhere: R = 4, x0 = 2 y / 4 = y / 2, and the GAP update
    x = v + 2 (y - 2 v) / 4 = y / 2 whatever the denoiser returned.  So the reconstruction is
    y / 2 exactly; a dropped R, R = sum A instead of sum A^2, or a flipped residual sign fails."""
    rng = synth.rng_for("gap-full-mask")
    y = rng.random((9, 11))
    masks = np.full((1, 9, 11), 2.0)
    x = O.glr_reconstruct(y, masks, 3, 12, 4, [0.3, 0.1], 4.0, 0.1)
    np.testing.assert_allclose(x, (y / 2.0)[None], rtol=0, atol=1e-12)


def test_glr_reconstruct_identity_denoiser_keeps_x0():
    """sigma_w = 0 makes the denoiser the identity (previous pin), and x0 = Phi^T(y/R) already
    satisfies Phi x0 = y where R > 0, so every GAP iteration returns x0 = A_t y / R (0 where
    no mask is set), computed here by hand."""
    rng = synth.rng_for("gap-identity")
    T, H, W = 3, 10, 12
    masks = (rng.random((T, H, W)) < 0.5).astype(np.float64)
    y = rng.random((H, W))
    R = masks.sum(0)
    x0 = masks * np.where(R > 0, y / np.where(R > 0, R, 1.0), 0.0)[None]
    x = O.glr_reconstruct(y, masks, 3, 15, 4, [0.0, 0.0], 4.0, 0.1)
    np.testing.assert_allclose(x, x0, rtol=0, atol=1e-12)


def _zero_denoiser_case(tag, T):
    """Random frames small enough that every position can be a key (N = Hq Wq): every pixel
    is then covered by its own key's patch (the unique distance-0 match of a random image),
    and with a huge sigma_w (sigma_hat = 0, tau = C sw^2 / eps) WNNM removes every group,
    so the denoiser returns exactly 0."""
    rng = synth.rng_for(tag)
    H, W, P = 7, 8, 2
    masks = (rng.random((T, H, W)) < 0.6).astype(np.float64) if T > 1 else np.full((1, H, W), 2.0)
    y = 0.2 + rng.random((H, W))
    N = (H - P + 1) * (W - P + 1)
    return y, masks, P, N


def test_glr_reconstruct_accelerated_with_zero_denoiser():
    """Accelerated GAP with v = 0: y_acc = y + (y - 0) = 2y after the first iteration and 3y after
    the second, so x_k = (k + 1) Phi^T(y / R) (by hand): pins the residual accumulation."""
    y, masks, P, N = _zero_denoiser_case("gap-acc-zero", 3)
    v, _ = O.glr_denoise(O.gap_init(y, masks)[:, None], P, N, 2, 1e3, 4.0, 0.1)
    assert np.all(v == 0)
    R = masks.sum(0)
    x0 = masks * np.where(R > 0, y / np.where(R > 0, R, 1.0), 0.0)[None]
    x = O.glr_reconstruct(y, masks, P, N, 2, [1e3, 1e3], 4.0, 0.1, accelerate=True)
    np.testing.assert_allclose(x, 3.0 * x0, rtol=1e-12, atol=1e-14)


def test_glr_reconstruct_admm_with_zero_denoiser_closed_form():
    """Scaled ADMM (reading A20), one frame behind a mask of 2 (R = 4), rho = 1, z = D(.) = 0:
    x0 = y/2; iteration 1: u = x0 = y/2, w = -y/2, x1 = w + 2 (y - 2 w) / 5 = 0.3 y;
    iteration 2: u = 0.5 y + 0.3 y = 0.8 y, w = -0.8 y, x2 = -0.8 y + 2 (y + 1.6 y) / 5 = 0.24 y."""
    y, masks, P, N = _zero_denoiser_case("admm-zero", 1)
    x1 = O.glr_reconstruct_admm(y, masks, P, N, 2, [1e3], 4.0, 0.1, 1.0)
    np.testing.assert_allclose(x1, (0.3 * y)[None], rtol=1e-12)
    x2 = O.glr_reconstruct_admm(y, masks, P, N, 2, [1e3, 1e3], 4.0, 0.1, 1.0)
    np.testing.assert_allclose(x2, (0.24 * y)[None], rtol=1e-12)
