"""Plain FP64 CPU oracle of the global low-rank (GLR) denoising step and its GAP projection.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The library's CUDA path
never calls it, and it shares no code with that path (no helpers, tables or
constants); the only thing both sides use is the seeded input generator.

Every function follows one step of the method in the paper's order and
notation, written for clarity, not speed:

* ``sobel`` / ``edge_maps``        -- Section 2 (Method), Eq. 2 and Eq. 3:
  Sobel horizontal / vertical gradients and the four signed binary edge maps.
* ``corner_response`` / ``nms3`` / ``select_keys`` -- Section 2: exemplar (key)
  patches are centred on corner points of the averaged edge map.
* ``edge_match_topk``              -- the paper's global-matching heat map (Eq. 4):
  correlation of binary edge patches over the four maps of Eq. 2.
* ``match_topk``                   -- Eq. 1 made global (Section 2): the K
  positions with the smallest squared L2 distance to each key over the whole
  image; the grouping operator R~_i of Eq. 5.
* ``gather_groups``                -- R~_i x of Eq. 5.
* ``wnnm``                         -- low-rank step of Eq. 5 solved by weighted
  nuclear-norm minimisation (the paper adopts WNNM, Section 2).
* ``aggregate``                    -- returns the low-rank patch estimates to
  the image by averaging overlapping patches.
* ``gap_project`` / ``gap_init``   -- the generalized-alternating-projection
  update for the coded-aperture model y = sum_t A_t x_t (Eq. 6).
* ``glr_reconstruct``              -- GAP iterations with the GLR denoiser.

Readings of points the paper leaves open (each also listed in the design notes):

A1  Eq. 2 prints T(abs(g)) and T(abs(-g)) for the "+" and "-" maps, which are
    identical; they are read as T(max(g,0)) and T(max(-g,0)) (rising and
    falling edges), matching the four-term sum of Eq. 4.
A2  th is an argument (default 0.1 on Sobel output for [0,1] images).  The
    threshold decision is taken on the gradient rounded to float32, the
    precision the CUDA path decides in.
A3  The corner detector is unnamed: Harris with k = 1/25 on the integer
    averaged edge map S (sum of the four 0/1 maps, OR-ed over channels),
    Sobel of S with replicated border, 5x5 box sums with zero outside the
    image, R = 25 (A B - C^2) - (A + B)^2 in exact integers; only R > 0
    qualifies; 3x3 non-maximum suppression keeps a pixel if it is strictly
    greater than neighbours with a smaller linear index and >= neighbours
    with a larger one.
A4  Key centre (r, c) -> patch top-left (r - P//2, c - P//2) clamped to the
    valid range; duplicates after clamping are dropped in rank order.
A5  Fewer corners than N: fill from a row-major grid of stride
    max(1, isqrt(Hq*Wq // N)), skipping positions already chosen.
A7  Search domain: every valid position of the same image, the key itself
    included; ties by smaller position id.
A8  Fixed K (no threshold T_i).
A9  WNNM single pass: sigma_hat_i = sqrt(max(s_i^2 - K sw^2, 0)),
    tau_i = C sw^2 / (sigma_hat_i + eps), s'_i = max(s_i - tau_i, 0),
    X^ = U diag(s') V^T; no mean removal.
A10 Aggregation weight 1; pixels no patch covers keep the input value.
A12 Plain GAP (accelerated is a flag); R = sum_t A_t^2 with R = 0 -> 1;
    x0 = Phi^T (y / R).
A19 Corner + uniform keys (Section 3, CACTI and the matching-strategy
    comparison): at most N - n_uniform corners, then the uniform grid of the
    smallest stride s with ceil(Hq/s) ceil(Wq/s) <= n_uniform (so the grid covers
    the image) in row-major order, skipping chosen positions.
A20 ADMM for y = Phi x (the paper uses GAP or ADMM): scaled form z = D(x + u),
    u = u + x - z, x = w + Phi^T((y - Phi w)/(R + rho)) with w = z - u.
A21 Block matching baseline: a (2w+1) x (2w+1) window of positions centred on
    the key, shifted inside the position grid at its borders (so every key sees
    (2w+1)^2 candidates); K smallest distances, ties by smaller id.
A18 The paper's own matching score (the heat map of Eq. 4, ``edge_match_topk``):
    Conv2d is a correlation summed over the four maps and the C channels (the
    per-channel maps, not the OR-ed ones of key selection); a larger value is a
    better match; the K largest are kept, ties by smaller position id.

Layouts: images x[F][C][H][W]; a patch vector is ordered channel, then row,
then column (index ch*P*P + dr*P + dc); a position id is q = r*Wq + c of the
patch's top-left corner, with Hq = H-P+1, Wq = W-P+1.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Eq. 2 / Eq. 3: Sobel gradients and signed binary edge maps
# ---------------------------------------------------------------------------


def sobel(img: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Horizontal and vertical Sobel derivatives of one channel, replicated border.

    g_h responds to change along columns (x), g_v to change along rows (y):
    g_h = [[-1,0,1],[-2,0,2],[-1,0,1]] (correlation), g_v = its transpose.
    A ramp of slope a per pixel gives 8a in the interior.
    """
    H, W = img.shape
    p = np.pad(np.asarray(img, dtype=np.float64), 1, mode="edge")

    def at(dr: int, dc: int) -> np.ndarray:  # image shifted so that out[r,c] = img[r+dr, c+dc]
        return p[1 + dr : 1 + dr + H, 1 + dc : 1 + dc + W]

    out_h = np.zeros((H, W))
    out_v = np.zeros((H, W))
    for k, w in ((-1, 1.0), (0, 2.0), (1, 1.0)):
        out_h += w * (at(k, 1) - at(k, -1))  # right column minus left column
        out_v += w * (at(1, k) - at(-1, k))  # bottom row minus top row
    return out_h, out_v


def threshold(z: np.ndarray, th: float) -> np.ndarray:
    """Eq. 3: T(z) = 1 if z > th else 0, decided in float32 (reading A2)."""
    return (np.asarray(z, dtype=np.float64).astype(np.float32) > np.float32(th)).astype(np.uint8)


def edge_maps(img: np.ndarray, th: float) -> dict[str, np.ndarray]:
    """Eq. 2 under reading A1: four 0/1 maps of rising / falling horizontal and vertical edges."""
    gh, gv = sobel(img)
    gh32 = gh.astype(np.float32).astype(np.float64)
    gv32 = gv.astype(np.float32).astype(np.float64)
    return {
        "h+": threshold(np.maximum(gh32, 0.0), th),
        "h-": threshold(np.maximum(-gh32, 0.0), th),
        "v+": threshold(np.maximum(gv32, 0.0), th),
        "v-": threshold(np.maximum(-gv32, 0.0), th),
    }


def edge_sum(x: np.ndarray, th: float) -> np.ndarray:
    """Integer averaged edge map S in 0..4 of one image x[C][H][W].

    Each of the four maps is OR-ed over channels, then the four are summed
    (the sum is 4x the averaged map; the scale does not change corner ranks).
    """
    C = x.shape[0]
    acc = {k: np.zeros(x.shape[1:], dtype=np.uint8) for k in ("h+", "h-", "v+", "v-")}
    for ch in range(C):
        m = edge_maps(x[ch], th)
        for k in acc:
            acc[k] |= m[k]
    return sum(acc[k].astype(np.int64) for k in acc)


# ---------------------------------------------------------------------------
# Corner points of the averaged edge map (reading A3)
# ---------------------------------------------------------------------------


def _box5_zero(a: np.ndarray) -> np.ndarray:
    """5x5 window sums, zero outside the image (direct double loop over offsets)."""
    H, W = a.shape
    p = np.zeros((H + 4, W + 4), dtype=np.int64)
    p[2 : 2 + H, 2 : 2 + W] = a
    out = np.zeros((H, W), dtype=np.int64)
    for dr in range(5):
        for dc in range(5):
            out += p[dr : dr + H, dc : dc + W]
    return out


def corner_response(S: np.ndarray) -> np.ndarray:
    """Integer Harris response R = 25 (A B - C^2) - (A + B)^2 (k = 1/25) of the edge map S."""
    ih, iv = sobel(S)
    ih = np.rint(ih).astype(np.int64)
    iv = np.rint(iv).astype(np.int64)
    A = _box5_zero(ih * ih)
    B = _box5_zero(iv * iv)
    Cc = _box5_zero(ih * iv)
    return 25 * (A * B - Cc * Cc) - (A + B) * (A + B)


def nms3(R: np.ndarray) -> np.ndarray:
    """3x3 non-maximum suppression with the index tie-break of reading A3; R > 0 only."""
    H, W = R.shape
    keep = R > 0
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == 0 and dc == 0:
                continue
            nb = np.full((H, W), np.iinfo(np.int64).min, dtype=np.int64)
            rs, re = max(0, -dr), min(H, H - dr)
            cs, ce = max(0, -dc), min(W, W - dc)
            nb[rs:re, cs:ce] = R[rs + dr : re + dr, cs + dc : ce + dc]
            lower_index = (dr < 0) or (dr == 0 and dc < 0)
            if lower_index:
                keep &= R > nb
            else:
                keep &= R >= nb
    return keep


def select_keys(x: np.ndarray, P: int, N: int, th: float, n_uniform: int = 0) -> tuple[np.ndarray, int]:
    """Key (exemplar) positions of one image x[C][H][W]: corners first, then a uniform grid.

    n_uniform > 0 mixes in uniformly placed keys (reading A19, the corner +
    uniform selections of Section 3): at most N - n_uniform corners, then the
    row-major grid of the smallest stride s with ceil(Hq/s) ceil(Wq/s) <= n_uniform
    (it covers the whole image), skipping chosen positions, then the reading-A5
    grid up to N keys.
    Returns (keys int32[N] position ids in rank order, number of corner keys kept).
    """
    C, H, W = x.shape
    Hq, Wq = H - P + 1, W - P + 1
    if N > Hq * Wq or N <= 0:
        raise ValueError("N must be in 1..Hq*Wq")
    if not 0 <= n_uniform <= N:
        raise ValueError("n_uniform must be in 0..N")
    S = edge_sum(x, th)
    R = corner_response(S)
    keep = nms3(R)
    rr, cc = np.nonzero(keep)
    pix = rr * W + cc
    resp = R[rr, cc]
    order = np.lexsort((pix, -resp))  # R descending, pixel id ascending
    top = order[:N - n_uniform]
    chosen: list[int] = []
    seen: set[int] = set()
    for i in top:
        tr = min(max(int(rr[i]) - P // 2, 0), Hq - 1)
        tc = min(max(int(cc[i]) - P // 2, 0), Wq - 1)
        q = tr * Wq + tc
        if q not in seen:
            seen.add(q)
            chosen.append(q)
    n_corner = len(chosen)
    if n_uniform > 0:
        su = 1
        while -(-Hq // su) * -(-Wq // su) > n_uniform:
            su += 1
        for gr in range(0, Hq, su):
            for gc in range(0, Wq, su):
                if len(chosen) == N:
                    break
                q = gr * Wq + gc
                if q not in seen:
                    seen.add(q)
                    chosen.append(q)
    s = max(1, math.isqrt((Hq * Wq) // N))
    if len(chosen) < N:
        for gr in range(0, Hq, s):
            for gc in range(0, Wq, s):
                q = gr * Wq + gc
                if q in seen:
                    continue
                seen.add(q)
                chosen.append(q)
                if len(chosen) == N:
                    break
            if len(chosen) == N:
                break
    return np.asarray(chosen, dtype=np.int32), n_corner


# ---------------------------------------------------------------------------
# Global matching: exact top-K of the squared L2 distance over all positions
# ---------------------------------------------------------------------------


def patch_matrix(x: np.ndarray, P: int) -> np.ndarray:
    """All patches of x[C][H][W] as rows [Hq*Wq][C*P*P] (float64), ordered by position id."""
    C, H, W = x.shape
    Hq, Wq = H - P + 1, W - P + 1
    xd = np.asarray(x, dtype=np.float64)
    Q = np.empty((Hq, Wq, C, P, P))
    for dr in range(P):
        for dc in range(P):
            Q[:, :, :, dr, dc] = np.moveaxis(xd[:, dr : dr + Hq, dc : dc + Wq], 0, -1)
    return Q.reshape(Hq * Wq, C * P * P)


def match_topk(x: np.ndarray, P: int, keys: np.ndarray, K: int, Q: np.ndarray | None = None):
    """For each key the K positions of smallest sum((p - q)^2), ordered by (distance, id).

    Distances are the direct FP64 sums (no expansion).  Returns (idx int32[N][K],
    dist float64[N][K]).
    """
    if Q is None:
        Q = patch_matrix(x, P)
    n_pos = Q.shape[0]
    ids = np.arange(n_pos)
    idx = np.empty((len(keys), K), dtype=np.int32)
    dist = np.empty((len(keys), K), dtype=np.float64)
    for i, k in enumerate(keys):
        diff = Q - Q[int(k)]
        d = np.einsum("ij,ij->i", diff, diff)
        order = np.lexsort((ids, d))[:K]
        idx[i] = order
        dist[i] = d[order]
    return idx, dist


def edge_planes(x: np.ndarray, th: float) -> np.ndarray:
    """The four binary edge maps of Eq. 2 (reading A1) for every channel of x[C][H][W]:
    planes[m * C + c] for m in (h+, h-, v+, v-), values 0/1 (float64)."""
    C = x.shape[0]
    out = np.zeros((4 * C,) + x.shape[1:])
    for c in range(C):
        e = edge_maps(x[c], th)
        for m, name in enumerate(("h+", "h-", "v+", "v-")):
            out[m * C + c] = e[name]
    return out


def edge_heatmap(x: np.ndarray, P: int, key: int, th: float, E: np.ndarray | None = None) -> np.ndarray:
    """Eq. 4: H(q) = sum over the four maps and the C channels of the Conv2d (a
    correlation) of the key's edge patch with the edge maps, at every valid
    position q (an integer: the number of edge pixels the two patches share)."""
    if E is None:
        E = edge_planes(x, th)
    Qe = patch_matrix(E, P)  # rows: every position's 4 C P^2 edge values
    return Qe @ Qe[key]


def edge_match_topk(x: np.ndarray, P: int, keys: np.ndarray, K: int, th: float):
    """Global matching by the heat map of Eq. 4: for each key the K positions of
    largest H, ties by smaller position id (reading A18); returns (idx, H values)."""
    E = edge_planes(x, th)
    Qe = patch_matrix(E, P)
    idx = np.empty((len(keys), K), dtype=np.int32)
    val = np.empty((len(keys), K))
    for i, k in enumerate(keys):
        h = Qe @ Qe[int(k)]
        order = np.lexsort((np.arange(len(h)), -h))[:K]
        idx[i] = order
        val[i] = h[order]
    return idx, val


def window_match_topk(x: np.ndarray, P: int, keys: np.ndarray, K: int, w: int, Q: np.ndarray | None = None):
    """Block matching (Eq. 1 in a local window, the baseline global matching replaces;
    reading A21): the (2w+1)^2 positions centred on the key, the window shifted inside
    the position grid at its borders; the K smallest distances, ties by smaller id."""
    C, H, W = x.shape
    Hq, Wq = H - P + 1, W - P + 1
    if Q is None:
        Q = patch_matrix(x, P)
    wl = 2 * w + 1
    idx = np.empty((len(keys), K), dtype=np.int32)
    dist = np.empty((len(keys), K))
    for i, k in enumerate(keys):
        kr, kc = divmod(int(k), Wq)
        r0 = min(max(kr - w, 0), Hq - wl)
        c0 = min(max(kc - w, 0), Wq - wl)
        cand = np.array([(r0 + a) * Wq + c0 + b for a in range(wl) for b in range(wl)])
        diff = Q[cand] - Q[int(k)]
        dd = np.einsum("ij,ij->i", diff, diff)
        order = np.lexsort((cand, dd))[:K]
        idx[i] = cand[order]
        dist[i] = dd[order]
    return idx, dist


def all_distances(x: np.ndarray, P: int, key: int, Q: np.ndarray | None = None) -> np.ndarray:
    """Direct FP64 distances from one key to every position (for separation checks)."""
    if Q is None:
        Q = patch_matrix(x, P)
    diff = Q - Q[int(key)]
    return np.einsum("ij,ij->i", diff, diff)


# ---------------------------------------------------------------------------
# Eq. 5: grouping, WNNM low-rank step, aggregation
# ---------------------------------------------------------------------------


def gather_groups(x: np.ndarray, P: int, idx: np.ndarray, Q: np.ndarray | None = None) -> np.ndarray:
    """R~_i x for every key: groups[N][K][d] (row j = the j-th matched patch)."""
    if Q is None:
        Q = patch_matrix(x, P)
    return Q[idx.astype(np.int64)]


def wnnm(Y: np.ndarray, sigma_w: float, c: float, eps: float = 1e-16):
    """Weighted nuclear-norm shrinkage of one group Y (d rows x K columns), reading A9.

    Returns (X_hat d x K, rank, singular values s, shrunk singular values s').
    """
    Yd = np.asarray(Y, dtype=np.float64)
    K = Yd.shape[1]
    U, s, Vt = np.linalg.svd(Yd, full_matrices=False)
    sig_hat = np.sqrt(np.maximum(s * s - K * sigma_w * sigma_w, 0.0))
    tau = c * sigma_w * sigma_w / (sig_hat + eps)
    s_new = np.maximum(s - tau, 0.0)
    X = (U * s_new) @ Vt
    return X, int(np.count_nonzero(s_new > 0)), s, s_new


def lowrank_groups(groups: np.ndarray, sigma_w: float, c: float, eps: float = 1e-16):
    """WNNM applied to every group [N][K][d]; returns (X_hat [N][K][d], rank[N])."""
    out = np.empty(groups.shape, dtype=np.float64)
    rank = np.empty(groups.shape[0], dtype=np.int32)
    for i in range(groups.shape[0]):
        X, r, _, _ = wnnm(groups[i].T, sigma_w, c, eps)
        out[i] = X.T
        rank[i] = r
    return out, rank


def aggregate(groups: np.ndarray, idx: np.ndarray, x: np.ndarray, P: int) -> np.ndarray:
    """Average every patch estimate back into image x[C][H][W] (weight 1, reading A10).

    v = num / den where some patch covers the pixel, else v = x.
    """
    C, H, W = x.shape
    Wq = W - P + 1
    num = np.zeros((C, H, W))
    den = np.zeros((C, H, W))
    flat_idx = idx.reshape(-1).astype(np.int64)
    flat_val = groups.reshape(-1, C, P, P)
    r0 = flat_idx // Wq
    c0 = flat_idx % Wq
    for ch in range(C):
        for dr in range(P):
            for dc in range(P):
                np.add.at(num[ch], (r0 + dr, c0 + dc), flat_val[:, ch, dr, dc])
                np.add.at(den[ch], (r0 + dr, c0 + dc), 1.0)
    v = np.asarray(x, dtype=np.float64).copy()
    m = den > 0
    v[m] = num[m] / den[m]
    return v


def glr_denoise(x: np.ndarray, P: int, N: int, K: int, sigma_w: float, c: float, th: float, eps: float = 1e-16):
    """One GLR denoising pass on every image of x[F][C][H][W]; returns v and per-image details."""
    out = np.empty(x.shape, dtype=np.float64)
    info = []
    for f in range(x.shape[0]):
        Q = patch_matrix(x[f], P)
        keys, n_corner = select_keys(x[f], P, N, th)
        idx, dist = match_topk(x[f], P, keys, K, Q)
        groups = gather_groups(x[f], P, idx, Q)
        xh, rank = lowrank_groups(groups, sigma_w, c, eps)
        out[f] = aggregate(xh, idx, x[f], P)
        info.append({"keys": keys, "n_corner": n_corner, "idx": idx, "dist": dist, "rank": rank})
    return out, info


# ---------------------------------------------------------------------------
# GAP projection for y = sum_t A_t x_t (Eq. 6 / Eq. 8)
# ---------------------------------------------------------------------------


def gap_normaliser(masks: np.ndarray) -> np.ndarray:
    """R = sum_t A_t^2 (the diagonal of Phi Phi^T), with 0 replaced by 1."""
    R = (np.asarray(masks, dtype=np.float64) ** 2).sum(0)
    R[R == 0] = 1.0
    return R


def gap_init(y: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """x0 = Phi^T (y / R)."""
    R = gap_normaliser(masks)
    return np.asarray(masks, dtype=np.float64) * (np.asarray(y, dtype=np.float64) / R)[None]


def gap_project(y: np.ndarray, masks: np.ndarray, v: np.ndarray, y_acc: np.ndarray | None = None):
    """x = v + Phi^T ((y - Phi v) / R).  With y_acc given (accelerated GAP),
    y_acc <- y_acc + (y - Phi v) and y_acc replaces y.  Returns (x, y_acc)."""
    A = np.asarray(masks, dtype=np.float64)
    vd = np.asarray(v, dtype=np.float64)
    R = gap_normaliser(A)
    yd = np.asarray(y, dtype=np.float64)
    phi_v = (A * vd).sum(0)
    if y_acc is not None:
        y_acc = np.asarray(y_acc, dtype=np.float64) + (yd - phi_v)
        yd = y_acc
    x = vd + A * ((yd - phi_v) / R)[None]
    return x, y_acc


def admm_sci_step(y, masks, z, x, u, rho):
    """One ADMM step for y = Phi x after the denoiser (reading A20, scaled form):
    u <- u + x - z;  x' = argmin ||y - Phi x||^2 + rho ||x - (z - u)||^2
    = w + Phi^T ((y - Phi w) / (R + rho)) with w = z - u (Phi Phi^T = diag(R));
    returns (x', u, the next denoiser input x' + u)."""
    A = np.asarray(masks, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64) + np.asarray(x, dtype=np.float64) - np.asarray(z, dtype=np.float64)
    w = np.asarray(z, dtype=np.float64) - u
    R = (A * A).sum(0)
    xn = w + A * ((np.asarray(y, dtype=np.float64) - (A * w).sum(0)) / (R + rho))[None]
    return xn, u, xn + u


def glr_reconstruct_admm(y, masks, P, N, K, sigmas, c, th, rho, eps=1e-16, n_uniform=0):
    """ADMM iterations with the GLR denoiser (reading A20): start x = Phi^T(y/R), u = 0;
    z = D(x + u), then admm_sci_step."""
    x = gap_init(y, masks)
    u = np.zeros_like(x)
    for sw in sigmas:
        z, _ = glr_denoise((x + u)[:, None], P, N, K, sw, c, th, eps)
        x, u, _ = admm_sci_step(y, masks, z[:, 0], x, u, rho)
    return x


def glr_reconstruct(y, masks, P, N, K, sigmas, c, th, accelerate=False, eps=1e-16, callback=None):
    """GAP iterations with the GLR denoiser for one snapshot (frames are the images).

    x_0 = Phi^T(y/R); for each sigma_w: v = D(x), x = project(v).
    """
    x = gap_init(y, masks)
    y_acc = np.asarray(y, dtype=np.float64).copy() if accelerate else None
    for k, sw in enumerate(sigmas):
        v, info = glr_denoise(x[:, None], P, N, K, sw, c, th, eps)
        x, y_acc = gap_project(y, masks, v[:, 0], y_acc)
        if callback is not None:
            callback(k, x, v[:, 0], info)
    return x


def psnr(a: np.ndarray, b: np.ndarray, peak: float = 1.0) -> float:
    mse = float(np.mean((np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)


def psnr_framewise(a: np.ndarray, b: np.ndarray, peak: float = 1.0) -> float:
    """Mean over frames of the per-frame PSNR (reading A16)."""
    return float(np.mean([psnr(a[i], b[i], peak) for i in range(a.shape[0])]))
