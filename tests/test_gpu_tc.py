"""Tensor-core (tcgen05, BF16) matching path.

* The raw scores of one position tile equal ||p~ - q~||^2 of the mean-shifted
  patches rounded to BF16, computed here on the host (checks the operand
  packing, the SW128 / SW32 shared-memory descriptors and the TMEM read-out).
* The full BF16 path (candidates by BF16 score, exact FP32 re-rank) agrees
  with the oracle: every reported distance is the exact distance of the
  reported id and the list is sorted.  Ids are bit-exact (where the FP32
  distances separate) for every key whose BF16 score error cannot move a true
  top-K position behind K' others: with p~, q~ the BF16-rounded mean-shifted
  patches, | ||p~ - q~||^2 - ||p - q||^2 | <= E(q) = 2 ||p - q|| dl + dl^2 +
  2.02e-6 (||p||^2 + ||q||^2), dl = 2^-9 (||p|| + ||q||) (BF16 rounding is
  within 2^-9 relative per value; the last term is the FP32 accumulation of the
  contraction, the bound the raw-score test uses).  If the largest d + E over
  the oracle's top K is below the smallest d - E beyond its top K', the K'
  candidates hold the whole top K and the exact re-rank returns it.  Other keys
  must still return distances within that bound.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("case", [("tc1", 2, 60, 300, 8, 150), ("tc2", 1, 40, 70, 5, 30), ("tc3", 1, 30, 30, 4, 128)])
def test_tc_raw_scores_match_host_bf16(case):
    tag, F, H, W, P, N = case
    rng = synth.rng_for(tag)
    x = synth.textured_frames(rng, F, H, W)[:, None].astype(np.float32)
    npos = (H - P + 1) * (W - P + 1)
    keys = np.stack([rng.choice(npos, size=N, replace=False) for _ in range(F)]).astype(np.int32)
    sc = glr.debug_match_scores(cuda(x), P, cuda(keys, torch.int32), cuda(np.full(F, N, np.int32), torch.int32), 8)
    torch.cuda.synchronize()
    sc = sc.cpu().numpy()
    ncol = min(256, npos)
    for f in range(F):
        mu = np.float32(np.float64(x[f]).mean())
        xs = (x[f] - mu).astype(np.float32)
        Q = bf16(O.patch_matrix(xs, P))
        for i in range(N):
            p = Q[keys[f, i]]
            want = ((Q[:ncol] - p) ** 2).sum(1)
            scale = (p * p).sum() + (Q[:ncol] ** 2).sum(1)
            err = np.abs(sc[f, i, :ncol] - want)
            assert np.all(err <= 2e-6 * scale + 1e-6), (f, i, err.max())


U_BF16 = 2.0**-9


def check_bf16_topk(x, P, keys, K, k_over, idx, dist):
    """Returns the fraction of keys the separation condition covers (all of them checked)."""
    covered = tot = 0
    for f in range(x.shape[0]):
        mu = np.float64(x[f]).mean()
        Q = O.patch_matrix(x[f], P)
        qn = np.sqrt((O.patch_matrix(np.float64(x[f]) - mu, P) ** 2).sum(1))
        for i in range(keys.shape[1]):
            d_all = O.all_distances(x[f], P, keys[f, i], Q)
            g = idx[f, i]
            np.testing.assert_allclose(dist[f, i], d_all[g], rtol=2e-5, atol=2e-6)
            assert np.all(np.diff(dist[f, i]) >= -1e-4) and len(set(g.tolist())) == K
            order = np.lexsort((np.arange(len(d_all)), d_all))
            dl = U_BF16 * (qn[keys[f, i]] + qn)
            E = 2 * np.sqrt(np.maximum(d_all, 0)) * dl + dl * dl + 2.02e-6 * (qn[keys[f, i]] ** 2 + qn**2)
            hi = (d_all[order[:K]] + E[order[:K]]).max()
            tot += 1
            if k_over < len(order) and (d_all[order[k_over:]] - E[order[k_over:]]).min() > hi:
                covered += 1
                ds = d_all[order]
                for j in range(K):
                    lo_gap = ds[j] - ds[j - 1] if j > 0 else np.inf
                    hi_gap = ds[j + 1] - ds[j] if j + 1 < len(ds) else np.inf
                    if lo_gap > 1e-4 and hi_gap > 1e-4:
                        assert g[j] == order[j], (f, i, j)
            else:
                assert np.all(d_all[g] <= hi + E[g] + 1e-6), (f, i)
    return covered / tot


@pytest.mark.parametrize("case", [("b1", 2, 70, 260, 8, 130, 40), ("b2", 1, 50, 60, 6, 40, 16), ("b3", 1, 40, 40, 8, 64, 64)])
@pytest.mark.parametrize("splits", [0, 2])
def test_match_bf16_exact_where_separated(case, splits):
    tag, F, H, W, P, N, K = case
    x = synth.textured_frames(synth.rng_for(tag), F, H, W)[:, None].astype(np.float32)
    rng = synth.rng_for(tag + "k")
    npos = (H - P + 1) * (W - P + 1)
    keys = np.stack([rng.choice(npos, size=N, replace=False) for _ in range(F)]).astype(np.int32)
    idx, dist = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.full(F, N, np.int32), torch.int32), K,
                               "bf16", splits=splits, k_over=K + 16)
    torch.cuda.synchronize()
    covered = check_bf16_topk(x, P, keys, K, K + 16, idx.cpu().numpy(), dist.cpu().numpy())
    assert covered >= 0.8, covered  # the condition covers 85-100 % of these keys


def test_match_bf16_vs_fp32_on_gap_start_image():
    """On the GAP start image (half the pixels masked) the BF16 and FP32 forms agree closely."""
    cfg = synth.scaled(synth.SCI_SMALL, T=2, H=96, W=96, N=100, K=40)
    prob = synth.sci_problem(cfg)
    x0 = O.gap_init(prob.y, prob.masks)[:, None].astype(np.float32)
    xt = cuda(x0)
    keys, nf, _ = glr.select_keys(xt, cfg.P, cfg.N)
    i32, d32 = glr.match_topk(xt, cfg.P, keys, nf, cfg.K, "fp32")
    i16, d16 = glr.match_topk(xt, cfg.P, keys, nf, cfg.K, "bf16")
    a, b = i32.cpu().numpy(), i16.cpu().numpy()
    same = np.mean([len(set(a[f, k]) & set(b[f, k])) / cfg.K for f in range(a.shape[0]) for k in range(a.shape[1])])
    assert same >= 0.99, same
