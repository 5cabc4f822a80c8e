"""The paper's heat-map matching (Eq. 4, GLR_MATCH_EDGE) against the FP64 oracle.

The operands are binary edge patches, exact in BF16, and the heat-map values
are integers, so the values are compared exactly.  Ids: the top-K by value is
unique except among positions tied at the K-th value; the ids above that value
must equal the oracle's, and every returned id must carry the value reported
for it (a valid choice among the ties).  Inputs are 8-bit quantised so the
FP32 Sobel sums, and hence the edge maps, are exact on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import glr_oracle as O  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.parametrize("case", [("e1", 1, 1, 40, 60, 4, 30, 16, 0), ("e2", 2, 1, 48, 70, 8, 40, 24, 0),
                                  ("e3", 1, 2, 40, 52, 6, 25, 12, 2), ("e4", 1, 3, 36, 40, 5, 20, 10, 0),
                                  ("e5", 1, 1, 64, 300, 8, 130, 32, 0)])
def test_edge_match_parity(case):
    tag, F, C, H, W, P, N, K, splits = case
    rng = synth.rng_for(tag)
    x = synth.quantize8(synth.textured_frames(rng, F * C, H, W)).reshape(F, C, H, W)
    th = 0.1
    npos = (H - P + 1) * (W - P + 1)
    keys = np.stack([rng.choice(npos, size=N, replace=False) for _ in range(F)]).astype(np.int32)
    idx, val = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.full(F, N, np.int32), torch.int32), K,
                              "edge", edge_th=th, splits=splits)
    torch.cuda.synchronize()
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    for f in range(F):
        E = O.edge_planes(x[f], th)
        Qe = O.patch_matrix(E, P)
        oi, ov = O.edge_match_topk(x[f], P, keys[f], K, th)
        for i in range(N):
            h = Qe @ Qe[keys[f, i]]
            np.testing.assert_array_equal(val[f, i], ov[i])          # the K values, exactly
            np.testing.assert_array_equal(h[idx[f, i]], val[f, i])   # each id carries its value
            assert len(set(idx[f, i].tolist())) == K
            hk = ov[i][-1]
            assert set(idx[f, i][val[f, i] > hk].tolist()) == set(oi[i][ov[i] > hk].tolist())
            # ties in order of id, as the oracle orders them
            for v in np.unique(val[f, i]):
                ids = idx[f, i][val[f, i] == v]
                assert np.all(np.diff(ids) > 0)


def test_edge_match_finds_the_key_itself_first():
    rng = synth.rng_for("e-self")
    x = synth.quantize8(synth.textured_frames(rng, 1, 50, 50))[None]
    P, N, K = 8, 20, 8
    npos = 43 * 43
    keys = rng.choice(npos, size=(1, N), replace=False).astype(np.int32)
    idx, val = glr.match_topk(cuda(x), P, cuda(keys, torch.int32), cuda(np.array([N], np.int32), torch.int32), K, "edge",
                              edge_th=0.6)
    torch.cuda.synchronize()
    idx, val = idx.cpu().numpy()[0], val.cpu().numpy()[0]
    E = O.edge_planes(x[0], 0.6)
    Qe = O.patch_matrix(E, P)
    for i in range(N):
        k = keys[0, i]
        h = Qe @ Qe[k]
        own = h[k]
        assert val[i, 0] == own  # nothing shares more edge entries than the key itself
        # the key is returned unless K positions of smaller id tie with it
        if np.count_nonzero(h[:k] == own) < K:
            assert k in idx[i][val[i] == own]


def test_denoiser_with_heat_map_matching_runs_and_groups_by_it():
    cfg = synth.scaled(synth.SCI_SMALL, T=2, H=64, W=64, N=40, K=16)
    x = synth.quantize8(synth.textured_frames(synth.rng_for("e-den"), 2, 64, 64))[:, None]
    den = glr.GlrDenoiser(glr.GlrShape(2, 1, 64, 64, cfg.P, cfg.N, cfg.K), mode="edge")
    v = den(cuda(x), 0.2, cfg.c_wnnm)
    torch.cuda.synchronize()
    assert torch.isfinite(v).all()
    keys = den.keys.cpu().numpy()
    for f in range(2):
        oi, ov = O.edge_match_topk(x[f], cfg.P, keys[f], cfg.K, 0.1)
        np.testing.assert_array_equal(den.dist.cpu().numpy()[f], ov)
