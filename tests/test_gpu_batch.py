"""Uneven batches: glr_match_topk_batch, one persistent tensor-core launch over images of
different sizes.

Per image the batch path packs the same BF16 operands as glr_match_topk (the image's own mean,
the same rows), keeps the K' best (score, id) pairs over all of a key's streams and re-ranks them
exactly, so its matches equal the single-image BF16 path's element by element whatever the
position splits; a sample of keys is also checked against the FP64 oracle (the BF16 separation
check of the tensor-core tests), and a CUDA-graph replay of the call equals the eager call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def make_batch(tag, sides, C, P, N):
    rng = synth.rng_for(tag)
    imgs = [synth.textured_frames(rng, C, h, w).astype(np.float32) for h, w in sides]
    x = torch.from_numpy(np.concatenate([im.reshape(-1) for im in imgs])).cuda()
    keys = []
    for (h, w), n in zip(sides, N):
        npos = (h - P + 1) * (w - P + 1)
        keys.append(rng.choice(npos, size=n, replace=False).astype(np.int32))
    kt = torch.from_numpy(np.concatenate(keys)).cuda()
    b = glr.Batch(sides, C, P, N)
    nf = torch.tensor(N, dtype=torch.int32, device="cuda")
    return imgs, keys, x, kt, b, nf


CASES = [
    # (tag, sides, C, P, N per image, K): sizes repeated out of order; the last key tile of an image ragged
    ("bt1", [(70, 90), (50, 60), (70, 90), (40, 44), (50, 60)], 4, 6, [150, 90, 150, 40, 90], 24),
    ("bt2", [(120, 100), (64, 64), (90, 80)], 1, 8, [200, 60, 130], 32),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("splits", [0, 3])
def test_batch_matches_single_image_path(case, splits):
    tag, sides, C, P, N, K = case
    imgs, keys, x, kt, b, nf = make_batch(tag, sides, C, P, N)
    idx, dist = glr.match_topk_batch(x, b, kt, nf, K, splits=splits)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    for i, (h, w) in enumerate(sides):
        xi = torch.from_numpy(imgs[i][None]).cuda()
        ki = torch.from_numpy(keys[i][None]).cuda()
        ref_i, ref_d = glr.match_topk(xi, P, ki, nf[i:i + 1].clone(), K, "bf16", bound_pass=-1)
        torch.cuda.synchronize()
        r0, r1 = int(b.key_off[i]), int(b.key_off[i + 1])
        np.testing.assert_array_equal(dist[r0:r1], ref_d.cpu().numpy()[0])
        np.testing.assert_array_equal(idx[r0:r1], ref_i.cpu().numpy()[0])


def test_batch_against_the_oracle():
    from test_gpu_tc import check_bf16_topk

    tag, sides, C, P, N, K = CASES[1]
    imgs, keys, x, kt, b, nf = make_batch(tag, sides, C, P, N)
    idx, dist = glr.match_topk_batch(x, b, kt, nf, K)
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    for i in range(len(sides)):
        r0 = int(b.key_off[i])
        sel = np.arange(0, N[i], max(1, N[i] // 12))
        covered = check_bf16_topk(imgs[i][None], P, keys[i][None][:, sel], K, K + 16, idx[None, r0 + sel],
                                  dist[None, r0 + sel])
        assert covered >= 0.5, covered


def test_batch_graph_replay_equals_eager():
    tag, sides, C, P, N, K = CASES[0]
    imgs, keys, x, kt, b, nf = make_batch(tag, sides, C, P, N)
    want_i, want_d = glr.match_topk_batch(x, b, kt, nf, K)
    lib = glr.L.load()
    o = glr.match_opts("bf16")
    import ctypes

    ws = torch.empty(int(lib.glr_workspace_size_batch(ctypes.byref(b.c), K, ctypes.byref(o))) + 256,
                     dtype=torch.uint8, device="cuda")
    idx = torch.empty_like(want_i)
    dist = torch.empty_like(want_d)
    glr.match_topk_batch(x, b, kt, nf, K, idx=idx, dist=dist, ws=ws)  # warm-up (kernel attributes) before capture
    torch.cuda.synchronize()
    idx.fill_(-1)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            glr.match_topk_batch(x, b, kt, nf, K, idx=idx, dist=dist, ws=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(idx, want_i) and torch.equal(dist, want_d)


def test_batch_rejects_what_it_does_not_cover():
    _, sides, C, P, N, K = CASES[0]
    b = glr.Batch(sides, C, P, N)
    x = torch.zeros(b.total_pixels, device="cuda")
    kt = torch.zeros(b.total_keys, dtype=torch.int32, device="cuda")
    nf = torch.tensor(N, dtype=torch.int32, device="cuda")
    lib = glr.L.load()
    import ctypes

    o = glr.match_opts("fp32")
    assert lib.glr_workspace_size_batch(ctypes.byref(b.c), K, ctypes.byref(o)) == 0
    bad = glr.Batch([(50, 60), (50, 60)], C, P, [90, 91])  # one size, two key counts
    assert lib.glr_workspace_size_batch(ctypes.byref(bad.c), K, None) == 0
    with pytest.raises(glr.GlrError):
        glr.match_topk_batch(x, b, kt, nf, 129)
