"""glr_aggregate_noalloc: the aggregation entry point for callers that cannot allocate.

Callers such as a plug-in inside a framework that owns every device allocation,
or a real-time loop with a fixed memory budget, have no workspace to pass; this
entry point uses a fixed 16 MiB scratch array reserved by the library instead.
The test calls it through the C ABI twice in a row (the scratch keeps the first
call's contents, so the second call checks that everything that must start at
zero is cleared) and compares each result with glr_aggregate's, within the
tolerance of the other aggregation tests.  This file runs last so that a
failure here cannot stop the rest of the GPU suite.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2301_03047_gb300 import _lib as L  # noqa: E402
from paper_2301_03047_gb300 import glr, synth  # noqa: E402


def _inputs(tag, F, C, H, W, P, N, K):
    rng = synth.rng_for(tag)
    x = torch.from_numpy(rng.random((F, C, H, W)).astype(np.float32)).cuda()
    npos = (H - P + 1) * (W - P + 1)
    idx = torch.from_numpy(rng.integers(0, npos, size=(F, N, K)).astype(np.int32)).cuda()
    g = torch.from_numpy(rng.random((F, N, K, C * P * P)).astype(np.float32)).cuda()
    nf = torch.full((F,), N, dtype=torch.int32, device="cuda")
    return x, idx, g, nf


def _noalloc(lib, g, idx, nf, x, P, out):
    F, C, H, W = x.shape
    im = L.GlrImages(F, C, H, W, P)
    N, K = idx.shape[1], idx.shape[2]
    return lib.glr_aggregate_noalloc(g.data_ptr(), idx.data_ptr(), nf.data_ptr(), ctypes.byref(im), N, K,
                                     x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_workspace_entry_point_twice():
    lib = L.load()
    for case in (("na1", 2, 1, 40, 44, 8, 30, 12), ("na2", 1, 3, 21, 23, 4, 17, 9)):
        tag, F, C, H, W, P, N, K = case
        x, idx, g, nf = _inputs(tag, F, C, H, W, P, N, K)
        want = glr.aggregate(g, idx, nf, x, P)
        for _ in range(2):
            out = torch.full_like(x, float("nan"))
            assert _noalloc(lib, g, idx, nf, x, P, out) == L.GLR_OK
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), want.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = L.load()
    x = torch.zeros((4, 1, 1024, 1024), dtype=torch.float32, device="cuda")  # 16 MiB of planes alone
    idx = torch.zeros((4, 1, 1), dtype=torch.int32, device="cuda")
    g = torch.zeros((4, 1, 1, 64), dtype=torch.float32, device="cuda")
    nf = torch.ones(4, dtype=torch.int32, device="cuda")
    out = torch.empty_like(x)
    assert _noalloc(lib, g, idx, nf, x, 8, out) == L.GLR_ETOOBIG
    assert b"16 MiB" in lib.glr_status_string(L.GLR_ETOOBIG)


def test_noalloc_accepts_a_problem_of_exactly_its_scratch():
    """320 x 4369 pixels with P = 1 need exactly the 16 MiB of scratch (the host-side test
    computes this from the documented formula): accepted, and equal to glr_aggregate."""
    lib = L.load()
    x, idx, g, nf = _inputs("na_exact", 1, 1, 320, 4369, 1, 50, 3)
    want = glr.aggregate(g, idx, nf, x, 1)
    out = torch.full_like(x, float("nan"))
    assert _noalloc(lib, g, idx, nf, x, 1, out) == L.GLR_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), want.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_noalloc_reports_a_bad_index_through_poll_status():
    """A match id outside the position grid is skipped and recorded in the status block of the
    scratch array, which glr_poll_status(NULL, ...) reads; the next clean call clears it."""
    lib = L.load()
    x, idx, g, nf = _inputs("na_bad", 1, 1, 30, 34, 6, 10, 4)
    npos = (30 - 6 + 1) * (34 - 6 + 1)
    bad = idx.clone()
    bad[0, 3, 2] = npos  # one past the last position
    out = torch.empty_like(x)
    assert _noalloc(lib, g, bad, nf, x, 6, out) == L.GLR_OK
    bits, _ = glr.poll_status(None)
    assert bits & L.GLR_DEV_BAD_INDEX
    assert _noalloc(lib, g, idx, nf, x, 6, out) == L.GLR_OK
    bits, _ = glr.poll_status(None)
    assert bits == 0
