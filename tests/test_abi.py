"""The C-ABI library loads here (no GPU), exports every symbol include/glr.h declares,
and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2301_03047_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_03047_gb300 import build_lib

    build_lib.build()
    return L.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "glr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glr_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.PROTOTYPES), "binding and header disagree"


def test_status_strings_and_version(lib):
    assert lib.glr_status_string(0) == b"GLR_OK"
    assert b"workspace" in lib.glr_status_string(3)
    assert b"sm_103a" in lib.glr_version()
    assert lib.glr_launch_count() == 0


def test_workspace_size_validation(lib):
    im = L.GlrImages(2, 1, 64, 64, 8)
    assert lib.glr_workspace_size(L.GLR_OP_SELECT, ctypes.byref(im), 100, 10, None) > 0
    assert lib.glr_workspace_size(L.GLR_OP_MATCH, ctypes.byref(im), 100, 10, None) > 0
    assert lib.glr_workspace_size(L.GLR_OP_MATCH, ctypes.byref(im), 100, 0, None) == 0
    bad = L.GlrImages(2, 1, 64, 64, 70)  # P > H
    assert lib.glr_workspace_size(L.GLR_OP_SELECT, ctypes.byref(bad), 10, 1, None) == 0
    assert lib.glr_workspace_size(L.GLR_OP_SELECT, ctypes.byref(im), 57 * 57 + 1, 1, None) == 0
    assert lib.glr_workspace_size(99, ctypes.byref(im), 10, 1, None) == 0
    # low-rank step: status block + the FP64 fallback's queue (one int32 per group)
    small = lib.glr_workspace_size(L.GLR_OP_LOWRANK, ctypes.byref(im), 100, 10, None)
    large = lib.glr_workspace_size(L.GLR_OP_LOWRANK, ctypes.byref(im), 4000, 10, None)
    assert 256 + 2 * 100 * 4 <= small < large and large >= 256 + 2 * 4000 * 4
    assert lib.glr_workspace_size(L.GLR_OP_LOWRANK, ctypes.byref(im), 0, 10, None) == 0


def test_entry_points_reject_bad_arguments_on_host(lib):
    im = L.GlrImages(1, 1, 32, 32, 8)
    p = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    assert lib.glr_select_keys(None, ctypes.byref(im), 0.1, 10, p, p, None, p, 1 << 20, None) == L.GLR_EINVAL
    assert lib.glr_select_keys(p, ctypes.byref(im), 0.1, 0, p, p, None, p, 1 << 20, None) == L.GLR_EINVAL
    assert lib.glr_select_keys(p, ctypes.byref(im), -1.0, 10, p, p, None, p, 1 << 20, None) == L.GLR_EINVAL
    assert lib.glr_select_keys(p, ctypes.byref(im), 0.1, 10, p, p, None, p, 16, None) == L.GLR_ENOMEM
    assert lib.glr_select_keys(p, ctypes.byref(im), 0.1, 10, p, p, None, ctypes.c_void_p(258), 1 << 30, None) == L.GLR_EINVAL
    o = L.GlrMatchOpts()
    o.mode = 7
    assert lib.glr_match_topk(p, ctypes.byref(im), p, p, 10, 5, ctypes.byref(o), p, p, p, 1 << 30, None) == L.GLR_EINVAL
    o.mode = 0
    assert lib.glr_match_topk(p, ctypes.byref(im), p, p, 10, 626, ctypes.byref(o), p, p, p, 1 << 30, None) == L.GLR_EINVAL
    assert lib.glr_match_topk(p, ctypes.byref(im), p, p, 10, 200, ctypes.byref(o), p, p, p, 1 << 30, None) == L.GLR_ENOTSUP
    assert lib.glr_lowrank_groups(p, ctypes.byref(im), p, p, 10, 5, -1.0, 1.0, p, None, p, 1 << 20, None) == L.GLR_EINVAL
    assert lib.glr_aggregate(p, p, p, ctypes.byref(im), 10, 5, p, p, p, 1 << 20, None) == L.GLR_EINVAL  # v_out aliases groups
    assert lib.glr_gap_step(p, p, 0, None, 1, 0, 8, 8, 0, None, p, None) == L.GLR_EINVAL
    assert lib.glr_gap_step(p, p, 0, None, 1, 2, 8, 8, 1, None, p, None) == L.GLR_EINVAL  # accelerate needs y_acc
    assert lib.glr_launch_count() == 0


def _noalloc_bytes(n, C, H, W, P):
    """Scratch of glr_aggregate_noalloc as its header states it: 256 + n C H W 8 + n Hq Wq 4,
    each part rounded up to 256 bytes."""
    up = lambda v: (v + 255) // 256 * 256
    return 256 + up(n * C * H * W * 8) + up(n * (H - P + 1) * (W - P + 1) * 4)


def test_noalloc_scratch_limit_on_host(lib):
    """One column past the 16 MiB scratch is rejected before anything touches the device.
    320 x 4369 with P = 1 needs exactly 16 MiB (accepted: checked on the GPU by
    tests/test_zz_no_alloc.py); 320 x 4370 needs 3840 bytes more."""
    assert _noalloc_bytes(1, 1, 320, 4369, 1) == 16 << 20
    assert _noalloc_bytes(1, 1, 320, 4370, 1) > 16 << 20
    p = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    over = L.GlrImages(1, 1, 320, 4370, 1)
    assert lib.glr_aggregate_noalloc(p, p, p, ctypes.byref(over), 1, 1, p, ctypes.c_void_p(512), None) == L.GLR_ETOOBIG
    # a second image doubles the planes: far over
    two = L.GlrImages(2, 1, 320, 4369, 1)
    assert lib.glr_aggregate_noalloc(p, p, p, ctypes.byref(two), 1, 1, p, ctypes.c_void_p(512), None) == L.GLR_ETOOBIG
    assert lib.glr_launch_count() == 0
