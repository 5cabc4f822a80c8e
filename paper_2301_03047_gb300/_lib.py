"""ctypes loader for the in-tree C-ABI library ``libglr.so`` (declarations mirror include/glr.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglr.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_size_t = ctypes.c_size_t
c_float = ctypes.c_float
c_void_p = ctypes.c_void_p
c_uint32_p = ctypes.POINTER(ctypes.c_uint32)

GLR_OK, GLR_EINVAL, GLR_ECUDA, GLR_ENOMEM, GLR_ETIMEDOUT, GLR_ENOTSUP, GLR_EDEVICE, GLR_ETOOBIG = range(8)
GLR_DEV_TIMEOUT, GLR_DEV_NONFINITE, GLR_DEV_SVD_NOCONV, GLR_DEV_CAND_OVERFLOW, GLR_DEV_BAD_INDEX = 1, 2, 4, 8, 16
GLR_MATCH_FP32, GLR_MATCH_BF16, GLR_MATCH_LEARNED, GLR_MATCH_EDGE, GLR_MATCH_WINDOW = 0, 1, 2, 3, 4
GLR_OP_SELECT, GLR_OP_MATCH, GLR_OP_LOWRANK, GLR_OP_AGGREGATE, GLR_OP_ENCODER, GLR_OP_ADMM = 1, 2, 3, 4, 5, 6
GLR_ENCODER_PARAMS = 5200


class GlrImages(ctypes.Structure):
    _fields_ = [("n_img", c_int32), ("C", c_int32), ("H", c_int32), ("W", c_int32), ("P", c_int32)]


class GlrMatchOpts(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("k_over", c_int32), ("splits", c_int32), ("cap", c_int32), ("encoder", c_void_p),
                ("epi_batch", c_int32), ("edge_th", c_float), ("window", c_int32), ("bound_pass", c_int32),
                ("emb_format", c_int32)]


class GlrBatch(ctypes.Structure):
    _fields_ = [("n_img", c_int32), ("C", c_int32), ("P", c_int32), ("H", c_void_p), ("W", c_void_p), ("N", c_void_p),
                ("d_H", c_void_p), ("d_W", c_void_p), ("d_pix_off", c_void_p), ("d_key_off", c_void_p)]


# name -> (restype, argtypes); every symbol declared in include/glr.h
PROTOTYPES = {
    "glr_workspace_size_batch": (c_size_t, [ctypes.POINTER(GlrBatch), c_int32, ctypes.POINTER(GlrMatchOpts)]),
    "glr_match_topk_batch": (c_int32, [c_void_p, ctypes.POINTER(GlrBatch), c_void_p, c_void_p, c_int32,
                                       ctypes.POINTER(GlrMatchOpts), c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_workspace_size": (c_size_t, [c_int32, ctypes.POINTER(GlrImages), c_int32, c_int32, ctypes.POINTER(GlrMatchOpts)]),
    "glr_select_keys": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_float, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_select_keys_mixed": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_float, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_admm_sci_step": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p, c_void_p]),
    "glr_match_topk": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, ctypes.POINTER(GlrMatchOpts), c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_debug_match_scores": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_debug_proposal_scores": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_debug_wnnm_sweep_cap": (c_int32, [c_int32]),
    "glr_debug_match_wait_ns": (ctypes.c_uint64, [ctypes.c_uint64]),
    "glr_encoder_embed": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_encoder_train_step": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_float, c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_lowrank_groups": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, c_float, c_float, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_lowrank_groups_complex": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, c_float, c_float, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_mosaic_init": (c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "glr_lowrank_aggregate": (c_int32, [c_void_p, ctypes.POINTER(GlrImages), c_void_p, c_void_p, c_int32, c_int32, c_float, c_float, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_fft2": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    "glr_admm_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_aggregate": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(GlrImages), c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "glr_aggregate_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(GlrImages), c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "glr_gap_step": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "glr_poll_status": (c_int32, [c_void_p, c_uint32_p, c_uint32_p, c_int32, c_void_p]),
    "glr_status_string": (ctypes.c_char_p, [c_int32]),
    "glr_launch_count": (ctypes.c_uint64, []),
    "glr_version": (ctypes.c_char_p, []),
    "glr_profile_enable": (c_int32, [c_int32]),
    "glr_profile_collect": (c_int32, [ctypes.c_char_p, ctypes.POINTER(c_float), ctypes.POINTER(c_int32), c_int32]),
}

_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the library (raises if it has not been built); never falls back to anything else."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
