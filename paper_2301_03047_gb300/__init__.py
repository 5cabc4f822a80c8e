"""GB300-native global low-rank (GLR) denoising for compressed imaging.

The compute path is the C-ABI library ``libglr.so`` (hand-written CUDA for
sm_103a, built in-tree by ``__graft_entry__.build()``); ``glr`` is its thin
Python binding (argument marshalling only).  PyTorch provides device memory
and streams.
"""
__all__ = ["glr", "synth"]
