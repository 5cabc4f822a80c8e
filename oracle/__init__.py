"""FP64 CPU oracle for the GLR hot path.

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users.  The library never imports
it and shares no code with it.
"""
from . import glr_oracle  # noqa: F401
from . import mri_oracle  # noqa: F401
from . import msfa_oracle  # noqa: F401
