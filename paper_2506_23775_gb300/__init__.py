"""GB300-native matrix-free Riemannian circuit optimiser (sm_103a CUDA).

The compute path lives in ``_lib/librq.so`` (C ABI in ``include/rq.h``);
``rq`` is its ctypes binding.  Build with ``_build.build()``.
"""
from .rq import Context, RQError, tr_state, load  # noqa: F401
