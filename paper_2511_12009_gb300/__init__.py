"""GB300-native exact N-Queens counting (Yao & Li, arXiv 2511.12009).

The counting path -- prefix enumeration, the persistent depth-first search
kernel, the per-prefix and per-warp reductions -- lives in libnq (C++/CUDA,
sm_103a), exposed through the C ABI in include/nq.h. ``nq`` is its thin
Python binding.
"""
from . import nq  # noqa: F401

__all__ = ["nq"]
