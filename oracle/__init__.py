"""FP64 CPU oracle of covariance-driven SSI with randomized SVD.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
arm of ``bench.py`` use it.  It shares no code with the CUDA library.
"""
from .ssi_oracle import *  # noqa: F401,F403
from .ssi_oracle import __all__  # noqa: F401
