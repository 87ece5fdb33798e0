"""GB300 (sm_103a) RSVD-based covariance-driven SSI: Python binding of libssi."""
from . import _lib  # noqa: F401  (fails loudly when libssi.so is missing)
from .api import *  # noqa: F401,F403
from ._lib import SsiError  # noqa: F401,E402
