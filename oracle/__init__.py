"""FP64 CPU oracle of the cavity-QED master equation: test infrastructure only.

Only the tests, the smoke check and the bench's CPU-baseline leg import this package.
"""
from .qme import *  # noqa: F401,F403
from . import qme  # noqa: F401
