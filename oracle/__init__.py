"""CPU oracle for exact butterfly counting.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline of the benchmark; the product path never imports it.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
