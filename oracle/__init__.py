"""FP64 CPU oracle for hyperedge effective-resistance estimation (HyperEF 2.0).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark import this package.  The GPU library never calls it and
shares no code with it.
"""
from .hef_oracle import *  # noqa: F401,F403
