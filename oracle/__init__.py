"""CPU oracle for the gDRR projection path (arXiv:1204.6367).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline and reference legs may import this package.  It shares no code
with the CUDA library and never imports it.

Parity status: every function here is pinned by a CPU test against something
other than itself (a library routine, a closed form, an invariant, or a value
printed in the paper); see tests/test_oracle_*.py.
"""
from .oracle import *  # noqa: F401,F403
