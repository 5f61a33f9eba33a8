"""FP64 CPU oracle of the relativistic particle-mesh step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path never does.
"""
from .oracle import OracleSim, build_oracle, lib  # noqa: F401
