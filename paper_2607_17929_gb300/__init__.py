"""GB300-native relativistic particle-mesh step (gevolution 2.0, arxiv 2607.17929).

The compute path is libpm.so (hand-written sm_103a CUDA behind the C ABI of
include/pm.h); ``paper_2607_17929_gb300.pm`` is its ctypes binding and
``paper_2607_17929_gb300.ics`` the seeded synthetic initial conditions.
"""
