"""Failure handling and determinism on the GPU: an injected allocation failure (host-side test hook)
leaves no leak and no broken state; the same FP64 step twice agrees to rounding (the order of
atomic additions is the only nondeterminism)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_17929_gb300 import ics

pytestmark = pytest.mark.gpu

OM, H = 0.31, 0.67


@pytest.fixture(scope="module")
def pm():
    import torch  # noqa: F401
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm as m
    return m


def test_injected_allocation_failure_releases_everything(pm):
    import torch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in (1, 6, 12, 18):
        os.environ["PM_TEST_FAIL_ALLOC"] = str(k)
        try:
            with pytest.raises(pm.PMError) as err:
                pm.PM(64, 64 ** 3, 640.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
            assert err.value.status == pm.PM_ERR_OOM
        finally:
            del os.environ["PM_TEST_FAIL_ALLOC"]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20, (free0, free1)
    g = pm.PM(64, 64 ** 3, 640.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)   # a normal context still works
    g.close()


def test_fp64_steps_are_deterministic_to_rounding(pm):
    n = 32
    s = O.OracleSim(n, n ** 3, OM, 320.0, 100.0, 0.0, 100)
    a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], OM, s.h0)
    pos, mom = ics.zeldovich_ics(n, 320.0, OM, H, s.a_n[0], a_m, 12)
    runs = []
    for _ in range(2):
        g = pm.PM(n, n ** 3, 320.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
        g.set_particles(pos, mom)
        for _ in range(3):
            g.step()
        p, u = g.particles()
        runs.append((p, u, g.field("phi"), g.field("chi")))
        g.close()
    (p1, u1, f1, c1), (p2, u2, f2, c2) = runs
    assert np.max(np.abs((p1 - p2 + 0.5) % 1.0 - 0.5)) < 1e-14
    for a, b in ((u1, u2), (f1, f2), (c1, c2)):
        assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(b)
