"""Column-pass shapes of the FFT (pm_fft_shapes): every shape computes the same transform, the tuner
keeps one of them, and contexts without a choice keep shape 0."""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def inputs(pm, n, box):
    probe = pm.PM(8, 8, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    a_n, dtau, _ = probe.schedule()
    probe.close()
    return ics.zeldovich_ics(n, box, OM, H, a_n[0], ics.a_half_step_before(a_n[0], dtau[0], OM, box), 8)


@pytest.mark.parametrize("n", [64, 128])
def test_every_shape_gives_the_same_step(pm, n):
    """Two steps with each y and z shape: the fields agree with the default shapes to the level at which
    two mixed-precision runs of the same shapes agree (the k = 0 sum is accumulated with atomics)."""
    box = 4.0 * n
    pos, mom = inputs(pm, n, box)
    out = {}
    for ys, zs in [(0, 0), (0, 0), (1, 0), (2, 0), (0, 1), (0, 2), (2, 2)]:
        s = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
        assert pm.pm_fft_shapes(s.ctx, ys, zs) == (ys, zs)
        s.set_particles(pos, mom)
        s.step()
        s.step()
        f = {k: s.field(k) for k in ("phi", "chi", "Bx")}
        s.close()
        out.setdefault((ys, zs), []).append(f)
    ref, rep = out[(0, 0)]
    noise = max(rel(rep[k], ref[k]) for k in ref)
    for key, (f,) in ((k, v) for k, v in out.items() if k != (0, 0)):
        for k in ref:
            assert rel(f[k], ref[k]) <= max(10 * noise, 1e-6), (key, k, rel(f[k], ref[k]), noise)


def test_tuner_keeps_a_valid_shape_and_fp64_has_no_choice(pm):
    s = pm.PM(128, 64 ** 3, 500.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    y, z = pm.pm_fft_shapes(s.ctx)
    assert 0 <= y <= 2 and 0 <= z <= 2
    assert pm.pm_fft_shapes(s.ctx, 1, 2) == (1, 2)
    assert pm.pm_fft_shapes(s.ctx, -2, -2) == (1, 2)
    with pytest.raises(pm.PMError):
        pm.pm_fft_shapes(s.ctx, 3, 0)
    s.close()
    d = pm.PM(64, 32 ** 3, 500.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
    assert pm.pm_fft_shapes(d.ctx, 2, 2) == (0, 0)
    d.close()
    r = pm.PM(48, 32 ** 3, 500.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    assert pm.pm_fft_shapes(r.ctx) == (0, 0)
    r.close()
