"""Batched ensemble (boxes of uneven size stepped together from one captured CUDA graph)
against the oracle box by box, and against the same boxes stepped alone, with per-box
steps and with the batched particle kernels (one deposit and one kick launch over the
(box, tile) work list of all boxes); the projection's bin shapes against each other."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_17929_gb300 import ics

pytestmark = pytest.mark.gpu

OM, H = 0.31, 0.67
BOXES = [(16, 160.0, 21), (24, 240.0, 22), (32, 300.0, 23)]


@pytest.fixture(scope="module")
def pm():
    import torch  # noqa: F401
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm as m
    return m


def _ics(n, box, seed):
    s = O.OracleSim(n, n ** 3, OM, box, 100.0, 0.0, 100)
    a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], OM, s.h0)
    pos, mom = ics.zeldovich_ics(n, box, OM, H, s.a_n[0], a_m, seed)
    return s, pos, mom


def _box_state(pm, e, b, n):
    ctx = pm.pm_ensemble_box(e, b)
    pos = np.zeros((n ** 3, 3)); mom = np.zeros((n ** 3, 3)); phi = np.zeros((n, n, n))
    pm.pm_get_particles(ctx, pos, mom)
    pm.pm_get_field(ctx, "phi", phi)
    return pos, mom, phi


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("batched", [False, True])
def test_fp64_ensemble_matches_oracle_per_box(pm, batched):
    cfgs = [dict(n_mesh=n, n_part=n ** 3, box_mpch=box, omega_m=OM, z_init=100.0, precision=pm.PM_FP64)
            for n, box, _ in BOXES]
    e = pm.pm_ensemble_init(cfgs)
    pm.pm_ensemble_set_batched(e, batched)
    sims = []
    for b, (n, box, seed) in enumerate(BOXES):
        s, pos, mom = _ics(n, box, seed)
        s.set_particles(pos, mom)
        pm.pm_ensemble_set_particles(e, b, pos, mom)
        sims.append(s)
    pm.pm_ensemble_step(e, use_graph=False)
    for _ in range(2):
        pm.pm_ensemble_step(e, use_graph=True)
    pm.pm_ensemble_sync(e)
    for b, (n, box, _) in enumerate(BOXES):
        for _ in range(3):
            sims[b].step()
        pos, mom, phi = _box_state(pm, e, b, n)
        p_o, u_o = sims[b].particles()
        dx = (pos - p_o + 0.5) % 1.0 - 0.5
        assert np.linalg.norm(dx) / np.linalg.norm(p_o) < 1e-11
        assert rel(mom, u_o) < 1e-11 and rel(phi, sims[b].field("phi")) < 1e-11
    pm.pm_ensemble_destroy(e)


@pytest.mark.parametrize("batched", [False, True])
def test_mixed_ensemble_matches_boxes_stepped_alone(pm, batched):
    specs = [(32, 300.0, 31), (64, 500.0, 32), (48, 400.0, 33), (32, 250.0, 34)]
    cfgs = [dict(n_mesh=n, n_part=n ** 3, box_mpch=box, omega_m=OM, z_init=100.0, precision=pm.PM_MIXED)
            for n, box, _ in specs]
    e = pm.pm_ensemble_init(cfgs)
    pm.pm_ensemble_set_batched(e, batched)
    pm.pm_ensemble_set_streams(e, 2)
    alone = []
    for b, (n, box, seed) in enumerate(specs):
        _, pos, mom = _ics(n, box, seed)
        pm.pm_ensemble_set_particles(e, b, pos, mom)
        g = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
        g.set_particles(pos, mom)
        alone.append(g)
    pm.pm_ensemble_step(e, use_graph=False)
    for _ in range(3):
        pm.pm_ensemble_step(e, use_graph=True)
    pm.pm_ensemble_sync(e)
    for b, (n, box, _) in enumerate(specs):
        for _ in range(4):
            alone[b].step()
        pos, mom, phi = _box_state(pm, e, b, n)
        pa, ua = alone[b].particles()
        dx = (pos - pa + 0.5) % 1.0 - 0.5
        assert np.sqrt(np.mean(dx ** 2)) * n < 1e-6
        assert rel(mom, ua) < 1e-5 and rel(phi, alone[b].field("phi")) < 1e-5
        alone[b].close()
    pm.pm_ensemble_destroy(e)


def test_fp64_deposit_shapes_agree(pm):
    """Both projection bin shapes on a clustered load (one tile holds several chunks of either size): the
    same sums up to the order of additions inside a cell."""
    n = 16
    rng = np.random.default_rng(5)
    pos = np.concatenate([(5.0 + 2.0 * rng.random((3000, 3))) / n, rng.random((1500, 3))])
    mom = rng.standard_normal(pos.shape) * 1e-4
    runs = []
    for shape in (0, 1):
        g = pm.PM(n, len(pos), 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
        g.set_particles(pos, mom)
        assert pm.pm_deposit_shape(g.ctx, shape) == shape
        for _ in range(2):
            g.step()
        runs.append((g.field("R"), g.field("Sxy"), g.particles()[1]))
        if shape == 1:
            assert pm.pm_deposit_shape(g.ctx, -1) in (0, 1)   # timing between steps changes nothing seen
            r2 = g.field("R")
            assert np.array_equal(r2, runs[1][0])
        g.close()
    for a, b in zip(runs[0], runs[1]):
        assert rel(a, b) < 1e-12


def test_mixed_ensemble_tunes(pm):
    specs = [(32, 300.0, 31), (64, 500.0, 32), (48, 400.0, 33), (32, 250.0, 34)]
    cfgs = [dict(n_mesh=n, n_part=n ** 3, box_mpch=box, omega_m=OM, z_init=100.0, precision=pm.PM_MIXED)
            for n, box, _ in specs]
    e = pm.pm_ensemble_init(cfgs)
    alone = []
    for b, (n, box, seed) in enumerate(specs):
        _, pos, mom = _ics(n, box, seed)
        pm.pm_ensemble_set_particles(e, b, pos, mom)
        g = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
        g.set_particles(pos, mom)
        alone.append(g)
    pm.pm_ensemble_step(e, use_graph=False)
    k = pm.pm_ensemble_tune(e)  # 1, 2, 4 streams, per-box and batched, three steps each
    assert k in (1, 2, 4) and pm.pm_ensemble_get_mode(e)[0] == k
    pm.pm_ensemble_step(e, use_graph=True)
    pm.pm_ensemble_sync(e)
    for b, (n, box, _) in enumerate(specs):
        done = pm.pm_get_time(pm.pm_ensemble_box(e, b))[0]
        while alone[b].time()[0] < done:
            alone[b].step()
        pos, mom, phi = _box_state(pm, e, b, n)
        pa, ua = alone[b].particles()
        dx = (pos - pa + 0.5) % 1.0 - 0.5
        # same kernels; only the summation order inside cells differs (FP32 rounding)
        assert np.sqrt(np.mean(dx ** 2)) * n < 1e-6
        assert rel(mom, ua) < 1e-5 and rel(phi, alone[b].field("phi")) < 1e-5
        alone[b].close()
    pm.pm_ensemble_destroy(e)
