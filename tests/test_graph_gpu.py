"""pm_step as one captured CUDA graph per step (pm_step_graph) against plain pm_step launches.

The graph holds the same kernels in the same order, so both contexts compute the same step; the only
freedom is the order of the particles inside a cell, which the counting sort leaves open (its slots
come from atomics), so the deposit's sums may round differently: FP64 within 1e-12, mixed within the
FP32 bounds of the per-field parity tests.  Also: switching graph steps off and on between steps,
a graph-stepped box inside the ensemble's own capture, and the argument check.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_17929_gb300 import ics

from mixed_bounds import MIXED_BOUND

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
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def wrapdiff(a, b):
    return (np.asarray(a) - np.asarray(b) + 0.5) % 1.0 - 0.5


def _ics(n, box, seed):
    s = O.OracleSim(n, n ** 3, OM, box, 100.0, 0.0, 100)
    a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], OM, s.h0)
    return ics.zeldovich_ics(n, box, OM, H, s.a_n[0], a_m, seed)


def _errors(a, b, n):
    out = {f: rel(b.field(f), a.field(f)) for f in ("phi", "chi", "R")}
    out["B"] = rel(np.stack([b.field(c) for c in ("Bx", "By", "Bz")]), np.stack([a.field(c) for c in ("Bx", "By", "Bz")]))
    pa, ua = a.particles()
    pb, ub = b.particles()
    out["x_cells_max"] = float(np.max(np.abs(wrapdiff(pb, pa))) * n)
    out["u"] = rel(ub, ua)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_steps_match_plain_steps(pm, precision):
    n, box = 32, 320.0
    prec = pm.PM_FP64 if precision == "fp64" else pm.PM_MIXED
    pos, mom = _ics(n, box, 41)
    a = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, prec)
    b = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, prec)
    a.set_particles(pos, mom)
    b.set_particles(pos, mom)
    b.step_graph(True)
    worst = {}
    for k in range(7):
        if k == 3:
            b.step_graph(False)   # one plain step between graph steps
        if k == 4:
            b.step_graph(True)    # the graph of step 2 is updated or re-instantiated for step 4
        a.step()
        b.step()
        for key, v in _errors(a, b, n).items():
            worst[key] = max(worst.get(key, 0.0), v)
    a.close()
    b.close()
    print(precision, "graph vs plain:", {k: f"{v:.2e}" for k, v in worst.items()})
    if precision == "fp64":
        assert worst["x_cells_max"] < 1e-10 and all(v < 1e-12 for k, v in worst.items() if k != "x_cells_max"), worst
    else:
        assert worst["x_cells_max"] < 1e-5, worst
        for key in ("phi", "chi", "R", "B", "u"):
            assert worst[key] < MIXED_BOUND[key], (key, worst)


def test_graph_stepped_box_inside_the_ensemble_capture(pm):
    """A box with graph steps on, stepped by an ensemble that captures its own graph: the box's step is
    recorded into the ensemble's capture as plain launches (no nested capture)."""
    n, box = 24, 240.0
    pos, mom = _ics(n, box, 42)
    cfg = dict(n_mesh=n, n_part=n ** 3, box_mpch=box, omega_m=OM, z_init=100.0, precision=pm.PM_FP64)
    e = pm.pm_ensemble_init([cfg])
    pm.pm_ensemble_set_particles(e, 0, pos, mom)
    pm.pm_step_graph(pm.pm_ensemble_box(e, 0), 1)
    ref = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_FP64)
    ref.set_particles(pos, mom)
    for _ in range(3):
        pm.pm_ensemble_step(e, use_graph=True)
        ref.step()
    pm.pm_ensemble_sync(e)
    ctx = pm.pm_ensemble_box(e, 0)
    p = np.zeros((n ** 3, 3)); u = np.zeros((n ** 3, 3)); phi = np.zeros((n, n, n))
    pm.pm_get_particles(ctx, p, u)
    pm.pm_get_field(ctx, "phi", phi)
    pr, ur = ref.particles()
    assert float(np.max(np.abs(wrapdiff(p, pr)))) * n < 1e-10
    assert rel(u, ur) < 1e-12 and rel(phi, ref.field("phi")) < 1e-12
    ref.close()
    pm.pm_ensemble_destroy(e)


def test_graph_step_switch_rejects_other_values(pm):
    g = pm.PM(16, 16 ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    with pytest.raises(pm.PMError):
        pm.pm_step_graph(g.ctx, 2)
    g.close()
