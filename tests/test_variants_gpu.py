"""Parity of the two solve variants with the FP64 oracle, through the C ABI:
PM_FULL_HC (the remainder of Eq. fullHc in the phi source) and PM_B_SPACESPACE
(B_i integrated from the spin-1 part of Eq. spacespace).  FP64 bar: 1e-11
relative L2 on every field, the tensor state and every particle coordinate;
mixed precision: the bounds of the plain mixed step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_17929_gb300 import ics

from mixed_bounds import mixed_violations

pytestmark = pytest.mark.gpu

OM, H = 0.31, 0.67


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def wrapdiff(a, b):
    return (np.asarray(a) - np.asarray(b) + 0.5) % 1.0 - 0.5


@pytest.fixture(scope="module")
def pm():
    import torch  # noqa: F401
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm as m
    return m


def make_pair(pm, n, n_side, box, seed, precision, full_hc=False, b_space=False):
    orc = O.OracleSim(n, n_side ** 3, OM, box, 100.0, 0.0, 100, full_hc=full_hc, b_space=b_space)
    a_m = O.a_after(orc.a_n[0], -0.5 * orc.dtau[0], OM, orc.h0)
    pos, mom = ics.zeldovich_ics(n_side, box, OM, H, orc.a_n[0], a_m, seed)
    orc.set_particles(pos, mom)
    flags = (pm.PM_FULL_HC if full_hc else 0) | (pm.PM_B_SPACESPACE if b_space else 0)
    g = pm.PM(n, len(pos), box, OM, 100.0, 0.0, 100, precision, flags)
    g.set_particles(pos, mom)
    return orc, g, pos


def compare(orc, g, n, with_f=True):
    h = n // 2 + 1
    out = {f: rel(g.field(f), orc.field(f)) for f in ("phi", "chi", "R", "Sxx", "Sxy", "Sxz", "Syy", "Syz")}
    out["B"] = rel(np.stack([g.field(c) for c in ("Bx", "By", "Bz")]),
                   np.stack([orc.field(c) for c in ("Bx", "By", "Bz")]))
    if with_f:
        for f in ("Fx", "Fy", "Fz"):
            out[f] = rel(g.field(f), orc.field(f))
    for t in ("h+", "hx", "h+'", "hx'"):
        out[t] = rel(g.tensor(t), orc.tensor(t)[:, :, :h])
    p_g, u_g = g.particles()
    p_o, u_o = orc.particles()
    out["x"] = float(np.linalg.norm(wrapdiff(p_g, p_o)) / np.linalg.norm(p_o))
    out["u"] = rel(u_g, u_o)
    return out


def run(orc, g, n, steps, b_space):
    worst = {}
    for k in range(steps):
        orc.step()
        g.step()
        # with B from Eq. spacespace, F is assembled only at step 0 (the seed of the integration)
        for key, v in compare(orc, g, n, with_f=not b_space or k == 0).items():
            worst[key] = max(worst.get(key, 0.0), v)
    return worst


@pytest.mark.parametrize("full_hc,b_space", [(True, False), (False, True), (True, True)])
def test_fp64_variants_ten_steps_32cubed(pm, full_hc, b_space):
    orc, g, _ = make_pair(pm, 32, 32, 320.0, 1, pm.PM_FP64, full_hc, b_space)
    worst = run(orc, g, 32, 10, b_space)
    g.close()
    bad = {k: v for k, v in worst.items() if not v < 1e-11}
    assert not bad, (bad, worst)


@pytest.mark.parametrize("n,n_side,box", [(24, 20, 240.0), (48, 30, 480.0)])
def test_fp64_variants_ragged_and_radix3(pm, n, n_side, box):
    orc, g, _ = make_pair(pm, n, n_side, box, 5, pm.PM_FP64, True, True)
    worst = run(orc, g, n, 3, True)
    g.close()
    assert all(v < 1e-11 for v in worst.values()), worst


def test_mixed_variants_32cubed(pm):
    """Both variants in the mixed form, the bounds of the plain mixed step (mixed_bounds.py; positions 1e-6
    cell rms)."""
    orc, g, pos = make_pair(pm, 32, 32, 320.0, 1, pm.PM_MIXED, True, True)
    worst = run(orc, g, 32, 10, True)
    p_g, _ = g.particles()
    p_o, _ = orc.particles()
    rms_cells = float(np.sqrt(np.mean(wrapdiff(p_g, p_o) ** 2)) * 32)
    g.close()
    print("mixed variants vs oracle:", {k: f"{v:.2e}" for k, v in worst.items()}, f"rms dx {rms_cells:.2e}")
    assert not mixed_violations(worst), mixed_violations(worst)
    assert rms_cells < 1e-6, rms_cells


def test_variants_act_on_the_step(pm):
    """The variants change what they should and nothing else: the full-Hc remainder moves phi by a
    second-order amount; B from Eq. spacespace equals the momentum-constraint B at step 0 and departs
    from it afterwards."""
    n = 32
    a_n, dtau, _ = O.schedule(100, 1.0 / 101.0, 1.0, OM, 320.0 / 2997.92458)
    a_m = O.a_after(a_n[0], -0.5 * dtau[0], OM, 320.0 / 2997.92458)
    pos, mom = ics.zeldovich_ics(n, 320.0, OM, H, a_n[0], a_m, 1)
    runs = {}
    for name, flags in (("plain", 0), ("hc", pm.PM_FULL_HC), ("bs", pm.PM_B_SPACESPACE)):
        g = pm.PM(n, n ** 3, 320.0, OM, 100.0, 0.0, 100, pm.PM_FP64, flags)
        g.set_particles(pos, mom)
        out = []
        for _ in range(3):
            g.step()
            out.append((g.field("phi"), np.stack([g.field(c) for c in ("Bx", "By", "Bz")])))
        runs[name] = out
        g.close()
    d_phi = rel(runs["hc"][2][0], runs["plain"][2][0])
    assert 1e-6 < d_phi < 1e-2, d_phi
    assert rel(runs["bs"][0][1], runs["plain"][0][1]) < 1e-14
    assert rel(runs["bs"][2][1], runs["plain"][2][1]) > 1e-3
    assert rel(runs["bs"][2][0], runs["plain"][2][0]) < 1e-4   # B does not feed phi within a step


def test_b_spacespace_checkpoint_resume(pm, tmp_path):
    """The integrated B_k state travels with the checkpoint."""
    n = 16
    _, g, _ = make_pair(pm, n, n, 160.0, 4, pm.PM_FP64, True, True)
    for _ in range(3):
        g.step()
    path = str(tmp_path / "variant.pmck")
    g.save(path)
    for _ in range(3):
        g.step()
    B_ref = np.stack([g.field(c) for c in ("Bx", "By", "Bz")])
    p_ref, _ = g.particles()
    h = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64, pm.PM_FULL_HC | pm.PM_B_SPACESPACE)
    h.load(path)
    for _ in range(3):
        h.step()
    B2 = np.stack([h.field(c) for c in ("Bx", "By", "Bz")])
    p2, _ = h.particles()
    assert rel(B2, B_ref) < 1e-12 and np.max(np.abs(wrapdiff(p2, p_ref))) < 1e-14
    g.close(); h.close()
