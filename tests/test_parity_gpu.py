"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Same seeded inputs on both sides; every field, the tensor state and every
particle coordinate are compared element by element.  FP64 tolerance: 1e-11
relative L2 (the bar the plain FP64 step must meet).  Mixed precision: the
per-field bounds derived from FP32 arithmetic (see test docstrings).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_17929_gb300 import ics

from mixed_bounds import mixed_violations

pytestmark = pytest.mark.gpu

OM, H = 0.31, 0.67


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()),
                                                                               1e-300))


def wrapdiff(a, b):
    return (np.asarray(a) - np.asarray(b) + 0.5) % 1.0 - 0.5


@pytest.fixture(scope="module")
def pm():
    import torch  # noqa: F401
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm as m
    return m


def make_pair(pm, n, n_side, box, seed, precision, newtonian=False, zi=100.0, nsteps=100, pos=None, mom=None):
    orc = O.OracleSim(n, n_side ** 3 if pos is None else len(pos), OM, box, zi, 0.0, nsteps, newtonian)
    if pos is None:
        a_m = O.a_after(orc.a_n[0], -0.5 * orc.dtau[0], OM, orc.h0)
        pos, mom = ics.zeldovich_ics(n_side, box, OM, H, orc.a_n[0], a_m, seed)
    orc.set_particles(pos, mom)
    g = pm.PM(n, len(pos), box, OM, zi, 0.0, nsteps, precision, pm.PM_NEWTONIAN if newtonian else 0)
    g.set_particles(pos, mom)
    return orc, g, pos, mom


def compare(orc, g, n, full=True):
    """Relative L2 errors of every field, the tensor state and the particles."""
    h = n // 2 + 1
    out = {"phi": rel(g.field("phi"), orc.field("phi"))}
    if full:
        out["chi"] = rel(g.field("chi"), orc.field("chi"))
        out["B"] = rel(np.stack([g.field(c) for c in ("Bx", "By", "Bz")]),
                       np.stack([orc.field(c) for c in ("Bx", "By", "Bz")]))
        for src in ("R", "Fx", "Fy", "Fz", "Sxx", "Sxy", "Sxz", "Syy", "Syz"):
            out[src] = rel(g.field(src), orc.field(src))
        for t in ("h+", "hx", "h+'", "hx'"):
            out[t] = rel(g.tensor(t), orc.tensor(t)[:, :, :h])
    p_g, u_g = g.particles()
    p_o, u_o = orc.particles()
    out["x"] = float(np.linalg.norm(wrapdiff(p_g, p_o)) / np.linalg.norm(p_o))
    out["u"] = rel(u_g, u_o)
    return out


def test_fp64_bootstrap_matches(pm):
    orc, g, *_ = make_pair(pm, 32, 32, 320.0, 1, pm.PM_FP64)
    assert rel(g.field("phi"), orc.field("phi")) < 1e-11
    assert rel(g.field("R"), orc.field("R")) < 1e-11
    g.close()


def test_fp64_ten_steps_32cubed(pm):
    """32^3 mesh and particles, 320 Mpc/h, z_i = 100, first 10 steps of the 100-step schedule."""
    orc, g, *_ = make_pair(pm, 32, 32, 320.0, 1, pm.PM_FP64)
    a_g, dt_g, ah_g = g.schedule()
    assert np.max(np.abs(a_g - orc.a_n) / orc.a_n) < 1e-14
    assert np.max(np.abs(dt_g - orc.dtau) / orc.dtau) < 1e-13
    assert np.max(np.abs(ah_g - orc.a_half) / orc.a_half) < 1e-14
    worst = {}
    for _ in range(10):
        orc.step()
        g.step()
        e = compare(orc, g, 32)
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
    g.close()
    bad = {k: v for k, v in worst.items() if not v < 1e-11}
    assert not bad, (bad, worst)


@pytest.mark.parametrize("n,n_side,box,newtonian", [(24, 20, 240.0, False), (16, 7, 160.0, False),
                                                    (24, 21, 240.0, True), (48, 30, 480.0, False),
                                                    (64, 40, 640.0, False), (128, 50, 1000.0, True)])
def test_fp64_ragged_and_radix3(pm, n, n_side, box, newtonian):
    """Mesh sizes with a factor 3, particle counts that are not n^3, sparse loads, Newtonian mode."""
    orc, g, *_ = make_pair(pm, n, n_side, box, 5, pm.PM_FP64, newtonian=newtonian)
    for _ in range(3 if n <= 48 else 2):
        orc.step()
        g.step()
    e = compare(orc, g, n, full=not newtonian)
    g.close()
    assert all(v < 1e-11 for v in e.values()), e


def test_fp64_clustered_tile_needs_several_chunks(pm):
    """5000 particles inside 2^3 cells: one tile holds far more particles than one shared-memory chunk."""
    n = 16
    rng = np.random.default_rng(3)
    pos = np.concatenate([(5.0 + 2.0 * rng.random((5000, 3))) / n, rng.random((2000, 3))])
    mom = rng.standard_normal(pos.shape) * 1e-4
    orc, g, *_ = make_pair(pm, n, 0, 160.0, 0, pm.PM_FP64, pos=pos, mom=mom)
    for _ in range(2):
        orc.step()
        g.step()
    e = compare(orc, g, n)
    g.close()
    assert all(v < 1e-11 for v in e.values()), e


def test_mixed_clustered_tile_needs_several_chunks(pm):
    """The mixed form on the clustered load above (5000 particles in 2^3 cells: one tile takes several
    960-particle chunks) against the FP64 oracle, with the mixed bounds of the 32^3 test."""
    n = 16
    rng = np.random.default_rng(3)
    pos = np.concatenate([(5.0 + 2.0 * rng.random((5000, 3))) / n, rng.random((2000, 3))])
    mom = rng.standard_normal(pos.shape) * 1e-4
    orc, g, *_ = make_pair(pm, n, 0, 160.0, 0, pm.PM_MIXED, pos=pos, mom=mom)
    worst = {}
    for _ in range(2):
        orc.step()
        g.step()
        for k, v in compare(orc, g, n).items():
            worst[k] = max(worst.get(k, 0.0), v)
    g.close()
    print("mixed clustered vs oracle worst rel L2:", {k: f"{v:.2e}" for k, v in worst.items()})
    assert not mixed_violations(worst), mixed_violations(worst)


def test_fp64_newtonian_zero_net_momentum(pm):
    n = 32
    orc, g, pos, mom = make_pair(pm, n, n, 320.0, 2, pm.PM_FP64, newtonian=True)
    g.step()
    _, u1 = g.particles()
    du = u1 - mom
    assert np.linalg.norm(du.sum(0)) <= 1e-12 * np.abs(du).sum()
    g.close()


def test_device_and_host_inputs_agree(pm):
    import torch
    n = 16
    orc = O.OracleSim(n, n ** 3, OM, 160.0, 100.0, 0.0, 100)
    pos, mom = ics.zeldovich_ics(n, 160.0, OM, H, orc.a_n[0], orc.a_n[0], 9)
    a = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
    b = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
    a.set_particles(pos, mom)
    b.set_particles(torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda())
    a.step(); b.step()
    pa, ua = a.particles()
    pd = torch.zeros((n ** 3, 3), dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(pd)
    pm.pm_get_particles(b.ctx, pd, ud)
    torch.cuda.synchronize()
    assert np.max(np.abs(wrapdiff(pa, pd.cpu().numpy()))) < 1e-14
    assert rel(ua, ud.cpu().numpy()) < 1e-13
    a.close(); b.close()


def test_pinned_host_buffers_agree_with_device_buffers(pm):
    """Pinned host arrays are read and written by the kernels in place (no staging copy): same result as
    device arrays, both directions, and non-finite input is still rejected."""
    import torch
    n = 16
    orc = O.OracleSim(n, n ** 3, OM, 160.0, 100.0, 0.0, 100)
    pos, mom = ics.zeldovich_ics(n, 160.0, OM, H, orc.a_n[0], orc.a_n[0], 10)
    a = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    b = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    a.set_particles(torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda())
    hp, hu = torch.from_numpy(pos).pin_memory(), torch.from_numpy(mom).pin_memory()
    b.set_particles(hp, hu)
    pd = torch.zeros((n ** 3, 3), dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(pd)
    ph = torch.zeros((n ** 3, 3), dtype=torch.float64).pin_memory()
    uh = torch.zeros_like(ph).pin_memory()
    pm.pm_get_particles(a.ctx, pd, ud)
    pm.pm_get_particles(b.ctx, ph, uh)
    torch.cuda.synchronize()
    assert torch.equal(pd.cpu(), ph) and torch.equal(ud.cpu(), uh)
    bad = hu.clone().pin_memory()
    bad[5, 1] = float("nan")
    with pytest.raises(pm.PMError):
        b.put_particles(hp, bad)
    a.close(); b.close()


def test_checkpoint_resume(pm, tmp_path):
    n = 16
    orc, g, pos, mom = make_pair(pm, n, n, 160.0, 4, pm.PM_FP64)
    for _ in range(3):
        g.step()
    path = str(tmp_path / "state.pmck")
    g.save(path)
    for _ in range(3):
        g.step()
    p_ref, u_ref = g.particles()
    phi_ref = g.field("phi")
    h = pm.PM(n, n ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
    h.load(path)
    assert h.time()[0] == 3
    for _ in range(3):
        h.step()
    p2, u2 = h.particles()
    assert np.max(np.abs(wrapdiff(p2, p_ref))) < 1e-14
    assert rel(u2, u_ref) < 1e-12 and rel(h.field("phi"), phi_ref) < 1e-12
    # a corrupted file is refused
    raw = bytearray(open(path, "rb").read())
    raw[-100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    with pytest.raises(pm.PMError):
        h.load(path)
    g.close(); h.close()


def test_power_spectrum_matches_oracle(pm):
    n = 32
    orc, g, pos, mom = make_pair(pm, n, n, 320.0, 6, pm.PM_FP64)
    k_g, pk_g, nm_g = g.power_spectrum(12)
    rho = O.deposit_mass(n, pos, OM / n ** 3)
    k_o, pk_o, nm_o = O.power_spectrum(rho, OM, 12)
    assert np.array_equal(nm_g, nm_o)
    assert rel(pk_g[1:], pk_o[1:]) < 1e-11
    assert rel(k_g[1:], k_o[1:]) < 1e-13
    g.close()


def test_mixed_precision_ten_steps_32cubed(pm):
    """Mixed form against the FP64 oracle, every field within its bound in mixed_bounds.py (about five
    times the worst measured value; each bound is derived there from the FP32 arithmetic).  Positions are
    cell + f32 offset: each drift rounds the offset to 2^-24 of a cell, so after 10 steps the rms
    position error stays below 10 * 2^-24 ~ 6e-7 cell plus the f32 velocity error times the displacement."""
    orc, g, pos, mom = make_pair(pm, 32, 32, 320.0, 1, pm.PM_MIXED)
    worst = {}
    for _ in range(10):
        orc.step()
        g.step()
        e = compare(orc, g, 32)
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
    p_g, _ = g.particles()
    p_o, _ = orc.particles()
    disp = np.linalg.norm(wrapdiff(p_o, pos))
    dx = np.linalg.norm(wrapdiff(p_g, p_o)) / disp
    rms_cells = float(np.sqrt(np.mean(wrapdiff(p_g, p_o) ** 2)) * 32)
    g.close()
    print("mixed vs oracle worst rel L2:", {k: f"{v:.2e}" for k, v in worst.items()},
          f"dx/disp {dx:.2e} rms dx {rms_cells:.2e} cell")
    assert not mixed_violations(worst), mixed_violations(worst)
    assert rms_cells < 1e-6 and dx < 1e-4


@pytest.mark.parametrize("n,n_side,box,newtonian", [(64, 64, 640.0, False), (128, 48, 1280.0, True)])
def test_mixed_precision_tuned_fft_sizes(pm, n, n_side, box, newtonian):
    """Mixed form at sizes whose FP32 column passes use the tuned shapes (16 points per thread on
    z lines), against the FP64 oracle with the bounds of the 32^3 mixed test."""
    orc, g, pos, mom = make_pair(pm, n, n_side, box, 8, pm.PM_MIXED, newtonian=newtonian)
    for _ in range(2):
        orc.step()
        g.step()
    e = compare(orc, g, n, full=not newtonian)
    p_g, _ = g.particles()
    p_o, _ = orc.particles()
    rms_cells = float(np.sqrt(np.mean(wrapdiff(p_g, p_o) ** 2)) * n)
    g.close()
    print(f"mixed {n}^3 vs oracle:", {k: f"{v:.2e}" for k, v in e.items()}, f"rms dx {rms_cells:.2e} cell")
    assert not mixed_violations(e), mixed_violations(e)
    assert rms_cells < 1e-6, rms_cells


def test_packed_particle_io(pm):
    """Packed records (int32 cell, f32 offsets, f32 momenta: the mixed form's own precision) in and out:
    they reproduce the f64 view exactly, a context started from them steps like one started from f64,
    pinned host records are read and written in place, and invalid records or an FP64 context are refused."""
    import torch
    n, box = 16, 160.0
    orc = O.OracleSim(n, n ** 3, OM, box, 100.0, 0.0, 100)
    pos, mom = ics.zeldovich_ics(n, box, OM, H, orc.a_n[0], orc.a_n[0], 12)
    a = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    a.set_particles(pos, mom)
    rec = np.zeros(n ** 3, dtype=pm.PACKED)
    pm.pm_get_particles_packed(a.ctx, n ** 3, rec)
    pa, ua = a.particles()
    c = rec["cell"].astype(np.int64)
    ijk = np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)
    assert np.array_equal((ijk + rec["f"].astype(np.float64)) * (1.0 / n), pa)
    assert np.array_equal(rec["u"].astype(np.float64), ua)
    assert np.all((rec["f"] >= 0) & (rec["f"] < 1))
    # a context started from the records steps like the one started from f64
    b = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    pm.pm_set_particles_packed(b.ctx, n ** 3, rec)
    for _ in range(2):
        a.step(); b.step()
    pa, ua = a.particles()
    pb, ub = b.particles()
    assert np.sqrt(np.mean(wrapdiff(pa, pb) ** 2)) * n < 1e-6 and rel(ub, ua) < 1e-5
    # pinned host records, in place, both directions, match the device-array path
    hrec = torch.from_numpy(rec.view(np.uint8).copy()).pin_memory()
    drec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    pm.pm_put_particles_packed(a.ctx, n ** 3, hrec)
    pm.pm_put_particles_packed(b.ctx, n ** 3, drec)
    a.step(); b.step()
    hout = torch.zeros(28 * n ** 3, dtype=torch.uint8).pin_memory()
    dout = torch.zeros(28 * n ** 3, dtype=torch.uint8, device="cuda")
    pm.pm_get_particles_packed(a.ctx, n ** 3, hout)
    pm.pm_get_particles_packed(b.ctx, n ** 3, dout)
    torch.cuda.synchronize()
    ra = hout.numpy().view(pm.PACKED)
    rb = dout.cpu().numpy().view(pm.PACKED)
    assert np.array_equal(ra["cell"], rb["cell"])
    assert np.max(np.abs(ra["f"] - rb["f"])) < 1e-5 and np.max(np.abs(ra["u"] - rb["u"])) < 1e-6 * np.abs(rb["u"]).max()
    # invalid records are refused
    for field, idx, value in (("f", (3, 1), 1.0), ("cell", 7, n ** 3), ("u", (5, 2), np.nan), ("f", (0, 0), -1e-8)):
        bad = rec.copy()
        bad[field][idx] = value
        with pytest.raises(pm.PMError) as ei:
            pm.pm_put_particles_packed(a.ctx, n ** 3, bad)
        assert ei.value.status == pm.PM_ERR_INVALID_ARG
        pm.pm_set_particles_packed(a.ctx, n ** 3, rec)   # the refused put left no valid state; start again
    a.close(); b.close()
    g = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_FP64)
    with pytest.raises(pm.PMError) as ei:
        pm.pm_set_particles_packed(g.ctx, n ** 3, rec)
    assert ei.value.status == pm.PM_ERR_INVALID_ARG
    g.close()


def test_overlapped_packed_io_matches_the_synchronous_calls(pm):
    """pm_put_particles_packed_async / pm_get_particles_packed_async / pm_io_wait: a loop that puts the same
    records, steps and gets the result every step, with the copies on the context's I/O streams, gives what
    the synchronous calls give; a bad record is reported by pm_io_wait and leaves no particles."""
    import torch
    n, box = 32, 320.0
    orc = O.OracleSim(n, n ** 3, OM, box, 100.0, 0.0, 100)
    pos, mom = ics.zeldovich_ics(n, box, OM, H, orc.a_n[0], orc.a_n[0], 13)
    a = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    b = pm.PM(n, n ** 3, box, OM, 100.0, 0.0, 100, pm.PM_MIXED)
    a.set_particles(pos, mom)
    b.set_particles(pos, mom)
    rec = np.zeros(n ** 3, dtype=pm.PACKED)
    pm.pm_get_particles_packed(a.ctx, n ** 3, rec)
    hin = torch.from_numpy(rec.view(np.uint8).copy()).pin_memory()
    outs_a = [np.zeros(n ** 3, dtype=pm.PACKED) for _ in range(3)]
    outs_b = [torch.zeros(28 * n ** 3, dtype=torch.uint8).pin_memory() for _ in range(3)]
    for k in range(3):
        pm.pm_put_particles_packed(a.ctx, n ** 3, hin)
        a.step()
        pm.pm_get_particles_packed(a.ctx, n ** 3, outs_a[k])
        pm.pm_put_particles_packed_async(b.ctx, n ** 3, hin)
        b.step()
        pm.pm_get_particles_packed_async(b.ctx, n ** 3, outs_b[k])
    pm.pm_io_wait(b.ctx)
    def positions(r):
        c = r["cell"].astype(np.int64)
        return (np.stack([c % n, (c // n) % n, c // (n * n)], axis=1) + r["f"].astype(np.float64)) / n

    for k in range(3):
        ra, rb = outs_a[k], outs_b[k].numpy().view(pm.PACKED)
        # the two runs may order the particles of a cell differently, so the deposits may round differently
        assert np.max(np.abs(wrapdiff(positions(ra), positions(rb)))) * n < 1e-5, k
        assert np.max(np.abs(ra["u"] - rb["u"])) < 1e-6 * np.abs(ra["u"]).max(), k
    # the same context still steps and reads back through the synchronous calls
    b.step()
    pb, _ = b.particles()
    assert np.all((pb >= 0) & (pb < 1))
    # a bad record: reported by the wait, after which the context has no particles
    bad = rec.copy()
    bad["f"][9, 1] = 1.5
    hbad = torch.from_numpy(bad.view(np.uint8).copy()).pin_memory()
    pm.pm_put_particles_packed_async(b.ctx, n ** 3, hbad)
    with pytest.raises(pm.PMError) as ei:
        pm.pm_io_wait(b.ctx)
    assert ei.value.status == pm.PM_ERR_INVALID_ARG
    with pytest.raises(pm.PMError) as ei:
        b.step()
    assert ei.value.status == pm.PM_ERR_STATE
    pm.pm_set_particles_packed(b.ctx, n ** 3, rec)
    pm.pm_io_wait(b.ctx)   # nothing latched any more
    a.close(); b.close()
    g = pm.PM(16, 16 ** 3, 160.0, OM, 100.0, 0.0, 100, pm.PM_FP64)
    with pytest.raises(pm.PMError) as ei:
        pm.pm_put_particles_packed_async(g.ctx, 16 ** 3, np.zeros(16 ** 3, dtype=pm.PACKED))
    assert ei.value.status == pm.PM_ERR_INVALID_ARG
    g.close()
