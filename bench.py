#!/usr/bin/env python
"""Benchmark of one full relativistic particle-mesh step on GB300.

Workload: 512^3 mesh and 512^3 particles, periodic box 2000 Mpc/h, flat LCDM
(Omega_m = 0.31, h = 0.67), Zel'dovich initial conditions at z = 100 from a
seeded BBKS Gaussian random field (sigma_8 = 0.8), 100-step schedule in ln a;
mixed precision (int32 cell + f32 offsets, f32 fields and FFTs, f64
background, compensated cell sums, f64 k = 0 mode).  One step = projection of
all stress-energy components, forward FFTs, scalar/vector/tensor solves,
inverse FFTs, gather + kick + drift, counting sort.

Metric: particle-updates/s = particles / step time (whole job over all ranks),
timed with CUDA events on the library's stream over K steps after W warm-up
steps.  The FP64 path is timed on the same workload for the mixed-vs-FP64
speed-up.  ``--impl reference`` times the FP64 CPU oracle instead.

Multi-GPU: independent replicas (the step does not shard without exchange
steps), one box per rank, weak scaling; no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OM, H, ZI, SEED = 0.31, 0.67, 100.0, 3
N_STEPS_SCHEDULE = 100
CELL_MPCH = 2000.0 / 512  # comoving cell size of the workload

# kernels whose compulsory DRAM bytes are modelled (per launch)
KERNELS = ["project", "fft_fwd_x", "fft_fwd_y", "fft_fwd_z", "solve", "fft_inv_z", "fft_inv_y", "fft_inv_x",
           "kick_drift", "scan", "scatter"]
KERNEL_SOURCE = {"project": "pm_particles.cu", "kick_drift": "pm_particles.cu", "scan": "pm_particles.cu",
                 "scatter": "pm_particles.cu", "solve": "pm_solve.cu"}


def kernel_bytes(name, n, n_part, mixed):
    """Compulsory DRAM bytes of one launch: every input read once, every output written once."""
    ts = 4 if mixed else 8
    cs = 2 * ts
    ps = 32 if mixed else 64
    nc = n ** 3
    nh = n * n * (n // 2 + 1)
    return {
        "project": ps * n_part + 4 * (nc + 1) + 3 * ts * nc + 9 * ts * nc,
        "fft_fwd_x": 9 * ts * nc + 9 * cs * nh,
        "fft_fwd_y": 2 * 9 * cs * nh,
        "fft_fwd_z": 2 * 9 * cs * nh,
        "solve": 9 * cs * nh + 5 * cs * nh + 2 * 4 * cs * nh,
        "fft_inv_z": 2 * 5 * cs * nh,
        "fft_inv_y": 2 * 5 * cs * nh,
        "fft_inv_x": 5 * cs * nh + 5 * ts * nc,
        "kick_drift": 2 * ps * n_part + 5 * ts * nc + 8 * nc,
        "scan": 4 * nc + 4 * (nc + 1),
        "scatter": 2 * ps * n_part + 4 * nc + 8 * nc,
    }[name]


def method_bytes_per_update(mixed):
    """Minimum bytes per particle update of the method (140 B/particle + 288 B/cell mixed; twice for FP64)."""
    return 428.0 if mixed else 816.0


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha(fname):
    p = os.path.join(ROOT, "paper_2607_17929_gb300", "csrc", fname)
    try:
        return hashlib.sha256(open(p, "rb").read()).hexdigest()[:12]
    except OSError:
        return None


def ncu_traffic(kernel, n, n_part, mixed):
    """DRAM bytes per launch from the committed ncu summary, scaled to this launch, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) < 6 or line.startswith("#"):
            continue
        kname, prec, ncap, bytes_cap, src, sha = parts[:6]
        if kname != kernel or prec != ("mixed" if mixed else "fp64"):
            continue
        if source_sha(src) != sha:
            return None
        scale = (n ** 3) / float(int(ncap) ** 3)
        return float(bytes_cap) * scale
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = str(device_index)
        try:  # address the physical GPU by PCI bus id when torch exposes it
            import torch
            pr = torch.cuda.get_device_properties(device_index)
            self.dev = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis and vis.split(",")[0].strip().isdigit():
                self.dev = vis.split(",")[0].strip()
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def make_ics(n, box, seed, a0, a_m):
    from paper_2607_17929_gb300 import ics
    return ics.zeldovich_ics(n, box, OM, H, a0, a_m, seed)


def half_step_back(a0, dtau0, box):
    """a at tau_0 - dtau_0/2 from the library's own schedule scalars."""
    from paper_2607_17929_gb300 import ics
    return ics.a_half_step_before(a0, dtau0, OM, box)


ENSEMBLE_SIDES = (64,) * 16 + (128,) * 16 + (192,) * 16


def ensemble_specs():
    """48 boxes of uneven size: 16 each at 64^3, 128^3 and 192^3 mesh with one particle per cell; box b has
    seed 1000 + b and a box length drawn uniformly from 200-1000 Mpc/h by a generator seeded with that seed."""
    import numpy as np
    return [(n, float(np.random.default_rng(1000 + b).uniform(200.0, 1000.0)), 1000 + b)
            for b, n in enumerate(ENSEMBLE_SIDES)]


def ensemble_bench(pm, torch, steps, warmup):
    """boxes*steps/s of the batched ensemble (one captured graph per step; the autotuner picks the FFT and
    deposit shapes per mesh size, the stream count and per-box or batched particle kernels) against looping
    the single-box pm_step over the same boxes on one stream, and the mode the tuner did not pick.  Inputs
    resident in HBM."""
    specs = ensemble_specs()
    inputs = []
    t_ic = time.perf_counter()
    for n, box, seed in specs:
        probe = pm.PM(8, 8, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED)
        a_n, dtau, _ = probe.schedule()
        probe.close()
        pos, mom = make_ics(n, box, seed, a_n[0], half_step_back(a_n[0], dtau[0], box))
        inputs.append((torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda()))
    t_ic = time.perf_counter() - t_ic
    nb = len(specs)

    # looping the single-box path: one context per box, all on one stream, pm_step box after box
    stream = torch.cuda.current_stream()
    sims = []
    for (n, box, _), (p, u) in zip(specs, inputs):
        g = pm.PM(n, n ** 3, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED, 0, stream)
        g.set_particles(p, u)
        sims.append(g)
    for _ in range(warmup):
        for g in sims:
            g.step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        for g in sims:
            g.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    loop_ms = ev0.elapsed_time(ev1) / steps
    for g in sims:
        g.close()
    del sims
    torch.cuda.empty_cache()

    # the ensemble: one graph per step on k streams
    cfgs = [dict(n_mesh=n, n_part=n ** 3, box_mpch=box, omega_m=OM, z_init=ZI, n_steps=N_STEPS_SCHEDULE,
                 precision=pm.PM_MIXED) for n, box, _ in specs]
    e = pm.pm_ensemble_init(cfgs)
    for b, (p, u) in enumerate(inputs):
        pm.pm_ensemble_set_particles(e, b, p, u)
    pm.pm_ensemble_step(e, use_graph=False)
    k = pm.pm_ensemble_tune(e)
    _, tuned_batched = pm.pm_ensemble_get_mode(e)
    shapes, dep_shapes = {}, {}
    for b, (n, _, _) in enumerate(specs):
        if n not in shapes:
            shapes[n] = pm.pm_fft_shapes(pm.pm_ensemble_box(e, b), -2, -2)
            dep_shapes[n] = pm.pm_deposit_shape(pm.pm_ensemble_box(e, b), -2)
    es = torch.cuda.ExternalStream(pm.pm_ensemble_stream(e))

    def run(batched, use_graph):
        pm.pm_ensemble_set_batched(e, batched)
        for _ in range(warmup):
            pm.pm_ensemble_step(e, use_graph=use_graph)
        pm.pm_ensemble_sync(e)
        ev0.record(es)
        t0 = time.perf_counter()
        for _ in range(steps):
            pm.pm_ensemble_step(e, use_graph=use_graph)
        ev1.record(es)
        pm.pm_ensemble_sync(e)
        wall = 1e3 * (time.perf_counter() - t0) / steps
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / steps, wall

    ens_ms, wall_ms = run(tuned_batched, True)            # the tuner's choice
    other_ms, _ = run(not tuned_batched, True)            # the other particle-kernel mode, same streams
    nog_ms, _ = run(tuned_batched, False)                 # the tuner's choice without graphs
    pm.pm_ensemble_destroy(e)
    del inputs
    torch.cuda.empty_cache()
    part = sum(n ** 3 for n, _, _ in specs)
    return {"metric": "boxes*steps/s", "value": nb / (ens_ms * 1e-3), "ms_per_step": ens_ms,
            "host_wall_ms_per_step": wall_ms, "loop_value": nb / (loop_ms * 1e-3), "loop_ms_per_step": loop_ms,
            "speedup_over_loop": loop_ms / ens_ms, "streams": k, "no_graph_ms_per_step": nog_ms,
            "batched_particle_kernels": tuned_batched,
            ("per_box_ms_per_step" if tuned_batched else "batched_ms_per_step"): other_ms,
            "fft_shapes": {str(n): list(v) for n, v in shapes.items()},
            "deposit_shapes": {str(n): v for n, v in dep_shapes.items()},
            "particle_updates_per_s": part / (ens_ms * 1e-3), "steps": steps, "warmup": warmup,
            "config": "48 boxes: 16 x 64^3, 16 x 128^3, 16 x 192^3 mesh, one particle per cell, box U(200,1000) "
                      "Mpc/h, seeds 1000+b, mixed precision, same Zel'dovich/BBKS recipe at z=100",
            "ic_seconds": round(t_ic, 1)}


def correction_bench(pm, torch, reps=20, train=True):
    """Learned force correction at its 256^3 workload (500 Mpc/h, Newtonian): network forward (4 conv layers on
    the tensor cores), one training step, and the plain vs corrected step, all timed with CUDA events; then a
    short training run and its gain on two held-out seeds (rms displacement and P(k) against the 512^3-mesh run
    of the same particles)."""
    n, box = 256, 500.0
    probe = pm.PM(8, 8, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED, pm.PM_NEWTONIAN)
    a_n, dtau, _ = probe.schedule()
    probe.close()
    pos, mom = make_ics(n, box, 1234, a_n[0], half_step_back(a_n[0], dtau[0], box))
    sim = pm.PM(n, n ** 3, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED, pm.PM_NEWTONIAN)
    sim.set_particles(torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda())
    net = pm.pm_net_create(n, 1)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(k):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / k

    plain_ms = timed(sim.step, reps)

    def corrected():
        sim.project()
        sim.solve()
        pm.pm_net_apply(net, sim.ctx)
        sim.update()
    corr_ms = timed(corrected, reps)
    fwd_ms = timed(lambda: pm.pm_net_forward(net), reps)
    tgt = torch.zeros((n ** 3, 8), dtype=torch.float32, device="cuda")
    train_ms = timed(lambda: pm.pm_net_backward(net, tgt, want_loss=False), 5)
    sim.close()
    pm.pm_net_destroy(net)
    gain = None
    if train:
        # what the trained network gains: trained on 8 seeds (snapshots at steps 90 and 99), evaluated on two
        # held-out seeds against the plain 256^3 run, both compared with the 512^3-mesh run of the same particles
        from paper_2607_17929_gb300 import correction as CR
        t0 = time.perf_counter()
        tnet = pm.pm_net_create(n, 1)
        snaps = {90, 99}
        CR.calibrate(pm, torch, tnet, 999, snaps, n, box)
        pairs = CR.make_pairs(pm, torch, tnet, list(range(1000, 1008)), snaps, n, box, log=lambda *_: None)
        losses = CR.train(pm, torch, tnet, pairs, 600, log=lambda *_: None)
        ev_val = CR.explained_variance(pm, torch, tnet, CR.make_pairs(pm, torch, tnet, [3000], snaps, n, box,
                                                                       log=lambda *_: None))
        del pairs
        torch.cuda.empty_cache()
        evals = [CR.evaluate(pm, torch, tnet, s, n, box, log=lambda *_: None) for s in (5000, 5001)]
        pm.pm_net_destroy(tnet)
        gain = {"training": "8 seeds (1000-1007), snapshots at steps 90 and 99, 600 Adam steps; validation seed 3000",
                "loss_first_last": [round(losses[0], 4), round(losses[-1], 4)],
                "explained_variance_validation": [round(e["explained"], 3) for e in ev_val],
                "held_out": [{"seed": e["seed"],
                              **{k: {kk: round(vv, 4) for kk, vv in e[k].items()} for k in ("plain", "corrected")},
                              "ms_per_step": {k: round(v, 3) for k, v in e["ms_per_step"].items()}} for e in evals],
                "seconds": round(time.perf_counter() - t0, 1)}
        torch.cuda.empty_cache()
    cells = n ** 3
    # algorithmic work of the network, and the MMA work the kernels issue: layer 1 packs 8 offsets x 2
    # channels per k16 step (4 steps), layers 2-3 16 x 16 per offset, layer 4 16 x 8 per offset
    useful = 2 * 27 * cells * (2 * 16 + 16 * 16 + 16 * 16 + 16 * 3)
    issued = 2 * cells * (64 * 16 + 2 * 27 * 16 * 16 + 27 * 16 * 8)
    peak = load_bf16_peak()
    return {"workload": "256^3 mesh and particles, 500 Mpc/h, Newtonian, mixed; network 2-16-16-16-3, 3^3 conv, "
                        "BF16/FP32, He-initialised weights (timing does not depend on them)",
            "plain_step_ms": round(plain_ms, 3), "corrected_step_ms": round(corr_ms, 3), "trained_gain": gain,
            "forward_ms": round(fwd_ms, 3), "forward_backward_ms": round(train_ms, 3),
            "roofline": {"bound": "tensor", "kernel": "k_conv_in2 + k_conv_tc (4 layers)",
                         "achieved": round(useful / (fwd_ms * 1e-3) / 1e12, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(useful / (fwd_ms * 1e-3) / 1e12 / peak, 4), "flops": useful,
                         "flops_issued": issued, "issued_tflops": round(issued / (fwd_ms * 1e-3) / 1e12, 1),
                         "note": "algorithmic FLOPs of measured bf16 burst peak; layers 2-4 tcgen05.mma M128 N16 K16 "
                                 "(FP32 in TMEM), layer 1 mma.sync; with 16 output channels each MMA re-reads its "
                                 "128x16 operand from shared memory, which bounds the kernel"}}


def host_cpu():
    """CPU model and logical core count of this host (recorded beside the CPU baseline)."""
    model, arm = "", {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" not in line:
                    continue
                key, val = (x.strip() for x in line.split(":", 1))
                key = key.lower()
                if key in ("model name", "cpu model", "hardware") and not model:
                    model = val
                elif key in ("cpu implementer", "cpu part") and key not in arm:
                    arm[key] = val
    except OSError:
        pass
    import platform
    if not model and arm:   # Arm cores name themselves by implementer and part number (0x41 0xd4f: Neoverse V2)
        model = f"{platform.machine()} implementer {arm.get('cpu implementer', '?')} part {arm.get('cpu part', '?')}"
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over the ranks (the job's time is its slowest rank's); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_max):
    """Units processed by all ranks per second, timed by the slowest rank (weak scaling: each rank its own box)."""
    return world * units_per_rank / (ms_max * 1e-3)


def replica_seed(rank):
    """Seed of a rank's replica: every rank steps its own box."""
    return SEED + rank


def schedule_phases(pm, torch, n, n_part, box, d_pos, d_mom, stream, block=10):
    """The whole 100-step schedule (z = 100 -> 0) in blocks of `block` steps, each timed with CUDA events
    with its per-kernel means: clustering makes late steps costlier for the deposit and the sort."""
    sim = pm.PM(n, n_part, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED, 0, stream)
    sim.set_particles(d_pos, d_mom)
    a_n, _, _ = sim.schedule()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for b0 in range(0, N_STEPS_SCHEDULE, block):
        k = min(block, N_STEPS_SCHEDULE - b0)
        torch.cuda.synchronize()
        pm.pm_get_timings(sim.ctx)
        ev0.record(stream)
        for _ in range(k):
            sim.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        per_kernel, _ = pm.pm_get_timings(sim.ctx)
        ms = ev0.elapsed_time(ev1) / k
        out.append({"steps": f"{b0}-{b0 + k - 1}", "z": [round(1 / a_n[b0] - 1, 2), round(1 / a_n[b0 + k - 1] - 1, 3)],
                    "ms_per_step": round(ms, 3),
                    "step_roofline_frac": round(method_bytes_per_update(True) * n_part / (ms * 1e-3) / 1e9 /
                                                load_peaks()[0], 4),
                    "kernels_ms": {key: round(per_kernel[key], 3) for key in
                                   ("project", "fft_fwd", "solve", "fft_inv", "kick_drift", "sort")}})
    sim.close()
    return out


def config2_bench(pm, torch, n=256, box=1000.0, seed=2, checkpoints=(10, 50, 100), nbins=None):
    """FP64 against mixed precision over the whole 100-step schedule (z = 100 -> 0) at 256^3 mesh and
    particles in a 1 Gpc/h box: per-stage ms and per-kernel GB/s of both forms, and the relative L2 of each
    mixed field against the FP64 GPU path at steps 10, 50 and 100, and P(k) at z = 0.  Both contexts step in
    lockstep from the same Zel'dovich/BBKS initial conditions; field differences are taken on the device."""
    stream = torch.cuda.current_stream()
    probe = pm.PM(8, 8, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, pm.PM_MIXED)
    a_n, dtau, _ = probe.schedule()
    probe.close()
    pos, mom = make_ics(n, box, seed, a_n[0], half_step_back(a_n[0], dtau[0], box))
    d_pos, d_mom = torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda()
    del pos, mom
    sims = {name: pm.PM(n, n ** 3, box, OM, ZI, 0.0, N_STEPS_SCHEDULE, prec, 0, stream)
            for name, prec in (("fp64", pm.PM_FP64), ("mixed", pm.PM_MIXED))}
    for g in sims.values():
        g.set_particles(d_pos, d_mom)
    nc = n ** 3
    nh = n * n * (n // 2 + 1)
    bufs = {k: torch.empty(nc, dtype=torch.float64, device="cuda") for k in ("fp64", "mixed")}
    tbufs = {k: torch.empty(2 * nh, dtype=torch.float64, device="cuda") for k in ("fp64", "mixed")}
    pbufs = {k: (torch.empty((n ** 3, 3), dtype=torch.float64, device="cuda"),
                 torch.empty((n ** 3, 3), dtype=torch.float64, device="cuda")) for k in ("fp64", "mixed")}

    def rel_field(get, names, bb):
        num = den = 0.0
        for nm in names:
            for k in ("fp64", "mixed"):
                get(sims[k].ctx, nm, bb[k])
            num += float(torch.sum((bb["mixed"] - bb["fp64"]) ** 2))
            den += float(torch.sum(bb["fp64"] ** 2))
        return math.sqrt(num / den) if den > 0 else 0.0

    errors = {}
    ms = {k: [] for k in sims}
    kern = {k: {} for k in sims}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in sims:
        pm.pm_get_timings(sims[k].ctx)
    done = 0
    for cp in checkpoints:
        for k, g in sims.items():
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(cp - done):
                g.step()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms[k].append((cp - done, ev0.elapsed_time(ev1)))
            per, _ = pm.pm_get_timings(g.ctx)
            for key, v in per.items():
                kern[k][key] = kern[k].get(key, 0.0) + v * (cp - done)
        done = cp
        e = {"phi": rel_field(pm.pm_get_field, ["phi"], bufs), "chi": rel_field(pm.pm_get_field, ["chi"], bufs),
             "B": rel_field(pm.pm_get_field, ["Bx", "By", "Bz"], bufs),
             "h": rel_field(pm.pm_get_tensor, ["h+", "hx"], tbufs)}
        for k in sims:
            pm.pm_get_particles(sims[k].ctx, *pbufs[k])
        torch.cuda.synchronize()
        dx = torch.remainder(pbufs["mixed"][0] - pbufs["fp64"][0] + 0.5, 1.0) - 0.5
        disp = torch.remainder(pbufs["fp64"][0] - d_pos + 0.5, 1.0) - 0.5
        e["x_rms_cells"] = float(torch.sqrt(torch.mean(dx ** 2))) * n
        e["x_rel_to_displacement"] = float(torch.linalg.norm(dx) / torch.linalg.norm(disp))
        e["u"] = float(torch.linalg.norm(pbufs["mixed"][1] - pbufs["fp64"][1]) / torch.linalg.norm(pbufs["fp64"][1]))
        errors[f"step_{cp}"] = {key: float(f"{v:.3e}") for key, v in e.items()}
    nb = nbins or n // 2
    pk = {k: pm.pm_power_spectrum(g.ctx, nb) for k, g in sims.items()}
    kk, p64, nm = pk["fp64"]
    _, pmx, _ = pk["mixed"]
    half = [b for b in range(1, nb) if nm[b] > 0 and b <= n // 4]
    dev = [abs(pmx[b] / p64[b] - 1.0) for b in half]
    peak = load_peaks()[0]
    out = {"workload": f"{n}^3 mesh, {n}^3 particles, box {box:.0f} Mpc/h, seed {seed}, LCDM Om={OM} h={H}, "
                       f"z = 100 -> 0 in {N_STEPS_SCHEDULE} steps, FP64 and mixed in lockstep from the same ICs",
           "errors_mixed_vs_fp64": errors,
           "pk_z0_max_rel_dev_to_half_nyquist": float(f"{max(dev):.3e}"),
           "pk_z0": {"k": [round(float(kk[b]), 4) for b in half], "fp64": [float(f"{p64[b]:.6e}") for b in half],
                     "mixed_over_fp64_minus_1": [float(f"{pmx[b] / p64[b] - 1.0:.3e}") for b in half]}}
    for k in sims:
        steps = sum(c for c, _ in ms[k])
        step_ms = sum(t for _, t in ms[k]) / steps
        km = {key: v / steps for key, v in kern[k].items()}
        mixed = k == "mixed"
        gbs = {key: round(kernel_bytes(key, n, n ** 3, mixed) / (km[key] * 1e-3) / 1e9, 1)
               for key in KERNELS if km.get(key, 0) > 0.01}
        out[k] = {"ms_per_step": round(step_ms, 3), "particle_updates_per_s": n ** 3 / (step_ms * 1e-3),
                  "kernels_ms": {key: round(v, 4) for key, v in km.items()},
                  "kernels_gbs": gbs, "step_roofline_frac": round(
                      method_bytes_per_update(mixed) * n ** 3 / (step_ms * 1e-3) / 1e9 / peak, 4)}
    out["speedup_mixed_over_fp64"] = round(out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"], 2)
    for g in sims.values():
        g.close()
    return out


def _load_cufft():
    import ctypes
    import glob
    import torch
    names = ["libcufft.so.12", "libcufft.so"]
    names += glob.glob(os.path.join(os.path.dirname(torch.__file__), "..", "nvidia", "*", "lib", "libcufft.so*"))
    names += glob.glob("/usr/local/cuda/lib64/libcufft.so*")
    for nm in names:
        try:
            return ctypes.CDLL(nm)
        except OSError:
            continue
    return None


def cufft_bench(torch, n, reps=5):
    """cuFFT on the transforms one step makes: batched r2c of the 9 source fields and c2r of the 5 force
    fields, n^3, out of place (c2r overwrites its input; the values do not change the timing).  A
    comparison for the hand-written passes only; the step never calls it."""
    import ctypes
    lib = _load_cufft()
    if lib is None:
        return {"unavailable": "libcufft not found"}
    R2C, C2R, D2Z, Z2D = 0x2A, 0x2C, 0x6A, 0x6C
    stream = torch.cuda.current_stream()
    out = {}
    for name, dt, kf, ki in (("f32", torch.float32, R2C, C2R), ("f64", torch.float64, D2Z, Z2D)):
        x = torch.randn((9, n, n, n), dtype=dt, device="cuda")
        X = torch.empty((9, n, n, n // 2 + 1), dtype=torch.complex64 if dt == torch.float32 else torch.complex128,
                        device="cuda")
        dims = (ctypes.c_int * 3)(n, n, n)
        plans = []
        for kind, batch in ((kf, 9), (ki, 5)):
            h = ctypes.c_int()
            rc = lib.cufftPlanMany(ctypes.byref(h), 3, dims, None, 1, 0, None, 1, 0, kind, batch)
            if rc != 0:
                return {"unavailable": f"cufftPlanMany returned {rc}"}
            lib.cufftSetStream(h, ctypes.c_void_p(stream.cuda_stream))
            plans.append(h)
        execf = lib.cufftExecR2C if dt == torch.float32 else lib.cufftExecD2Z
        execi = lib.cufftExecC2R if dt == torch.float32 else lib.cufftExecZ2D
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        res = {}
        for key, fn in (("fwd_ms", lambda: execf(plans[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(X.data_ptr()))),
                        ("inv_ms", lambda: execi(plans[1], ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(x.data_ptr())))):
            for _ in range(3):
                if fn() != 0:
                    return {"unavailable": f"cuFFT exec failed ({name} {key})"}
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            res[key] = round(ev0.elapsed_time(ev1) / reps, 4)
        for h in plans:
            lib.cufftDestroy(h)
        out[name] = res
        del x, X
        torch.cuda.empty_cache()
    return out


def load_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def cpu_oracle_rate(n, steps, box, threads=1):
    """Particle updates per second of the FP64 C oracle on an n^3 sample; threads = 0 uses every core (the
    oracle's independent loops carry OpenMP pragmas; results do not depend on the thread count)."""
    from oracle import oracle as O
    O.set_threads(threads)
    s = O.OracleSim(n, n ** 3, OM, box, ZI, 0.0, N_STEPS_SCHEDULE)
    a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], OM, s.h0)
    pos, mom = make_ics(n, box, SEED, s.a_n[0], a_m)
    s.set_particles(pos, mom)
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step()
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt, dt, O.set_threads(threads)


METRIC = "particle-updates/s per full PM step at 512^3 (mixed precision)"


def workload_config(n, box, warmup, steps, world, n_sched=N_STEPS_SCHEDULE):
    return {"workload": f"relativistic PM step, {n}^3 mesh, {n}^3 particles, box {box:.0f} Mpc/h, "
                        f"LCDM Om={OM} h={H}, Zel'dovich/BBKS ICs z={ZI:.0f}, seed {SEED}, "
                        f"steps {warmup}..{warmup + steps - 1} of a {n_sched}-step schedule",
            "precision": "mixed: int32 cell + f32 offset, f32 fields/FFT, f64 background and k=0, "
                         "compensated cell sums",
            "components": "T00, 3 T0i, 5 trace-free Tij; phi, chi, B_i, h (2 helicities)",
            "parallelism": f"replicas x{world}", "l2": "working set ~25 GB >> 129 MB L2, no flush"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on all host cores, on a bounded sample of the workload (a 64^3
    box with the benchmark's cell size, same recipe); config.workload names that sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 64
    box = CELL_MPCH * n
    from oracle import oracle as O
    cores = O.set_threads(0)
    s = O.OracleSim(n, n ** 3, OM, box, ZI, 0.0, N_STEPS_SCHEDULE)
    a_m = O.a_after(s.a_n[0], -0.5 * s.dtau[0], OM, s.h0)
    pos, mom = make_ics(n, box, SEED, s.a_n[0], a_m)
    s.set_particles(pos, mom)
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt
    sample = (f"{args.steps} oracle steps of the same recipe at {n}^3 (box {box:.0f} Mpc/h, the cell size of the "
              f"{args.n}^3 benchmark box), steps {args.warmup}..{args.warmup + args.steps - 1}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "particle-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(n, box, args.warmup, args.steps, args.gpus),
                       precision="FP64 throughout (the oracle's plain C loops and FFT)",
                       l2="host run, no GPU", parallelism=f"OpenMP, {cores} host threads",
                       sampled_from=f"the {args.n}^3 mesh / {args.n}^3 particle benchmark workload"),
        "cpu_baseline": {"value": value, "unit": "particle-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample + f"; the FP64 CPU oracle on {cores} threads", "host": host_cpu()},
        "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pm", choices=["pm", "reference"])
    ap.add_argument("--n", type=int, default=512, help="mesh side (particles = n^3)")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=10, help="steps of the synchronous end-to-end loops")
    ap.add_argument("--e2e-async-steps", type=int, default=None,
                    help="steps of the overlapped end-to-end loop (the line's e2e; default: --steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-correction", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="correction leg without its training run and gain")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-phases", action="store_true")
    ap.add_argument("--no-config2", action="store_true")
    ap.add_argument("--variant-steps", type=int, default=5)
    ap.add_argument("--ensemble-steps", type=int, default=10)
    args = ap.parse_args(argv)
    if args.e2e_async_steps is None:
        args.e2e_async_steps = args.steps
    return args


def schedule_length(args):
    """Steps of the z = 100 -> 0 schedule: the 100 of the benchmark configuration, longer only when the
    requested warm-up, timed and end-to-end steps of one context do not fit in it."""
    used = args.warmup + args.steps + 2 * (args.e2e_steps + 1) + (args.e2e_async_steps + 1) + 2
    return max(N_STEPS_SCHEDULE, used)


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2607_17929_gb300 import build
    build.build()
    from paper_2607_17929_gb300 import pm

    n = args.n
    n_part = n ** 3
    box = CELL_MPCH * n
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_ranks(x):
        return max_over_ranks(x, dist, "cuda")

    n_sched = schedule_length(args)
    # inputs: the same seeded initial conditions for every rank's replica (seed offset per rank)
    probe = pm.PM(8, 8, box, OM, ZI, 0.0, n_sched, pm.PM_MIXED)
    a_n, dtau, _ = probe.schedule()
    probe.close()
    a_m = half_step_back(a_n[0], dtau[0], box)
    t_ic = time.perf_counter()
    pos, mom = make_ics(n, box, replica_seed(rank), a_n[0], a_m)
    t_ic = time.perf_counter() - t_ic
    d_pos = torch.from_numpy(pos).cuda()
    d_mom = torch.from_numpy(mom).cuda()

    def timed_run(precision, warmup, steps, flags=0):
        sim = pm.PM(n, n_part, box, OM, ZI, 0.0, n_sched, precision, flags, stream)
        sim.set_particles(d_pos, d_mom)
        for _ in range(warmup):
            sim.step()
        torch.cuda.synchronize()
        pm.pm_get_timings(sim.ctx)  # open a fresh timing window
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(steps):
                sim.step()
            ev1.record(stream)
            torch.cuda.synchronize()
            barrier()
        ms = ev0.elapsed_time(ev1) / steps
        per_kernel, launches = pm.pm_get_timings(sim.ctx)
        return sim, ms, per_kernel, launches, clk.summary()

    sim, ms_mixed, kern, launches, clocks = timed_run(pm.PM_MIXED, args.warmup, args.steps)
    ms_max = max_ranks(ms_mixed)
    value = whole_job_rate(world, n_part, ms_max)


    # end to end through the C ABI with pinned host buffers: upload the state, step, read it back
    h_pos = torch.from_numpy(pos).pin_memory()
    h_mom = torch.from_numpy(mom).pin_memory()
    o_pos = torch.empty_like(h_pos).pin_memory()
    o_mom = torch.empty_like(h_mom).pin_memory()
    sim.put_particles(h_pos, h_mom)
    sim.step()
    pm.pm_get_particles(sim.ctx, o_pos, o_mom)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sim.put_particles(h_pos, h_mom)
        sim.step()
        pm.pm_get_particles(sim.ctx, o_pos, o_mom)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_ranks(1e3 * (time.perf_counter() - t0) / args.e2e_steps)
    # the same through the packed records (int32 cell + f32 offsets + f32 momenta, 28 bytes a particle): the
    # mixed step's own precision, so nothing it uses is lost on the way
    h_rec = torch.empty(28 * n_part, dtype=torch.uint8).pin_memory()
    pm.pm_get_particles_packed(sim.ctx, n_part, h_rec)
    o_rec = torch.empty_like(h_rec).pin_memory()
    pm.pm_put_particles_packed(sim.ctx, n_part, h_rec)
    sim.step()
    pm.pm_get_particles_packed(sim.ctx, n_part, o_rec)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pm.pm_put_particles_packed(sim.ctx, n_part, h_rec)
        sim.step()
        pm.pm_get_particles_packed(sim.ctx, n_part, o_rec)
    torch.cuda.synchronize()
    barrier()
    e2e_packed_ms = max_ranks(1e3 * (time.perf_counter() - t0) / args.e2e_steps)
    # the same loop through the overlapped calls: each step's upload and the previous step's download run
    # on copy engines beside the steps (pinned host records; every step still moves its inputs in and its
    # result out).  The loop's first upload and last download have no step beside them, so it runs as many
    # steps as the device-timed region unless told otherwise.
    pm.pm_put_particles_packed_async(sim.ctx, n_part, h_rec)
    sim.step()
    pm.pm_get_particles_packed_async(sim.ctx, n_part, o_rec)
    pm.pm_io_wait(sim.ctx)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_async_steps):
        pm.pm_put_particles_packed_async(sim.ctx, n_part, h_rec)
        sim.step()
        pm.pm_get_particles_packed_async(sim.ctx, n_part, o_rec)
    pm.pm_io_wait(sim.ctx)
    barrier()
    e2e_async_ms = max_ranks(1e3 * (time.perf_counter() - t0) / args.e2e_async_steps)
    del h_rec, o_rec
    sim.close()
    del sim

    # the same steps of the schedule as graph-replayed pm_step calls (one captured graph per step)
    gsim = pm.PM(n, n_part, box, OM, ZI, 0.0, n_sched, pm.PM_MIXED, 0, stream)
    gsim.set_particles(d_pos, d_mom)
    for _ in range(args.warmup - 1):
        gsim.step()
    gsim.step_graph(True)
    gsim.step()   # instantiates the executable graphs
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        gsim.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    graph_ms = max_ranks(ev0.elapsed_time(ev1) / args.steps)
    gsim.close()
    del gsim

    # the whole schedule in blocks of 10 steps (early vs late, clustered steps)
    phases = None
    if not args.no_phases:
        phases = schedule_phases(pm, torch, n, n_part, box, d_pos, d_mom, stream)
        torch.cuda.empty_cache()

    # FP64 vs mixed over the whole schedule at 256^3 / 1 Gpc/h
    config2 = None
    if not args.no_config2:
        config2 = config2_bench(pm, torch)
        torch.cuda.empty_cache()

    # FP64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        sim64, ms64, kern64, _, _ = timed_run(pm.PM_FP64, 2, args.fp64_steps)
        sim64.close()
        ms64 = max_ranks(ms64)
        fp64 = {"ms_per_step": ms64, "value": world * n_part / (ms64 * 1e-3),
                "speedup_mixed_over_fp64": ms64 / ms_max,
                "kernels_ms": {k: round(v, 4) for k, v in kern64.items()},
                "step_roofline_frac": method_bytes_per_update(False) * n_part / (ms64 * 1e-3) / 1e9 /
                load_peaks()[0]}
        del sim64
    torch.cuda.empty_cache()

    # the solve variants on the same workload (mixed)
    variants = None
    if not args.no_variants:
        variants = {}
        for name, flags in (("full_hc", pm.PM_FULL_HC), ("b_spacespace", pm.PM_B_SPACESPACE),
                            ("full_hc+b_spacespace", pm.PM_FULL_HC | pm.PM_B_SPACESPACE)):
            simv, msv, kernv, _, _ = timed_run(pm.PM_MIXED, 3, args.variant_steps, flags)
            simv.close()
            del simv
            msv = max_ranks(msv)
            variants[name] = {"ms_per_step": round(msv, 3), "value": world * n_part / (msv * 1e-3),
                              "kernels_ms": {k: round(v, 4) for k, v in kernv.items()}}
        torch.cuda.empty_cache()

    correction = None
    if not args.no_correction:
        correction = correction_bench(pm, torch, train=not args.no_train)
        torch.cuda.empty_cache()

    cufft = None
    if not args.no_cufft:
        cufft = cufft_bench(torch, n)
        cufft["ours_f32"] = {"fwd_ms": round(kern["fft_fwd"], 4), "inv_ms": round(kern["fft_inv"], 4)}
        if fp64 is not None:
            cufft["ours_f64"] = {"fwd_ms": fp64["kernels_ms"]["fft_fwd"], "inv_ms": fp64["kernels_ms"]["fft_inv"]}
        cufft["what"] = (f"batched 9 r2c and 5 c2r transforms of {n}^3, out of place, cuFFT plans made once; "
                         "comparison only (the step runs the hand-written passes)")

    ensemble = None
    if not args.no_ensemble:
        ensemble = ensemble_bench(pm, torch, args.ensemble_steps, 3)

    # roofline of the dominant kernel
    peak, peak_kind = load_peaks()
    dom = max(KERNELS, key=lambda k: kern.get(k, 0.0))
    alg = kernel_bytes(dom, n, n_part, True)
    achieved = alg / (kern[dom] * 1e-3) / 1e9
    src = KERNEL_SOURCE.get(dom, "pm_fft.cu")
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": ncu_traffic(dom, n, n_part, True), "algorithmic_bytes": alg,
                "launch_ms": round(kern[dom], 4)}
    live = [k for k in KERNELS if kern.get(k, 0) > 0.02]   # fused passes read ~0 ms
    per_kernel_frac = {k: round(kernel_bytes(k, n, n_part, True) / (kern[k] * 1e-3) / 1e9 / peak, 3) for k in live}
    design_bytes = sum(kernel_bytes(k, n, n_part, True) for k in live)

    cpu = None
    if rank == 0 and not args.no_cpu:
        nc_ = 96
        rate, dt, cores = cpu_oracle_rate(nc_, 2, CELL_MPCH * nc_, threads=0)
        rate1, dt1, _ = cpu_oracle_rate(nc_, 1, CELL_MPCH * nc_, threads=1)
        cpu = {"value": rate, "unit": "particle-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"2 steps of the same recipe at {nc_}^3 (box {CELL_MPCH * nc_:.0f} Mpc/h, same cell "
                         f"size) after its bootstrap, all {cores} host threads, {dt:.1f} s", "host": host_cpu(),
               "single_thread": {"value": rate1, "cores": 1, "seconds": round(dt1, 1),
                                 "sample": f"1 step at {nc_}^3 after its bootstrap"}}

    if rank == 0:
        h2d = 2 * 3 * 8 * n_part
        line = {
            "metric": METRIC,
            "value": value, "unit": "particle-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "graph_ms_per_step": round(graph_ms, 4),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(n, box, args.warmup, args.steps, world, n_sched), ic_seconds=round(t_ic, 1)),
            "kernels_ms": {k: round(v, 4) for k, v in kern.items()},
            "kernels_roofline_frac": per_kernel_frac,
            "step_roofline_frac": method_bytes_per_update(True) * n_part / (ms_max * 1e-3) / 1e9 / peak,
            "design_bytes_per_step": design_bytes,
            "design_roofline_frac": design_bytes / (ms_max * 1e-3) / 1e9 / peak,
            "roofline": roofline,
            "fp64": fp64,
            "variants": variants,
            "ensemble": ensemble,
            "correction": correction,
            "cufft_comparison": cufft,
            "schedule_phases": phases,
            "config2_fp64_vs_mixed": config2,
            "e2e": {"value": world * n_part / (e2e_async_ms * 1e-3), "unit": "particle-updates/s",
                    "ms_per_step": e2e_async_ms, "h2d_bytes_per_step": 28 * n_part, "d2h_bytes_per_step": 28 * n_part,
                    "how": "every step: pm_put_particles_packed_async from pinned host records (int32 cell, 3 f32 "
                           "offsets, 3 f32 momenta: the state the mixed step holds) + pm_step + "
                           "pm_get_particles_packed_async into pinned host memory; the copies run on copy engines "
                           "beside the steps; pm_io_wait closes the timed region",
                    "loop_steps": args.e2e_async_steps},
            "e2e_sync": {"value": world * n_part / (e2e_packed_ms * 1e-3), "unit": "particle-updates/s",
                         "ms_per_step": e2e_packed_ms, "h2d_bytes_per_step": 28 * n_part,
                         "d2h_bytes_per_step": 28 * n_part,
                         "how": "the same loop through the synchronous pm_put_particles_packed / "
                                "pm_get_particles_packed", "loop_steps": args.e2e_steps},
            "e2e_f64": {"value": world * n_part / (e2e_ms * 1e-3), "unit": "particle-updates/s", "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                        "how": "every step: pm_put_particles(pinned host f64 pos, mom) + pm_step + "
                               "pm_get_particles(pinned host f64)", "loop_steps": args.e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
