"""Training and evaluation of the learned sub-mesh force correction.

Workload: 256^3 particles in a 500 Mpc/h box on a 256^3 mesh, Newtonian mode,
Zel'dovich/BBKS initial conditions at z = 100, the 100-step schedule to z = 0.
Training pairs: for each seed, at the chosen steps, the network inputs of the
coarse step and the target from the same particles solved on a 512^3 mesh.
Evaluation on a held-out seed: the plain 256^3-mesh run, the corrected run and
the 512^3-mesh run of the same particles, compared at z = 0 by P(k) (all three
measured on one 256^3 mesh) and by the rms particle displacement from the
512^3-mesh run, with the step times of the three.

Every computation runs in libpm's kernels through the C ABI; this module only
marshals buffers and runs the loops.

    python -m paper_2607_17929_gb300.correction --seeds 32 --iters 600 --out result.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

N, BOX, OM, H, ZI, NSTEPS = 256, 500.0, 0.31, 0.67, 100.0, 100


def _wrap(torch, ptr, nbytes):
    """uint8 CUDA tensor over a device buffer owned by the library (no copy)."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


def initial_conditions(pm, torch, n, box, seed):
    probe = pm.PM(8, 8, box, OM, ZI, 0.0, NSTEPS, pm.PM_MIXED, pm.PM_NEWTONIAN)
    a_n, dtau, _ = probe.schedule()
    probe.close()
    from . import ics
    pos, mom = ics.zeldovich_ics(n, box, OM, H, a_n[0], ics.a_half_step_before(a_n[0], dtau[0], OM, box), seed)
    return torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda(), a_n


def make_pairs(pm, torch, net, seeds, snap_steps, n=N, box=BOX, log=print):
    """[(inputs BF16 [cell][16] as uint8 bytes, target FP32 [cell][8])] for every seed and snapshot step."""
    pairs = []
    inp = _wrap(torch, pm.pm_net_buffer(net, pm.PM_NET_INPUT), 32 * n ** 3)
    p = torch.empty((n ** 3, 3), dtype=torch.float64, device="cuda")
    u = torch.empty_like(p)
    for seed in seeds:
        t0 = time.perf_counter()
        pos, mom, a_n = initial_conditions(pm, torch, n, box, seed)
        coarse = pm.PM(n, n ** 3, box, OM, ZI, 0.0, NSTEPS, pm.PM_MIXED, pm.PM_NEWTONIAN)
        coarse.set_particles(pos, mom)
        del pos, mom
        for k in range(NSTEPS):
            coarse.project()
            coarse.solve()
            if k in snap_steps:
                pm.pm_get_particles(coarse.ctx, p, u)
                a = a_n[k]
                fine = pm.PM(2 * n, n ** 3, box, OM, 1.0 / a - 1.0, 0.0, NSTEPS - k, pm.PM_MIXED, pm.PM_NEWTONIAN)
                fine.set_particles(p, u)
                fine.project()
                fine.solve()
                tgt = torch.empty((n ** 3, 8), dtype=torch.float32, device="cuda")
                pm.pm_net_target(net, coarse.ctx, fine.ctx, tgt)
                pm.pm_net_features(net, coarse.ctx)
                torch.cuda.synchronize()
                pairs.append((inp.clone(), tgt, seed, k))
                fine.close()
                del fine
            coarse.update()
        coarse.close()
        torch.cuda.synchronize()
        log(f"seed {seed}: {len(snap_steps)} pairs in {time.perf_counter() - t0:.1f} s")
    return pairs


def calibrate(pm, torch, net, seed, snap_steps, n=N, box=BOX):
    """Set the network's input and target normalisation to the inverse rms of one seed's pairs."""
    pm.pm_net_set_scales(net, 1.0, 1.0, 1.0)
    pairs = make_pairs(pm, torch, net, [seed], snap_steps, n, box, log=lambda *_: None)
    x = np.concatenate([p[0].view(torch.bfloat16).view(-1, 16)[:, :2].float().cpu().numpy() for p in pairs])
    t = np.concatenate([p[1][:, :3].cpu().numpy() for p in pairs])
    rms = np.sqrt(np.mean(x.astype(np.float64) ** 2, axis=0))
    rt = float(np.sqrt(np.mean(t.astype(np.float64) ** 2)))
    scales = (1.0 / rms[0], 1.0 / rms[1], 1.0 / rt)
    pm.pm_net_set_scales(net, *scales)
    return scales


def train(pm, torch, net, pairs, iters, lr0=1e-3, lr1=3e-5, seed=0, log=print):
    """Adam on random pairs with a cosine learning-rate schedule; returns the loss history."""
    inp = _wrap(torch, pm.pm_net_buffer(net, pm.PM_NET_INPUT), pairs[0][0].numel())
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(iters):
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * it / max(iters - 1, 1)))
        x, t, _, _ = pairs[rng.integers(len(pairs))]
        inp.copy_(x)
        losses.append(pm.pm_net_train_step(net, t, lr, want_loss=(it % 10 == 0 or it == iters - 1)))
        if it % 100 == 0:
            log(f"iter {it}: loss {losses[-1]:.4e} lr {lr:.2e}")
    return [l for l in losses if l is not None]


def explained_variance(pm, torch, net, pairs):
    """1 - MSE / mean(target^2) of the network on pairs (the fraction of the force error it removes)."""
    inp = _wrap(torch, pm.pm_net_buffer(net, pm.PM_NET_INPUT), pairs[0][0].numel())
    out = []
    for x, t, seed, k in pairs:
        inp.copy_(x)
        mse = pm.pm_net_backward(net, t)   # forward + loss; the accumulated gradient is discarded below
        var = float((t[:, :3].double() ** 2).mean())
        out.append({"seed": seed, "step": k, "mse": mse, "target_ms": var, "explained": 1.0 - mse / var})
    grad = _wrap(torch, pm.pm_net_buffer(net, pm.PM_NET_GRAD), 4 * pm.pm_net_param_count())
    grad.zero_()
    return out


def evaluate(pm, torch, net, seed, n=N, box=BOX, log=print):
    """Plain, corrected and 2x-mesh runs of one seed to z = 0: P(k) and displacement errors, step times."""
    pos, mom, _ = initial_conditions(pm, torch, n, box, seed)
    runs = {}
    for name in ("plain", "corrected", "fine"):
        nm = 2 * n if name == "fine" else n
        sim = pm.PM(nm, n ** 3, box, OM, ZI, 0.0, NSTEPS, pm.PM_MIXED, pm.PM_NEWTONIAN)
        sim.set_particles(pos, mom)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(NSTEPS):
            sim.project()
            sim.solve()
            if name == "corrected":
                pm.pm_net_apply(net, sim.ctx)
            sim.update()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / NSTEPS
        p = torch.empty((n ** 3, 3), dtype=torch.float64, device="cuda")
        u = torch.empty_like(p)
        pm.pm_get_particles(sim.ctx, p, u)
        runs[name] = {"pos": p, "ms_per_step": ms}
        sim.close()
        log(f"{name}: {ms:.2f} ms/step")
    # P(k) of the three particle sets on one 256^3 mesh
    meas = pm.PM(n, n ** 3, box, OM, ZI, 0.0, NSTEPS, pm.PM_MIXED, pm.PM_NEWTONIAN)
    meas.set_particles(pos, mom)
    zero = torch.zeros_like(mom)
    nb = n // 2 + 1
    spectra = {}
    for name, r in runs.items():
        meas.put_particles(r["pos"], zero)
        k, pk, nmodes = meas.power_spectrum(nb)
        spectra[name] = pk
    meas.close()
    kny = n // 2
    res = {"seed": seed, "ms_per_step": {k: v["ms_per_step"] for k, v in runs.items()}}
    for name in ("plain", "corrected"):
        ratio = spectra[name][1:] / spectra["fine"][1:]
        d = (runs[name]["pos"] - runs["fine"]["pos"] + 0.5) % 1.0 - 0.5
        res[name] = {
            "rms_displacement_error_cells": float(torch.sqrt((d ** 2).sum(1).mean()) * n),
            "pk_ratio_max_dev_k_le_kny_2": float(np.max(np.abs(ratio[: kny // 2] - 1.0))),
            "pk_ratio_max_dev_k_le_kny": float(np.max(np.abs(ratio[:kny] - 1.0))),
            "pk_ratio_at_kny_2": float(ratio[kny // 2 - 1]),
            "pk_ratio_at_kny": float(ratio[kny - 1]),
        }
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--val-seeds", type=int, default=2)
    ap.add_argument("--snap-steps", default="90,99")
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--eval-seed", type=int, default=5000)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    from . import pm
    n = args.n
    box = BOX * n / N
    snaps = {int(s) for s in args.snap_steps.split(",")}
    net = pm.pm_net_create(n, 1)
    t0 = time.perf_counter()
    scales = calibrate(pm, torch, net, 999, snaps, n, box)
    pairs = make_pairs(pm, torch, net, list(range(1000, 1000 + args.seeds)), snaps, n, box)
    val = make_pairs(pm, torch, net, list(range(3000, 3000 + args.val_seeds)), snaps, n, box)
    t_pairs = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(pm, torch, net, pairs, args.iters)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    ev_train = explained_variance(pm, torch, net, pairs[:4])
    ev_val = explained_variance(pm, torch, net, val)
    del pairs, val
    torch.cuda.empty_cache()
    result = evaluate(pm, torch, net, args.eval_seed, n, box)
    out = {"n": n, "box_mpch": box, "seeds": args.seeds, "scales": scales, "snap_steps": sorted(snaps), "iters": args.iters,
           "pairs_seconds": round(t_pairs, 1), "train_seconds": round(t_train, 1),
           "train_ms_per_iter": round(1e3 * t_train / args.iters, 2),
           "loss_first_last": [losses[0], losses[-1]], "explained_train": ev_train, "explained_val": ev_val,
           "eval": result}
    print(json.dumps(out), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    pm.pm_net_destroy(net)


if __name__ == "__main__":
    main()
