"""Benchmark of the FDTD hot path on one GB300 (or N replicas under torchrun).

Workload (one "step"): the soft-core Coulomb problem V = -1/sqrt(r^2 + a^2)
in a box of L = 40 Bohr radii, solved for two symmetry sectors -- the
all-symmetric sector (1s, E -> -1/2) and the A_x sector (2p_x, E -> -1/8) --
by the multi-resolution bootstrap 64^3 -> 128^3 -> 256^3 (Sec. VI): random
start on 64^3, FP32 stencil, FP64/compensated sums, check every 100 steps,
convergence of the binding energy to a part in 10^6 at every level
(Sec. V), trilinear transfer to the next level.  Every row of the hot path
runs inside the step: potential upload, symmetric random start, update
steps, sums, renormalisation + symmetry re-imposition, transfer.

metric: site updates per second (interior sites x update steps, all levels,
both sectors), whole job; "value" times the device work with V already
resident in HBM, "e2e" the same call with V in pinned host memory
(host->device copies inside the timed region) and the observables read back.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (update steps with checks on the 256^3 lattice).
"""
from __future__ import annotations

import argparse
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

METRIC = "Gsite-updates/s"
LEVELS = (64, 128, 256)
LENGTH = 40.0
SECTORS = (("1s", 0b010101), ("2p_x", 0b000010))
TOL = 1e-6
SEED = 904939
# dram__bytes_read.sum + dram__bytes_write.sum of one 256^3 stencil launch
# from an ncu capture of the current kernel, by (depth, span, tile width,
# tile height); a tuned configuration without a capture reports traffic null
TRAFFIC_256 = {(3, 54, 128, 16): 238_210_048, (3, -1, 128, 16): 237_899_008}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def potentials(resident: bool, device):
    import numpy as np
    import torch

    import workloads as wl

    out = []
    for n in LEVELS:
        v = wl.coulomb_soft(n, LENGTH).astype(np.float32)
        # host-resident: pinned (page-locked) memory, so each step's copies are plain DMA
        out.append(torch.from_numpy(v).to(device) if resident else torch.from_numpy(v).pin_memory())
    return out


def run_step(fd, pots, seed, opts):
    """Both sectors, three levels each: one handle per level holding the two
    sectors' lattices (their evolve loops run concurrently, each lattice
    upsampled from its own sector's coarser level).  Returns a dict of
    totals: site updates, kernel launches, and the stencil time / algorithmic
    bytes of the finest level (the dominant kernel), plus per-level results."""
    import torch

    tot = {"updates": 0, "launches": 0, "fine_ms": 0.0, "fine_bytes": 0.0, "fine_updates": 0,
           "fine_launches": 0, "fine_timed": 0, "results": {}, "config": None, "level_ms": {}}
    prev = None
    for lvl, n in enumerate(LEVELS):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        s = fd.Solver([fd.Lattice(n, LENGTH, fd.F32) for _ in SECTORS], opts)
        s.set_profiling(n == LEVELS[-1])
        for i, (name, mask) in enumerate(SECTORS):
            s.set_potential(pots[lvl], lat=i)
            if prev is None:
                s.init_symmetric(seed, mask, lat=i)
            else:
                s.upsample_from(prev, lat_src=i, lat=i)
        _, conv = s.evolve(2_000_000)
        st = s.stats()
        tot["launches"] += st["launches"]
        if n == LEVELS[-1]:
            tot["fine_ms"] += st["stencil_ms"]
            tot["fine_bytes"] += st["stencil_bytes"]
            tot["fine_updates"] += st["stencil_site_updates"]
            tot["fine_launches"] += st["stencil_launches"]
            tot["fine_timed"] += st["stencil_timed_launches"]
            tot["config"] = s.tuned_config() + s.tuned_kernel()
        ev1.record()
        ev1.synchronize()
        tot["level_ms"][str(n)] = ev0.elapsed_time(ev1)
        tuned = list(s.tuned_config()) + list(s.tuned_kernel())
        for i, (name, _) in enumerate(SECTORS):
            o = s.last_check(lat=i)
            tot["updates"] += n**3 * o["steps"]
            tot["results"][f"{name}_{n}"] = {"E": o["energy"], "r2": o["r2"], "steps": o["steps"],
                                             "converged": bool(o["converged"]), "level_ms": ev0.elapsed_time(ev1),
                                             "stencil": tuned}
        if prev is not None:
            prev.close()
        prev = s
    prev.close()
    return tot


def time_to_e0(fd, pots, seed, opts, dev):
    """Wall time until |E - E_ref| < 1e-6 |E_ref| per sector, E_ref being the
    plain FP64 256^3 solve converged to 1e-11 (relative): the FP32
    multi-resolution path (coarse levels to a part in 10^6, the 256^3 level in
    chunks of 100 steps until within 1e-6 of E_ref) against the plain FP64
    form from a random start on the same GB300, both timed with CUDA events
    (the checks against E_ref run on the host between chunks)."""
    import torch

    import workloads as wl

    out = {}
    v64 = torch.from_numpy(wl.coulomb_soft(LEVELS[-1], LENGTH)).to(dev)
    ref_opts = fd.default_options(check_every=100, tol=1e-11, tol_relative=1)
    chunk_opts = fd.default_options(check_every=100, tol=0.0)

    def until_within(s, e_ref, limit=400_000):
        steps, t_ms = 0, 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while steps < limit:
            e0.record()
            s.evolve(100)
            e1.record()
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            steps += 100
            if abs(s.last_check()["energy"] - e_ref) < 1e-6 * abs(e_ref):
                break
        return steps, t_ms * 1e-3

    for name, mask in SECTORS:
        r = fd.Solver(fd.Lattice(LEVELS[-1], LENGTH, fd.F64), ref_opts)
        r.set_potential(v64)
        r.init_symmetric(seed + 17, mask)
        ref_steps, _ = r.evolve(1_000_000)
        e_ref = r.last_check()["energy"]
        r.close()
        # FP32 multi-resolution
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prev = None
        for lvl, n in enumerate(LEVELS[:-1]):
            s = fd.Solver(fd.Lattice(n, LENGTH, fd.F32), opts)
            s.set_potential(pots[lvl])
            if prev is None:
                s.init_symmetric(seed, mask)
            else:
                s.upsample_from(prev)
            s.evolve(2_000_000)
            prev = s
        fine = fd.Solver(fd.Lattice(LEVELS[-1], LENGTH, fd.F32), chunk_opts)
        fine.set_potential(pots[-1])
        fine.upsample_from(prev)
        e1.record()
        torch.cuda.synchronize()
        coarse_s = e0.elapsed_time(e1) * 1e-3
        mr_steps, mr_s = until_within(fine, e_ref)
        e_mr = fine.last_check()["energy"]
        # plain FP64 from a random start
        p64 = fd.Solver(fd.Lattice(LEVELS[-1], LENGTH, fd.F64), chunk_opts)
        e0.record()
        p64.set_potential(v64)
        p64.init_symmetric(seed, mask)
        e1.record()
        torch.cuda.synchronize()
        p_steps, p_s = until_within(p64, e_ref)
        p_s += e0.elapsed_time(e1) * 1e-3
        e_p = p64.last_check()["energy"]
        out[name] = {"E_ref_fp64": e_ref, "E_ref_steps": ref_steps,
                     "fp32_multires_s": coarse_s + mr_s, "fp32_multires_fine_steps": mr_steps,
                     "fp32_multires_rel_err": abs(e_mr - e_ref) / abs(e_ref),
                     "fp64_plain_s": p_s, "fp64_plain_steps": p_steps,
                     "fp64_plain_rel_err": abs(e_p - e_ref) / abs(e_ref),
                     "speedup": p_s / (coarse_s + mr_s)}
    return out


def anisotropic_multires(fd, dev, seed):
    """The 512^3, L = 16 anisotropic workload (oscillator + 32 Gaussians):
    128^3 and 256^3 levels with BF16 storage (to 1e-4), the 512^3 level in
    FP32 to a part in 10^6."""
    import torch

    import workloads as wl

    L = 16.0
    plan = ((128, fd.BF16, 1e-4), (256, fd.BF16, 1e-4), (512, fd.F32, TOL))
    pots = [wl.anisotropic_device(n, L, dev, dtype=torch.float32) for n, _, _ in plan]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    prev, upd, levels = None, 0, {}
    for (n, prec, tol), v in zip(plan, pots):
        s = fd.Solver(fd.Lattice(n, L, prec), fd.default_options(check_every=100, tol=tol, tol_relative=1))
        s.set_potential(v)
        if prev is None:
            s.init_symmetric(seed, 0)
        else:
            s.upsample_from(prev)
        steps, conv = s.evolve(2_000_000)
        o = s.last_check()
        upd += n**3 * steps
        levels[f"{n}_{'bf16' if prec == fd.BF16 else 'f32'}"] = {"steps": steps, "E": o["energy"], "r2": o["r2"],
                                                                  "converged": conv}
        prev = s
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"levels": levels, "ms": ms, "site_updates": upd, "gsite_per_s": upd / (ms * 1e-3) / 1e9}


def backward_run(fd, dev):
    """Gradient of E w.r.t. V through 4000 unrolled FP32 steps on 128^3
    (V_theta = r^2/2 + 16 Gaussians, L = 10), sqrt(T) checkpointing: forward,
    segment recompute and adjoint, all inside fdtd_backward."""
    import numpy as np
    import torch

    import workloads as wl

    n, L, T = 128, 10.0, 4000
    g, th = wl.config_theta(n, L)
    v = torch.from_numpy(wl.v_theta(n, L, th, g).astype(np.float32)).to(dev)
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=100, tol=0.0, backward_steps=T))
    s.set_potential(v)
    s.set_psi(torch.from_numpy(np.exp(-0.5 * wl.radius2(n, L))).to(dev))
    out = torch.empty((n, n, n), dtype=torch.float64, device=dev)
    s.backward(T, 1.0, 0.0, out=out)  # warm-up
    s.set_psi(torch.from_numpy(np.exp(-0.5 * wl.radius2(n, L))).to(dev))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, obs = s.backward(T, 1.0, 0.0, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dtheta = torch.tensordot(torch.from_numpy(g).to(dev), out, dims=3).cpu().numpy()
    s.close()
    return {"n": n, "T": T, "checkpoint_every": int(np.ceil(np.sqrt(T))), "ms": ms,
            "forward_equivalent_gsite_per_s": 3 * n**3 * T / (ms * 1e-3) / 1e9, "E_T": obs["energy"],
            "dE_dtheta_first4": [float(x) for x in dtheta[:4]]}


def batched_run(fd, dev, seed):
    """The 64-lattice batch (sizes 48..160, oscillator or soft Coulomb,
    four symmetry sectors), FP32, one persistent launch to a part in 10^6."""
    import numpy as np
    import torch

    import workloads as wl

    lats = wl.config_batch()
    opts = fd.default_options(check_every=100, tol=TOL, tol_relative=1, batched=1)
    s = fd.Solver([fd.Lattice(l.n, l.length, fd.F32) for l in lats], opts)
    pots = [torch.from_numpy(l.potential().astype(np.float32)).to(dev) for l in lats]

    def start():
        for i, l in enumerate(lats):
            s.set_potential(pots[i], lat=i)
            s.init_symmetric(seed, l.mask, lat=i)

    # first solve: the autotuner times its candidates on slices of the run
    # and keeps the fastest; the timed solve uses it in one launch
    start()
    s.evolve(200_000)
    start()
    s.reset_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    steps, conv = s.evolve(200_000)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    graph_launches = s.stats()["graph_launches"]
    upd = 0
    worst = 0
    for i, l in enumerate(lats):
        o = s.last_check(lat=i)
        upd += l.n**3 * o["steps"]
        worst = max(worst, o["steps"])
    tuned = s.tuned_config()
    s.close()
    return {"lattices": len(lats), "sites": int(sum(l.n**3 for l in lats)), "site_updates": upd, "ms": ms,
            "gsite_per_s": upd / (ms * 1e-3) / 1e9, "max_steps_taken": worst, "all_converged": bool(conv),
            "launches": graph_launches, "launch": "cooperative kernel in a CUDA graph",
            "tuned": tuned}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(target_s: float = 12.0):
    """The FP64 oracle on the host cores: update steps with checks on the
    256^3 Coulomb lattice (a bounded sample of the workload)."""
    import numpy as np

    import oracle
    import workloads as wl

    n = LEVELS[-1]
    a = LENGTH / n
    v = wl.coulomb_soft(n, LENGTH)
    psi = oracle.init_symmetric(n, SEED, SECTORS[0][1])
    # per-step cost from two short runs (each call also pads/unpads the field)
    t0 = time.perf_counter()
    psi, _, _ = oracle.evolve(psi, v, a, a * a / 4, 2, 100, 0.0, False, SECTORS[0][1])
    t1 = time.perf_counter()
    psi, _, _ = oracle.evolve(psi, v, a, a * a / 4, 6, 100, 0.0, False, SECTORS[0][1])
    t2 = time.perf_counter()
    per = max((t2 - t1) - (t1 - t0), 1e-3) / 4
    steps = max(4, min(2000, int(target_s / per)))
    t0 = time.perf_counter()
    oracle.evolve(psi, v, a, a * a / 4, steps, 100, 0.0, False, SECTORS[0][1])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n**3 * steps / dt / 1e9, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 update steps with checks on the 256^3 Coulomb lattice ({dt:.1f} s)"}


def workload_config(ws: int) -> dict:
    """The workload both arms report (the reference arm times a bounded
    sample of it, described in its cpu_baseline)."""
    return {"workload": "coulomb_soft_L40_multires_64-128-256_1s+2px", "levels": list(LEVELS), "length": LENGTH,
            "tol_rel": TOL, "check_every": 100, "l2": "flushed (512 MiB write) between timed steps",
            "parallelism": f"replicas{ws}"}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; each step is independent
    vals = []
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(target_s=max(3.0, 60.0 / max(1, args.steps)))
        vals.append(cb["value"])
    value = statistics.mean(vals)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(ws),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def reduce_over_ranks(times, counts, device, world_size):
    """Whole-job figures: the slowest rank's times (max) and the units all
    ranks processed (sum).  With one rank the inputs come back unchanged."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(times, dtype=torch.float64, device=device)
    u = torch.tensor(counts, dtype=torch.float64, device=device)
    if world_size > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.tolist(), u.tolist()


def backward_case(args):
    """The differentiable workload (V_theta, L = 10, FP32, checks every 100
    steps, sqrt(T) checkpoints) on an n^3 lattice through T = --iters
    unrolled steps: three fdtd_backward calls (the first includes the
    autotuner's first-use timings), wall time of each with a synchronise on
    both sides.  Small enough to run under ncu."""
    import numpy as np
    import torch

    import paper_0904_0939_gb300 as fd
    import workloads as wl

    n, L, T = args.n, 10.0, args.iters
    dev = torch.device("cuda:0")
    g, th = wl.config_theta(n, L)
    v = torch.from_numpy(wl.v_theta(n, L, th, g).astype(np.float32)).to(dev)
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=100, tol=0.0, backward_steps=T))
    s.set_potential(v)
    psi0 = torch.from_numpy(np.exp(-0.5 * wl.radius2(n, L))).to(dev)
    out = torch.empty((n, n, n), dtype=torch.float64, device=dev)
    ms = []
    for _ in range(3):
        s.set_psi(psi0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.backward(T, 1.0, 0.0, out=out)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    s.close()
    print(json.dumps({"case": "backward", "n": n, "T": T, "ms_per_call": ms, "us_per_step": ms[-1] * 1e3 / T}))


def stencil_case(args):
    """Fixed number of update steps on one lattice (512^3, L = 16 by default,
    the size of the anisotropic-oscillator workload; the kernel's time does
    not depend on V's values, so the oscillator r^2/2 stands in for it):
    per-launch stencil time with CUDA events and the HBM fraction.  Small
    enough to run under ncu."""
    import numpy as np
    import torch

    import paper_0904_0939_gb300 as fd
    import workloads as wl

    n = args.n
    prec = {"f32": fd.F32, "bf16": fd.BF16, "f64": fd.F64}[args.precision]
    opts = fd.default_options(check_every=1 << 30, tol=0.0, temporal_depth=args.depth, zchunk=args.zc)
    s = fd.Solver(fd.Lattice(n, 16.0, prec), opts)
    v = torch.from_numpy(wl.harmonic(n, 16.0).astype(np.float32)).cuda()
    s.set_potential(v)
    s.init_symmetric(SEED, 0)
    s.evolve(args.iters)  # warm-up
    s.reset_stats()
    s.set_profiling(True)
    s.evolve(args.iters)
    st = s.stats()
    ms = st["stencil_ms"] / max(1, st["stencil_timed_launches"])
    upd = st["stencil_site_updates"] / (st["stencil_ms"] * 1e-3) / 1e9
    gbs = st["stencil_bytes"] / (st["stencil_ms"] * 1e-3) / 1e9
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    print(json.dumps({"case": "stencil", "n": n, "precision": args.precision, "depth": args.depth,
                      "tuned": s.tuned_config(),
                      "launches": st["stencil_launches"], "ms_per_launch": ms, "gsite_per_s": upd,
                      "achieved_gbs": gbs, "hbm_frac": gbs / peak, "effective_frac_12B": upd * 12 / peak}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="0: every evolve through the stream (for launch lists under ncu)")
    ap.add_argument("--case", default="solve", choices=["solve", "stencil", "backward"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--zc", type=int, default=0)
    ap.add_argument("--precision", default="f32", choices=["f32", "bf16", "f64"])
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.case == "stencil":
        return stencil_case(args)
    if args.case == "backward":
        return backward_case(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_0904_0939_gb300 as fd

    opts = fd.default_options(check_every=100, tol=TOL, tol_relative=1, graphs=args.graphs)
    seed = SEED + rank
    pots_dev = potentials(True, dev)
    pots_host = potentials(False, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        run_step(fd, pots_dev, seed, opts)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    tot_ms, tot_upd, tot_launch = 0.0, 0, 0
    fine_ms, fine_bytes, fine_upd, fine_launches, fine_timed = 0.0, 0.0, 0, 0, 0
    tot = None
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tot = run_step(fd, pots_dev, seed, opts)
        e1.record()
        torch.cuda.synchronize()
        tot_ms += e0.elapsed_time(e1)
        tot_upd += tot["updates"]
        tot_launch += tot["launches"]
        fine_ms += tot["fine_ms"]
        fine_bytes += tot["fine_bytes"]
        fine_upd += tot["fine_updates"]
        fine_launches += tot["fine_launches"]
        fine_timed += tot["fine_timed"]
    barrier()
    clk = clocks.stop()

    # end to end: host-resident V, copies and read-back inside the region
    e2e_ms = 0.0
    e2e_upd = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_upd += run_step(fd, pots_host, seed, opts)["updates"]
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3

    (ms_max, e2e_max), (upd_all, e2e_upd_all) = reduce_over_ranks([tot_ms, e2e_ms],
                                                                  [float(tot_upd), float(e2e_upd)], dev, ws)
    extra = {}
    if not args.no_extras:
        extra["time_to_E0"] = time_to_e0(fd, pots_dev, seed, opts, dev)
        extra["batched_64_lattices"] = batched_run(fd, dev, seed)
        extra["anisotropic_512_multires_bf16_coarse"] = anisotropic_multires(fd, dev, seed)
        extra["backward_128_T4000"] = backward_run(fd, dev)
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    value = upd_all / (ms_max * 1e-3) / 1e9
    e2e_value = e2e_upd_all / (e2e_max * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # the dominant kernel's average launch: duration over the launches timed
    # with CUDA events, algorithmic bytes and site updates over all of them
    ms_launch = fine_ms / fine_timed if fine_timed else None
    bytes_launch = fine_bytes / max(1, fine_launches)
    achieved = bytes_launch / (ms_launch * 1e-3) / 1e9 if ms_launch else None
    eff = fine_upd / max(1, fine_launches) * 12.0 / (ms_launch * 1e-3) / 1e9 / hbm if ms_launch else None
    depth, zc, tx, ty = tot["config"] if tot and tot["config"] else (None, None, None, None)
    h2d = sum(n**3 * 4 for n in LEVELS) * len(SECTORS)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(ws),
        "path": {"evolve": "cuda graph per lattice (device-side loop), the two sectors concurrently" if args.graphs
                 else "stream", "precision": "fp32 stencil, fp64 sums"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": TRAFFIC_256.get((depth, zc, tx, ty)),
                     "kernel": (f"k_step_tma (256^3 level, depth {depth}, "
                                f"{'balanced one-wave partition' if zc < 0 else f'span {zc}'}, tile {tx}x{ty})" if zc
                                else "k_step_f32 (256^3 level, one-step z-marching)"),
                     "launches": fine_launches, "timed_launches": fine_timed, "ms_per_launch": ms_launch,
                     "bytes_per_launch": bytes_launch, "peak_kind": peak_note,
                     "effective_frac": eff},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 6 * 96},
        "gpu_launches": tot_launch,
        "clocks": clk,
        "results": tot["results"] if tot else None,
        "extra": extra,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
