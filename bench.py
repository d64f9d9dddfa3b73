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
resident in HBM, "e2e" the same call with host-resident V (host->device
copies inside the timed region) and the observables read back.

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
        out.append(torch.from_numpy(v).to(device) if resident else v)
    return out


def run_step(fd, pots, seed, opts):
    """Both sectors, three levels each.  Returns (site_updates, launches, stencil_ms, stencil_bytes, results)."""
    updates, launches, st_ms, st_bytes = 0, 0, 0.0, 0.0
    results = {}
    for name, mask in SECTORS:
        prev = None
        for lvl, n in enumerate(LEVELS):
            s = fd.Solver(fd.Lattice(n, LENGTH, fd.F32), opts)
            s.set_profiling(True)
            s.set_potential(pots[lvl])
            if prev is None:
                s.init_symmetric(seed, mask)
            else:
                s.upsample_from(prev)
            steps, conv = s.evolve(2_000_000)
            o = s.last_check()
            st = s.stats()
            updates += n**3 * steps
            launches += st["launches"]
            st_ms += st["stencil_ms"]
            st_bytes += st["stencil_bytes"]
            results[f"{name}_{n}"] = {"E": o["energy"], "r2": o["r2"], "steps": steps, "converged": conv}
            if prev is not None:
                prev.close()
            prev = s
        prev.close()
    return updates, launches, st_ms, st_bytes, results


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
    t0 = time.perf_counter()
    psi, _, _ = oracle.evolve(psi, v, a, a * a / 4, 2, 100, 0.0, False, SECTORS[0][1])
    t1 = time.perf_counter()
    per = (t1 - t0) / 2
    steps = max(2, min(200, int(target_s / max(per, 1e-3))))
    t0 = time.perf_counter()
    oracle.evolve(psi, v, a, a * a / 4, steps, 100, 0.0, False, SECTORS[0][1])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n**3 * steps / dt / 1e9, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 update steps with checks on the 256^3 Coulomb lattice ({dt:.1f} s)"}


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
            "config": {"workload": "coulomb_soft_L40_multires_64-128-256_1s+2px (oracle sample: 256^3 steps)"},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


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
    opts = fd.default_options(check_every=1 << 30, tol=0.0, temporal_depth=args.depth)
    s = fd.Solver(fd.Lattice(n, 16.0, prec), opts)
    v = torch.from_numpy(wl.harmonic(n, 16.0).astype(np.float32)).cuda()
    s.set_potential(v)
    s.init_symmetric(SEED, 0)
    s.evolve(args.iters)  # warm-up
    s.reset_stats()
    s.set_profiling(True)
    s.evolve(args.iters)
    st = s.stats()
    ms = st["stencil_ms"] / max(1, st["stencil_launches"])
    upd = st["stencil_site_updates"] / (st["stencil_ms"] * 1e-3) / 1e9
    gbs = st["stencil_bytes"] / (st["stencil_ms"] * 1e-3) / 1e9
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    print(json.dumps({"case": "stencil", "n": n, "precision": args.precision, "depth": args.depth,
                      "launches": st["stencil_launches"], "ms_per_launch": ms, "gsite_per_s": upd,
                      "achieved_gbs": gbs, "hbm_frac": gbs / peak, "effective_frac_12B": upd * 12 / peak}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="solve", choices=["solve", "stencil"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--precision", default="f32", choices=["f32", "bf16", "f64"])
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.case == "stencil":
        return stencil_case(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_0904_0939_gb300 as fd

    opts = fd.default_options(check_every=100, tol=TOL, tol_relative=1)
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
    tot_ms, tot_upd, tot_launch, st_ms, st_bytes = 0.0, 0, 0, 0.0, 0.0
    results = None
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        upd, nl, sms, sb, results = run_step(fd, pots_dev, seed, opts)
        e1.record()
        torch.cuda.synchronize()
        tot_ms += e0.elapsed_time(e1)
        tot_upd += upd
        tot_launch += nl
        st_ms += sms
        st_bytes += sb
    barrier()
    clk = clocks.stop()

    # end to end: host-resident V, copies and read-back inside the region
    e2e_ms = 0.0
    e2e_upd = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upd, _, _, _, _ = run_step(fd, pots_host, seed, opts)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_upd += upd

    t_local = torch.tensor([tot_ms, e2e_ms], dtype=torch.float64, device=dev)
    u_local = torch.tensor([float(tot_upd), float(e2e_upd)], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(u_local, op=dist.ReduceOp.SUM)
    ms_max, e2e_max = t_local.tolist()
    upd_all, e2e_upd_all = u_local.tolist()
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
    achieved = st_bytes / (st_ms * 1e-3) / 1e9 if st_ms > 0 else None
    h2d = sum(n**3 * 4 for n in LEVELS) * len(SECTORS)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "coulomb_soft_L40_multires_64-128-256_1s+2px", "levels": list(LEVELS),
                   "length": LENGTH, "tol_rel": TOL, "check_every": 100, "precision": "fp32 stencil, fp64 sums",
                   "l2": "flushed (512 MiB write) between timed steps", "parallelism": f"replicas{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": None,
                     "kernel": "stencil (all levels)", "peak_kind": peak_note},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 6 * 96},
        "gpu_launches": tot_launch,
        "clocks": clk,
        "results": results,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
