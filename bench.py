#!/usr/bin/env python
"""Benchmark of the masked-domain multigrid Poisson solve on GB300.

One step is one pass of the whole solver path on the 256^3 union-of-spheres
workload (40 spheres, 8 Gaussian sources, Dirichlet 0): rebuild the mask
hierarchy from the device-resident mask (hierarchy build), load rho and the
Dirichlet values (fold into the right-hand side), reset the guess to 0 and
solve to relative residual 1e-8 with the run-time order switch.

`value` is GS cell-updates per second of the whole job (updates of active
cells at every level, from the solver's own count), with inputs already in
HBM.  `e2e` is the same metric through the public C ABI with host buffers:
the mask and rho are copied from pinned host memory and the solution is read
back every step.  `ms_per_step` is the time to the tolerance per solve.

--impl reference times the FP64 CPU oracle on the host cores (bounded
sample: hierarchy build + right-hand side + one multigrid iteration of the
same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1104_1703_gb300 import workloads as W  # noqa: E402

METRIC = "GS cell-updates/s, FP64 multigrid solve to rel. residual 1e-8"
UNIT = "cell-updates/s"
TOL = 1e-8
N = 256


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=N)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    return p.parse_args()


def config(size):
    return {"workload": "sphere_union_%d^3: union of 40 spheres (centres U[0.2,0.8]^3, radii U[0.05,0.2]), "
                        "rho = 8 Gaussians sigma 0.03, Dirichlet 0, tol 1e-8, seed 2" % size,
            "grid": [size, size, size], "tol": TOL, "n_pre": 2, "n_post": 2, "coarse_sweeps": 50,
            "order": "auto (Section 4 switch, eta 0.5, hold 10)",
            "l2": "working set (Phi, b, codes of all levels, ~%.2f GB) exceeds the 129 MB L2; no flush"
                  % (size ** 3 * 17.5 / 1e9)}


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# distributed plumbing (independent replicas; no collective on the data path)
# --------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------
# oracle (CPU) timing: the cpu_baseline leg and the reference arm
# --------------------------------------------------------------------------

def oracle_step(O, w, order):
    """Hierarchy build + rhs + one multigrid iteration of the workload on the
    host cores; returns (seconds, cell updates)."""
    t0 = time.perf_counter()
    R = O.Hierarchy(w["mask"], w["h"])
    R.set_rhs(w["rho"])
    R.vcycle(order=order)
    r = R.residual_norm()
    dt = time.perf_counter() - t0
    assert np.isfinite(r)
    upd = 0
    deep = R.deepest(order)
    for l in range(deep + 1):
        act = R.level_active(l, 2 if l == 0 else order)
        upd += act * (50 if l == deep else 4)
    R.close()
    return dt, upd


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    w = W.sphere_union(args.size)
    for _ in range(args.warmup):
        oracle_step(O, w, 1)
    secs, upd = 0.0, 0
    for _ in range(args.steps):
        dt, u = oracle_step(O, w, 1)
        secs += dt
        upd += u
    value = upd / secs
    cores = O.num_threads()
    sample = ("per step: mask hierarchy + rhs + one first-order multigrid iteration of the %d^3 workload "
              "(the order the solve settles in)" % args.size)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args.size),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(size):
    from oracle import oracle as O
    O.build()
    w = W.sphere_union(size)
    oracle_step(O, w, 1)  # page in
    secs, upd, n = 0.0, 0, 0
    while secs < 10.0 and n < 6:
        dt, u = oracle_step(O, w, 1)
        secs += dt
        upd += u
        n += 1
    return {"value": upd / secs, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d x (mask hierarchy + rhs + one first-order multigrid iteration) of the %d^3 workload, "
                      "%.1f s" % (n, size, secs)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    from paper_1104_1703_gb300 import binding as B

    w = W.sphere_union(args.size)
    mask_d = torch.from_numpy(w["mask"]).to(device)
    rho_d = torch.from_numpy(w["rho"]).to(device)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=device)
    H = B.Hierarchy(mask_d, w["h"], stream=stream.cuda_stream)
    n_active = H.level_info(0)[1]

    def step(mask, rho, out=None):
        H.update_mask(mask)
        H.set_rhs(rho)
        H.set_dirichlet(None, None, None)
        H.set_solution(None)
        st, info = H.solve(TOL, 200)
        if st != 0:
            raise RuntimeError("solve failed: status %d rel %.3e" % (st, info["rel"]))
        if out is not None:
            H.get_solution(out)
        return info

    # ---- device-resident timing ----
    for _ in range(max(3, args.warmup)):
        step(mask_d, rho_d)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    B.mg_timing_enable(H.handle, True)
    B.mg_timing_read(H.handle)  # reset accumulators
    l0 = B.mg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    updates, cycles, orders = 0, 0, []
    for _ in range(args.steps):
        info = step(mask_d, rho_d)
        updates += info["cell_updates"]
        cycles += info["cycles"]
        orders.append(info["order"])
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = B.mg_launch_count() - l0
    n_gs, gs_ms = B.mg_timing_read(H.handle)
    B.mg_timing_enable(H.handle, False)
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed = max_over_ranks(elapsed, world, device)
    total_updates = sum_over_ranks(updates, world, device)
    barrier(world)

    # ---- end to end through the C ABI with host buffers ----
    if args.no_e2e:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": total_updates / elapsed, "unit": UNIT,
                              "ms_per_step": 1e3 * elapsed / args.steps, "gpu_launches": launches,
                              "note": "profiling run without the e2e pass"}), flush=True)
        return
    mask_h = torch.from_numpy(w["mask"]).pin_memory()
    rho_h = torch.from_numpy(w["rho"]).pin_memory()
    out_h = torch.empty(w["rho"].shape, dtype=torch.float64).pin_memory()
    step(mask_h, rho_h, out_h)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_updates = 0
    for _ in range(args.steps):
        e2e_updates += step(mask_h, rho_h, out_h)["cell_updates"]
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, device)
    e2e_total = sum_over_ranks(e2e_updates, world, device)
    h2d = w["mask"].nbytes + w["rho"].nbytes
    d2h = w["rho"].nbytes

    if rank != 0:
        return
    gs_avg_s = gs_ms / 1e3 / max(n_gs, 1)
    # algorithmic content of one level-0 half-sweep (one colour of the active
    # cells): 7 FP64 instructions and 12.5 bytes per active cell on average
    # (25 B per cell-update over the full red+black sweep)
    half_cells = n_active / 2.0
    fp64_instr = 7.0 * half_cells
    alg_bytes = 25.0 * half_cells
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64_peak = 2 * 152 * 2.07e9 / 1e12  # T FP64 instructions/s: 2 per clock per SM at 2070 MHz
    line = {
        "metric": METRIC, "value": total_updates / elapsed, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(args.size),
        "time_to_tol_ms": 1e3 * elapsed / args.steps,
        "cycles_per_solve": cycles / args.steps, "orders": sorted(set(orders)),
        "roofline": {"bound": "alu", "kernel": "half_sweep_kernel<0> (level-0 red/black Gauss-Seidel)",
                     "achieved": fp64_instr / gs_avg_s / 1e12, "peak": fp64_peak,
                     "unit": "T FP64 instr/s", "frac": fp64_instr / gs_avg_s / 1e12 / fp64_peak,
                     "traffic": None, "launches": n_gs, "avg_launch_us": gs_avg_s * 1e6,
                     "peak_source": "nominal FP64 rate (1.25 TFLOP/s = 2 DFMA/clk/SM x 152 SMs x 2.07 GHz)",
                     "hbm_view": {"achieved_gbs": alg_bytes / gs_avg_s / 1e9, "peak_gbs": hbm_peak,
                                  "frac": alg_bytes / gs_avg_s / 1e9 / hbm_peak,
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks
                                  else "fallback 6.8 TB/s"}},
        "e2e": {"value": e2e_total / e2e_elapsed, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk,
        "gpu_launches": launches,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.size)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        try:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()
        except Exception:
            pass


if __name__ == "__main__":
    main()
