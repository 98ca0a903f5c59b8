#!/usr/bin/env python
"""Benchmark of the masked-domain multigrid Poisson solve on GB300.

One step is one pass of the whole solver path on the 256^3 union-of-spheres
workload (40 spheres, 8 Gaussian sources, Dirichlet 0): rebuild the mask
hierarchy from the device-resident mask (hierarchy build), load rho and the
Dirichlet values (fold into the right-hand side), reset the guess to 0 and
solve to relative residual 1e-8 with the run-time order switch.

`value` is GS cell-updates per second of the whole job (updates of active
cells at every level, from the solver's own count), with inputs already in
HBM, timed with CUDA events and no instrumentation inside the steps.  The
dominant kernel's launches are timed in a second pass of the same steps
with CUDA events around each launch (`roofline`).  `e2e` is the same metric
through the public C ABI with host buffers: the mask and rho are copied from
pinned host memory and the solution is read back every step.
`ms_per_step` is the time to the tolerance per solve.

More is timed in the same run and reported beside the headline:
- 96 AMR patches solved as one batch (`batched_96_patches`), with the same
  patches solved one after the other for comparison;
- the 512^3 cube with 20000 sub-cell holes (`holes_512`, both forms);
- the headline workload in the FP64 method with N_cycles = 1, 2 and 3
  coarse iterations per level (`w_cycles`, Section 5.3).

--impl reference times the FP64 CPU oracle on the host cores (bounded
sample: hierarchy build + right-hand side + one multigrid iteration of the
same workload per step, so its ms_per_step is that sample, not a solve),
and then one whole oracle solve of the workload to 1e-8 (`time_to_tol_ms`).
The CPU-baseline leg of our arm times the same whole solve, continues it to
1e-13, and reports each GPU form's error against that converged solution
(`error_vs_oracle`).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
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

METRIC = "GS cell-updates/s of the multigrid solve to rel. residual 1e-8"
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
    p.add_argument("--no-batch", action="store_true", help="skip the 96-patch batched workload")
    p.add_argument("--inner-cycles", type=int, default=0,
                   help="mixed form: FP32 V-cycles per FP64 refinement step (0: the fastest of 1..8, "
                        "measured before the timed run)")
    p.add_argument("--batch-only", action="store_true", help="time only the 96-patch batched workload")
    p.add_argument("--learned-only", action="store_true", help="run only the learned-guess training and evaluation")
    p.add_argument("--no-holes", action="store_true", help="skip the 512^3 complex-boundary workload")
    p.add_argument("--no-wcycles", action="store_true", help="skip the W-cycle schedules (N_cycles = 2, 3)")
    p.add_argument("--profile", action="store_true",
                   help="profiling runs: time the headline form only (no second form, e2e or CPU leg)")
    p.add_argument("--precision", type=int, default=1, choices=[0, 1],
                   help="form timed for the headline: 1 = FP32 V-cycles in FP64 refinement, 0 = FP64")
    p.add_argument("--smoother-pass", type=int, default=0, choices=[0, 1],
                   help="mixed form: 1 = fine-level FP32 sweep pairs as temporal-blocked passes (the headline "
                        "otherwise runs the faster list half-sweeps and times the pass beside it)")
    p.add_argument("--no-pass-probe", action="store_true", help="skip timing the temporal-blocked pass")
    p.add_argument("--no-learned", action="store_true", help="skip training and evaluating the learned guess")
    p.add_argument("--learned-train", type=int, default=4096, help="method-generated training solves (128^3)")
    p.add_argument("--learned-eval", type=int, default=512, help="held-out patches evaluated (128^3)")
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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait for its first sample so that
        # the samples cover the timed steps that follow
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

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


def oracle_solve(O, w, tol):
    """One whole oracle solve of the workload from a zero guess to `tol`
    (hierarchy build and right-hand side included, as in the GPU step);
    returns (seconds, info, hierarchy)."""
    t0 = time.perf_counter()
    R = O.Hierarchy(w["mask"], w["h"])
    R.set_rhs(w["rho"])
    st, info = R.solve(tol, 400)
    dt = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError("oracle solve failed: status %d" % st)
    return dt, info, R


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
              "(the order the solve settles in); ms_per_step is that sample" % args.size)
    t_solve, info, R = oracle_solve(O, w, TOL)
    R.close()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args.size),
            "time_to_tol_ms": 1e3 * t_solve, "cycles_per_solve": info["cycles"],
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "time_to_tol_ms": 1e3 * t_solve},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(size, gpu_solutions=None):
    """The oracle on the host cores: a bounded sample of the per-step work
    (throughput), one whole solve of the workload to 1e-8 (time to
    tolerance), and that solve continued to 1e-13, against which the GPU
    forms' solutions at 1e-8 are compared (max-norm error relative to the
    converged solution's max norm)."""
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
    t_solve, info, R = oracle_solve(O, w, TOL)
    out = {"value": upd / secs, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "%d x (mask hierarchy + rhs + one first-order multigrid iteration) of the %d^3 workload, "
                     "%.1f s; then one whole solve to 1e-8" % (n, size, secs),
           "time_to_tol_ms": 1e3 * t_solve, "cycles_per_solve": info["cycles"]}
    errors = None
    if gpu_solutions:
        st, _ = R.solve(1e-13, 400)
        if st == 0:
            star = R.get_phi()
            scale = float(np.abs(star).max())
            errors = {k: float(np.abs(v - star).max() / scale) for k, v in gpu_solutions.items()}
            errors["reference"] = ("oracle solution converged to rel. residual 1e-13; max-norm error / "
                                   "max |Phi|, GPU solves stopped at 1e-8")
    R.close()
    return out, errors


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

FORMS = {0: "fp64", 1: "mixed"}


class Form:
    """One solver form (precision 0 = FP64 method, 1 = FP32 V-cycles inside
    FP64 iterative refinement) on the resident workload."""

    def __init__(self, B, precision, mask_d, rho_d, h, stream, inner_cycles=1, smoother_pass=0, **extra):
        self.B = B
        self.precision = precision
        opts = dict(extra, precision=precision)
        if precision == 1:
            opts["inner_cycles"] = inner_cycles
            opts["smoother_pass"] = smoother_pass
        self.H = B.Hierarchy(mask_d, h, stream=stream, **opts)
        self.n_active = self.H.level_info(0)[1]
        # the fine level's FP32 sweep pairs run as temporal-blocked passes
        self.pass_on = precision == 1 and self.H.smoother_pass
        d = B.mg_default_options()
        # FP32 level-0 sweeps over row segments; FP64 ones with the integer neighbour sum
        seg = int(extra.get("fine_segments", d.fine_segments))
        self.seg_on = seg if (precision == 1 and not self.pass_on) else 0  # 0: cell lists
        self.exact_on = precision == 0 and int(extra.get("fp64_sum", d.fp64_sum)) == 1
        self.kinds = (self.pass_on, self.seg_on, self.exact_on)

    def step(self, mask, rho, out=None):
        H = self.H
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


def time_form(f, args, mask, rho, stream, world, device, out=None, timing=False):
    """W untimed warm-up steps, then K steps between CUDA events on the
    library's stream; returns elapsed seconds (max over ranks) and stats."""
    import torch
    B = f.B
    # at least 3 warm-up steps for any timed number; the ncu profiling pass
    # (--profile) may ask for fewer so that its launch list stays short
    warm = args.warmup if getattr(args, "profile", False) else max(3, args.warmup)
    for _ in range(max(1, warm)):
        f.step(mask, rho, out)
    torch.cuda.synchronize()
    barrier(world)
    if timing:
        B.mg_timing_enable(f.H.handle, True)
        B.mg_timing_read(f.H.handle)
    l0 = B.mg_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    updates, cycles, orders = 0, 0, set()
    for _ in range(args.steps):
        info = f.step(mask, rho, out)
        updates += info["cell_updates"]
        cycles += info["cycles"]
        orders.add(info["order"])
    ev1.record(stream)
    torch.cuda.synchronize()
    st = {"launches": B.mg_launch_count() - l0, "cycles": cycles / args.steps, "orders": sorted(orders)}
    if timing:
        st["gs_n"], st["gs_ms"] = B.mg_timing_read(f.H.handle)
        B.mg_timing_enable(f.H.handle, False)
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, device)
    st["elapsed"] = elapsed
    st["updates"] = sum_over_ranks(updates, world, device)
    barrier(world)
    return st


KERNEL_SRCS = [os.path.join(ROOT, "paper_1104_1703_gb300", "csrc", f)
               for f in ("kernels_cycle.cu", "cycle_device.cuh", "kernels_pass.cu", "exact_sum.cuh")]


def kernel_source_hash():
    """sha256 over the sources of the single-hierarchy cycle kernels."""
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(profile):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu summary `profiles/<profile>`, or None when the summary is
    missing or the kernel source has changed since it was captured."""
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        digest = kernel_source_hash()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not (m_hash and m_bytes) or digest != m_hash.group(1):
        return None
    return int(m_bytes.group(1))


def roofline(st, n_active, precision, peaks, fp64_rate=None, pass_on=False, seg_on=False, exact_on=True):
    """Roofline of the dominant kernel, the level-0 Gauss-Seidel smoother,
    from its CUDA-event-timed launches inside the timed region.  A
    half-sweep launch updates one colour of the unknowns (n_active / 2 on
    average); a temporal-blocked pass launch runs two red-black sweeps (four
    half-sweeps, 2 n_active updates).  Algorithmic bytes are counted per
    active update as for the unfused half-sweeps (a row-segment sweep also
    touches the inactive slots of its segments; those are not counted), so
    the pass's `achieved` is the bandwidth the half-sweeps would need to
    match it."""
    gs_s = st["gs_ms"] / 1e3 / max(st["gs_n"], 1)
    half = n_active / 2.0
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    if precision == 0:
        # 25 B per update over the red+black sweep: read the other colour 8,
        # b/D 8, code 1, write 8.  The method's 7 FP64 operations per update
        # (6 adds, 1 multiply) issue as 1 fused multiply-add when the
        # neighbour sum is formed in integer arithmetic (fp64_sum), else 6
        ops = 1.0 if exact_on else 6.0
        if fp64_rate:
            peak, psrc = fp64_rate / 1e12, "measured DFMA rate on this GPU (mg_probe_fp64_rate)"
        else:
            peak, psrc = 2 * 152 * 2.07e9 / 1e12, "nominal: 2 FP64 lane-ops/clk/SM x 152 SMs x 2.07 GHz"
        ach = 25.0 * half / gs_s / 1e9
        name = ("gs_list_kernel<0,double,...,exact> (level-0 red/black Gauss-Seidel, FP64, integer neighbour sum)"
                if exact_on else "gs_list_kernel<0,double> (level-0 red/black Gauss-Seidel, FP64)")
        return {"bound": "hbm", "kernel": name,
                "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": profiled_traffic("gs_list_fp64_exact_level0_sphere_union_256.md" if exact_on
                                            else "gs_list_fp64_level0_sphere_union_256.md"),
                "launches": st["gs_n"], "avg_launch_us": gs_s * 1e6, "peak_source": src,
                "fp64_pipe_view": {"achieved": ops * half / gs_s / 1e12, "peak": peak, "unit": "T FP64 instr/s",
                                   "frac": ops * half / gs_s / 1e12 / peak, "issued_fp64_ops_per_update": ops,
                                   "method_fp64_ops_per_update": 7, "peak_source": psrc}}
    # FP32: read the other colour 4 + b 4 + code 1, write 4 = 13 B per update
    if pass_on:
        upd = 2.0 * n_active
        ach = 13.0 * upd / gs_s / 1e9
        return {"bound": "hbm", "kernel": "smooth_pass_kernel (level-0 FP32, two red-black sweeps per launch, "
                                          "temporal-blocked z-wavefront)",
                "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "updates_per_launch": upd, "bytes_per_update": 13,
                "traffic": profiled_traffic("smooth_pass_fp32_level0_sphere_union_256.md"),
                "launches": st["gs_n"], "avg_launch_us": gs_s * 1e6, "peak_source": src}
    ach = 13.0 * half / gs_s / 1e9
    if seg_on == 3:
        return {"bound": "hbm", "kernel": "gs_seg_pair_kernel (level-0 red/black Gauss-Seidel over 16-slot row "
                                          "segments, two slots per thread, FP32 inner cycle)",
                "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": profiled_traffic("gs_seg_pair_fp32_level0_sphere_union_256.md"),
                "launches": st["gs_n"], "avg_launch_us": gs_s * 1e6, "peak_source": src}
    if seg_on:
        return {"bound": "hbm", "kernel": "gs_seg_kernel<float> (level-0 red/black Gauss-Seidel over %d-slot row "
                                          "segments, FP32 inner cycle)" % (8 if seg_on == 1 else 16),
                "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": profiled_traffic("gs_seg_fp32_level0_sphere_union_256.md") if seg_on == 1 else None,
                "launches": st["gs_n"], "avg_launch_us": gs_s * 1e6, "peak_source": src}
    return {"bound": "hbm", "kernel": "gs_list_kernel<0,float> (level-0 red/black Gauss-Seidel, FP32 inner cycle)",
            "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": profiled_traffic("gs_list_fp32_level0_sphere_union_256.md"),
            "launches": st["gs_n"], "avg_launch_us": gs_s * 1e6, "peak_source": src}


def peaks_of():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


BATCH_PATCHES = 96


def run_batched(args, B, device, stream, world):
    """The batched workload: 96 AMR patches (edges from {32,48,64,96,128}
    per axis, blob masks, Dirichlet values from a half-resolution coarse
    potential) solved together to 1e-8 by mg_batch_solve after the
    autotuner has picked the launch parameters.  One step resets every
    patch's guess to 0 and solves the whole batch.  Also timed: the same 96
    problems solved one after the other by mg_solve on separate hierarchies."""
    import torch
    ws = W.amr_patches(BATCH_PATCHES, seed=4)
    masks = [torch.from_numpy(w["mask"]).to(device) for w in ws]
    bt = B.Batch(masks, [w["h"] for w in ws], stream=stream.cuda_stream)
    singles = []
    for p, w in enumerate(ws):
        rho = torch.from_numpy(w["rho"]).to(device)
        phi_c = torch.from_numpy(w["phi_c"]).to(device)
        P = bt.patch(p)
        P.set_rhs(rho)
        P.set_dirichlet_from_coarse(phi_c, w["origin"])
        H = B.Hierarchy(masks[p], w["h"], stream=stream.cuda_stream)
        H.set_rhs(rho)
        H.set_dirichlet_from_coarse(phi_c, w["origin"])
        singles.append(H)
    t0 = time.time()
    # launch parameters, then the smoother schedule (n_pre, n_post) by time to tolerance
    tune = bt.autotune(reps=3, tol=TOL, max_cycles=200, flags=B.MG_TUNE_SCHEDULE)
    tune_s = time.time() - t0

    def batch_step():
        for p in range(BATCH_PATCHES):
            bt.patch(p).set_solution(None)
        st, infos = bt.solve(TOL, 200)
        if st != 0:
            raise RuntimeError("batched solve failed: status %d" % st)
        return infos

    def single_step():
        infos = []
        for H in singles:
            H.set_solution(None)
            st, info = H.solve(TOL, 200)
            if st != 0:
                raise RuntimeError("solve failed: status %d" % st)
            infos.append(info)
        return infos

    out = {}
    legs = (("batched", batch_step),) if args.profile else (("batched", batch_step), ("sequential", single_step))
    for name, fn in legs:
        for _ in range(max(1, args.warmup) if args.profile else max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        l0 = B.mg_launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        updates, cycles = 0, []
        for _ in range(args.steps):
            infos = fn()
            updates += sum(i["cell_updates"] for i in infos)
            cycles.append(max(i["cycles"] for i in infos))
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, device)
        out[name] = {"time_to_tol_ms": 1e3 * elapsed / args.steps,
                     "value": sum_over_ranks(updates, world, device) / elapsed,
                     "max_cycles_per_solve": max(cycles), "gpu_launches": B.mg_launch_count() - l0}
    n_cells = sum(int(w["mask"].size) for w in ws)
    n_act = sum(int((w["mask"] > 0).sum()) for w in ws)
    res = {"workload": "%d AMR patches, edges from {32,48,64,96,128}^3, blob masks (correlation 8 cells), "
                       "Dirichlet from a half-resolution coarse potential; %.1f M cells, %.1f M active"
                       % (BATCH_PATCHES, n_cells / 1e6, n_act / 1e6),
           "unit": UNIT, "tol": TOL, **out["batched"],
           "launches_per_cycle": bt.launches_per_cycle(),
           "tuning": {"threads": tune.threads, "persistent_ctas": tune.persistent_ctas,
                      "bottom_slots": tune.bottom_slots, "n_pre": tune.n_pre, "n_post": tune.n_post,
                      "chunk_entries": tune.chunk or 2 * tune.threads,
                      "ms_per_cycle": tune.ms_per_cycle, "autotune_s": tune_s},
           "sequential_mg_solve": out.get("sequential"),
           "speedup_vs_sequential": (out["sequential"]["time_to_tol_ms"] / out["batched"]["time_to_tol_ms"]
                                     if "sequential" in out else None)}
    for H in singles:
        H.close()
    bt.close()
    return res


def run_holes(args, B, device, stream, world):
    """The complex-boundary workload: the 512^3 unit cube minus 20000 balls of
    0.5-4 cells (holes below the coarse cell size, so Section 4's switch
    selects first order), rho ~ U[-1,1], Dirichlet 0, solved to 1e-8 in
    both forms from a zero guess (the same step as the headline)."""
    import torch
    w = W.holes(512)
    mask_d = torch.from_numpy(w["mask"]).to(device)
    rho_d = torch.from_numpy(w["rho"]).to(device)
    out = {"workload": "holes_512^3: unit cube minus 20000 balls (centres U[0,1]^3, radii U[0.5,4] cells), "
                       "rho ~ U[-1,1], Dirichlet 0, tol 1e-8, seed 3",
           "active_cells": int((w["mask"] > 0).sum()), "unit": UNIT}
    del w
    probe = argparse.Namespace(steps=min(args.steps, 3), warmup=args.warmup)
    for prec in (1, 0):
        f = Form(B, prec, mask_d, rho_d, 1.0 / 512, stream.cuda_stream, args.inner_cycles)
        st = time_form(f, probe, mask_d, rho_d, stream, world, device)
        out[FORMS[prec]] = {"time_to_tol_ms": 1e3 * st["elapsed"] / probe.steps,
                            "value": st["updates"] / st["elapsed"], "cycles_per_solve": st["cycles"],
                            "orders": st["orders"], "steps": probe.steps}
        del f
    return out


def run_learned(args):
    """The learned initial guess (a 4-level 3D U-Net, 16 base channels, BF16
    weights and activations, FP32 accumulation, tcgen05 convolutions):
    trained on --learned-train solves at 128^3 that the method generates
    (blob patches with one-way-interface boundary values, solved to 1e-10;
    one Adam step per solve), then evaluated on --learned-eval held-out
    patches: V-cycles and wall time to 1e-8 of the mixed form from the
    learned guess (inference inside the timed region) against the mixed form
    and the plain FP64 method from a zero guess."""
    from paper_1104_1703_gb300 import learned as Lg
    s, losses, records = Lg.run(n=128, levels=4, base=16, n_train=args.learned_train, n_eval=args.learned_eval)
    s["workload"] = ("blob patches 128^3 (white noise smoothed over 8 cells, thresholded; rho ~ U[-1,1]; Dirichlet "
                     "values interpolated from a half-resolution coarse potential), GPU-generated from seeds")
    s["tol"] = 1e-8
    return s


def run_wcycles(args, B, device, stream, world, mask_d, rho_d, h):
    """The multigrid schedules of Section 5.3 on the headline workload: the
    plain FP64 method with N_cycles = 1 (V), 2 and 3 (W) coarse iterations
    per level, each solved to 1e-8 from a zero guess (the headline step)."""
    probe = argparse.Namespace(steps=min(args.steps, 3), warmup=args.warmup)
    out = {"workload": "the headline workload, FP64 method, tol 1e-8", "unit": UNIT}
    for nc in (1, 2, 3):
        f = Form(B, 0, mask_d, rho_d, h, stream.cuda_stream, n_cycles=nc)
        st = time_form(f, probe, mask_d, rho_d, stream, world, device)
        out["n_cycles_%d" % nc] = {"time_to_tol_ms": 1e3 * st["elapsed"] / probe.steps,
                                   "value": st["updates"] / st["elapsed"], "cycles_per_solve": st["cycles"],
                                   "orders": st["orders"], "steps": probe.steps}
        del f
    return out


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

    if args.learned_only:
        res = run_learned(args)
        if rank == 0:
            print(json.dumps({"learned_guess": res}), flush=True)
        return

    if args.batch_only:
        stream = torch.cuda.Stream(device=device)
        res = run_batched(args, B, device, stream, world)
        if rank == 0:
            print(json.dumps({"batched_96_patches": res}), flush=True)
        return

    w = W.sphere_union(args.size)
    mask_d = torch.from_numpy(w["mask"]).to(device)
    rho_d = torch.from_numpy(w["rho"]).to(device)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=device)
    ic_ms = {}
    if args.inner_cycles == 0:
        # pick the refinement step length of the mixed form by its time to
        # tolerance (same workload, untimed here; the chosen form is then
        # timed from scratch below)
        for ic in range(1, 9):
            f = Form(B, 1, mask_d, rho_d, w["h"], stream.cuda_stream, ic, args.smoother_pass)
            probe = argparse.Namespace(steps=3, warmup=1)
            ic_ms[ic] = 1e3 * time_form(f, probe, mask_d, rho_d, stream, world, device)["elapsed"] / 3
            del f
        args.inner_cycles = min(ic_ms, key=ic_ms.get)
    main = Form(B, args.precision, mask_d, rho_d, w["h"], stream.cuda_stream, args.inner_cycles, args.smoother_pass)
    n_active = main.n_active

    # clocks are sampled through the headline form's timed passes (steps
    # without and with kernel events); the steps are short, so both passes
    # are covered to get more than one sample
    clocks = ClockSampler(local)
    clocks.start()
    st_main = time_form(main, args, mask_d, rho_d, stream, world, device)
    # the dominant kernel's launches are timed in a second pass of the same
    # steps: the event pairs around every level-0 half-sweep add their own
    # cost to the step, so the step time above is taken without them
    st_main_k = st_main if args.profile else time_form(main, args, mask_d, rho_d, stream, world, device,
                                                       timing=True)
    clk = clocks.stop()
    clk["span"] = "warm-up and timed steps of the headline form, without and with kernel events"

    if args.profile:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "form": FORMS[args.precision],
                              "value": st_main["updates"] / st_main["elapsed"], "unit": UNIT,
                              "ms_per_step": 1e3 * st_main["elapsed"] / args.steps,
                              "cycles_per_solve": st_main["cycles"], "inner_cycles": args.inner_cycles,
                              "gpu_launches": st_main["launches"], "note": "profiling run without the e2e pass"}),
                  flush=True)
        return

    other = Form(B, 1 - args.precision, mask_d, rho_d, w["h"], stream.cuda_stream, args.inner_cycles,
                 args.smoother_pass)
    st_other = time_form(other, args, mask_d, rho_d, stream, world, device)
    st_other_k = time_form(other, args, mask_d, rho_d, stream, world, device, timing=True)

    # end to end through the C ABI with host buffers: mask and rho copied from
    # pinned host memory and the solution read back every step
    mask_h = torch.from_numpy(w["mask"]).pin_memory()
    rho_h = torch.from_numpy(w["rho"]).pin_memory()
    out_h = torch.empty(w["rho"].shape, dtype=torch.float64).pin_memory()
    st_e2e = time_form(main, args, mask_h, rho_h, stream, world, device, out=out_h)
    h2d = w["mask"].nbytes + w["rho"].nbytes
    d2h = w["rho"].nbytes
    # the last step's solutions of both forms (each a solve to 1e-8 from a
    # zero guess), for their error against the oracle's converged solution
    solutions = {FORMS[args.precision]: main.H.get_solution(), FORMS[1 - args.precision]: other.H.get_solution()}
    fp64_rate = B.mg_probe_fp64_rate(4096)
    main_kinds, other_kinds = main.kinds, other.kinds
    del main, other
    pass_probe = None
    if not args.no_pass_probe and not args.smoother_pass:
        # the mixed form with the temporal-blocked smoothing pass, same inner
        # cycles (bit-identical results), timed beside the headline
        fp = Form(B, 1, mask_d, rho_d, w["h"], stream.cuda_stream, args.inner_cycles, 1)
        probe = argparse.Namespace(steps=min(args.steps, 5), warmup=args.warmup)
        st_p = time_form(fp, probe, mask_d, rho_d, stream, world, device)
        st_pk = time_form(fp, probe, mask_d, rho_d, stream, world, device, timing=True)
        pass_probe = {"time_to_tol_ms": 1e3 * st_p["elapsed"] / probe.steps, "steps": probe.steps,
                      "active": fp.pass_on,
                      "roofline": roofline(st_pk, n_active, 1, peaks_of(), fp64_rate, *fp.kinds)}
        del fp
    wcyc = None if args.no_wcycles else run_wcycles(args, B, device, stream, world, mask_d, rho_d, w["h"])
    batched = None if args.no_batch else run_batched(args, B, device, stream, world)
    holes = None if args.no_holes else run_holes(args, B, device, stream, world)
    learned = None if args.no_learned else run_learned(args)

    if rank != 0:
        return
    peaks = peaks_of()
    ms = lambda st: 1e3 * st["elapsed"] / args.steps  # noqa: E731
    line = {
        "metric": METRIC, "value": st_main["updates"] / st_main["elapsed"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms(st_main), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 in f64 refinement" if args.precision == 1 else "f64",
        "data": "synthetic", "config": config(args.size),
        "form": FORMS[args.precision],
        "inner_cycles": args.inner_cycles,
        "inner_cycles_probe_ms": ic_ms or None,
        "time_to_tol_ms": ms(st_main), "cycles_per_solve": st_main["cycles"], "orders": st_main["orders"],
        # active fine cells x multigrid V-cycles (the mixed form's FP32 cycles: steps x inner cycles) per second
        "fine_cell_vcycles_per_s": world * n_active * st_main["cycles"] * (args.inner_cycles if args.precision == 1 else 1)
                                   * args.steps / st_main["elapsed"],
        "roofline": roofline(st_main_k, n_active, args.precision, peaks, fp64_rate, *main_kinds),
        FORMS[1 - args.precision]: {"time_to_tol_ms": ms(st_other),
                                     "value": st_other["updates"] / st_other["elapsed"],
                                     "cycles_per_solve": st_other["cycles"],
                                     "roofline": roofline(st_other_k, n_active, 1 - args.precision, peaks,
                                                          fp64_rate, *other_kinds)},
        "e2e": {"value": st_e2e["updates"] / st_e2e["elapsed"], "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms(st_e2e)},
        "clocks": clk,
        "gpu_launches": st_main["launches"],
        "fp64_dfma_rate_measured": fp64_rate,
    }
    if batched is not None:
        line["batched_96_patches"] = batched
    if holes is not None:
        line["holes_512"] = holes
    if wcyc is not None:
        line["w_cycles"] = wcyc
    if pass_probe is not None:
        line["smoother_pass_probe"] = pass_probe
    if learned is not None:
        line["learned_guess"] = learned
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"], line["error_vs_oracle"] = cpu_baseline(args.size, solutions)
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
