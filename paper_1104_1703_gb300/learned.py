"""The learned initial guess: training on solves the method generates, and
its evaluation against the plain V-cycle.

Every step runs in the library's kernels through the C ABI (binding.py):
synthetic patches are generated on the GPU (mg_generate_blob_patch), their
boundary values come from the coarse potential by the one-way interface
(mg_faces_from_coarse), the training target is the method's own solution
(mg_solve), and the network trains and predicts with mg_unet_*.  This module
only sequences those calls and times them.

The guess never changes what the solve accepts: mg_solve starts from it and
stops at the same relative residual (the residual of Phi = 0 is the
reference), so a poor guess costs cycles, not accuracy.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B

ORIGIN = (-2, -2, -2)


def init_params(seed: int, levels: int, base: int, c_in: int = 3) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)) and zero biases in the
    network's parameter order, from numpy's seeded generator."""
    rng = np.random.default_rng(seed)
    ch = [base << l for l in range(levels)]
    out = []

    def conv(ci, co, k=3):
        out.append(rng.normal(0.0, np.sqrt(2.0 / (ci * k ** 3)), co * ci * k ** 3))
        out.append(np.zeros(co))

    for l in range(levels):
        conv(c_in if l == 0 else ch[l - 1], ch[l])
        conv(ch[l], ch[l])
    for l in range(levels - 1):
        conv(ch[l] + ch[l + 1], ch[l])
        conv(ch[l], ch[l])
    conv(ch[0], 1, k=1)
    return np.concatenate(out)


class Patches:
    """Device buffers of one synthetic patch of an n^3 grid and a hierarchy
    to solve it (precision 1: the mixed form, or 0: FP64)."""

    def __init__(self, n: int, device, precision: int = 1, inner_cycles: int = 1, corr_cells: float = 8.0):
        import torch
        self.n = n
        self.h = 1.0 / n
        self.corr = corr_cells
        cn = (n + 1) // 2 + 2
        V = n ** 3
        self.shape = (n, n, n)
        self.mask = torch.zeros(self.shape, dtype=torch.int8, device=device)
        self.rho = torch.zeros(self.shape, dtype=torch.float64, device=device)
        self.phi_c = torch.zeros((cn, cn, cn), dtype=torch.float64, device=device)
        self.scratch = torch.zeros(2 * V + int(8 * corr_cells) + 8, dtype=torch.float32, device=device)
        self.bx = torch.zeros((n, n, n + 1), dtype=torch.float64, device=device)
        self.by = torch.zeros((n, n + 1, n), dtype=torch.float64, device=device)
        self.bz = torch.zeros((n + 1, n, n), dtype=torch.float64, device=device)
        self.phi = torch.zeros(self.shape, dtype=torch.float64, device=device)
        self.guess = torch.zeros(self.shape, dtype=torch.float64, device=device)
        self.load(12345)  # a non-empty mask to build the hierarchy on
        self.H = B.Hierarchy(self.mask, self.h, precision=precision, inner_cycles=inner_cycles)

    @property
    def faces(self):
        return self.bx, self.by, self.bz

    def load(self, seed: int) -> None:
        B.mg_generate_blob_patch(seed, self.shape, self.scratch, self.mask, self.rho, self.phi_c, self.corr)

    def setup(self, seed: int) -> bool:
        """Generates patch `seed` and hands it to the hierarchy; False for a
        patch without an active cell."""
        self.load(seed)
        try:
            self.H.update_mask(self.mask)
        except B.MGError as e:
            if e.status == B.MG_ERR_EMPTY_DOMAIN:
                return False
            raise
        self.H.set_rhs(self.rho)
        self.H.faces_from_coarse(self.phi_c, ORIGIN, self.bx, self.by, self.bz)
        self.H.set_dirichlet(self.bx, self.by, self.bz)
        return True


def train(net: B.UNet, patches: Patches, seeds, lr: float = 1e-3, lr_end: float = 1e-4, target_tol: float = 1e-10,
          log_every: int = 0):
    """One pass over `seeds`: each patch is solved by the method to
    target_tol and the network takes one Adam step towards that solution
    (learning rate decaying geometrically from lr to lr_end).  Returns the
    losses."""
    losses = []
    n = len(seeds)
    for i, seed in enumerate(seeds):
        if not patches.setup(seed):
            continue
        patches.H.set_solution(None)
        st, info = patches.H.solve(target_tol, 400)
        if st != 0:
            continue
        patches.H.get_solution(patches.phi)
        rate = lr * (lr_end / lr) ** (i / max(1, n - 1))
        losses.append(net.train_patch(patches.mask, patches.rho, patches.faces, patches.h, patches.phi, rate))
        if log_every and (i + 1) % log_every == 0:
            print("train %d/%d loss %.4f" % (i + 1, n, float(np.mean(losses[-log_every:]))), flush=True)
    return losses


def evaluate(net: B.UNet, patches: Patches, seeds, tol: float = 1e-8, max_cycles: int = 200, fp64: "Patches" = None):
    """For each patch: the solve to tol from a zero guess and from the
    learned guess (the guess's inference inside the timed region), timed
    with CUDA events on the library's stream; with `fp64` (Patches of the
    plain FP64 method) also the FP64 solve from a zero guess.  Returns
    per-patch records."""
    import torch
    out = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    stream = torch.cuda.current_stream()
    for seed in seeds:
        if not patches.setup(seed):
            continue
        H = patches.H
        rec = {"seed": int(seed)}
        if fp64 is not None:
            fp64.setup(seed)
            torch.cuda.synchronize()
            ev[4].record(stream)
            fp64.H.set_solution(None)
            st2, i2 = fp64.H.solve(tol, max_cycles)
            ev[5].record(stream)
        torch.cuda.synchronize()
        ev[0].record(stream)
        H.set_solution(None)
        st0, i0 = H.solve(tol, max_cycles)
        ev[1].record(stream)
        ev[2].record(stream)
        net.predict(patches.mask, patches.rho, patches.faces, patches.h, patches.guess)
        H.set_solution(patches.guess)
        st1, i1 = H.solve(tol, max_cycles)
        ev[3].record(stream)
        torch.cuda.synchronize()
        rec.update({"status": (st0, st1), "cycles_zero": i0["cycles"], "cycles_learned": i1["cycles"],
                    "ms_zero": ev[0].elapsed_time(ev[1]), "ms_learned": ev[2].elapsed_time(ev[3]),
                    "rel_init_learned": i1["r_init"] / i1["r_zero"], "order": (i0["order"], i1["order"])})
        if fp64 is not None:
            rec.update({"status_fp64": st2, "cycles_fp64": i2["cycles"], "ms_fp64": ev[4].elapsed_time(ev[5])})
        out.append(rec)
    return out


def summary(records, inner_cycles: int = 1):
    """Cycle counts (multigrid iterations: steps x inner cycles) and wall
    times of the evaluation records."""
    if not records:
        return {}
    cz = np.array([r["cycles_zero"] for r in records]) * inner_cycles
    cl = np.array([r["cycles_learned"] for r in records]) * inner_cycles
    mz = np.array([r["ms_zero"] for r in records])
    ml = np.array([r["ms_learned"] for r in records])
    saved = cz - cl
    return {"patches": len(records), "cycles_zero_mean": float(cz.mean()), "cycles_learned_mean": float(cl.mean()),
            "cycles_saved_mean": float(saved.mean()),
            "cycles_saved_hist": {int(k): int(v) for k, v in zip(*np.unique(saved, return_counts=True))},
            "ms_zero_mean": float(mz.mean()), "ms_learned_mean": float(ml.mean()),
            "wall_time_ratio_learned_over_zero": float(ml.mean() / mz.mean()),
            "initial_rel_residual_learned_median": float(np.median([r["rel_init_learned"] for r in records])),
            "all_converged": all(r["status"] == (0, 0) for r in records) and
                             all(r.get("status_fp64", 0) == 0 for r in records),
            **({"cycles_fp64_mean": float(np.mean([r["cycles_fp64"] for r in records])),
                "ms_fp64_mean": float(np.mean([r["ms_fp64"] for r in records])),
                "wall_time_ratio_learned_over_fp64": float(ml.mean() / np.mean([r["ms_fp64"] for r in records]))}
               if "ms_fp64" in records[0] else {})}


def run(n: int = 128, levels: int = 4, base: int = 16, n_train: int = 4096, n_eval: int = 512, lr: float = 1e-3,
        lr_end: float = 1e-4, seed: int = 5, inner_cycles: int = 1, log_every: int = 0):
    """Trains on n_train method-generated solves (seeds seed * 10^6 + i) and
    evaluates on n_eval held-out patches (seeds seed * 10^6 + 500000 + i).
    Returns (summary dict, training losses, evaluation records)."""
    import torch
    device = torch.device("cuda", torch.cuda.current_device())
    net = B.UNet(levels, base, (n, n, n))
    net.set_params(init_params(seed, levels, base))
    patches = Patches(n, device, precision=1, inner_cycles=inner_cycles)
    base_seed = seed * 1000000
    t0 = time.time()
    losses = train(net, patches, [base_seed + i for i in range(n_train)], lr, lr_end, log_every=log_every)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    fp64 = Patches(n, device, precision=0)
    records = evaluate(net, patches, [base_seed + 500000 + i for i in range(n_eval)], fp64=fp64)
    s = summary(records, inner_cycles)
    s.update({"grid": [n, n, n], "levels": levels, "base_channels": base, "train_patches": len(losses),
              "train_seconds": t_train, "loss_first_64": float(np.mean(losses[:64])) if losses else None,
              "loss_last_64": float(np.mean(losses[-64:])) if losses else None, "inner_cycles": inner_cycles})
    return s, losses, records
