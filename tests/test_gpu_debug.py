"""Debugging aids of the library (failure detection without a GPU fault):
- the allocation-failure hook (mg_debug_fail_alloc): every device or pinned
  allocation of mg_create_hierarchy, mg_set_rhs's staging buffer and
  mg_batch_create in turn fails as if the device were out of memory; each
  call returns MG_ERR_OOM and the device's free memory is what it was before
  (nothing leaked), and the next call succeeds;
- the bounds-checked build (MG_CHECKED, libgbmg_checked.so): the small and
  odd-sized parity cases (single hierarchy, W-cycles, mixed form, batch) run
  through it in a child process and still match the oracle, with no kernel
  reporting an entry outside its level.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_forced_allocation_failure_is_oom_and_leaks_nothing(dev):
    w = W.ball(32)
    with B.Hierarchy(w["mask"], w["h"]):  # loads the kernels first
        pass
    free0 = _free()
    try:
        for nth in (1, 2):  # the arena, then the pinned host scalars
            B.mg_debug_fail_alloc(nth)
            with pytest.raises(B.MGError) as ei:
                B.Hierarchy(w["mask"], w["h"])
            assert ei.value.status == B.MG_ERR_OOM, ei.value
            B.mg_debug_fail_alloc(0)
            assert _free() == free0, nth
        with B.Hierarchy(w["mask"], w["h"]) as H:
            B.mg_debug_fail_alloc(1)  # the staging buffer of a host-side right-hand side
            with pytest.raises(B.MGError) as ei:
                H.set_rhs(w["rho"])
            assert ei.value.status == B.MG_ERR_OOM
            B.mg_debug_fail_alloc(0)
            H.set_rhs(w["rho"])  # the hierarchy is still usable
            H.set_dirichlet(w["bx"], w["by"], w["bz"])
            st, info = H.solve(1e-10, 50)
            assert st == 0 and info["rel"] < 1e-10
        assert _free() == free0
        ws = [W.blob_patch(s, seed=q) for s, q in [((12, 10, 14), 5), ((9, 16, 7), 61), ((20, 12, 16), 62)]]
        masks = [x["mask"] for x in ws]
        hs = [x["h"] for x in ws]
        n_alloc = 2 + 2 * len(ws) + 1  # pinned state and norms, each patch's arena and scalars, the tables
        for nth in range(1, n_alloc + 1):
            B.mg_debug_fail_alloc(nth)
            with pytest.raises(B.MGError) as ei:
                B.Batch(masks, hs)
            assert ei.value.status == B.MG_ERR_OOM, (nth, ei.value)
            B.mg_debug_fail_alloc(0)
            assert _free() == free0, nth
        B.mg_debug_fail_alloc(n_alloc + 1)  # one past the last allocation: creation succeeds
        bt = B.Batch(masks, hs)
        B.mg_debug_fail_alloc(0)
        bt.close()
        assert _free() == free0
    finally:
        B.mg_debug_fail_alloc(0)


def test_checked_build_runs_the_small_parity_cases_clean():
    env = dict(os.environ, MG_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c",
                            "from paper_1104_1703_gb300 import binding as B; print(B.mg_checked_build())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert probe.returncode == 0 and probe.stdout.strip().endswith("True"), probe.stdout + probe.stderr
    sel = ("tests/test_gpu_parity.py::test_tiny_grids tests/test_gpu_parity.py::test_vcycle_parity "
           "tests/test_gpu_parity.py::test_solve_parity tests/test_gpu_parity.py::test_smoother_parity "
           "tests/test_gpu_parity.py::test_prolongation_parity tests/test_gpu_parity.py::test_restriction_parity "
           "tests/test_gpu_wcycles.py::test_wcycle_solve_parity tests/test_gpu_mixed.py::test_mixed_solve_against_oracle "
           "tests/test_gpu_batch.py::test_batch_solve_matches_oracle").split()
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu and not slow", "-p", "no:cacheprovider"]
                       + sel, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0 and " passed" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
