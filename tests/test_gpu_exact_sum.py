"""The FP64 form's integer neighbour sum (option fp64_sum, exact_sum.cuh) on
the GPU:
  - the device computes bit for bit what the host build of the same
    function computes (which tests/test_exact_sum.py checks against exact
    arithmetic);
  - a level-0 Gauss-Seidel sweep with it agrees with the oracle's sweep to
    1e-14 (one rounding of the sum plus the fused multiply-add: both
    variants are held to the same per-update bound);
  - whole solves with it take the oracle's cycle counts and order decisions
    and agree with its solution to the parity tolerance."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

from test_exact_sum import build_checker, run_checker, sum_cases  # noqa: E402
from test_gpu_parity import CASES, make_pair, relerr, _level_state  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def test_device_sum_equals_host_sum():
    rng = np.random.default_rng(99)
    extra = rng.standard_normal((200000, 6)) * np.exp2(rng.integers(-60, 60, (200000, 6)))
    extra[rng.random((200000, 6)) < 0.2] = 0.0
    sets = np.concatenate([sum_cases(), extra])
    with tempfile.TemporaryDirectory() as d:
        exe = build_checker(d)
        host = run_checker(exe, "host", sets, d)
        devv = run_checker(exe, "device", sets, d)
    same = (host.view(np.uint64) == devv.view(np.uint64)) | (np.isnan(host) & np.isnan(devv))
    assert same.all(), np.flatnonzero(~same)[:5]


@pytest.mark.parametrize("name", ["ball64", "random17x12x10", "blob48x32x40"])
@pytest.mark.parametrize("fp64_sum", [0, 1])
def test_level0_sweep_per_update_bound(dev, name, fp64_sum):
    w = CASES[name]
    H, R = make_pair(w, dev, fp64_sum=fp64_sum)
    _level_state(w, H, R, 0, 2, seed=910)
    for sweeps in (1, 2):
        H.smooth(0, 2, sweeps)
        R.smooth(0, 2, sweeps)
        assert relerr(H.level_get(0, B.MG_FIELD_PHI), R.phi(0)) < 1e-14


@pytest.mark.parametrize("name", ["ball64", "holes32", "blob48x32x40"])
def test_solves_with_the_integer_sum_match_the_oracle(dev, name):
    w = CASES[name]
    H, R = make_pair(w, dev, fp64_sum=1)
    st, info = H.solve(1e-10, 100)
    st_o, info_o = R.solve(1e-10, 100)
    assert st == st_o == 0
    assert (info["cycles"], info["order"], info["switched"]) == (info_o["cycles"], info_o["order"], info_o["switched"])
    assert relerr(H.get_solution(), R.get_phi()) < 1e-12
