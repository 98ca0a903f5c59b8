"""The temporal-blocked FP32 smoothing pass of the fine level (option
smoother_pass, kernels_pass.cu) against the four list half-sweeps it
replaces: whole mixed-form solves with the pass on and off take the same
decisions and produce bit-identical residual histories and solutions, on
odd-sized and partly filled grids (partial tiles at every edge), with one and
eight inner cycles, with an uneven smoother schedule (a pass plus a single
list sweep, and an odd number of passes per cycle), and in W-cycles.  Also
the pass's bounded wait: a forced stall makes the solve return
MG_ERR_INTERNAL after about a second and leaves the GPU usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _cases():
    return {
        "ball64": W.ball(64),
        "union64": W.sphere_union(64),
        "blob48x32x40": W.blob_patch((40, 32, 48), seed=104),
        "holes64": W.holes(64),
        "blob37x70x45": W.blob_patch((45, 70, 37), seed=7),
    }


CASES = _cases()


def _solve(oracle, w, **opts):
    H = B.Hierarchy(w["mask"], w["h"], precision=1, **opts)
    assert H.smoother_pass == (opts.get("smoother_pass", 0) == 1)
    H.set_rhs(w["rho"])
    if "phi_c" in w:
        H.set_dirichlet(*oracle.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"]))
    elif "bx" in w:
        H.set_dirichlet(w["bx"], w["by"], w["bz"])
    st, info = H.solve(w.get("tol", 1e-8), 200)
    phi = H.get_solution()
    H.close()
    return st, info, phi


def _same(a, b):
    st_a, ia, pa = a
    st_b, ib, pb = b
    assert st_a == st_b == 0
    assert ia["cycles"] == ib["cycles"] and ia["order"] == ib["order"] and ia["switched"] == ib["switched"]
    assert np.array_equal(ia["hist"], ib["hist"]), (ia["hist"], ib["hist"])
    assert np.array_equal(pa, pb)


@pytest.mark.parametrize("inner", [1, 8])
@pytest.mark.parametrize("name", list(CASES))
def test_pass_is_bit_identical_to_list_half_sweeps(dev, oracle, name, inner):
    w = CASES[name]
    _same(_solve(oracle, w, inner_cycles=inner, smoother_pass=1), _solve(oracle, w, inner_cycles=inner, smoother_pass=0))


@pytest.mark.parametrize("pre,post", [(3, 1), (2, 1), (4, 2), (1, 3)])
def test_pass_with_uneven_schedules(dev, oracle, pre, post):
    w = CASES["blob48x32x40"]
    _same(_solve(oracle, w, n_pre=pre, n_post=post, smoother_pass=1),
          _solve(oracle, w, n_pre=pre, n_post=post, smoother_pass=0))


def test_pass_in_w_cycles_and_without_graphs(dev, oracle):
    w = CASES["union64"]
    _same(_solve(oracle, w, n_cycles=2, smoother_pass=1), _solve(oracle, w, n_cycles=2, smoother_pass=0))
    _same(_solve(oracle, w, use_graphs=0, smoother_pass=1), _solve(oracle, w, use_graphs=0, smoother_pass=0))


@pytest.mark.slow
def test_pass_full_size_sphere_union_256(dev, oracle):
    w = W.sphere_union(256)
    mask = torch.from_numpy(w["mask"]).to(dev)
    rho = torch.from_numpy(w["rho"]).to(dev)
    out = []
    for sp in (1, 0):
        H = B.Hierarchy(mask, w["h"], precision=1, inner_cycles=8, smoother_pass=sp)
        H.set_rhs(rho)
        st, info = H.solve(1e-8, 200)
        out.append((st, info, H.get_solution()))
        H.close()
    _same(out[0], out[1])


def test_pass_follows_a_mask_update(dev, oracle):
    """After mg_update_mask the pass walks the new mask's tiles (and cells
    the new mask made inactive read 0)."""
    a, b = CASES["ball64"], CASES["union64"]
    res = []
    for sp in (1, 0):
        H = B.Hierarchy(a["mask"], a["h"], precision=1, smoother_pass=sp)
        H.set_rhs(a["rho"])
        H.set_dirichlet(a["bx"], a["by"], a["bz"])
        assert H.solve(1e-8, 100)[0] == 0
        H.update_mask(b["mask"])
        H.set_rhs(b["rho"])
        st, info = H.solve(1e-8, 100)
        res.append((st, info, H.get_solution()))
        H.close()
    _same(res[0], res[1])
    H = B.Hierarchy(b["mask"], b["h"], precision=1, smoother_pass=1)
    H.set_rhs(b["rho"])
    st, info = H.solve(1e-8, 100)
    _same(res[0], (st, info, H.get_solution()))


def test_pass_stall_returns_internal_error(dev, oracle):
    w = CASES["ball64"]
    B.mg_debug_stall_pass(True)
    try:
        H = B.Hierarchy(w["mask"], w["h"], precision=1, smoother_pass=1)
        H.set_rhs(w["rho"])
        with pytest.raises(B.MGError) as ei:
            H.solve(1e-8, 5)
        assert ei.value.status == B.MG_ERR_INTERNAL and "did not complete" in ei.value.message
        H.close()
    finally:
        B.mg_debug_stall_pass(False)
    torch.cuda.synchronize()
    st, info, _ = _solve(oracle, w, smoother_pass=1)  # the context is still usable
    assert st == 0
