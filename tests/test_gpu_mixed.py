"""The mixed-precision form: FP32 V-cycles on the error equation inside FP64
iterative refinement (option precision = 1).

Its results are not bitwise those of the FP64 oracle, so it is held to what
the method guarantees at a residual tolerance:
  - the returned solution has relative residual below the tolerance when
    the residual is re-evaluated by the oracle's own FP64 operator;
  - its error against the oracle's fully converged solution (tol 1e-13) is
    of the size the tolerance allows: at most 10x the error of the plain
    FP64 GPU solve stopped at the same tolerance (plus 1e-12 relative);
  - it needs about as many multigrid iterations as the FP64 form (the FP32
    inner cycle contracts the error like the FP64 one), and the order switch
    takes the same decision.
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
    m = W.random_mask((10, 12, 17), seed=101, p_active=0.7)
    return {
        "ball32": W.ball(32),
        "ball64": W.ball(64),
        "random17x12x10": {"mask": m, "rho": W.random_field(m.shape, 102), "h": 0.07,
                           "faces": W.random_faces(m.shape, 103), "tol": 1e-9},
        "holes64": W.holes(64),
        "blob48x32x40": W.blob_patch((40, 32, 48), seed=104),
        "union64": W.sphere_union(64),
    }


CASES = _cases()


def _faces(oracle, w):
    if "phi_c" in w:
        return oracle.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"])
    if "faces" in w:
        return w["faces"]
    return w.get("bx"), w.get("by"), w.get("bz")


def _gpu(w, faces, **opts):
    H = B.Hierarchy(w["mask"], w["h"], **opts)
    H.set_rhs(w["rho"])
    if faces[0] is not None:
        H.set_dirichlet(*faces)
    return H


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_solve_against_oracle(dev, oracle, name):
    w = CASES[name]
    tol = w.get("tol", 1e-8)
    faces = _faces(oracle, w)
    Hm = _gpu(w, faces, precision=1)
    st, info = Hm.solve(tol, 200)
    assert st == 0 and info["rel"] < tol
    phi = Hm.get_solution()

    # residual of the returned solution, by the oracle's FP64 operator
    S0 = np.where(w["mask"] > 0, 1, -1).astype(np.int64)
    R = oracle.Hierarchy(w["mask"], w["h"])
    R.set_rhs(w["rho"])
    if faces[0] is not None:
        R.set_faces(*faces)
    r0 = R.residual_norm_zero()
    r = oracle.residual(S0, 0, 2, w["h"], phi, w["rho"], *faces)
    rel_o = np.sqrt((r ** 2).sum()) / r0
    assert rel_o < tol * (1 + 1e-6)
    assert rel_o == pytest.approx(info["rel"], rel=1e-6)

    # error against the oracle's converged solution, next to the FP64 form's
    st_o, _ = R.solve(1e-13, 400)
    assert st_o == 0
    phi_star = R.get_phi()
    scale = np.abs(phi_star).max()
    err_mixed = np.abs(phi - phi_star).max() / scale
    H64 = _gpu(w, faces, precision=0)
    st64, info64 = H64.solve(tol, 200)
    assert st64 == 0
    err_64 = np.abs(H64.get_solution() - phi_star).max() / scale
    assert err_mixed <= 10 * err_64 + 1e-12, (err_mixed, err_64)
    assert abs(info["cycles"] - info64["cycles"]) <= 2, (info["cycles"], info64["cycles"])
    assert info["order"] == info64["order"] and info["switched"] == info64["switched"]


@pytest.mark.parametrize("inner", [3, 6, 8, 13])
@pytest.mark.parametrize("name", ["ball64", "holes64", "blob48x32x40", "union64"])
def test_mixed_several_inner_cycles(dev, oracle, name, inner):
    """Several FP32 V-cycles per refinement step: the same tolerance as
    checked by the oracle's operator, the same order decision as the FP64
    form (the switch compares a step's ratio with eta^inner), about 1/inner
    of the steps, and the update count of `inner` V-cycles per step."""
    w = CASES[name]
    tol = w.get("tol", 1e-8)
    faces = _faces(oracle, w)
    Hm = _gpu(w, faces, precision=1, inner_cycles=inner)
    st, info = Hm.solve(tol, 200)
    assert st == 0 and info["rel"] < tol
    R = oracle.Hierarchy(w["mask"], w["h"])
    R.set_rhs(w["rho"])
    if faces[0] is not None:
        R.set_faces(*faces)
    R.set_phi(Hm.get_solution())
    assert R.residual_norm() / R.residual_norm_zero() < tol * (1 + 1e-6)
    H64 = _gpu(w, faces, precision=0)
    st64, info64 = H64.solve(tol, 200)
    assert info["order"] == info64["order"] and info["switched"] == info64["switched"]
    # the switch is tested once per step, so a switching solve can spend up
    # to a step of second-order cycles (and restart) before it trips; and a
    # step's FP32 cycles reduce the error equation's residual by at most
    # about the FP32 precision, so two steps are the least for these
    # tolerances however many cycles a step has
    slack = inner + 2 if not info["switched"] else 3 * inner
    assert info64["cycles"] - 2 <= inner * info["cycles"] <= max(info64["cycles"] + slack, 2 * inner), (
        info["cycles"], info64["cycles"])
    per = []
    for order in (1, 2):   # updates of one V-cycle in each order
        Ho = _gpu(w, faces, precision=1, order=order)
        _, io = Ho.solve(1e-300, 1)
        per.append(io["cell_updates"])
    u = info["cell_updates"]
    assert u % inner == 0 and info["cycles"] * min(per) <= u // inner <= info["cycles"] * max(per)


def test_mixed_inner_cycles_and_graphs_agree(dev, oracle):
    w = CASES["ball64"]
    faces = _faces(oracle, w)
    sols = []
    for graphs in (1, 0):
        H = _gpu(w, faces, precision=1, use_graphs=graphs)
        st, info = H.solve(1e-10, 100)
        assert st == 0
        sols.append(H.get_solution())
    assert np.array_equal(sols[0], sols[1])  # graph replay = eager launches, bit for bit
    H2 = _gpu(w, faces, precision=1, inner_cycles=2)
    st2, info2 = H2.solve(1e-10, 100)
    assert st2 == 0 and info2["cycles"] < info["cycles"]


def test_mixed_vcycle_api_and_restart(dev, oracle):
    """mg_vcycle in the mixed form reduces the FP64 residual; setting a new
    solution or right-hand side re-prepares the FP32 problem."""
    w = CASES["ball32"]
    faces = _faces(oracle, w)
    H = _gpu(w, faces, precision=1)
    rels = [H.vcycle() for _ in range(3)]
    assert rels[0] < 0.5 and rels[2] < rels[1] < rels[0]
    H.set_solution(None)
    rel = H.vcycle()
    assert rel == pytest.approx(rels[0], rel=1e-5)
    H.set_rhs(2.0 * w["rho"])
    H.set_solution(None)
    rel2 = H.vcycle()
    assert rel2 < 0.5


@pytest.mark.slow
def test_mixed_full_size_sphere_union_256(dev, oracle):
    """The benchmark workload: the mixed form reaches 1e-8 (checked by the
    oracle's operator) and lands within the tolerance's error of the FP64
    GPU solution converged to 1e-12 (itself within 1e-12 of the oracle)."""
    w = W.sphere_union(256)
    mask = torch.from_numpy(w["mask"]).to(dev)
    rho = torch.from_numpy(w["rho"]).to(dev)
    Hm = B.Hierarchy(mask, w["h"], precision=1)
    Hm.set_rhs(rho)
    st, info = Hm.solve(1e-8, 200)
    assert st == 0
    phi = Hm.get_solution()
    S0 = np.where(w["mask"] > 0, 1, -1).astype(np.int64)
    r = oracle.residual(S0, 0, 2, w["h"], phi, w["rho"])
    act = w["mask"] > 0
    rel_o = np.sqrt((r ** 2).sum()) / np.sqrt((w["rho"][act] ** 2).sum())
    assert rel_o < 1e-8 * (1 + 1e-6)
    H64 = B.Hierarchy(mask, w["h"], precision=0)
    H64.set_rhs(rho)
    st64, info64 = H64.solve(1e-12, 300)
    assert st64 == 0
    ref = H64.get_solution()
    err = np.abs(phi - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    assert abs(info["cycles"] - 23) <= 3


@pytest.mark.slow
def test_mixed_headline_config_against_oracle_256(dev, oracle):
    """The benchmark's exact configuration: the 256^3 union of spheres,
    8 FP32 V-cycles per FP64 refinement step, tol 1e-8 from a zero guess.
    The residual of the returned solution, re-evaluated by the oracle's FP64
    operator, is below the tolerance; its max-norm error against the
    oracle's own solution converged to 1e-13 is at most 10x that of the plain
    FP64 GPU solve stopped at the same tolerance (both errors printed)."""
    w = W.sphere_union(256)
    mask = torch.from_numpy(w["mask"]).to(dev)
    rho = torch.from_numpy(w["rho"]).to(dev)
    Hm = B.Hierarchy(mask, w["h"], precision=1, inner_cycles=8)
    Hm.set_rhs(rho)
    st, info = Hm.solve(1e-8, 200)
    assert st == 0 and info["rel"] < 1e-8
    phi = Hm.get_solution()
    H64 = B.Hierarchy(mask, w["h"], precision=0)
    H64.set_rhs(rho)
    st64, info64 = H64.solve(1e-8, 200)
    assert st64 == 0
    phi64 = H64.get_solution()
    S0 = np.where(w["mask"] > 0, 1, -1).astype(np.int64)
    act = w["mask"] > 0
    r0 = np.sqrt((w["rho"][act] ** 2).sum())
    for sol in (phi, phi64):
        r = oracle.residual(S0, 0, 2, w["h"], sol, w["rho"])
        assert np.sqrt((r ** 2).sum()) / r0 < 1e-8 * (1 + 1e-6)
    R = oracle.Hierarchy(w["mask"], w["h"])
    R.set_rhs(w["rho"])
    st_o, _ = R.solve(1e-13, 400)
    assert st_o == 0
    star = R.get_phi()
    scale = np.abs(star).max()
    err_mixed = np.abs(phi - star).max() / scale
    err_64 = np.abs(phi64 - star).max() / scale
    print("256^3 union, tol 1e-8: max-norm error vs the oracle's converged solution: mixed (8 inner) %.3e, "
          "FP64 %.3e" % (err_mixed, err_64))
    assert err_mixed <= 10 * err_64 + 1e-12, (err_mixed, err_64)
    assert err_mixed < 1e-6
