"""GPU parity of the multigrid schedules with N_cycles = 2 and 3 (Section 5.3)
and of the one-way interface under a strong boundary gradient (Section 5.1),
against the FP64 oracle.  Same bar as the V-cycle: 1e-12 relative after
every cycle, identical decisions in mg_solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
HIST_REL, HIST_FLOOR = 1e-10, 1e-15


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def relerr(a, b):
    return np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300)


def _cases():
    m = W.random_mask((10, 12, 17), seed=101, p_active=0.7)
    return {
        "ball32": W.ball(32),
        "random17x12x10": {"mask": m, "rho": W.random_field(m.shape, 102), "h": 0.07,
                           "faces": W.random_faces(m.shape, 103)},
        "holes32": W.holes(32),
        "blob48x32x40": W.blob_patch((40, 32, 48), seed=104),
    }


CASES = _cases()


def make_pair(w, dev, **opts):
    from oracle import oracle as O
    H = B.Hierarchy(torch.from_numpy(w["mask"]).to(dev), w["h"], **opts)
    R = O.Hierarchy(w["mask"], w["h"])
    H.set_rhs(torch.from_numpy(w["rho"]).to(dev))
    R.set_rhs(w["rho"])
    if "phi_c" in w:
        H.set_dirichlet_from_coarse(torch.from_numpy(w["phi_c"]).to(dev), w["origin"])
        R.set_faces(*O.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"]))
    else:
        f = w["faces"] if "faces" in w else (w.get("bx"), w.get("by"), w.get("bz"))
        if f[0] is not None:
            H.set_dirichlet(*(torch.from_numpy(a).to(dev) for a in f))
            R.set_faces(*f)
    return H, R


@pytest.mark.parametrize("n_cycles", [2, 3])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_wcycle_parity(dev, name, order, n_cycles):
    w = CASES[name]
    H, R = make_pair(w, dev, order=order, n_cycles=n_cycles)
    r0 = R.residual_norm_zero()
    for k in range(3):
        rel = H.vcycle()
        R.vcycle(order=order, n_cycles=n_cycles)
        assert relerr(H.get_solution(), R.get_phi()) < TOL, "cycle %d" % (k + 1)
        rel_o = R.residual_norm() / r0
        assert abs(rel - rel_o) <= HIST_REL * rel_o + HIST_FLOOR


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("name", ["holes32", "blob48x32x40"])
def test_wcycle_solve_parity(dev, name, graphs):
    w = CASES[name]
    H, R = make_pair(w, dev, n_cycles=2, use_graphs=graphs)
    st, info = H.solve(1e-9, 80)
    st_o, info_o = R.solve(1e-9, 80, n_cycles=2)
    assert st == st_o == 0
    for key in ("cycles", "order", "switched"):
        assert info[key] == info_o[key], key
    ho, hg = info_o["hist"], info["hist"]
    assert (np.abs(hg - ho) <= HIST_REL * ho + HIST_FLOOR * info_o["r_zero"]).all()
    assert relerr(H.get_solution(), R.get_phi()) < TOL


def test_wcycle_fewer_iterations_and_update_count(dev):
    """W-cycles need fewer iterations than V-cycles, and the solver's
    cell-update count follows the N_cycles recursion."""
    w = CASES["ball32"]
    out = {}
    for nc in (1, 2):
        H, _ = make_pair(w, dev, order=2, n_cycles=nc)
        st, info = H.solve(1e-10, 60)
        assert st == 0
        out[nc] = info
    assert out[2]["cycles"] < out[1]["cycles"]
    per = [out[nc]["cell_updates"] / out[nc]["cycles"] for nc in (1, 2)]
    assert per[1] > per[0]


def test_wcycle_mixed_precision(dev, oracle):
    """The mixed form with W-cycles reaches the tolerance as checked by the
    oracle's FP64 operator."""
    w = CASES["blob48x32x40"]
    H, R = make_pair(w, dev, precision=1, n_cycles=2)
    st, info = H.solve(1e-9, 80)
    assert st == 0
    R.set_phi(H.get_solution())
    assert R.residual_norm() / R.residual_norm_zero() < 1e-9 * (1 + 1e-6)


R0, NC, RADIUS = 0.04, 64, 0.2


def test_boundary_gradient_chain_on_device(dev, oracle):
    """Section 5.1's boundary-gradient test run as the one-way interface on
    the device: the coarse level is solved on the GPU, its solution stays in
    device memory and gives each refined patch its Dirichlet values through
    mg_set_dirichlet_from_coarse.  Every step matches the oracle's chain, and
    the error behaves as the paper describes (flat while the border is more
    than 3 r0 from the mass, larger at the mass)."""
    c = W.concentrated_coarse(NC, R0)
    Hc = B.Hierarchy(torch.from_numpy(c["mask"]).to(dev), c["h"])
    Hc.set_rhs(torch.from_numpy(c["rho"]).to(dev))
    Hc.set_dirichlet(*(torch.from_numpy(a).to(dev) for a in (c["bx"], c["by"], c["bz"])))
    st, info = Hc.solve(1e-11, 100)
    assert st == 0
    phi_c = torch.empty(c["mask"].shape, dtype=torch.float64, device=dev)
    Hc.get_solution(phi_c)
    Rc = oracle.Hierarchy(c["mask"], c["h"])
    Rc.set_rhs(c["rho"])
    Rc.set_faces(c["bx"], c["by"], c["bz"])
    st_o, info_o = Rc.solve(1e-11, 100)
    assert info["cycles"] == info_o["cycles"]
    phi_c_o = Rc.get_phi()
    assert relerr(phi_c.cpu().numpy(), phi_c_o) < TOL

    errs = {}
    for d in (0.2, 0.12, 0.0):
        p = W.concentrated_patch(NC, R0, RADIUS, d)
        H = B.Hierarchy(torch.from_numpy(p["mask"]).to(dev), p["h"])
        H.set_rhs(torch.from_numpy(p["rho"]).to(dev))
        H.set_dirichlet_from_coarse(phi_c, p["origin"])
        st, info = H.solve(1e-7, 50)
        R = oracle.Hierarchy(p["mask"], p["h"])
        R.set_rhs(p["rho"])
        R.set_faces(*oracle.dirichlet_from_coarse(p["mask"], phi_c_o, p["origin"]))
        st_o, info_o = R.solve(1e-7, 50)
        assert st == st_o == 0 and info["cycles"] == info_o["cycles"]
        phi = H.get_solution()
        assert relerr(phi, R.get_phi()) < 1e-11
        errs[d] = np.abs(phi - p["phi_exact"])[p["mask"] > 0].max()
    assert max(errs[0.2], errs[0.12]) <= 1.1 * min(errs[0.2], errs[0.12])
    assert errs[0.0] >= 2.0 * errs[0.2]


@pytest.mark.parametrize("name", ["ball32", "holes32", "blob48x32x40"])
@pytest.mark.parametrize("n_cycles,precision", [(1, 0), (2, 0), (3, 0), (1, 1), (2, 1)])
def test_coarsest_map_matches_the_sweeps(dev, name, n_cycles, precision):
    """The coarsest solve through its precomputed map (option coarse_matrix)
    against the coarse_sweeps sweeps it tabulates, in V- and W-cycles of both
    forms: the same decisions and cycle counts, solutions and residual
    histories within rounding."""
    w = CASES[name]
    res = []
    for cm in (0, 1):
        H, _ = make_pair(w, dev, n_cycles=n_cycles, precision=precision, coarse_matrix=cm)
        st, info = H.solve(1e-10, 60)
        assert st == 0
        res.append((info, H.get_solution()))
    (i0, s0), (i1, s1) = res
    assert (i0["cycles"], i0["order"], i0["switched"]) == (i1["cycles"], i1["order"], i1["switched"])
    assert relerr(s1, s0) < 1e-12
    assert np.abs(i1["hist"] - i0["hist"]).max() <= 1e-9 * i0["r_zero"]


def test_coarsest_map_follows_a_mask_update(dev):
    """The map is rebuilt with the hierarchy: after update_mask a W(2) solve
    equals a fresh hierarchy's."""
    a, b = CASES["blob48x32x40"], W.blob_patch((40, 32, 48), seed=105)
    H, _ = make_pair(a, dev, n_cycles=2)
    H.solve(1e-10, 60)
    H.update_mask(torch.from_numpy(b["mask"]).to(dev))
    H.set_rhs(torch.from_numpy(b["rho"]).to(dev))
    H.set_dirichlet_from_coarse(torch.from_numpy(b["phi_c"]).to(dev), b["origin"])
    H.set_solution(None)
    st, info = H.solve(1e-10, 60)
    F, _ = make_pair(b, dev, n_cycles=2)
    st2, info2 = F.solve(1e-10, 60)
    assert st == st2 == 0 and info["cycles"] == info2["cycles"]
    assert np.array_equal(H.get_solution(), F.get_solution())
