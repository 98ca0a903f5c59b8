"""The batched multi-patch solve (mg_batch_*) against the FP64 oracle, patch
by patch: every patch of a batch must do exactly what the oracle does when
it solves that patch alone (same cycle count, order, switch decision and
hold counter; solution to 1e-12 relative; residual history to 1e-10).  The
launch parameters must not change the results, and the autotuner must leave
the batch's solutions and hold counters as it found them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
HIST_REL, HIST_FLOOR = 1e-10, 1e-13


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def relerr(a, b):
    return np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300)


def _sieve(shape, seed):
    """Every cell active except the (even, even, even) ones: each coarse cell
    has 7 active children, so level 1 has unknowns in second order but none
    in first order (the first-order hierarchy ends at level 0)."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mask = (~((i % 2 == 0) & (j % 2 == 0) & (k % 2 == 0))).astype(np.int8)
    return {"mask": mask, "rho": W.random_field(shape, seed), "h": 0.05, "faces": W.random_faces(shape, seed + 1)}


def _line(n, seed):
    """A single row of active cells: no coarse level has an unknown."""
    mask = np.zeros((4, 5, n), np.int8)
    mask[2, 2, :] = 1
    return {"mask": mask, "rho": W.random_field(mask.shape, seed), "h": 0.1,
            "faces": W.random_faces(mask.shape, seed + 1)}


def _patches():
    m = W.random_mask((10, 12, 17), seed=101, p_active=0.7)
    return [
        W.ball(24),
        {"mask": m, "rho": W.random_field(m.shape, 102), "h": 0.07, "faces": W.random_faces(m.shape, 103)},
        W.holes(32),
        W.blob_patch((40, 32, 48), seed=104),
        _sieve((18, 20, 16), 105),
        _line(13, 107),
    ]


PATCHES = _patches()


def _faces(oracle, w):
    if "phi_c" in w:
        return oracle.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"])
    if "faces" in w:
        return w["faces"]
    return w.get("bx"), w.get("by"), w.get("bz")


def make_batch(dev, oracle, patches, **opts):
    masks = [torch.from_numpy(w["mask"]).to(dev) for w in patches]
    Bt = B.Batch(masks, [w["h"] for w in patches], **opts)
    refs = []
    for p, w in enumerate(patches):
        P = Bt.patch(p)
        P.set_rhs(torch.from_numpy(w["rho"]).to(dev))
        if "phi_c" in w:
            P.set_dirichlet_from_coarse(torch.from_numpy(w["phi_c"]).to(dev), w["origin"])
        else:
            f = _faces(oracle, w)
            if f[0] is not None:
                P.set_dirichlet(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in f))
        R = oracle.Hierarchy(w["mask"], w["h"])
        R.set_rhs(w["rho"])
        f = _faces(oracle, w)
        if f[0] is not None:
            R.set_faces(*f)
        refs.append(R)
    return Bt, refs


def test_degenerate_patches_are_what_they_claim(oracle):
    s, l = PATCHES[4], PATCHES[5]
    R = oracle.Hierarchy(s["mask"], s["h"])
    assert R.deepest(1) == 0 and R.deepest(2) >= 1
    R = oracle.Hierarchy(l["mask"], l["h"])
    assert R.deepest(1) == 0 and R.deepest(2) == 0


@pytest.mark.parametrize("order", [1, 2])
def test_batch_vcycles_match_oracle(dev, oracle, order):
    Bt, refs = make_batch(dev, oracle, PATCHES, order=order)
    r0 = [R.residual_norm_zero() for R in refs]
    for k in range(3):
        rel = Bt.vcycle()
        for p, R in enumerate(refs):
            R.vcycle(order=order)
            assert relerr(Bt.patch(p).get_solution(), R.get_phi()) < TOL, (p, k)
            rel_o = R.residual_norm() / r0[p]
            assert abs(rel[p] - rel_o) <= HIST_REL * rel_o + 1e-15, (p, k)


@pytest.mark.parametrize("order_opt", [0, 1, 2])
def test_batch_solve_matches_oracle(dev, oracle, order_opt):
    Bt, refs = make_batch(dev, oracle, PATCHES, order=order_opt)
    for rep in range(2):   # the second solve starts from the first's solution and hold counters
        st, infos = Bt.solve(1e-9, 80)
        sts = []
        for p, R in enumerate(refs):
            st_o, io = R.solve(1e-9, 80, order=order_opt)
            ig = infos[p]
            # forced second order does not converge on the holes cube (Section 4)
            assert ig["status"] == {0: 0, 1: 5, 2: 6}[st_o], (rep, p)
            sts.append(ig["status"])
            for key in ("cycles", "order", "switched"):
                assert ig[key] == io[key], (rep, p, key)
            assert ig["r_zero"] == pytest.approx(io["r_zero"], rel=1e-13)
            ho, hg = io["hist"], ig["hist"]
            assert hg.shape == ho.shape
            assert (np.abs(hg - ho) <= HIST_REL * ho + HIST_FLOOR * io["r_zero"]).all(), (rep, p)
            assert relerr(Bt.patch(p).get_solution(), R.get_phi()) < TOL, (rep, p)
            assert Bt.patch(p).hold == R.hold
        assert st == max(sts)
        if order_opt != 2:
            assert st == 0


def test_batch_small_islands_switch(dev, oracle):
    """Three copies of the holes cube with different right-hand sides: each
    trips the switch on its own and holds first order for 10 solves."""
    ws = [W.holes(32, seed=s) for s in (5, 6, 7)]
    Bt, refs = make_batch(dev, oracle, ws)
    for s in range(3):
        for p, R in enumerate(refs):
            Bt.patch(p).set_solution(None)
            R.set_phi(None)
        st, infos = Bt.solve(1e-8, 80)
        for p, R in enumerate(refs):
            st_o, io = R.solve(1e-8, 80)
            assert (infos[p]["cycles"], infos[p]["order"], infos[p]["switched"]) == (io["cycles"], io["order"],
                                                                                    io["switched"])
            assert Bt.patch(p).hold == R.hold
            assert relerr(Bt.patch(p).get_solution(), R.get_phi()) < TOL


def test_launch_parameters_do_not_change_results(dev, oracle):
    sols = None
    for threads, pers, bots, chunk in ((256, 0, 4096, 0), (128, 0, 1024, 0), (512, 152 * 4, 2048, 0),
                                       (256, 152 * 8, 64, 0), (128, 0, 4096, 1024), (256, 152 * 4, 2048, 64),
                                       (512, 0, 4096, 4096)):
        Bt, _ = make_batch(dev, oracle, PATCHES)
        t = Bt.tuning
        t.threads, t.persistent_ctas, t.bottom_slots, t.chunk = threads, pers, bots, chunk
        Bt.tuning = t
        for _ in range(3):
            Bt.vcycle(want_rel=False)
        got = [Bt.patch(p).get_solution() for p in range(len(PATCHES))]
        if sols is None:
            sols = got
        else:
            for a, b in zip(sols, got):
                assert np.array_equal(a, b)
        Bt.close()


def test_batch_equals_single_hierarchy_solves(dev, oracle):
    """The batch and mg_solve on each patch alone take the same decisions and
    land on the same solution (to rounding of the norm's summation order)."""
    Bt, _ = make_batch(dev, oracle, PATCHES)
    st, infos = Bt.solve(1e-9, 80)
    for p, w in enumerate(PATCHES):
        H = B.Hierarchy(torch.from_numpy(w["mask"]).to(dev), w["h"])
        H.set_rhs(torch.from_numpy(w["rho"]).to(dev))
        if "phi_c" in w:
            H.set_dirichlet_from_coarse(torch.from_numpy(w["phi_c"]).to(dev), w["origin"])
        else:
            f = _faces(oracle, w)
            if f[0] is not None:
                H.set_dirichlet(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in f))
        st1, i1 = H.solve(1e-9, 80)
        assert (i1["cycles"], i1["order"], i1["switched"]) == (infos[p]["cycles"], infos[p]["order"],
                                                              infos[p]["switched"])
        assert i1["cell_updates"] == infos[p]["cell_updates"]
        assert relerr(Bt.patch(p).get_solution(), H.get_solution()) < TOL


def test_autotune_restores_state_and_keeps_parity(dev, oracle):
    Bt, refs = make_batch(dev, oracle, PATCHES[:4])
    for p in range(4):
        Bt.patch(p).set_solution(torch.from_numpy(W.random_field(PATCHES[p]["mask"].shape, 900 + p)).to(dev))
    before = [Bt.patch(p).get_solution() for p in range(4)]
    holds = [Bt.patch(p).hold for p in range(4)]
    best = Bt.autotune(reps=2, tol=1e-8, max_cycles=60, flags=B.MG_TUNE_SCHEDULE)
    assert best.threads in (128, 256, 512) and best.bottom_slots in (1024, 2048, 4096)
    assert best.chunk in (0, best.threads, 2 * best.threads, 4 * best.threads, 8 * best.threads)
    assert (best.n_pre, best.n_post) in ((1, 1), (2, 1), (2, 2), (3, 3)) and best.ms_per_cycle > 0
    for p in range(4):
        assert np.array_equal(Bt.patch(p).get_solution(), before[p])
        assert Bt.patch(p).hold == holds[p]
    # the chosen schedule is the method with those sweep counts: the oracle
    # with the same counts takes the same path
    st, infos = Bt.solve(1e-9, 80)
    for p, R in enumerate(refs):
        R.set_phi(before[p])
        st_o, io = R.solve(1e-9, 80, n_pre=best.n_pre, n_post=best.n_post)
        assert infos[p]["cycles"] == io["cycles"] and infos[p]["order"] == io["order"]
        assert relerr(Bt.patch(p).get_solution(), R.get_phi()) < TOL


def test_batch_launch_count_and_errors(dev, oracle):
    Bt, _ = make_batch(dev, oracle, PATCHES[:3])
    Bt.vcycle(want_rel=False)  # the first cycle also computes each patch's b / D
    c0 = B.mg_launch_count()
    Bt.vcycle(want_rel=False)
    nodes = Bt.launches_per_cycle()
    assert nodes > 0 and B.mg_launch_count() - c0 == nodes
    with pytest.raises(B.MGError) as e:
        t = Bt.tuning
        t.threads = 100
        Bt.tuning = t
    assert e.value.status == B.MG_ERR_INVALID_ARG
    masks = [torch.from_numpy(w["mask"]).to(dev) for w in PATCHES[:2]]
    with pytest.raises(B.MGError) as e:
        B.Batch(masks, [0.1, 0.1], precision=1)
    assert e.value.status == B.MG_ERR_INVALID_ARG
    empty = torch.zeros((4, 4, 4), dtype=torch.int8, device=dev)
    with pytest.raises(B.MGError) as e:
        B.Batch([masks[0], empty], [0.1, 0.1])
    assert e.value.status == B.MG_ERR_EMPTY_DOMAIN and "patch 1" in e.value.message


@pytest.mark.slow
def test_full_size_96_patches_sampled(dev, oracle):
    """The 96-patch workload (edges from {32, 48, 64, 96, 128}): every patch
    converges, and sampled patches match the oracle's solve of that patch."""
    ws = W.amr_patches(96, seed=4)
    masks = [torch.from_numpy(w["mask"]).to(dev) for w in ws]
    Bt = B.Batch(masks, [w["h"] for w in ws])
    for p, w in enumerate(ws):
        P = Bt.patch(p)
        P.set_rhs(torch.from_numpy(w["rho"]).to(dev))
        P.set_dirichlet_from_coarse(torch.from_numpy(w["phi_c"]).to(dev), w["origin"])
    st, infos = Bt.solve(1e-8, 100)
    assert st == 0 and all(i["rel"] < 1e-8 for i in infos)
    for p in (0, 37, 95):
        w = ws[p]
        R = oracle.Hierarchy(w["mask"], w["h"])
        R.set_rhs(w["rho"])
        R.set_faces(*oracle.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"]))
        st_o, io = R.solve(1e-8, 100)
        assert (infos[p]["cycles"], infos[p]["order"], infos[p]["switched"]) == (io["cycles"], io["order"],
                                                                                io["switched"])
        assert relerr(Bt.patch(p).get_solution(), R.get_phi()) < TOL
