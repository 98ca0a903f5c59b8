"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: worked
numbers printed in the paper's figures, closed forms (exactness of the
stencil on quadratics, of the ghost extrapolation and of P2 on linear
fields), a dense direct solve, the observed order of the discretisation
error, and the convergence behaviour the paper reports.  No expected value
comes from the CUDA library.
"""
import json
import os

import numpy as np
import pytest

from paper_1104_1703_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Fig. 5 (ghost value) and Fig. 6 (mask restriction): worked numbers
# ---------------------------------------------------------------------------

def test_fig5_theta_and_ghost(oracle):
    g = _golden("fig5_ghost.json")
    th = oracle.theta(g["m_i"], g["m_j"])
    assert th == pytest.approx(g["theta"], rel=1e-15)
    # boundary position: cell spacing 2 in the figure, cell i at x = 5
    xb = g["x_i"] - th * (g["x_i"] - g["x_j"])
    assert xb == pytest.approx(g["x_boundary"], abs=1e-3)
    assert oracle.ghost(g["phi_i"], g["phi_b"], th) == pytest.approx(g["ghost"], rel=1e-15)


def test_fig5_configuration_in_coarse_operator(oracle):
    """The coarse-level operator uses theta from the level's mask: a level-1
    neighbour with m = -0.5 next to a full cell (m = 1) sits at theta = 2/3;
    with Phi_b = 0 on coarse levels the ghost is Phi_i - Phi_i/theta."""
    S = np.full((3, 3, 3), 8, dtype=np.int64)
    S[1, 1, 0] = -4  # m = -4/8 = -0.5
    hl = 0.125
    phi = np.full((3, 3, 3), -0.5)
    phi[S <= 0] = 0.0
    lap = oracle.laplacian(S, 1, 2, hl, phi)
    # only the -x face differs from a constant field: (ghost - Phi_i)/h^2
    expected = (oracle.ghost(-0.5, 0.0, 2.0 / 3.0) - (-0.5)) / hl ** 2
    assert expected == pytest.approx(0.75 / hl ** 2, rel=1e-15)
    assert lap[1, 1, 1] == pytest.approx(expected, rel=1e-13)


def test_fig6_island_restriction(oracle):
    g = _golden("fig6_island.json")
    # 2D figure: one -1 among four children gives 1/2; the 3D analogue is 3/4
    assert (3 * 1 + (-1)) / 4 == g["m_coarse_2d"]
    S0 = np.ones((4, 4, 4), dtype=np.int64)
    S0[1, 0, 1] = -1
    S1 = oracle.mask_restrict(S0, 0)
    assert S1[0, 0, 0] / 8 == g["m_coarse_3d"]
    assert (S1.ravel()[1:] == 8).all()
    assert oracle.is_active(int(S1[0, 0, 0]), 1, 2)       # island lost in second order
    assert not oracle.is_active(int(S1[0, 0, 0]), 1, 1)   # kept as a constraint in first order (m < 1)


def test_mask_restriction_odd_dims(oracle):
    """Missing children of an odd dimension are outside the box (m = -1)."""
    S0 = np.ones((2, 2, 3), dtype=np.int64)
    S1 = oracle.mask_restrict(S0, 0)
    assert S1.shape == (1, 1, 2)
    assert S1[0, 0, 0] == 8 and S1[0, 0, 1] == 0          # 4 inside, 4 missing
    S2 = oracle.mask_restrict(np.full((1, 1, 3), 8, dtype=np.int64), 1)
    assert S2.shape == (1, 1, 2)
    assert S2[0, 0, 0] == 2 * 8 - 6 * 8 and S2[0, 0, 1] == 8 - 7 * 8


# ---------------------------------------------------------------------------
# Fig. 3: R1 and P2
# ---------------------------------------------------------------------------

def test_r1_average(oracle):
    r = np.arange(1.0, 9.0).reshape(2, 2, 2)
    assert oracle.restrict(r)[0, 0, 0] == 4.5
    r = np.ones((3, 3, 3))
    rc = oracle.restrict(r)
    assert rc.shape == (2, 2, 2)
    assert rc[0, 0, 0] == 1.0 and rc[1, 1, 1] == 1.0 / 8 and rc[0, 1, 1] == 2.0 / 8


def test_p2_weights_fig3(oracle):
    g = _golden("fig3_p2.json")
    ec = np.zeros((5, 5, 5))
    ec[2, 2, 2] = 1.0
    Sf = np.ones((10, 10, 10), dtype=np.int64)
    fine = oracle.prolong_add(ec, Sf, 0, 2, np.zeros((10, 10, 10)))
    w1 = g["weights_1d"]  # fine cells 2I-1, 2I, 2I+1, 2I+2 around coarse I
    for a, i in enumerate(range(3, 7)):
        for b, j in enumerate(range(3, 7)):
            for c, k in enumerate(range(3, 7)):
                assert fine[k, j, i] == pytest.approx(w1[a] * w1[b] * w1[c], rel=1e-15)
    # the 2D weights of the figure are the products of the 1D ones
    assert w1[1] * w1[1] == g["weights_2d"][0] and w1[1] * w1[0] == g["weights_2d"][1]
    assert w1[0] * w1[0] == g["weights_2d"][3]
    assert fine[4, 4, 4] == pytest.approx(27 / 64) and fine[3, 3, 3] == pytest.approx(1 / 64)
    assert fine.sum() == pytest.approx(8.0)  # P2 conserves: 8 fine cells per coarse cell


def test_p2_reproduces_linear_fields(oracle):
    cz, cy, cx = 6, 5, 7
    K, J, I = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    lin = lambda x, y, z: 0.3 * x - 1.7 * y + 0.9 * z + 2.5  # noqa: E731
    ec = lin(2 * I + 1.0, 2 * J + 1.0, 2 * K + 1.0)        # coarse centres in fine units
    nz, ny, nx = 2 * cz, 2 * cy, 2 * cx
    fine = oracle.prolong_add(ec, np.ones((nz, ny, nx), dtype=np.int64), 0, 2, np.zeros((nz, ny, nx)))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    exact = lin(i + 0.5, j + 0.5, k + 0.5)
    interior = (i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1) & (k > 0) & (k < nz - 1)
    np.testing.assert_allclose(fine[interior], exact[interior], rtol=1e-13, atol=1e-13)
    # prolongation only corrects active fine cells
    Sf = np.ones((nz, ny, nx), dtype=np.int64)
    Sf[0, 0, 0] = -1
    f2 = oracle.prolong_add(ec, Sf, 0, 2, np.zeros((nz, ny, nx)))
    assert f2[0, 0, 0] == 0.0 and f2[0, 0, 1] == fine[0, 0, 1]


# ---------------------------------------------------------------------------
# Section 2: 7-point stencil; Section 3: ghost reconstruction
# ---------------------------------------------------------------------------

def test_stencil_exact_on_quadratics(oracle):
    n, h = 10, 0.1
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    q = 1.5 * x * x - 0.25 * y * y + 0.75 * z * z + 0.3 * x * y - 0.6 * y * z + 0.2 * z * x + x - 2 * z + 3
    S = np.ones((n, n, n), dtype=np.int64)
    lap = oracle.laplacian(S, 0, 2, h, q)
    inner = lap[1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(inner, 2 * (1.5 - 0.25 + 0.75), rtol=1e-11)
    # the same at a coarse level (cell size 4h, all active)
    S2 = np.full((n, n, n), 64, dtype=np.int64)
    lap2 = oracle.laplacian(S2, 2, 2, 4 * h, q.copy())
    # the field was sampled with spacing h, so the coarse stencil sees (4h)^2 scaling
    np.testing.assert_allclose(lap2[1:-1, 1:-1, 1:-1], 2 * (1.5 - 0.25 + 0.75) / 16, rtol=1e-11)


def test_linear_fields_exact_with_ghosts(oracle):
    """Linear extrapolation through the face value is exact for linear fields:
    with Phi_b = Phi(face centre), Laplacian(Phi) = 0 at every active cell of
    an arbitrary mask, boundary cells included."""
    shape = (9, 10, 12)
    mask = W.random_mask(shape, seed=11, p_active=0.6)
    h = 0.05
    lin = lambda x, y, z: 0.7 * x - 1.1 * y + 0.4 * z + 0.25  # noqa: E731
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = lin((i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h)
    bx, by, bz = W.faces_from_function(lin, nx, ny, nz, h)
    S = np.where(mask > 0, 1, -1).astype(np.int64)
    lap = oracle.laplacian(S, 0, 2, h, phi, bx, by, bz)
    assert np.abs(lap[mask > 0]).max() < 1e-11 / h ** 2
    # a quadratic is NOT reproduced at boundary cells (first-order truncation
    # of the ghost there), so the test above is not vacuous
    phi2 = ((i + 0.5) * h) ** 2
    q = lambda x, y, z: x * x + 0 * y + 0 * z  # noqa: E731
    lap2 = oracle.laplacian(S, 0, 2, h, phi2, *W.faces_from_function(q, nx, ny, nz, h))
    assert np.abs(lap2[mask > 0] - 2.0).max() > 0.1


@pytest.mark.parametrize("face,levels", [(3, (1,)), (4, (1, 2))])
def test_coarse_boundary_position_half_space(oracle, face, levels):
    """A fine domain {x > face} (boundary on a fine face).  Where the mask
    averaging puts the coarse zero crossing exactly on that face, a linear
    field vanishing there has zero coarse Laplacian: this fixes theta from
    the mask values at coarse levels (Section 3)."""
    nx, ny, nz = 16, 16, 16
    mask = np.zeros((nz, ny, nx), dtype=np.int8)
    mask[:, :, face:] = 1
    S = np.where(mask > 0, 1, -1).astype(np.int64)
    for level in range(1, max(levels) + 1):
        S = oracle.mask_restrict(S, level - 1)
        if level not in levels:
            continue
        cz, cy, cx = S.shape
        cell = 2 ** level
        X = cell * (np.arange(cx) + 0.5)           # coarse centres in fine units
        phi = np.broadcast_to(X - face, (cz, cy, cx)).copy()
        phi[S <= 0] = 0.0
        lap = oracle.laplacian(S, level, 2, cell * 0.1, phi)
        act = S > 0
        inner = np.zeros_like(act)
        inner[1:-1, 1:-1, :-1] = True   # the +x box edge has its own Phi_b = 0 face
        sel = act & inner
        assert sel.sum() > 0
        assert np.abs(lap[sel]).max() < 1e-12 / (cell * 0.1) ** 2
        # and theta = 1/2 everywhere (the fine-level value) would be wrong here
        # unless the crossing happens to sit half a cell out
        if face == 3:
            edge = act & inner & (np.roll(S, 1, axis=2) <= 0)
            th = oracle.theta(S[edge][0] / 8 ** level, np.roll(S, 1, axis=2)[edge][0] / 8 ** level)
            assert th == 1.0


def test_gs_update_solves_its_row(oracle):
    """After a red-black sweep every black cell satisfies its own equation
    (Laplacian(Phi) - rho = 0) exactly up to rounding, for all three kinds of
    neighbour: active, ghost with face values, NGP zero."""
    shape = (7, 9, 11)
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    black = ((i + j + k) & 1) == 1
    mask = W.random_mask(shape, seed=5, p_active=0.65)
    rho = W.random_field(shape, seed=6)
    phi0 = W.random_field(shape, seed=7)
    bx, by, bz = W.random_faces(shape, seed=8)
    S = np.where(mask > 0, 1, -1).astype(np.int64)
    cases = [(S, 0, 2, (bx, by, bz))]
    S1 = np.where(mask > 0, 8, np.where(W.random_mask(shape, 9) > 0, 3, -5)).astype(np.int64)
    cases += [(S1, 1, 2, (None, None, None)), (S1, 1, 1, (None, None, None))]
    for Sx, level, order, faces in cases:
        act = np.vectorize(lambda s: oracle.is_active(int(s), level, order))(Sx)
        p0 = np.where(act, phi0, 0.0)
        hl = 0.1 * 2 ** level
        p1 = oracle.gs_sweeps(Sx, level, order, hl, p0, rho, 1, *faces)
        r = oracle.residual(Sx, level, order, hl, p1, rho, *faces)
        scale = np.abs(rho).max() + np.abs(p1).max() / hl ** 2
        assert np.abs(r[black & act]).max() < 1e-13 * scale
        assert np.abs(r[~black & act]).max() > 1e-3 * scale   # red cells moved afterwards
        assert (p1[~act] == 0).all()


# ---------------------------------------------------------------------------
# Whole discrete problem: dense direct solve, symmetry, definiteness
# ---------------------------------------------------------------------------

def _assemble(oracle, S, level, order, hl):
    act = np.vectorize(lambda s: oracle.is_active(int(s), level, order))(S)
    idx = np.flatnonzero(act.ravel())
    A = np.zeros((idx.size, idx.size))
    for col, c in enumerate(idx):
        e = np.zeros(S.size)
        e[c] = 1.0
        A[:, col] = oracle.laplacian(S, level, order, hl, e.reshape(S.shape)).ravel()[idx]
    return A, idx


def test_dense_direct_solve_8cube(oracle):
    shape = (8, 8, 8)
    w = W.ball(8, radius=0.45)
    mask = w["mask"].copy()
    mask[W.random_mask(shape, seed=21, p_active=0.15) > 0] = 0    # punch a few holes
    mask[4, 4, 4] = 1
    rho = W.random_field(shape, seed=22)
    bx, by, bz = W.random_faces(shape, seed=23)
    h = 1.0 / 8
    S = np.where(mask > 0, 1, -1).astype(np.int64)
    A, idx = _assemble(oracle, S, 0, 2, h)
    c0 = oracle.laplacian(S, 0, 2, h, np.zeros(shape), bx, by, bz).ravel()[idx]
    x = np.linalg.solve(A, rho.ravel()[idx] - c0)
    H = oracle.Hierarchy(mask, h)
    H.set_rhs(rho)
    H.set_faces(bx, by, bz)
    st, info = H.solve(1e-13, 200, order=2)
    assert st == 0
    phi = H.get_phi().ravel()[idx]
    assert np.abs(phi - x).max() <= 1e-11 * np.abs(x).max()


@pytest.mark.parametrize("level,order", [(0, 2), (1, 2), (1, 1), (2, 2), (2, 1)])
def test_operator_symmetric_negative_definite(oracle, level, order):
    w = W.holes(16, seed=31, n_spheres=12, r_min=0.5, r_max=2.5)
    S = np.where(w["mask"][:, :, :12] > 0, 1, -1).astype(np.int64)
    for l in range(level):
        S = oracle.mask_restrict(S, l)
    A, idx = _assemble(oracle, S, level, order, 0.1)
    assert idx.size > 10
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).max() < 0


# ---------------------------------------------------------------------------
# Convergence: discretisation order, V-cycle rate, small islands
# ---------------------------------------------------------------------------

def _solve_ball(oracle, n, **kw):
    w = W.ball(n)
    H = oracle.Hierarchy(w["mask"], w["h"])
    H.set_rhs(w["rho"])
    H.set_faces(w["bx"], w["by"], w["bz"])
    st, info = H.solve(1e-10, 60, **kw)
    return w, H, st, info


def test_second_order_potential_error_ball(oracle):
    """The potential error against the manufactured solution falls at second
    order on a Cartesian grid (Section 5.1)."""
    errs = []
    for n in (16, 32, 64):
        w, H, st, info = _solve_ball(oracle, n)
        assert st == 0
        m = w["mask"] > 0
        e = (H.get_phi() - w["phi_exact"])[m]
        errs.append((np.abs(e).max(), np.sqrt((e ** 2).mean())))
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert (orders >= 1.8).all(), orders


def test_vcycle_rate_grid_independent_ball(oracle):
    """Smooth boundary, second order: textbook, grid-independent convergence
    with a monotone residual (Section 4, disk case)."""
    rates = []
    for n in (16, 32, 64):
        _, _, st, info = _solve_ball(oracle, n, order=2)
        hist = info["hist"]
        assert st == 0 and info["order"] == 2
        ratio = hist[1:] / hist[:-1]
        assert (ratio < 0.25).all(), ratio
        rates.append(ratio[2:].max())
    assert max(rates) - min(rates) < 0.05


def test_small_islands_first_order_fix_and_switch(oracle):
    """Many sub-cell holes: second-order coarse reconstruction fails (ratio
    above eta, no convergence), first order converges, and the run-time
    switch picks first order and holds it for the next 10 solves (Section 4)."""
    w = W.holes(64)
    H = oracle.Hierarchy(w["mask"], w["h"])
    H.set_rhs(w["rho"])
    st2, i2 = H.solve(1e-8, 40, order=2)
    assert st2 != 0 and (i2["hist"][1:] / i2["hist"][:-1]).max() > 0.5
    H.set_phi(None)
    st1, i1 = H.solve(1e-8, 60, order=1)
    assert st1 == 0 and (np.diff(i1["hist"]) < 0).all()
    H.set_phi(None)
    assert H.hold == 0
    st0, i0 = H.solve(1e-8, 60, order=0)
    assert st0 == 0 and i0["switched"] == 1 and i0["order"] == 1 and H.hold == 10
    for expect in range(9, -1, -1):
        H.set_phi(None)
        st, info = H.solve(1e-3, 60, order=0)
        assert st == 0 and info["order"] == 1 and info["switched"] == 0 and H.hold == expect
    H.set_phi(None)
    st, info = H.solve(1e-8, 60, order=0)
    assert info["switched"] == 1  # back to second order first, which trips again


def diverging_guess(oracle, w, scale=1e-3):
    """Initial guess Phi* + e on `w`: Phi* is the converged discrete solution
    (first order, 1e-13) and e the error mode that second-order V-cycles
    amplify most, found by 30 normalised V-cycles on rho = 0 from a seeded
    random field; e is scaled so that ||r(guess)|| = scale * ||r(0)||."""
    act = w["mask"] > 0
    H = oracle.Hierarchy(w["mask"], w["h"])
    H.set_rhs(np.zeros_like(w["rho"]))
    H.set_phi(W.random_field(w["mask"].shape, seed=11) * act)
    for _ in range(30):
        H.vcycle(order=2)
        e = H.get_phi()
        H.set_phi(e / np.abs(e).max())
    e, r_e = H.get_phi(), H.residual_norm()
    H.set_rhs(w["rho"])
    H.set_phi(None)
    st, _ = H.solve(1e-13, 200, order=1)
    assert st == 0
    return H.get_phi() + e * (scale * H.residual_norm_zero() / r_e)


def test_switch_restart_from_initial_guess(oracle):
    """Reading of Section 4 (the paper does not say what becomes of the
    iterate when the switch trips): if the tripping residual is above the
    initial one, the solve restarts in first order from the initial guess.
    On the 64^3 holes domain the second-order V-cycle amplifies its dominant
    error mode (ratio > 1), so a guess carrying that mode trips the switch
    on the first cycle above r_init; every later residual must then be, to
    rounding, the history of a first-order solve from the same guess."""
    w = W.holes(64)
    g = diverging_guess(oracle, w)
    H = oracle.Hierarchy(w["mask"], w["h"])
    H.set_rhs(w["rho"])
    H.set_phi(g)
    st0, i0 = H.solve(1e-10, 80, order=0)
    h0 = i0["hist"]
    assert st0 == 0 and i0["switched"] == 1 and i0["order"] == 1 and H.hold == 10
    assert h0[1] > h0[0]
    phi0 = H.get_phi()
    H.hold = 0
    H.set_phi(g)
    st1, i1 = H.solve(1e-10, 80, order=1)
    h1 = i1["hist"]
    assert st1 == 0 and i1["cycles"] == i0["cycles"] - 1
    np.testing.assert_allclose(h0[2:], h1[1:], rtol=1e-12, atol=0)
    np.testing.assert_allclose(phi0, H.get_phi(), rtol=0, atol=1e-12 * np.abs(phi0).max())


def test_relative_residual_reference(oracle):
    """||r(Phi=0)|| with zero Dirichlet values on an all-active box is
    ||rho||: the reference of the relative residual."""
    rho = W.random_field((6, 5, 4), seed=41)
    H = oracle.Hierarchy(np.ones((6, 5, 4), dtype=np.int8), 0.25)
    H.set_rhs(rho)
    assert H.residual_norm_zero() == pytest.approx(np.linalg.norm(rho), rel=1e-14)


def test_zero_problem_returns_zero(oracle):
    H = oracle.Hierarchy(np.ones((4, 4, 4), dtype=np.int8), 0.25)
    H.set_rhs(np.zeros((4, 4, 4)))
    H.set_phi(np.ones((4, 4, 4)))
    st, info = H.solve(1e-8, 10)
    assert st == 0 and info["cycles"] == 0 and (H.get_phi() == 0).all()


def test_non_finite_data_is_divergence(oracle):
    rho = np.ones((4, 4, 4))
    rho[1, 2, 3] = np.nan
    H = oracle.Hierarchy(np.ones((4, 4, 4), dtype=np.int8), 0.25)
    H.set_rhs(rho)
    st, info = H.solve(1e-8, 10)
    assert st == 2 and info["cycles"] == 0


def test_deepest_levels_ball32(oracle):
    """The r = 0.4 ball at 32^3 has no active cell at 2^3 (second order) and
    no full cell at 4^3 (first order)."""
    w = W.ball(32)
    H = oracle.Hierarchy(w["mask"], w["h"])
    assert H.num_levels == 5
    assert H.deepest(2) == 3 and H.deepest(1) == 2


# ---------------------------------------------------------------------------
# One-way interface: boundary values from the coarser AMR level
# ---------------------------------------------------------------------------

def test_dirichlet_from_coarse_linear_exact(oracle):
    shape = (6, 8, 10)
    nz, ny, nx = shape
    mask = W.random_mask(shape, seed=51, p_active=0.6)
    cz, cy, cx = nz // 2 + 2, ny // 2 + 2, nx // 2 + 2
    K, J, I = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    lin = lambda x, y, z: 0.5 * x - 0.25 * y + 0.125 * z + 1.0  # noqa: E731
    o = (-2, -2, -2)
    pc = lin(o[0] + 2 * I + 1.0, o[1] + 2 * J + 1.0, o[2] + 2 * K + 1.0)
    bx, by, bz = oracle.dirichlet_from_coarse(mask, pc, o)
    ex = W.faces_from_function(lin, nx, ny, nz, 1.0)
    act = mask > 0
    pad = np.pad(act, 1)
    need_x = pad[1:-1, 1:-1, :-1] != pad[1:-1, 1:-1, 1:]
    need_y = pad[1:-1, :-1, 1:-1] != pad[1:-1, 1:, 1:-1]
    need_z = pad[:-1, 1:-1, 1:-1] != pad[1:, 1:-1, 1:-1]
    for got, want, need in ((bx, ex[0], need_x), (by, ex[1], need_y), (bz, ex[2], need_z)):
        assert need.any()
        np.testing.assert_allclose(got[need], want[need], rtol=1e-14, atol=1e-14)
        assert (got[~need] == 0).all()
    with pytest.raises(ValueError):
        oracle.dirichlet_from_coarse(np.ones(shape, np.int8), pc[1:, 1:, 1:], (0, 0, 0))
