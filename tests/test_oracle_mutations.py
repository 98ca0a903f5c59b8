"""The oracle's pins catch plausible single-point mistakes in the oracle.

Each entry below plants one mistake against the paper in a copy of
`oracle/mg_oracle.c`: a dropped term, a wrong sign, index or weight, a
skipped rule of Section 4.  The test builds that copy in a temporary folder
under the oracle's build folder, points the oracle loader at it
(MG_ORACLE_SRC, MG_ORACLE_BUILD) and runs the pins listed for it in a child
pytest, which must report failures.  The unmodified source runs the union
of those pins as a control and must pass, so a failure is the planted
mistake's doing.  Everything runs on the CPU.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mg_oracle.c")
PINS = "tests/test_oracle_pins.py::"
CYCLES = "tests/test_oracle_cycles.py::"

# name: (text in mg_oracle.c, its replacement, pins that must fail)
MUTATIONS = {
    # Fig. 5: theta measured from the inactive neighbour's centre
    "theta_from_j": ("return m_i / (m_i - m_j); }", "return -m_j / (m_i - m_j); }",
                     [PINS + "test_fig5_theta_and_ghost"]),
    # Fig. 5: ghost extrapolated away from the boundary value
    "ghost_sign": ("return phi_i + (phi_b - phi_i) / theta;", "return phi_i - (phi_b - phi_i) / theta;",
                   [PINS + "test_fig5_theta_and_ghost"]),
    # Section 3: the smoother's diagonal ignores theta at ghost faces
    "gs_ghost_coef": ("sum_c += 1.0 / nb.theta;", "sum_c += 1.0;",
                      [PINS + "test_gs_update_solves_its_row"]),
    # Fig. 1: the +x boundary face read from the -x face's slot
    "face_index": ("bx[((size_t)k * ny + j) * (nx + 1) + i + 1]", "bx[((size_t)k * ny + j) * (nx + 1) + i]",
                   [PINS + "test_linear_fields_exact_with_ghosts"]),
    # Section 4: first-order neighbours treated as second-order ghosts
    "ngp_off": ("if (level >= 1 && order == 1) {", "if (0) {",
                [CYCLES + "test_schedule_rates_ball"]),
    # Section 4: first-order unknowns taken as m > 0 instead of m = 1
    "first_order_active": ("if (level >= 1 && order == 1) return S == pow8(level);",
                           "if (level >= 1 && order == 1) return S > 0;",
                           [PINS + "test_deepest_levels_ball32"]),
    # Section 3: cells outside the box counted as m = 0 instead of -1
    "missing_child": ("sum += inside ? S[cell(i, j, k, nx, ny)] : -p8;",
                      "sum += inside ? S[cell(i, j, k, nx, ny)] : 0;",
                      [PINS + "test_mask_restriction_odd_dims"]),
    # Fig. 3: the 2D R1 weight used in 3D
    "r1_quarter": ("rc[cell(I, J, K, cx, cy)] = sum / 8.0;", "rc[cell(I, J, K, cx, cy)] = sum / 4.0;",
                   [PINS + "test_r1_average"]),
    # Fig. 3: P2's near and far weights swapped on even cells
    "p2_swap": ("*lo = I - 1;\n    *w_lo = 0.25;\n    *w_hi = 0.75;",
                "*lo = I - 1;\n    *w_lo = 0.75;\n    *w_hi = 0.25;",
                [PINS + "test_p2_weights_fig3"]),
    # Section 2: the correction also added to inactive fine cells
    "p2_inactive": ("if (!orc_is_active(Sf[c], level_f, order)) continue;\n        int xi", "int xi",
                    [PINS + "test_p2_reproduces_linear_fields"]),
    # Boundary values from the coarse level: centres off by half a cell in x
    "dir_tri": ("double u = (px - ox) / 2.0 - 0.5,", "double u = (px - ox) / 2.0,",
                [PINS + "test_dirichlet_from_coarse_linear_exact"]),
    # Section 2: coarse right-hand side +R1(r) instead of -R1(r)
    "rhs_sign": ("H->rhs[l + 1][c] = -H->rhs[l + 1][c];", "H->rhs[l + 1][c] = H->rhs[l + 1][c];",
                 [PINS + "test_vcycle_rate_grid_independent_ball"]),
    # Section 2: residual rho - Laplacian instead of Laplacian - rho
    "res_sign": ("if (orc_is_active(S[c], level, order)) r[c] -= rho[c];",
                 "if (orc_is_active(S[c], level, order)) r[c] += rho[c];",
                 [PINS + "test_dense_direct_solve_8cube"]),
    # Section 2: the smoother drops h^2 on the right-hand side
    "gs_h2": ("phi[c] = (sum_a - h2 * rho[c]) / sum_c;", "phi[c] = (sum_a - rho[c]) / sum_c;",
              [PINS + "test_gs_update_solves_its_row"]),
    # Section 2: every level uses the fine cell size
    "coarse_h": ("return ldexp(H->h, l); }", "return H->h; }",
                 [PINS + "test_vcycle_rate_grid_independent_ball"]),
    # Section 4: a first-order neighbour enters the operator as Phi_i, not 0
    "lap_ngp_ghost": ("          else\n            phi_star = 0.0;", "          else\n            phi_star = phi_i;",
                      [PINS + "test_operator_symmetric_negative_definite[2-1]"]),
    # Section 4: the switch never trips
    "switch_never": ("r_n / r_prev > eta)", "r_n / r_prev > 1e300)",
                     [PINS + "test_small_islands_first_order_fix_and_switch"]),
    # Section 4: first order not held for the following solves
    "no_hold": ("H->hold = hold_solves;", "H->hold = 0;",
                [PINS + "test_small_islands_first_order_fix_and_switch"]),
    # Section 4 reading: no restart from the initial guess after a divergent trip
    "no_restart": ("if (r_n > r_init) {", "if (0) {",
                   [PINS + "test_switch_restart_from_initial_guess"]),
}


def _run_pins(tmp, name, src_text, pins, threads):
    d = os.path.join(tmp, name)
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "mg_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    env = dict(os.environ, MG_ORACLE_SRC=src, MG_ORACLE_BUILD=os.path.join(d, "_build"),
               OMP_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    lines = out.stdout.strip().splitlines()
    return name, out.returncode, lines[-1] if lines else out.stderr[-500:]


def test_pins_catch_planted_mistakes():
    with open(SRC) as f:
        text = f.read()
    jobs = []
    for name, (old, new, pins) in MUTATIONS.items():
        assert text.count(old) == 1, "%s: the planted site must occur once in the oracle" % name
        jobs.append((name, text.replace(old, new), pins))
    control_pins = sorted({p for _, _, pins in MUTATIONS.values() for p in pins})
    jobs.append(("control", text, control_pins))
    workers = max(1, min(4, (os.cpu_count() or 2) // 2))
    threads = max(1, (os.cpu_count() or 2) // workers)
    # the mutants build in the oracle's own (git-ignored) build folder
    base = os.path.join(ROOT, "oracle", "_build")
    os.makedirs(base, exist_ok=True)
    tmp = tempfile.mkdtemp(prefix="mutants_", dir=base)
    try:
        with cf.ThreadPoolExecutor(workers) as ex:
            results = list(ex.map(lambda j: _run_pins(tmp, *j, threads), jobs))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    missed = []
    for name, rc, last in results:
        if name == "control":
            assert rc == 0 and "passed" in last and "failed" not in last, "control run: " + last
        elif not (rc == 1 and re.search(r"\b\d+ failed\b", last) and "error" not in last):
            missed.append("%s (exit %d): %s" % (name, rc, last))
    assert not missed, "planted mistakes not caught:\n" + "\n".join(missed)
