"""The integer neighbour sum of the FP64 sweep (exact_sum.cuh), run on the
host through tests/host/exact_sum_check.cu, against exact arithmetic:
  - wherever no term loses bits to the window (every non-zero term within 7
    binades of the largest), the result is the correctly rounded sum (the
    exact rational sum converted by Python's correctly rounded int / int
    division, cross-checked against math.fsum where fsum does not overflow);
  - everywhere else it is within half an ulp of the result plus 5 units of
    2^(e_max - 1082) of the exact rational sum (fractions.Fraction);
  - the documented edge cases: subnormal terms count as zero, sums whose
    largest term is below 2^-959 are zero, overflow gives an infinity, and
    non-finite terms give the non-finite value IEEE addition gives.
tests/test_gpu_exact_sum.py checks that the GPU computes the same bits."""
import math
import os
import shutil
import struct
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GUARD = 7


def nvcc_path():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    return nvcc


def build_checker(d, gencode=True):
    exe = os.path.join(d, "exact_sum_check")
    cmd = [nvcc_path(), "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", "exact_sum_check.cu")]
    if gencode:
        cmd[3:3] = ["-gencode", "arch=compute_103a,code=sm_103a"]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def run_checker(exe, mode, sets, d):
    sets = np.ascontiguousarray(sets, dtype=np.float64).reshape(-1, 6)
    fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<q", sets.shape[0]))
        f.write(sets.tobytes())
    subprocess.run([exe, mode, fin, fout], check=True, timeout=300)
    return np.fromfile(fout, dtype=np.float64)


def biased_exponent(x):
    return (struct.unpack("<Q", struct.pack("<d", float(x)))[0] >> 52) & 0x7FF


def sum_cases(seed=20240611):
    """Seeded sets of six doubles covering the regimes of the sweep and the
    edge cases (shared with the GPU test)."""
    rng = np.random.default_rng(seed)
    out = []
    n = 4000
    # stencil-like: six neighbours of similar size and sign
    out.append(1.0 + 1e-3 * rng.standard_normal((n, 6)))
    # mixed signs and magnitudes within a few binades
    out.append(rng.standard_normal((n, 6)) * np.exp2(rng.integers(-3, 4, (n, 6))))
    # exponent spreads up to 120 binades
    out.append(rng.choice([-1.0, 1.0], (n, 6)) * rng.random((n, 6)) * np.exp2(rng.integers(-120, 1, (n, 6))))
    # zeros among the terms (inactive neighbours hold 0)
    z = rng.standard_normal((n, 6))
    z[rng.random((n, 6)) < 0.4] = 0.0
    out.append(z)
    # cancellation: pairs x, -x plus small terms
    c = rng.standard_normal((n, 6))
    c[:, 1] = -c[:, 0] * (1 + np.exp2(-40) * rng.standard_normal(n))
    c[:, 3] = -c[:, 2]
    c[:, 4:] *= np.exp2(-30)
    out.append(c)
    # wide absolute scales (the window floats with the largest exponent)
    out.append(rng.standard_normal((n, 6)) * np.exp2(rng.integers(-900, 900, (n, 1))))
    edge = [
        [0.0] * 6,
        [-0.0] * 6,
        [5e-324, 1e-310, 0.0, 0.0, 0.0, 0.0],           # subnormals only
        [1e-300, 2e-300, -1e-300, 0, 0, 0],             # below 2^-959: zero
        [2.0 ** -958, 2.0 ** -958, 0, 0, 0, 0],         # just inside the range
        [1.7e308, 1.7e308, 0, 0, 0, 0],                 # overflow
        [-1.7e308, -1.7e308, -1e308, 0, 0, 0],
        [1.7976931348623157e308, -1.7976931348623157e308, 1.0, 0, 0, 0],
        [math.inf, 1.0, 0, 0, 0, 0],
        [-math.inf, 1.0, 0, 0, 0, 0],
        [math.inf, -math.inf, 0, 0, 0, 0],
        [math.nan, 1.0, 0, 0, 0, 0],
        [1.0, 2.0 ** -53, 0, 0, 0, 0],                  # a tie: rounds to even
        [1.0, 2.0 ** -53, 2.0 ** -60, 0, 0, 0],         # just above the tie
        [1.0 + 2.0 ** -52, 2.0 ** -53, 0, 0, 0, 0],     # tie on an odd significand
        [1.0, -2.0 ** -54, 0, 0, 0, 0],
        [3.0, 3.0, 3.0, 3.0, 3.0, 3.0],
        [2.0 ** 1023, 2.0 ** 1023, -2.0 ** 1023, 0, 0, 0],
    ]
    out.append(np.array(edge, dtype=np.float64))
    return np.concatenate(out)


def check_against_exact(sets, got):
    fails = []
    for x, r in zip(sets, got):
        x = [float(v) for v in x]
        if not all(math.isfinite(v) for v in x):
            plain = x[0]
            for v in x[1:]:
                plain += v
            # NaN, or the infinity IEEE addition gives
            ok = (math.isnan(plain) and math.isnan(r)) or plain == r
            if not ok:
                fails.append((x, r, "non-finite"))
            continue
        emax = max(biased_exponent(v) for v in x)
        if emax < 64:
            if r != 0.0:
                fails.append((x, r, "tiny"))
            continue
        terms = [v if biased_exponent(v) > 0 else 0.0 for v in x]
        exact = sum(Fraction(v) for v in terms)
        if abs(exact) >= Fraction(2) ** 1024 * (1 - Fraction(2) ** -54):
            if not (math.isinf(r) and (r > 0) == (exact > 0)):
                fails.append((x, r, "overflow"))
            continue
        if abs(exact) < Fraction(2) ** -1022:
            if not (r == 0.0 or abs(Fraction(r) - exact) <= Fraction(2) ** -1022):
                fails.append((x, r, "underflow"))
            continue
        if not math.isfinite(r):
            fails.append((x, r, "spurious overflow"))
            continue
        nz = [biased_exponent(v) for v in terms if v != 0.0]
        if nz and min(nz) >= emax - GUARD:
            # nothing truncated: the correctly rounded sum
            rounded = exact.numerator / exact.denominator
            if r != rounded:
                fails.append((x, r, "not correctly rounded: %r" % rounded))
            try:
                assert math.fsum(terms) == rounded
            except OverflowError:
                pass
            continue
        bound = Fraction(math.ulp(r)) / 2 + 5 * Fraction(2) ** (emax - 1075 - GUARD)
        if abs(Fraction(r) - exact) > bound:
            fails.append((x, r, "outside the bound"))
    return fails


def test_exact_sum_on_the_host_against_exact_arithmetic():
    sets = sum_cases()
    with tempfile.TemporaryDirectory() as d:
        exe = build_checker(d, gencode=True)
        got = run_checker(exe, "host", sets, d)
    assert got.shape[0] == sets.shape[0]
    fails = check_against_exact(sets, got)
    assert not fails, fails[:5]


def test_exact_sum_is_more_accurate_than_the_plain_sum_on_stencil_values():
    """On cancelling sums the integer sum's largest and mean errors are below
    those of the left-to-right FP64 sum (it rounds once)."""
    rng = np.random.default_rng(7)
    c = rng.standard_normal((2000, 6))
    c[:, 1] = -c[:, 0] * (1 + np.exp2(-40) * rng.standard_normal(2000))
    with tempfile.TemporaryDirectory() as d:
        exe = build_checker(d, gencode=True)
        got = run_checker(exe, "host", c, d)
    err_int, err_plain = [], []
    for x, r in zip(c, got):
        exact = sum(Fraction(float(v)) for v in x)
        plain = 0.0
        for v in x:
            plain += float(v)
        err_int.append(float(abs(Fraction(r) - exact)))
        err_plain.append(float(abs(Fraction(plain) - exact)))
    assert max(err_int) <= max(err_plain)
    assert np.mean(err_int) < np.mean(err_plain)
