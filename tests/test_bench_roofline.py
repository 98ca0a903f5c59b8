"""The roofline arithmetic of bench.py on given launch timings (no GPU):
achieved = algorithmic bytes per launch / the launch's average duration,
frac against the measured copy bandwidth, the kernel named after the sweep
variant that ran, and the ncu DRAM traffic taken from a committed profile
summary only while its kernel-source hash matches the sources."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6685.8}
ST = {"gs_ms": 12.8 * 100 / 1e3, "gs_n": 100}  # 100 launches of 12.8 us
N_ACTIVE = 4_400_000


def test_fp32_segment_pair_sweep():
    r = bench.roofline(ST, N_ACTIVE, 1, PEAKS, seg_on=3)
    assert "gs_seg_pair_kernel" in r["kernel"] and r["bound"] == "hbm" and r["unit"] == "GB/s"
    want = 13.0 * (N_ACTIVE / 2) / 12.8e-6 / 1e9  # 13 B per update, one colour per launch
    assert r["achieved"] == pytest.approx(want, rel=1e-12)
    assert r["frac"] == pytest.approx(want / 6685.8, rel=1e-12)
    assert r["avg_launch_us"] == pytest.approx(12.8, rel=1e-12)


@pytest.mark.parametrize("seg,name", [(0, "gs_list_kernel<0,float>"), (1, "8-slot"), (2, "16-slot")])
def test_fp32_other_sweeps_are_named(seg, name):
    assert name in bench.roofline(ST, N_ACTIVE, 1, PEAKS, seg_on=seg)["kernel"]


def test_fp64_sweep_counts_25_bytes_and_one_issued_fp64_op():
    r = bench.roofline(ST, N_ACTIVE, 0, PEAKS, fp64_rate=0.53e12, exact_on=True)
    half = N_ACTIVE / 2
    assert r["achieved"] == pytest.approx(25.0 * half / 12.8e-6 / 1e9, rel=1e-12)
    v = r["fp64_pipe_view"]
    assert v["issued_fp64_ops_per_update"] == 1.0 and v["method_fp64_ops_per_update"] == 7
    assert v["achieved"] == pytest.approx(half / 12.8e-6 / 1e12, rel=1e-12) and v["peak"] == pytest.approx(0.53)


def test_traffic_follows_the_profile_hash():
    """The committed summary of the headline kernel carries the hash of the
    current kernel sources, so its DRAM bytes are reported; any other hash
    would give None."""
    text = open(os.path.join(ROOT, "profiles", "gs_seg_pair_fp32_level0_sphere_union_256.md")).read()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text).group(1)
    b = int(re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text).group(1))
    got = bench.profiled_traffic("gs_seg_pair_fp32_level0_sphere_union_256.md")
    if h == bench.kernel_source_hash():
        assert got == b
    else:
        assert got is None
    assert bench.profiled_traffic("no_such_profile.md") is None
