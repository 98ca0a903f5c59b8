"""Level-0 sweeps by row segments (option fine_segments) against the
per-cell compact lists: the two visit the same cells with the same
arithmetic, so smoothing, whole solves (FP64 with either neighbour sum, and
the mixed form) and their residual histories are bit-identical.  Cases cover
odd sizes, rows whose length is not a multiple of the segment, and masks
with isolated cells."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import CASES, make_pair, _level_state  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def extra_cases():
    out = {}
    m = W.random_mask((21, 19, 67), seed=31, p_active=0.35)
    out["sparse67x19x21"] = {"mask": m, "rho": W.random_field(m.shape, 32), "h": 0.05,
                             "faces": W.random_faces(m.shape, 33)}
    out["union64"] = W.sphere_union(64)
    return out


ALL = dict(CASES, **extra_cases())


@pytest.mark.parametrize("name", ["ball64", "random17x12x10", "blob48x32x40", "sparse67x19x21"])
@pytest.mark.parametrize("fp64_sum", [0, 1])
def test_smoothing_bit_identical(dev, name, fp64_sum):
    w = ALL[name]
    got = []
    for seg in (0, 1):
        H, R = make_pair(w, dev, fine_segments=seg, fp64_sum=fp64_sum)
        _level_state(w, H, R, 0, 2, seed=77)
        H.smooth(0, 2, 2)
        got.append(H.level_get(0, B.MG_FIELD_PHI))
    assert np.array_equal(got[0].view(np.uint64), got[1].view(np.uint64))


@pytest.mark.parametrize("name", ["ball64", "blob48x32x40", "sparse67x19x21", "union64", "holes32"])
@pytest.mark.parametrize("precision,fp64_sum", [(0, 0), (0, 1), (1, 1)])
def test_solves_bit_identical(dev, name, precision, fp64_sum):
    w = ALL[name]
    res = []
    for seg in (0, 1):
        H, _ = make_pair(w, dev, fine_segments=seg, fp64_sum=fp64_sum, precision=precision)
        st, info = H.solve(1e-9, 100)
        assert st == 0
        res.append((info, H.get_solution()))
    (i0, s0), (i1, s1) = res
    assert (i0["cycles"], i0["order"], i0["switched"]) == (i1["cycles"], i1["order"], i1["switched"])
    assert np.array_equal(i0["hist"], i1["hist"])
    assert np.array_equal(s0.view(np.uint64), s1.view(np.uint64))


def test_segment_lists_follow_a_mask_update(dev):
    """After update_mask the segment lists are rebuilt: a solve on the new
    mask equals a fresh hierarchy's bit for bit."""
    a, b = ALL["blob48x32x40"], W.blob_patch((40, 32, 48), seed=105)
    H, _ = make_pair(a, dev, fine_segments=1)
    H.solve(1e-9, 100)
    H.update_mask(torch.from_numpy(b["mask"]).to(dev))
    H.set_rhs(torch.from_numpy(b["rho"]).to(dev))
    H.set_dirichlet_from_coarse(torch.from_numpy(b["phi_c"]).to(dev), b["origin"])
    H.set_solution(None)
    st, info = H.solve(1e-9, 100)
    F, _ = make_pair(b, dev, fine_segments=0)
    st2, info2 = F.solve(1e-9, 100)
    assert st == st2 == 0 and info["cycles"] == info2["cycles"]
    assert np.array_equal(H.get_solution().view(np.uint64), F.get_solution().view(np.uint64))
