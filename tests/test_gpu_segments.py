"""Level-0 sweeps by row segments of 8 and 16 slots, one or two slots per
thread (option fine_segments)
against the per-cell compact lists, in the mixed form's FP32 cycles: the
two visit the same cells with the same arithmetic, so whole solves and
their residual histories are bit-identical.  Cases cover
odd sizes, rows whose length is not a multiple of the segment, and masks
with isolated cells."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import CASES, make_pair  # noqa: E402

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


@pytest.mark.parametrize("name", ["ball64", "blob48x32x40", "sparse67x19x21", "union64", "holes32"])
@pytest.mark.parametrize("inner", [1, 3])
def test_solves_bit_identical(dev, name, inner):
    w = ALL[name]
    res = []
    for seg in (0, 1, 2, 3):
        H, _ = make_pair(w, dev, fine_segments=seg, precision=1, inner_cycles=inner)
        st, info = H.solve(1e-9, 100)
        assert st == 0
        res.append((info, H.get_solution()))
    i0, s0 = res[0]
    for i1, s1 in res[1:]:
        assert (i0["cycles"], i0["order"], i0["switched"]) == (i1["cycles"], i1["order"], i1["switched"])
        assert np.array_equal(i0["hist"], i1["hist"])
        assert np.array_equal(s0.view(np.uint64), s1.view(np.uint64))


@pytest.mark.parametrize("seg", [2, 3])
def test_segment_lists_follow_a_mask_update(dev, seg):
    """After update_mask the segment lists are rebuilt: a solve on the new
    mask equals a fresh hierarchy's bit for bit."""
    a, b = ALL["blob48x32x40"], W.blob_patch((40, 32, 48), seed=105)
    H, _ = make_pair(a, dev, fine_segments=seg, precision=1)
    H.solve(1e-9, 100)
    H.update_mask(torch.from_numpy(b["mask"]).to(dev))
    H.set_rhs(torch.from_numpy(b["rho"]).to(dev))
    H.set_dirichlet_from_coarse(torch.from_numpy(b["phi_c"]).to(dev), b["origin"])
    H.set_solution(None)
    st, info = H.solve(1e-9, 100)
    F, _ = make_pair(b, dev, fine_segments=0, precision=1)
    st2, info2 = F.solve(1e-9, 100)
    assert st == st2 == 0 and info["cycles"] == info2["cycles"]
    assert np.array_equal(H.get_solution().view(np.uint64), F.get_solution().view(np.uint64))
