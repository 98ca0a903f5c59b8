"""The middle coarse levels run as one thread-block cluster (option
coarse_cluster = 1) or as one launch per step (0, the default).  Both do the
same arithmetic in the same order, so their results agree bit for bit, in
both precisions and both orders (the launch path is the one every other
parity test holds to the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


CASES = {
    "ball64": W.ball(64),
    "holes64": W.holes(64),
    "union128": W.sphere_union(128),
    "blob96x80x72": W.blob_patch((72, 80, 96), seed=11),
}


def _run(w, dev, n, **opts):
    H = B.Hierarchy(torch.from_numpy(w["mask"]).to(dev), w["h"], **opts)
    H.set_rhs(torch.from_numpy(w["rho"]).to(dev))
    if "phi_c" in w:
        H.set_dirichlet_from_coarse(torch.from_numpy(w["phi_c"]).to(dev), w["origin"])
    elif w.get("bx") is not None:
        H.set_dirichlet(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w["bx"], w["by"], w["bz"])))
    rels = [H.vcycle() for _ in range(n)]
    return H, rels


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_cluster_path_is_bitwise_the_launch_path(dev, name, order, precision):
    w = CASES[name]
    Ha, ra = _run(w, dev, 3, order=order, precision=precision, coarse_cluster=1)
    Hb, rb = _run(w, dev, 3, order=order, precision=precision, coarse_cluster=0)
    assert ra == rb
    assert np.array_equal(Ha.get_solution(), Hb.get_solution())
    n_lev, _, _ = Ha.levels()
    for level in range(1, n_lev):
        assert np.array_equal(Ha.level_get(level, B.MG_FIELD_PHI), Hb.level_get(level, B.MG_FIELD_PHI))


def test_cluster_path_fewer_launches(dev):
    w = CASES["union128"]
    counts = []
    for cc in (1, 0):
        H, _ = _run(w, dev, 1, coarse_cluster=cc, use_graphs=0)
        c0 = B.mg_launch_count()
        H.vcycle()
        counts.append(B.mg_launch_count() - c0)
    assert counts[0] < counts[1]
