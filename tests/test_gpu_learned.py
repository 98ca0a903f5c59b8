"""The learned initial guess wired to the method (paper_1104_1703_gb300/
learned.py and the patch-level mg_unet_* / mg_generate_blob_patch /
mg_faces_from_coarse entry points):
  - the GPU patch generator follows the host recipe of workloads.blob_patch:
    the same rho and coarse potential (same SplitMix64 streams; libm-level
    differences only) and the same mask except where the smoothed noise is
    within rounding of the threshold (real-space instead of FFT filtering);
  - the face arrays of the one-way interface equal the oracle's trilinear
    interpolation of the coarse potential;
  - the network's input channels and scale equal the oracle's features()
    (FP32 channels, FP64 scale);
  - the guess is the scale times the network's forward pass on them;
  - a solve from the learned guess reaches the same tolerance, checked by
    the oracle's FP64 operator (the plain V-cycle stays the judge).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_oracle as U  # noqa: E402
from paper_1104_1703_gb300 import binding as B  # noqa: E402
from paper_1104_1703_gb300 import learned as Lg  # noqa: E402
from paper_1104_1703_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.mark.parametrize("shape,seed", [((32, 32, 32), 11), ((20, 24, 28), 12)])
def test_gpu_generator_follows_the_host_recipe(device, shape, seed):
    w = W.blob_patch(shape, seed=seed)
    nz, ny, nx = shape
    cn = ((nz + 1) // 2 + 2, (ny + 1) // 2 + 2, (nx + 1) // 2 + 2)
    mask = torch.zeros(shape, dtype=torch.int8, device=device)
    rho = torch.zeros(shape, dtype=torch.float64, device=device)
    phi_c = torch.zeros(cn, dtype=torch.float64, device=device)
    scratch = torch.zeros(2 * nx * ny * nz + 80, dtype=torch.float32, device=device)
    B.mg_generate_blob_patch(seed, shape, scratch, mask, rho, phi_c)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rho.cpu().numpy(), w["rho"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(phi_c.cpu().numpy(), w["phi_c"], rtol=0, atol=1e-12)
    agree = (mask.cpu().numpy() == w["mask"]).mean()
    assert agree > 0.99, agree


def test_faces_and_features_match_the_oracle(device, oracle):
    w = W.blob_patch((24, 32, 40), seed=21)
    nz, ny, nx = w["mask"].shape
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    mask, rho = dev(w["mask"]), dev(w["rho"])
    H = B.Hierarchy(mask, w["h"])
    bx = torch.zeros((nz, ny, nx + 1), dtype=torch.float64, device=device)
    by = torch.zeros((nz, ny + 1, nx), dtype=torch.float64, device=device)
    bz = torch.zeros((nz + 1, ny, nx), dtype=torch.float64, device=device)
    H.faces_from_coarse(dev(w["phi_c"]), w["origin"], bx, by, bz)
    fo = oracle.dirichlet_from_coarse(w["mask"], w["phi_c"], w["origin"])
    act = w["mask"] > 0
    pad = np.pad(act, 1)
    got = [bx.cpu().numpy(), by.cpu().numpy(), bz.cpu().numpy()]
    # compare on the boundary faces (the only ones the method reads); the
    # library writes 0 elsewhere
    for axis, g in enumerate(got):
        lo = [slice(1, -1)] * 3
        hi = [slice(1, -1)] * 3
        lo[2 - axis] = slice(0, -2)
        hi[2 - axis] = slice(2, None)
        gm = np.zeros_like(g, dtype=bool)
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[2 - axis] = slice(0, -1)
        b[2 - axis] = slice(1, None)
        gm[tuple(a)] |= act & ~pad[tuple(lo)]
        gm[tuple(b)] |= act & ~pad[tuple(hi)]
        np.testing.assert_allclose(g[gm], fo[axis][gm], rtol=0, atol=1e-12)
        assert not g[~gm].any()
    # the network's channels and scale
    net = B.UNet(1, 16, (nz, ny, nx))
    x, s = net.features(mask, rho, (bx, by, bz), w["h"])
    xo, so = U.features(w["mask"], w["rho"], tuple(np.asarray(f) for f in got), w["h"])
    assert s == pytest.approx(so, rel=1e-12)
    np.testing.assert_allclose(x, xo, rtol=0, atol=2e-6 * np.abs(xo).max())
    # the guess is s times the forward pass on those channels
    net.set_params(Lg.init_params(3, 1, 16))
    guess = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
    net.predict(mask, rho, (bx, by, bz), w["h"], guess)
    pred = net.forward(x)
    np.testing.assert_allclose(guess.cpu().numpy(), s * pred.astype(np.float64), rtol=1e-6, atol=1e-12)


def test_learned_guess_solve_reaches_the_tolerance(device, oracle):
    """A short training run at 32^3 (the loss falls) and solves from the
    learned guess: every held-out patch reaches 1e-8, the last one checked by
    the oracle's operator.  How much a trained guess saves is measured by the
    benchmark, not asserted here."""
    n = 32
    net = B.UNet(3, 16, (n, n, n))
    net.set_params(Lg.init_params(7, 3, 16))
    P = Lg.Patches(n, device, precision=1)
    losses = Lg.train(net, P, list(range(100, 164)), lr=2e-3, lr_end=5e-4)
    assert len(losses) >= 48 and np.mean(losses[-16:]) < np.mean(losses[:16])
    recs = Lg.evaluate(net, P, list(range(900, 906)))
    assert recs and all(r["status"] == (0, 0) for r in recs)
    # the last solve (from the learned guess) by the oracle's FP64 operator
    phi = P.H.get_solution()
    mask = P.mask.cpu().numpy()
    faces = tuple(f.cpu().numpy() for f in P.faces)
    S0 = np.where(mask > 0, 1, -1).astype(np.int64)
    r = oracle.residual(S0, 0, 2, P.h, phi, P.rho.cpu().numpy(), *faces)
    R = oracle.Hierarchy(mask, P.h)
    R.set_rhs(P.rho.cpu().numpy())
    R.set_faces(*faces)
    assert np.sqrt((r ** 2).sum()) / R.residual_norm_zero() < 1e-8 * (1 + 1e-6)
