"""Pins of the learned-guess network's CPU definition (oracle/unet_oracle.py)
against what fixes it from outside: SciPy's correlate for the convolution,
central finite differences for every gradient, the adjoint relations of
pooling and upsampling, shift equivariance, the mask on the head, and the
closed form of Adam's first step."""
import numpy as np
import pytest

from oracle import unet_oracle as U

ndimage = pytest.importorskip("scipy.ndimage")


def _input(rng, n, p_active=0.7):
    x = rng.normal(size=(3, n, n, n))
    x[1] = np.where(rng.random((n, n, n)) < p_active, 1.0, -1.0)
    return x


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 6, 7))
    w = rng.normal(size=(3, 2, 3, 3, 3))
    b = rng.normal(size=3)
    out = U.conv3d(x, w, b)
    for o in range(3):
        ref = b[o] + sum(ndimage.correlate(x[i], w[o, i], mode="constant", cval=0.0) for i in range(2))
        np.testing.assert_allclose(out[o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_is_shift_equivariant_in_the_interior():
    rng = np.random.default_rng(2)
    x = np.zeros((1, 12, 12, 12))
    x[0, 4:7, 3:6, 5:8] = rng.normal(size=(3, 3, 3))
    w = rng.normal(size=(2, 1, 3, 3, 3))
    b = np.zeros(2)
    a = U.conv3d(x, w, b)
    s = U.conv3d(np.roll(x, (1, 2, -1), axis=(1, 2, 3)), w, b)
    np.testing.assert_allclose(np.roll(a, (1, 2, -1), axis=(1, 2, 3)), s, rtol=0, atol=1e-13)


def test_pool_and_upsample_are_adjoint():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 8, 6, 4))
    y = rng.normal(size=(2, 4, 3, 2))
    assert np.vdot(U.avg_pool2(x), y) == pytest.approx(np.vdot(x, U.upsample2(y)) / 8.0, rel=1e-13)
    assert np.vdot(U.upsample2(y), x) == pytest.approx(np.vdot(y, U.upsample2_backward(x)), rel=1e-13)
    np.testing.assert_allclose(U.avg_pool2_backward(y), U.upsample2(y) / 8.0)


def test_head_predicts_zero_on_inactive_cells():
    rng = np.random.default_rng(4)
    P = U.init_params(5, levels=3, base=2)
    x = _input(rng, 8)
    p, _ = U.forward(P, x)
    assert p.shape == (1, 8, 8, 8)
    assert not p[0][x[1] <= 0].any()


@pytest.mark.parametrize("levels", [2, 3])
def test_backward_matches_finite_differences(levels):
    """Every parameter tensor, at sampled entries, for a random output
    weighting: a dropped skip gradient, a swapped concatenation order, a
    wrong pooling scale or a missing ReLU mask all fail here."""
    rng = np.random.default_rng(10 + levels)
    P = U.init_params(6, levels=levels, base=2)
    # random biases keep every pre-activation off the ReLU kink (with zero
    # biases a zero neighbourhood gives exactly 0, where a difference
    # quotient straddles the kink)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(0.0, 0.1, P[k].shape)
    x = _input(rng, 8)
    p, cache = U.forward(P, x)
    g = rng.normal(size=p.shape)
    G = U.backward(P, cache, g)
    assert set(G) == set(P)

    def f():
        return float((U.forward(P, x)[0] * g).sum())

    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            fp = f()
            flat[idx] = old - 1e-6
            fm = f()
            flat[idx] = old
            fd = (fp - fm) / 2e-6
            assert abs(fd - G[k].reshape(-1)[idx]) <= 1e-6 * max(1e-3, abs(fd)), (k, idx)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    p, y = rng.normal(size=(1, 4, 4, 4)), rng.normal(size=(1, 4, 4, 4))
    act = rng.random((1, 4, 4, 4)) < 0.6
    loss, g = U.loss_and_grad(p, y, act)
    assert loss == pytest.approx(((p - y)[act] ** 2).sum() / (y[act] ** 2).sum(), rel=1e-14)
    assert not g[~act].any()
    for idx in [(0, 1, 2, 3), (0, 0, 0, 0), (0, 3, 1, 2)]:
        q = p.copy()
        q[idx] += 1e-6
        lp = U.loss_and_grad(q, y, act)[0]
        q[idx] -= 2e-6
        lm = U.loss_and_grad(q, y, act)[0]
        assert (lp - lm) / 2e-6 == pytest.approx(g[idx], rel=1e-6, abs=1e-9)


def test_adam_first_step_closed_form():
    """With zero moments the bias-corrected first step is lr * g / (|g| + eps)
    for every entry (Kingma & Ba, Algorithm 1)."""
    rng = np.random.default_rng(8)
    P = {"a": rng.normal(size=(3, 4)), "b": rng.normal(size=5)}
    G = {k: rng.normal(size=v.shape) for k, v in P.items()}
    before = {k: v.copy() for k, v in P.items()}
    state = {}
    U.adam_step(P, G, state, lr=0.01, eps=1e-8)
    for k in P:
        np.testing.assert_allclose(before[k] - P[k], 0.01 * G[k] / (np.abs(G[k]) + 1e-8), rtol=1e-12)
    assert state["t"] == 1


def _backward_agrees(mod, levels):
    rng = np.random.default_rng(10 + levels)
    P = mod.init_params(6, levels=levels, base=2)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(0.0, 0.1, P[k].shape)
    x = _input(rng, 8)
    p, cache = mod.forward(P, x)
    g = rng.normal(size=p.shape)
    G = mod.backward(P, cache, g)

    def f():
        return float((mod.forward(P, x)[0] * g).sum())

    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            fp = f()
            flat[idx] = old - 1e-6
            fm = f()
            flat[idx] = old
            if abs((fp - fm) / 2e-6 - G[k].reshape(-1)[idx]) > 1e-6 * max(1e-3, abs((fp - fm) / 2e-6)):
                return False
    return True


@pytest.mark.parametrize("old,new", [
    ("            g = g + g_skip[l]\n", "            g = g\n"),                      # skip gradient dropped
    ("        g_skip[l] = g[:cs]\n        g = upsample2_backward(g[cs:])\n",
     "        g_skip[l] = g[-cs:]\n        g = upsample2_backward(g[:-cs])\n"),        # concatenation order swapped
    ("    return upsample2(g) / 8.0\n", "    return upsample2(g)\n"),              # pooling scale lost
    ('            name = "up%d.%d" % (l, j)\n            g = g * (cache[name + ".z"] > 0)\n',
     '            name = "up%d.%d" % (l, j)\n'),                                   # ReLU mask dropped
])
def test_planted_backward_mistakes_are_caught(old, new):
    """The finite-difference pin fails on an in-memory copy of the module
    with one plausible backward mistake planted."""
    import types
    src = open(U.__file__).read()
    assert src.count(old) == 1
    mod = types.ModuleType("unet_mutant")
    exec(compile(src.replace(old, new), "unet_mutant", "exec"), mod.__dict__)
    assert not (_backward_agrees(mod, 2) and _backward_agrees(mod, 3))


def test_features_scale_invariance_and_channels():
    """Scaling rho and the boundary values by c leaves the channels unchanged
    and scales s by c; inactive cells carry 0 in channels 0 and 2; the mask
    channel is +-1."""
    rng = np.random.default_rng(20)
    shape = (5, 6, 7)
    mask = (rng.random(shape) < 0.6).astype(np.int8)
    rho = rng.normal(size=shape)
    faces = (rng.normal(size=(5, 6, 8)), rng.normal(size=(5, 7, 7)), rng.normal(size=(6, 6, 7)))
    x, s = U.features(mask, rho, faces, 0.1)
    x3, s3 = U.features(mask, 3.0 * rho, tuple(3.0 * f for f in faces), 0.1)
    np.testing.assert_allclose(x3, x, rtol=1e-13, atol=1e-15)
    assert s3 == pytest.approx(3.0 * s, rel=1e-14)
    act = mask > 0
    assert not x[0][~act].any() and not x[2][~act].any()
    assert set(np.unique(x[1])) <= {-1.0, 1.0} and (x[1] > 0).sum() == act.sum()


def test_features_boundary_channel_single_cell():
    """One active cell alone in the box: all six faces are ghost faces and the
    boundary channel is their mean over s; with rho = 0, s is their root mean
    square."""
    mask = np.zeros((3, 3, 3), np.int8)
    mask[1, 1, 1] = 1
    bx, by, bz = np.zeros((3, 3, 4)), np.zeros((3, 4, 3)), np.zeros((4, 3, 3))
    vals = [1.0, 2.0, -3.0, 4.0, 5.0, -6.0]
    bx[1, 1, 1], bx[1, 1, 2] = vals[0], vals[1]
    by[1, 1, 1], by[1, 2, 1] = vals[2], vals[3]
    bz[1, 1, 1], bz[2, 1, 1] = vals[4], vals[5]
    x, s = U.features(mask, np.zeros((3, 3, 3)), (bx, by, bz), 0.5)
    assert s == pytest.approx(np.sqrt(np.mean(np.square(vals))), rel=1e-14)
    assert x[2][1, 1, 1] == pytest.approx(np.mean(vals) / s, rel=1e-14)
    assert np.count_nonzero(x[2]) == 1 and not x[0].any()
