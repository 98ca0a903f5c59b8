"""The learned initial guess's network on the GPU (mg_unet_*: tcgen05
convolutions, BF16 weights and activations, FP32 accumulation) against its
FP64 definition in oracle/unet_oracle.py.

Tolerances, from the arithmetic.  The network rounds its weights and every
activation to BF16 (relative error at most 2^-9 per value) and accumulates
in FP32 (K <= 27 x 192 products; relative error well below 1e-4 of the sum
of magnitudes).  So
  - per layer: the oracle's convolution applied to the network's own BF16
    input and BF16-rounded weights, then ReLU, matches the layer's output to
    |got - want| <= 2^-8 |want| + 2e-4 max|want| (one output rounding plus
    the accumulation);
  - end to end: the oracle's forward pass on BF16-rounded weights and input
    differs from the network's by the BF16 roundings of the intermediate
    activations, each of relative size 2^-9 and propagated through at most
    4 levels x 4 convolutions: relative L2 error <= 2e-2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_oracle as U  # noqa: E402
from paper_1104_1703_gb300 import binding as B  # noqa: E402

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(P):
    return np.concatenate([P[k].ravel() for k in P])


def _params(levels, base, seed):
    P = U.init_params(seed, levels=levels, base=base)
    rng = np.random.default_rng(seed + 1)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(0.0, 0.1, P[k].shape)
    return P


def _input(n, seed):
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(3,) + shape)
    x[1] = np.where(rng.random(shape) < 0.7, 1.0, -1.0)
    return x.astype(np.float32)


def _pool(t):
    c, d, h, w = t.shape
    return t.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(axis=(2, 4, 6)) * 0.125


def _names(levels):
    return ["down%d.%d" % (l, j) for l in range(levels) for j in range(2)] + \
           ["up%d.%d" % (l, j) for l in range(levels - 1) for j in range(2)]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


# grids with rows of 128 and 256 voxels take the halo-row path of the
# convolution at level 0 (and level 1 of the 256-voxel rows)
@pytest.mark.parametrize("levels,n", [(1, 16), (2, 16), (3, 16), (4, 16), (2, 24), (3, 32), (1, (4, 6, 128)),
                                      (2, (8, 4, 256)), (3, (4, 8, 128))])
def test_each_convolution_matches_the_oracle(dev, levels, n):
    P = _params(levels, 16, 11 + levels)
    x = _input(n, 5 + (n if np.isscalar(n) else n[2]))
    net = B.UNet(levels, 16, x.shape[1:])
    net.set_params(flat(P))
    net.forward(x)
    names = _names(levels)
    out = {name: net.layer_output(i).astype(np.float64) for i, name in enumerate(names)}
    for i, name in enumerate(names):
        l, j = int(name[-3]), int(name[-1])
        if name.startswith("down"):
            if j == 1:
                inp = out["down%d.0" % l]
            elif l == 0:
                inp = bf16(x)
            else:
                inp = bf16(_pool(out["down%d.1" % (l - 1)]))
        else:
            if j == 1:
                inp = out["up%d.0" % l]
            else:
                below = out["down%d.1" % (levels - 1)] if l == levels - 2 else out["up%d.1" % (l + 1)]
                inp = np.concatenate([out["down%d.1" % l], U.upsample2(below)], axis=0)
        want = U.relu(U.conv3d(inp, bf16(P[name + ".w"]), P[name + ".b"]))
        got = out[name]
        assert got.shape == want.shape, name
        bound = 2.0 ** -8 * np.abs(want) + 2e-4 * np.abs(want).max()
        bad = np.abs(got - want) > bound
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(got - want).max()), float(np.abs(want).max()))


@pytest.mark.parametrize("levels,n", [(2, 16), (4, 32)])
def test_forward_matches_the_oracle_end_to_end(dev, levels, n):
    P = _params(levels, 16, 21)
    x = _input(n, 9)
    net = B.UNet(levels, 16, (n, n, n))
    net.set_params(flat(P))
    pred = net.forward(x).astype(np.float64)
    Pb = {k: (bf16(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in P.items()}
    ref, _ = U.forward(Pb, bf16(x))
    ref = ref[0]
    assert not pred[x[1] <= 0].any()
    err = np.linalg.norm(pred - ref) / np.linalg.norm(ref)
    assert err < 2e-2, err


def test_params_round_trip(dev):
    P = _params(3, 16, 4)
    net = B.UNet(3, 16, (16, 16, 16))
    f = flat(P)
    net.set_params(f)
    back = net.get_params()
    assert back.shape == f.shape
    np.testing.assert_allclose(back, f.astype(np.float32).astype(np.float64), rtol=0, atol=0)


def _grad_case(levels, n, seed):
    P = _params(levels, 16, seed)
    x = _input(n, seed + 2)
    g = np.random.default_rng(seed + 3).normal(size=x.shape[1:]).astype(np.float32)
    net = B.UNet(levels, 16, x.shape[1:])
    net.set_params(flat(P))
    net.forward(x)
    net.backward(g)
    G = net.get_grads()
    return P, x, g, net, G


def _own_cache(levels, P, x, net):
    """The oracle's forward cache rebuilt from the network's own BF16
    activations (each layer's input and its ReLU output, whose sign gives the
    same mask as the pre-activation)."""
    names = _names(levels)
    out = {nm: net.layer_output(i).astype(np.float64) for i, nm in enumerate(names)}
    cache = {"x": bf16(x), "act": (x[1:2] > 0).astype(np.float64)}
    for nm in names:
        l, j = int(nm[-3]), int(nm[-1])
        if nm.startswith("down"):
            inp = out["down%d.0" % l] if j == 1 else (bf16(x) if l == 0 else bf16(_pool(out["down%d.1" % (l - 1)])))
        elif j == 1:
            inp = out["up%d.0" % l]
        else:
            below = out["down%d.1" % (levels - 1)] if l == levels - 2 else out["up%d.1" % (l + 1)]
            inp = np.concatenate([out["down%d.1" % l], U.upsample2(below)], axis=0)
        cache[nm + ".in"] = inp
        cache[nm + ".z"] = out[nm]
    cache["head.in"] = out["up0.1" if levels > 1 else "down0.1"]
    return cache, out


def _split(P, G):
    d, k0 = {}, 0
    for k in P:
        d[k] = G[k0:k0 + P[k].size].reshape(P[k].shape)
        k0 += P[k].size
    return d


@pytest.mark.parametrize("levels,n", [(2, 16), (3, 16), (2, (4, 4, 128))])
def test_each_backward_step_matches_the_oracle(dev, levels, n):
    """Per layer, on the network's own tensors: the weight and bias
    gradients are the oracle's convolution backward of the layer's input and
    pre-activation gradient (FP32 sums of BF16 products: relative 1e-5), the
    pre-activation gradient of the layer below is its backward-data output
    times the ReLU mask (one BF16 rounding), and the head, upsampling and
    pooling gradients likewise."""
    P, x, g, net, G = _grad_case(levels, n, 70 + levels)
    Pb = {k: (bf16(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in P.items()}
    cache, out = _own_cache(levels, P, x, net)
    names = _names(levels)
    gz = {nm: net.layer_grad(i).astype(np.float64) for i, nm in enumerate(names)}
    Gd = _split(P, G)

    def close(got, want, what, mag=None):
        # one BF16 rounding of each summand (mag: the sum of the summands'
        # magnitudes, where rounded terms are added) and of the result
        mag = np.abs(want) if mag is None else mag
        bound = 2.0 ** -8 * (mag + np.abs(want)) + 2e-3 * np.abs(want).max()
        assert not (np.abs(got - want) > bound).any(), (what, float(np.abs(got - want).max()))

    top = cache["head.in"]
    w_h = P["head.w"].ravel()
    close(gz["up0.1"], (top > 0) * w_h[:, None, None, None] * (g * (x[1] > 0))[None], "head")
    for nm in names:
        l, j = int(nm[-3]), int(nm[-1])
        gx, gw, gb = U.conv3d_backward(cache[nm + ".in"], Pb[nm + ".w"], gz[nm])
        assert np.linalg.norm(Gd[nm + ".w"] - gw) <= 1e-5 * np.linalg.norm(gw), nm
        assert np.linalg.norm(Gd[nm + ".b"] - gb) <= 1e-5 * np.linalg.norm(gb) + 1e-12, nm
        if j == 1:
            lower = nm[:-1] + "0"
            close(gz[lower], gx * (out[lower] > 0), nm + " backward data")
        elif nm.startswith("up"):
            gcat = gx * (cache[nm + ".in"] > 0)
            c = out["down%d.1" % l].shape[0]
            below = "down%d.1" % (levels - 1) if l == levels - 2 else "up%d.1" % (l + 1)
            close(gz[below], U.upsample2_backward(gcat[c:]), nm + " upsampling backward",
                  U.upsample2_backward(np.abs(gcat[c:])))
            gx1, _, _ = U.conv3d_backward(cache["down%d.0.in" % (l + 1)], Pb["down%d.0.w" % (l + 1)],
                                          gz["down%d.0" % (l + 1)])
            pool_part = U.avg_pool2_backward(gx1) * (out["down%d.1" % l] > 0)
            close(gz["down%d.1" % l], gcat[:c] + pool_part, nm + " skip and pooling backward",
                  np.abs(gcat[:c]) + np.abs(pool_part))


@pytest.mark.parametrize("levels,n", [(1, 16), (2, 16), (3, 16), (4, 32)])
def test_gradients_match_the_oracle_on_the_networks_activations(dev, levels, n):
    """The whole gradient against the oracle's backward pass on the
    network's own forward activations: the remaining differences are the
    BF16 roundings of the gradient tensors (relative L2 <= 2e-2)."""
    P, x, g, net, G = _grad_case(levels, n, 40 + levels)
    Pb = {k: (bf16(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in P.items()}
    cache, _ = _own_cache(levels, P, x, net)
    Gr = U.backward(Pb, cache, g[None].astype(np.float64))
    ref = flat({k: Gr[k] for k in P})
    err = np.linalg.norm(G - ref) / np.linalg.norm(ref)
    assert err < 2e-2, err


@pytest.mark.parametrize("levels,n", [(2, 16), (4, 32)])
def test_gradients_near_the_fp64_network(dev, levels, n):
    """Against the oracle's own FP64 forward and backward: about 1% of the
    ReLU masks differ between BF16 and FP64 activations, and gradient sums
    that mostly cancel magnify that to several per cent; the gradient keeps
    its direction."""
    P, x, g, net, G = _grad_case(levels, n, 40 + levels)
    Pb = {k: (bf16(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in P.items()}
    _, cache = U.forward(Pb, bf16(x))
    Gr = U.backward(Pb, cache, g[None].astype(np.float64))
    ref = flat({k: Gr[k] for k in P})
    assert np.linalg.norm(G - ref) / np.linalg.norm(ref) < 0.2
    assert np.dot(G, ref) / np.dot(ref, ref) > 0.9


def test_adam_step_matches_the_oracle(dev):
    P, _, _, net, G = _grad_case(2, 16, 50)
    theta0 = net.get_params()
    net.adam_step(lr=1e-3)
    theta1 = net.get_params()
    Q = {}
    k0 = 0
    for k in P:
        Q[k] = theta0[k0:k0 + P[k].size].reshape(P[k].shape).copy()
        k0 += P[k].size
    Gd, k0 = {}, 0
    for k in P:
        Gd[k] = G[k0:k0 + P[k].size].reshape(P[k].shape)
        k0 += P[k].size
    U.adam_step(Q, Gd, {}, lr=1e-3)
    want = flat(Q)
    np.testing.assert_allclose(theta1 - theta0, want - theta0, rtol=1e-4, atol=1e-9)


def test_training_reduces_the_loss_on_a_fixed_sample(dev):
    n = 16
    P = _params(2, 16, 60)
    x = _input(n, 62)
    y = (x[0] * (x[1] > 0)).astype(np.float32)  # a target the convolutions can represent
    net = B.UNet(2, 16, (n, n, n))
    net.set_params(flat(P))
    pred = net.forward(x).astype(np.float64)
    loss_ref, _ = U.loss_and_grad(pred, y.astype(np.float64), x[1])
    losses = [net.train_step(x, y, lr=1e-3) for _ in range(60)]
    assert losses[0] == pytest.approx(loss_ref, rel=1e-5)
    assert losses[-1] < 0.3 * losses[0], losses
