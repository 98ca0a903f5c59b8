"""Plain FP64 CPU definition of the learned initial guess's network: its
input channels, a 3D U-Net forward and backward pass, and its Adam update.

TEST INFRASTRUCTURE ONLY.  The paper has no network; this module writes out
the definition of the one the learned-guess form uses, so that its GPU
kernels can be held to it.  Only the tests may import it.  It shares no code
with the CUDA library.

The network (all tensors [C, D, H, W], z slowest, x fastest; D, H and W
divisible by 2^(levels - 1)):
- level l has c_l = base * 2^l channels, l = 0 .. levels - 1;
- down path: level 0 takes the input; level l > 0 takes the 2x2x2 average
  pool of level l - 1's output; each level applies two 3x3x3 convolutions
  (zero padding 1, bias), each followed by ReLU;
- up path, l = levels - 2 .. 0: nearest-neighbour upsampling by 2 of the
  level below, concatenated after level l's down output (skip first), then
  two 3x3x3 convolutions with ReLU;
- head: a 1x1x1 convolution to one channel, multiplied by the active mask
  (input channel 1 > 0), so inactive cells predict 0.

Loss: sum over active cells of (p - y)^2 divided by the sum of y^2 there
(relative squared error).  Adam: the textbook update (Kingma & Ba, 2015,
Algorithm 1) with bias correction.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Inputs and target
# --------------------------------------------------------------------------

def features(mask, rho, faces, h):
    """The network's three input channels for one fine level, and the scale s
    that maps its output back to Phi (Phi = s * prediction).
    - channel 0: h^2 rho n^2 / s on active cells (n = the largest dimension,
      so h^2 n^2 is the squared box size: Phi ~ rho L^2), 0 elsewhere;
    - channel 1: +1 on active cells, -1 elsewhere;
    - channel 2: the mean Dirichlet value over the cell's ghost faces (faces
      toward an inactive or out-of-box neighbour) / s, 0 where there are none;
    - s: the root of the mean square of channel 0's numerator over active
      cells plus the mean square of the ghost-face values, so that scaling rho
      and the boundary values by c > 0 leaves the channels unchanged and
      scales s by c (the problem is linear in both).
    faces = (bx, by, bz) as in mg_set_dirichlet: bx [nz, ny, nx+1], by
    [nz, ny+1, nx], bz [nz+1, ny, nx]; None for zero values."""
    act = mask > 0
    nz, ny, nx = act.shape
    bx, by, bz = faces
    bx = np.zeros((nz, ny, nx + 1)) if bx is None else bx
    by = np.zeros((nz, ny + 1, nx)) if by is None else by
    bz = np.zeros((nz + 1, ny, nx)) if bz is None else bz
    pad = np.pad(act, 1, constant_values=False)
    nbr_and_face = [(pad[1:-1, 1:-1, :-2], bx[:, :, :-1]), (pad[1:-1, 1:-1, 2:], bx[:, :, 1:]),
                    (pad[1:-1, :-2, 1:-1], by[:, :-1, :]), (pad[1:-1, 2:, 1:-1], by[:, 1:, :]),
                    (pad[:-2, 1:-1, 1:-1], bz[:-1, :, :]), (pad[2:, 1:-1, 1:-1], bz[1:, :, :])]
    total = np.zeros(act.shape)
    count = np.zeros(act.shape)
    sq, nfaces = 0.0, 0
    for nbr_active, face in nbr_and_face:
        ghost = act & ~nbr_active
        total += np.where(ghost, face, 0.0)
        count += ghost
        sq += float((face[ghost] ** 2).sum())
        nfaces += int(ghost.sum())
    n = max(act.shape)
    src = np.where(act, h * h * n * n * rho, 0.0)
    ms_src = float((src[act] ** 2).mean()) if act.any() else 0.0
    ms_face = sq / nfaces if nfaces else 0.0
    s = np.sqrt(ms_src + ms_face)
    if not s > 0:
        s = 1.0
    bval = np.where(count > 0, total / np.maximum(count, 1), 0.0)
    return np.stack([src / s, np.where(act, 1.0, -1.0), bval / s]), s


# --------------------------------------------------------------------------
# Layers
# --------------------------------------------------------------------------

def conv3d(x, w, b):
    """out[o, z, y, x] = b[o] + sum_{i, dz, dy, dx} w[o, i, dz, dy, dx] *
    xp[i, z + dz, y + dy, x + dx], with xp = x zero-padded by k // 2."""
    co, ci, k, _, _ = w.shape
    p = k // 2
    _, d, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (p, p)))
    out = np.broadcast_to(b[:, None, None, None], (co, d, h, wd)).astype(np.float64).copy()
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                sl = xp[:, dz:dz + d, dy:dy + h, dx:dx + wd]
                out += np.tensordot(w[:, :, dz, dy, dx], sl, axes=([1], [0]))
    return out


def conv3d_backward(x, w, g):
    """Gradients of sum(g * conv3d(x, w, b)) with respect to x, w and b."""
    co, ci, k, _, _ = w.shape
    p = k // 2
    _, d, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (p, p)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                sl = xp[:, dz:dz + d, dy:dy + h, dx:dx + wd]
                gw[:, :, dz, dy, dx] = np.tensordot(g, sl, axes=([1, 2, 3], [1, 2, 3]))
                gxp[:, dz:dz + d, dy:dy + h, dx:dx + wd] += np.tensordot(w[:, :, dz, dy, dx], g, axes=([0], [0]))
    gx = gxp[:, p:p + d, p:p + h, p:p + wd]
    return gx, gw, g.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def avg_pool2(x):
    c, d, h, w = x.shape
    return x.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).mean(axis=(2, 4, 6))


def avg_pool2_backward(g):
    return upsample2(g) / 8.0


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_backward(g):
    c, d, h, w = g.shape
    return g.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(axis=(2, 4, 6))


# --------------------------------------------------------------------------
# The network
# --------------------------------------------------------------------------

def init_params(seed, levels=4, base=16, c_in=3):
    """He-normal weights (std sqrt(2 / fan_in)) and zero biases, drawn from
    numpy's seeded generator in a fixed order: down blocks, up blocks, head."""
    rng = np.random.default_rng(seed)
    ch = [base * 2 ** l for l in range(levels)]
    P = {}

    def conv(name, ci, co, k=3):
        P[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (ci * k ** 3)), (co, ci, k, k, k))
        P[name + ".b"] = np.zeros(co)

    for l in range(levels):
        conv("down%d.0" % l, c_in if l == 0 else ch[l - 1], ch[l])
        conv("down%d.1" % l, ch[l], ch[l])
    for l in range(levels - 1):
        conv("up%d.0" % l, ch[l] + ch[l + 1], ch[l])
        conv("up%d.1" % l, ch[l], ch[l])
    conv("head", ch[0], 1, k=1)
    return P


def _levels(P):
    return sum(1 for k in P if k.startswith("down") and k.endswith(".0.w"))


def forward(P, x):
    """Returns (prediction [1, D, H, W], cache for backward)."""
    L = _levels(P)
    cache = {"x": x}
    h = x
    skips = []
    for l in range(L):
        if l:
            h = avg_pool2(h)
        for j in range(2):
            name = "down%d.%d" % (l, j)
            cache[name + ".in"] = h
            z = conv3d(h, P[name + ".w"], P[name + ".b"])
            cache[name + ".z"] = z
            h = relu(z)
        skips.append(h)
    for l in range(L - 2, -1, -1):
        h = np.concatenate([skips[l], upsample2(h)], axis=0)
        for j in range(2):
            name = "up%d.%d" % (l, j)
            cache[name + ".in"] = h
            z = conv3d(h, P[name + ".w"], P[name + ".b"])
            cache[name + ".z"] = z
            h = relu(z)
    cache["head.in"] = h
    act = (x[1:2] > 0).astype(np.float64)
    cache["act"] = act
    return conv3d(h, P["head.w"], P["head.b"]) * act, cache


def backward(P, cache, g_out):
    """Gradients of sum(g_out * forward(P, x)[0]) with respect to every
    parameter; returns a dict with the keys of P."""
    L = _levels(P)
    G = {}
    g = g_out * cache["act"]
    g, G["head.w"], G["head.b"] = conv3d_backward(cache["head.in"], P["head.w"], g)
    g_skip = [None] * L
    # up path, in reverse of the forward order (l = 0 .. L-2); what reaches
    # the concatenated input splits into the skip's part and the upsampled
    # part
    for l in range(0, L - 1):
        for j in (1, 0):
            name = "up%d.%d" % (l, j)
            g = g * (cache[name + ".z"] > 0)
            g, G[name + ".w"], G[name + ".b"] = conv3d_backward(cache[name + ".in"], P[name + ".w"], g)
        cs = P["down%d.1.w" % l].shape[0]
        g_skip[l] = g[:cs]
        g = upsample2_backward(g[cs:])
    # down path, deepest level first
    for l in range(L - 1, -1, -1):
        if g_skip[l] is not None:
            g = g + g_skip[l]
        for j in (1, 0):
            name = "down%d.%d" % (l, j)
            g = g * (cache[name + ".z"] > 0)
            g, G[name + ".w"], G[name + ".b"] = conv3d_backward(cache[name + ".in"], P[name + ".w"], g)
        if l:
            g = avg_pool2_backward(g)
    return G


def loss_and_grad(p, y, act):
    """Relative squared error over the active cells and its gradient in p."""
    m = (act > 0).astype(np.float64)
    den = float((y * y * m).sum())
    r = (p - y) * m
    return float((r * r).sum()) / den, 2.0 * r / den


def adam_step(P, G, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter in place; state holds t, m and v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m." + k, np.zeros_like(P[k]))
        v = state.setdefault("v." + k, np.zeros_like(P[k]))
        m *= beta1
        m += (1.0 - beta1) * G[k]
        v *= beta2
        v += (1.0 - beta2) * G[k] * G[k]
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        P[k] -= lr * mhat / (np.sqrt(vhat) + eps)
