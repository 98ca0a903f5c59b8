"""Seeded synthetic inputs for the masked-domain Poisson solver.

This module holds no part of the multigrid method: it only draws masks,
right-hand sides and boundary data.  Both the CUDA library's tests and the
CPU oracle's tests take their inputs from here, so both sides see identical
arrays.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014): the state
advances by 0x9E3779B97F4A7C15 and each output is the state passed through
the published two-multiply finaliser.  Uniforms use the top 53 bits; normals
use the Box-Muller transform.  Arrays are indexed [k, j, i] with x fastest;
cell (i, j, k) of an N-cell unit box has its centre at ((i+1/2)h, (j+1/2)h,
(k+1/2)h), h = 1/N.

The workloads stand in for the paper's RAMSES grids, which are not
available: a ball (the 3D analogue of the disk of the residual-history
test), a union of spheres, a cube riddled with sub-cell holes (the "small
islands" regime of Section 4), and random-blob AMR patches.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
            z = self.state + steps
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def cell_centres(n: int, h: float):
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def faces_from_function(fn, nx: int, ny: int, nz: int, h: float):
    """Face-centre samples of fn(x, y, z) on the three face families:
    bx[k, j, i] at (i h, (j+1/2) h, (k+1/2) h) for i in 0..nx, and likewise
    by, bz."""
    xc, yc, zc = cell_centres(nx, h), cell_centres(ny, h), cell_centres(nz, h)
    xf, yf, zf = np.arange(nx + 1) * h, np.arange(ny + 1) * h, np.arange(nz + 1) * h
    bx = fn(xf[None, None, :], yc[None, :, None], zc[:, None, None])
    by = fn(xc[None, None, :], yf[None, :, None], zc[:, None, None])
    bz = fn(xc[None, None, :], yc[None, :, None], zf[:, None, None])
    return (np.ascontiguousarray(np.broadcast_to(bx, (nz, ny, nx + 1)), dtype=np.float64),
            np.ascontiguousarray(np.broadcast_to(by, (nz, ny + 1, nx)), dtype=np.float64),
            np.ascontiguousarray(np.broadcast_to(bz, (nz + 1, ny, nx)), dtype=np.float64))


def _sin3(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def ball(n: int = 32, radius: float = 0.4):
    """Ball workload: an n^3 box on [0,1]^3, active cells are those whose
    centre lies strictly inside the ball of the given radius centred at
    (1/2,1/2,1/2).  Manufactured solution phi = sin(pi x) sin(pi y) sin(pi z),
    rho = Laplacian(phi) = -3 pi^2 phi at cell centres, Dirichlet values phi at
    the face centres."""
    h = 1.0 / n
    c = cell_centres(n, h)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    mask = (r2 < radius * radius).astype(np.int8)
    phi = _sin3(x, y, z)
    rho = -3.0 * np.pi ** 2 * phi
    bx, by, bz = faces_from_function(_sin3, n, n, n, h)
    return {"name": "ball_%d" % n, "mask": mask, "rho": rho, "bx": bx, "by": by, "bz": bz, "h": h,
            "phi_exact": phi, "tol": 1e-10}


def _sphere_mask(n, centres, radii, h, inside_value, base_value):
    """Marks cells whose centre lies strictly inside any sphere."""
    mask = np.full((n, n, n), base_value, dtype=np.int8)
    c = cell_centres(n, h)
    for (cx, cy, cz), r in zip(centres, radii):
        lo = [max(0, int(math.floor((v - r) / h - 1))) for v in (cx, cy, cz)]
        hi = [min(n, int(math.ceil((v + r) / h + 1))) for v in (cx, cy, cz)]
        xs, ys, zs = c[lo[0]:hi[0]], c[lo[1]:hi[1]], c[lo[2]:hi[2]]
        d2 = ((xs[None, None, :] - cx) ** 2 + (ys[None, :, None] - cy) ** 2 + (zs[:, None, None] - cz) ** 2)
        sub = mask[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[d2 < r * r] = inside_value
    return mask


def sphere_union(n: int = 256, seed: int = 2, n_spheres: int = 40, n_gauss: int = 8, sigma: float = 0.03):
    """Union-of-spheres workload: the active domain is the union of
    n_spheres balls with centres U[0.2,0.8]^3 and radii U[0.05,0.2];
    rho is a sum of n_gauss Gaussians of width sigma with amplitudes N(0,1)
    and centres U[0.2,0.8]^3; Dirichlet value 0.  Draw order: sphere
    centres (x,y,z per sphere), radii, Gaussian amplitudes, Gaussian centres."""
    h = 1.0 / n
    rng = SplitMix64(seed)
    centres = rng.uniform(3 * n_spheres, 0.2, 0.8).reshape(n_spheres, 3)
    radii = rng.uniform(n_spheres, 0.05, 0.2)
    amps = rng.normal(n_gauss)
    gcent = rng.uniform(3 * n_gauss, 0.2, 0.8).reshape(n_gauss, 3)
    mask = _sphere_mask(n, centres, radii, h, 1, 0)
    c = cell_centres(n, h)
    rho = np.zeros((n, n, n))
    for a, (gx, gy, gz) in zip(amps, gcent):
        ex = np.exp(-((c - gx) ** 2) / (2 * sigma * sigma))
        ey = np.exp(-((c - gy) ** 2) / (2 * sigma * sigma))
        ez = np.exp(-((c - gz) ** 2) / (2 * sigma * sigma))
        rho += a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return {"name": "sphere_union_%d" % n, "mask": mask, "rho": rho, "bx": None, "by": None, "bz": None,
            "h": h, "tol": 1e-8}


def holes(n: int = 512, seed: int = 3, n_spheres: int | None = None, r_min: float = 0.5, r_max: float = 4.0):
    """Cube-with-holes workload: the unit cube minus n_spheres excluded balls
    with centres U[0,1]^3 and radii U[r_min, r_max] cells; a cell is excluded
    if its centre is inside a ball.  rho ~ U[-1,1] (drawn for every cell,
    ignored on excluded ones); Dirichlet value 0.  n_spheres defaults to
    20000 (n/512)^3 so that the hole density matches the 512^3 case."""
    if n_spheres is None:
        n_spheres = max(1, int(round(20000 * (n / 512.0) ** 3)))
    h = 1.0 / n
    rng = SplitMix64(seed)
    centres = rng.uniform(3 * n_spheres).reshape(n_spheres, 3)
    radii = rng.uniform(n_spheres, r_min, r_max) * h
    mask = _sphere_mask(n, centres, radii, h, 0, 1)
    rho = rng.uniform(n * n * n, -1.0, 1.0).reshape(n, n, n)
    return {"name": "holes_%d" % n, "mask": mask, "rho": rho, "bx": None, "by": None, "bz": None, "h": h,
            "tol": 1e-8}


def random_mask(shape, seed: int, p_active: float = 0.7):
    """Independent random cells, active with probability p_active."""
    rng = SplitMix64(seed)
    n = int(np.prod(shape))
    return (rng.uniform(n) < p_active).astype(np.int8).reshape(shape)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0):
    rng = SplitMix64(seed)
    return rng.uniform(int(np.prod(shape)), lo, hi).reshape(shape)


def random_faces(shape, seed: int):
    nz, ny, nx = shape
    rng = SplitMix64(seed)
    bx = rng.uniform(nz * ny * (nx + 1), -1, 1).reshape(nz, ny, nx + 1)
    by = rng.uniform(nz * (ny + 1) * nx, -1, 1).reshape(nz, ny + 1, nx)
    bz = rng.uniform((nz + 1) * ny * nx, -1, 1).reshape(nz + 1, ny, nx)
    return bx, by, bz


def coarse_potential(shape_c, seed: int, n_modes: int = 6):
    """A smooth coarse-level potential on a grid of shape_c (indexed
    [K, J, I]): a sum of n_modes random low Fourier modes with N(0,1)
    amplitudes, wave numbers 1..3 per axis and U[0, 2 pi) phases."""
    cz, cy, cx = shape_c
    rng = SplitMix64(seed)
    amps = rng.normal(n_modes)
    waves = 1 + np.floor(rng.uniform(3 * n_modes) * 3).reshape(n_modes, 3)
    phases = rng.uniform(3 * n_modes, 0.0, 2 * math.pi).reshape(n_modes, 3)
    X = (np.arange(cx) + 0.5) / cx
    Y = (np.arange(cy) + 0.5) / cy
    Z = (np.arange(cz) + 0.5) / cz
    out = np.zeros(shape_c)
    for a, w, p in zip(amps, waves, phases):
        out += (a * np.cos(2 * math.pi * w[2] * Z + p[2])[:, None, None]
                * np.cos(2 * math.pi * w[1] * Y + p[1])[None, :, None]
                * np.cos(2 * math.pi * w[0] * X + p[0])[None, None, :])
    return out


def blob_patch(shape, seed: int, corr_cells: float = 8.0):
    """AMR-patch workload: a random blob mask (white noise smoothed by a
    Gaussian of width corr_cells, thresholded at 0), rho ~ U[-1,1] and a
    half-resolution coarse potential covering the patch with one coarse
    ghost cell on every side (origin (-2,-2,-2) in fine-cell units)."""
    nz, ny, nx = shape
    rng = SplitMix64(seed)
    noise = rng.normal(nx * ny * nz).reshape(shape)
    f = noise
    for axis, n in ((0, nz), (1, ny), (2, nx)):
        k = np.fft.fftfreq(n)
        g = np.exp(-0.5 * (2 * math.pi * k * corr_cells) ** 2)
        f = np.real(np.fft.ifft(np.fft.fft(f, axis=axis) * g.reshape([-1 if a == axis else 1 for a in range(3)]),
                                axis=axis))
    mask = (f > 0).astype(np.int8)
    rho = rng.uniform(nx * ny * nz, -1.0, 1.0).reshape(shape)
    shape_c = ((nz + 1) // 2 + 2, (ny + 1) // 2 + 2, (nx + 1) // 2 + 2)
    phi_c = coarse_potential(shape_c, seed + 1000003)
    return {"name": "blob_%dx%dx%d" % (nx, ny, nz), "mask": mask, "rho": rho, "phi_c": phi_c,
            "origin": (-2, -2, -2), "h": 1.0 / max(shape), "tol": 1e-8}


# ---------------------------------------------------------------------------
# Concentrated mass at a refined-level boundary (Section 5.1, last test)
# ---------------------------------------------------------------------------

def concentrated_phi(x, y, z, r0: float):
    """The concentrated potential of Section 5.1, ln(r^2 / r0^2 + 1), with r
    the distance to the box centre (1/2, 1/2, 1/2)."""
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    return np.log(r2 / (r0 * r0) + 1.0)


def concentrated_rho(x, y, z, r0: float):
    """The 3D Laplacian of concentrated_phi: with f(r) = ln(r^2/r0^2 + 1),
    f'' + 2 f'/r = (2 r^2 + 6 r0^2) / (r^2 + r0^2)^2 (the paper's 2D test has
    4 r0^2 / (r^2 + r0^2)^2 for the same potential)."""
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    return (2.0 * r2 + 6.0 * r0 * r0) / (r2 + r0 * r0) ** 2


def concentrated_coarse(nc: int, r0: float):
    """The coarse AMR level of the boundary-gradient test: the whole unit box
    at spacing 1/nc, every cell active, rho = concentrated_rho and Dirichlet
    values concentrated_phi at the box faces."""
    h = 1.0 / nc
    c = cell_centres(nc, h)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    fn = lambda a, b, d: concentrated_phi(a, b, d, r0)  # noqa: E731
    bx, by, bz = faces_from_function(fn, nc, nc, nc, h)
    return {"name": "concentrated_coarse_%d" % nc, "mask": np.ones((nc, nc, nc), np.int8),
            "rho": concentrated_rho(x, y, z, r0), "bx": bx, "by": by, "bz": bz, "h": h,
            "phi_exact": concentrated_phi(x, y, z, r0)}


def concentrated_patch(nc: int, r0: float, radius: float, d: float):
    """A refined patch at spacing 1/(2 nc) whose active cells are those with
    centre inside a ball of the given radius; the ball is shifted along +x so
    that its boundary passes at distance d from the mass at the box centre
    (d = radius: centred).  The patch starts one coarse cell outside the ball's
    bounding box, on a coarse-cell corner; ``origin`` is the corner of coarse
    cell (0,0,0) in the patch's fine-cell units, as the one-way interface
    (Dirichlet values from the coarse solution) takes it."""
    hc = 1.0 / nc
    h = hc / 2
    cx = 0.5 + (radius - d)
    centre = (cx, 0.5, 0.5)
    lo = [int(math.floor((v - radius) / hc)) - 1 for v in centre]
    hi = [int(math.ceil((v + radius) / hc)) + 1 for v in centre]
    if min(lo) < 0 or max(hi) > nc:
        raise ValueError("the patch must lie inside the coarse box")
    n = [2 * (b - a) for a, b in zip(lo, hi)]
    xs, ys, zs = [(2 * lo[a] + np.arange(n[a]) + 0.5) * h for a in range(3)]
    z, y, x = np.meshgrid(zs, ys, xs, indexing="ij")
    mask = (((x - cx) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) < radius * radius).astype(np.int8)
    return {"name": "concentrated_patch_d%.3f" % d, "mask": mask, "rho": concentrated_rho(x, y, z, r0),
            "h": h, "origin": (-2 * lo[0], -2 * lo[1], -2 * lo[2]),
            "phi_exact": concentrated_phi(x, y, z, r0), "corner": tuple(2 * v for v in lo)}


# ---------------------------------------------------------------------------
# Many AMR patches of one level (batched solve)
# ---------------------------------------------------------------------------

PATCH_EDGES = (32, 48, 64, 96, 128)


def amr_patches(n: int = 96, seed: int = 4, edges=PATCH_EDGES, h: float = 1.0 / 512):
    """n patches of one AMR level: each axis edge drawn uniformly from
    `edges`, each patch a blob_patch (thresholded smoothed noise of
    correlation length 8 cells, rho ~ U[-1,1], Dirichlet values from a
    half-resolution coarse potential); all patches share the cell size h."""
    rng = SplitMix64(seed)
    picks = np.floor(rng.uniform(3 * n) * len(edges)).astype(int).reshape(n, 3)
    out = []
    for p in range(n):
        nx, ny, nz = (edges[i] for i in picks[p])
        w = blob_patch((nz, ny, nx), seed=seed * 100003 + p)
        w["h"] = h
        w["name"] = "patch%d_%dx%dx%d" % (p, nx, ny, nz)
        out.append(w)
    return out
