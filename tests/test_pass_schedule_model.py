"""CPU model of the temporal-blocked smoothing pass's schedule (the wavefront
of kernels_pass.cu), checked bit for bit in FP32 against four sequential
red-black half-sweeps (two sweeps of Section 2's smoother), with nothing
shared with the CUDA code.

The model walks tiles of TQ x TJ slots (a slot holds the two x-neighbours
2q and 2q+1) and z-segments of Z planes exactly as the kernel does: each tile
starts from a private copy of the pass's input in which every red value is
NaN (the pass never reads red values from before it), runs the stages S1
(red) .. S4 (black) at planes t+3 .. t for t from six planes below the
segment, each stage on a ring of 3, 2, 1, 0 slots and rows around the tile
and of the same widths in z around the segment, and keeps only its interior.
Narrowing any ring, in-plane or in z, makes some tile read a value that is
not yet in the state the sequential half-sweeps would see, which the
bitwise comparison catches.
"""
import numpy as np
import pytest


def _problem(shape, seed, p_active=0.85):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    act = rng.random(shape) < p_active
    pad = np.pad(act, 1)
    nbr = [pad[1:-1, 1:-1, :-2], pad[1:-1, 1:-1, 2:], pad[1:-1, :-2, 1:-1], pad[1:-1, 2:, 1:-1],
           pad[:-2, 1:-1, 1:-1], pad[2:, 1:-1, 1:-1]]
    ghosts = sum((act & ~n).astype(np.int64) for n in nbr)
    invd = np.where(act, np.float32(1) / (np.float32(6) + ghosts.astype(np.float32)), np.float32(0))
    b = np.where(act, rng.normal(size=shape), 0).astype(np.float32)
    phi = np.where(act, rng.normal(size=shape), 0).astype(np.float32)
    k, j, i = np.indices(shape)
    colour = (i + j + k) & 1
    return act, invd.astype(np.float32), b, phi, colour


def _update(phi, act, invd, b, colour, c, sel):
    """Colour c's Gauss-Seidel update of the cells in `sel`, in the list
    kernel's order: (same-slot x + other x) + (y- + y+) + (z- + z+)."""
    nz, ny, nx = phi.shape
    p = np.pad(phi, 1)
    k, j, i = np.nonzero(sel & act & (colour == c))
    if k.size == 0:
        return
    same = np.where(i & 1, i - 1, i + 1)        # the other cell of the slot
    other = np.where(i & 1, i + 1, i - 1)       # the x-neighbour in the adjacent slot
    s = (p[k + 1, j + 1, same + 1] + p[k + 1, j + 1, other + 1]) + (p[k + 1, j, i + 1] + p[k + 1, j + 2, i + 1])
    s = s + (p[k, j + 1, i + 1] + p[k + 2, j + 1, i + 1])
    phi[k, j, i] = (s - b[k, j, i]) * invd[k, j, i]


def _sequential(phi0, act, invd, b, colour):
    phi = phi0.copy()
    allc = np.ones(phi.shape, bool)
    for c in (0, 1, 0, 1):
        _update(phi, act, invd, b, colour, c, allc)
    return phi


def _tiled(phi0, act, invd, b, colour, TQ, TJ, Z, rings=(3, 2, 1, 0), zrings=(3, 2, 1, 0), lead=6):
    nz, ny, nx = phi0.shape
    hx = (nx + 1) // 2
    k, j, i = np.indices(phi0.shape)
    q = i >> 1
    out = np.zeros_like(phi0)
    for k0 in range(0, nz, Z):
        for j0 in range(0, ny, TJ):
            for q0 in range(0, hx, TQ):
                st = np.where(colour == 1, phi0, np.float32(np.nan)).astype(np.float32)
                for t in range(k0 - lead, k0 + Z):
                    for s, c in enumerate((0, 1, 0, 1)):
                        plane = t + 3 - s
                        if not (k0 - zrings[s] <= plane < k0 + Z + zrings[s]) or not (0 <= plane < nz):
                            continue
                        r = rings[s]
                        region = ((k == plane) & (q >= q0 - r) & (q < q0 + TQ + r) & (j >= j0 - r) &
                                  (j < j0 + TJ + r))
                        if s == 0:  # S1 also zeroes the inactive red cells of its region
                            st[region & ~act & (colour == 0)] = 0
                        _update(st, act, invd, b, colour, c, region)
                inner = (q >= q0) & (q < q0 + TQ) & (j >= j0) & (j < j0 + TJ) & (k >= k0) & (k < k0 + Z)
                out[inner] = st[inner]
    return out


CASES = [((11, 14, 13), 1, (2, 3, 3)), ((9, 8, 17), 2, (3, 2, 4)), ((12, 10, 9), 3, (1, 4, 5))]


@pytest.mark.parametrize("shape,seed,tile", CASES)
def test_wavefront_schedule_is_bit_identical_to_sequential_half_sweeps(shape, seed, tile):
    act, invd, b, phi, colour = _problem(shape, seed)
    ref = _sequential(phi, act, invd, b, colour)
    got = _tiled(phi, act, invd, b, colour, *tile)
    assert not np.isnan(got).any()
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))


@pytest.mark.parametrize("rings,zrings,lead", [((2, 2, 1, 0), (3, 2, 1, 0), 6), ((3, 1, 1, 0), (3, 2, 1, 0), 6),
                                               ((3, 2, 0, 0), (3, 2, 1, 0), 6), ((3, 2, 1, 0), (2, 2, 1, 0), 6),
                                               ((3, 2, 1, 0), (3, 1, 1, 0), 6), ((3, 2, 1, 0), (3, 2, 0, 0), 6),
                                               ((3, 2, 1, 0), (3, 2, 1, 0), 5)])
def test_narrower_rings_or_a_shorter_lead_in_break_the_schedule(rings, zrings, lead):
    shape, seed, tile = CASES[0]
    act, invd, b, phi, colour = _problem(shape, seed)
    ref = _sequential(phi, act, invd, b, colour)
    got = _tiled(phi, act, invd, b, colour, *tile, rings=rings, zrings=zrings, lead=lead)
    assert not np.array_equal(np.nan_to_num(got).view(np.int32), ref.view(np.int32))
