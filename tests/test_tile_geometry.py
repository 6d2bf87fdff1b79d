"""Tile classes of the fused step and the index arithmetic of its TMA tiles,
on the CPU.

`lbm_tile_kinds` returns the library's own classification (the host/device
`tile_kind` and `seam_bits` of csrc/cplbm_internal.h).  These tests check it
against the rules it documents and then, for every tile the library sends to
a TMA path, check a model of that path's global index arithmetic (the
formulas of csrc/step_impl.cuh: staged partial sums, the seam fix-ups, the
wrapped writes and the neighbour tiles of the density hand-over):

* every index stays inside its array (populations 8 planes of nyf x pitch,
  densities nyf x pitch, partial sums as allocated by capi.cu);
* every staged entry the step reads that a TMA box fills with zeros (it lies
  across a periodic edge) is replaced from the wrapped node;
* every neighbour tile the hand-over writes to is the tile that holds the
  neighbour node;
* the launch that asks only for the TMA path's shared memory has no general
  tile.

A wrong index here is a wrong result or a fault on the GPU, where the
parity tests would meet it; this catches it without one.
"""
import random

import numpy as np
import pytest

from paper_1611_00907_gb300 import LbmError, _build, _lib, tile_kinds

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
R_L, R_R, R_B, R_T, R_BL, R_BR, R_TL, R_TR = range(8)
SHAPES = [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)]


@pytest.fixture(scope="module", autouse=True)
def library():
    _build.build()
    return _lib.load()


def wrap(v, n):
    return v + n if v < 0 else (v - n if v >= n else v)


class Geometry:
    """Lattice layout as capi.cu allocates it."""

    def __init__(self, nx, ny, walls):
        self.nx, self.ny, self.walls = nx, ny, walls
        self.nyf = ny - 2 if walls else ny
        self.pitch = (nx + 31) // 32 * 32
        self.nyf_pad = (self.nyf + 31) // 32 * 32

    def ring_elems(self, c):
        ncx, ncy = (self.nx + 31) // 32, (self.nyf + 15) // 16
        if c in (R_L, R_R):
            return ncx * self.nyf_pad
        if c in (R_B, R_T):
            return ncy * self.pitch
        return ncy * ncx

    def ring_index(self, c, bx, by, r, x):
        if c in (R_L, R_R):
            return bx * self.nyf_pad + r
        if c in (R_B, R_T):
            return by * self.pitch + x
        return by * ((self.nx + 31) >> 5) + bx


def rule_kind(g, tx, ty, bx, by, seams):
    """The classification as cplbm.h and cplbm_internal.h state it."""
    nfx, nfy = g.nx // tx, g.nyf // ty
    rx, ry = g.nx - nfx * tx, g.nyf - nfy * ty
    sx = seams and nfx >= 3 and (rx == 0 or rx >= 4)
    sy = seams and not g.walls and nfy >= 3 and (ry == 0 or ry >= 4)
    xhi = nfx - 1 if rx >= 4 else nfx - 2
    yhi = nfy - 1 if ry >= 4 else nfy - 2
    ix, iy = 1 <= bx <= xhi, 1 <= by <= yhi
    if ix and iy:
        return 2
    if (ix or (sx and bx < nfx)) and (iy or (sy and by < nfy)):
        return 1
    return 0


def edge_tile(ci):
    return -1 if ci == 0 else (1 if ci == 3 else 0)


def neighbour_tile(c0, d, t, n, seam):
    c = c0 - 1 if d < 0 else (c0 + t if d > 0 else c0)
    return (wrap(c, n) if seam else c) // t


def pin_col(px, i):   # odd steps
    return px - 1 if EX[i] == 1 else (1 if EX[i] == -1 else 0)


def check_tile(g, tx, ty, bx, by, seam):
    x0, y0 = bx * tx, by * ty
    nx, nyf = g.nx, g.nyf
    assert x0 + tx <= nx and y0 + ty <= nyf, "TMA tiles are full"
    # the four (or, wrapped, more distant) neighbour tiles across the halo
    # are full or at least 4 nodes wide
    for c in (x0 - 1, x0 + tx):
        if seam or 0 <= c < nx:
            t = wrap(c, nx) // tx
            assert min(tx, nx - t * tx) >= 4
    for c in (y0 - 1, y0 + ty):
        if seam or 0 <= c < nyf:
            t = wrap(c, nyf) // ty
            assert min(ty, nyf - t * ty) >= 4
    cl, rl = ty + 8, tx + 8
    if not seam:
        assert x0 >= 2 and x0 + tx + 1 < nx and y0 >= 2 and y0 + ty + 1 < nyf
        # bulk copies of the partial sums: contiguous runs inside the arrays
        for ci in range(4):
            c = R_L if ci & 1 else R_R
            i0 = g.ring_index(c, bx + edge_tile(ci), by, y0 - 4, x0)
            assert 0 <= i0 and i0 + cl <= g.ring_elems(c)
        for ri in range(4):
            c = R_B if ri & 1 else R_T
            i0 = g.ring_index(c, bx, by + edge_tile(ri), y0, x0 - 4)
            assert 0 <= i0 and i0 + rl <= g.ring_elems(c)
        return
    # seam tiles: partial sums staged element by element, wrapped
    for ci in range(4):
        c = R_L if ci & 1 else R_R
        t = neighbour_tile(x0, edge_tile(ci), tx, nx, True)
        for j in range(cl):
            assert 0 <= g.ring_index(c, t, 0, wrap(y0 - 4 + j, nyf), 0) < g.ring_elems(c)
    for ri in range(4):
        c = R_B if ri & 1 else R_T
        t = neighbour_tile(y0, edge_tile(ri), ty, nyf, True)
        for j in range(rl):
            assert 0 <= g.ring_index(c, 0, t, 0, wrap(x0 - 4 + j, nx)) < g.ring_elems(c)
    xl, xr, yb, yt = x0 == 0, x0 + tx >= nx, y0 == 0, y0 + ty >= nyf
    # density fix-ups (seam_rho_slot) cover every zero-filled entry read
    fixed = set()
    for t in range(2 * (ty + 4) + 2 * (tx + 4)):
        if t < 2 * (ty + 4):
            if not (xl or xr):
                continue
            ly, c = t >> 1, (2 if xl else tx + 4) + (t & 1)
        else:
            if not (yb or yt):
                continue
            q = t - 2 * (ty + 4)
            sel = q // (tx + 4)
            ly, c = (0 if yb else ty + 2) + sel, 2 + q - sel * (tx + 4)
        x, r = wrap(x0 - 4 + c, nx), wrap(y0 - 2 + ly, nyf)
        assert 0 <= x < nx and 0 <= r < nyf
        fixed.add((ly, c))
    for ly in range(ty + 4):
        for c in range(2, tx + 6):
            if not (0 <= x0 - 4 + c < nx and 0 <= y0 - 2 + ly < nyf):
                assert (ly, c) in fixed
    # odd-step population fix-ups (seam_pop_slot) cover every source across
    # an edge; only boundary nodes can have one
    fixed = set()
    for t in range(3 * ty + 3 * tx):
        if t < 3 * ty:
            if not (xl or xr):
                continue
            d, ly = t // ty, t % ty
            lx = 0 if xl else tx - 1
            i = ([1, 5, 8] if xl else [3, 6, 7])[d]
        else:
            if not (yb or yt):
                continue
            q = t - 3 * ty
            d, lx = q // tx, q % tx
            ly = 0 if yb else ty - 1
            i = ([2, 5, 6] if yb else [4, 7, 8])[d]
        xs, rs = wrap(x0 + lx - EX[i], nx), wrap(y0 + ly - EY[i], nyf)
        assert 0 <= xs < nx and 0 <= rs < nyf
        fixed.add((i, ly, lx))
    border = {(lx, ly) for lx in (0, tx - 1) for ly in range(ty)} | \
             {(lx, ly) for ly in (0, ty - 1) for lx in range(tx)}
    for lx, ly in border:
        for i in range(1, 9):
            if not (0 <= x0 + lx - EX[i] < nx and 0 <= y0 + ly - EY[i] < nyf):
                assert (i, ly, lx) in fixed
            # the staged column matches the box's start
            px = 4
            start = x0 - px if EX[i] == 1 else x0
            assert start + lx + pin_col(px, i) == x0 + lx - EX[i]
        # odd-step writes: the offset correction (lanes 0 / TX-1, rows 0 /
        # TY-1 at an edge) brings every target back into the lattice
        for i in range(1, 9):
            x, r = x0 + lx + EX[i], y0 + ly + EY[i]
            if EX[i] < 0 and xl and lx == 0:
                x += nx
            if EX[i] > 0 and xr and lx == tx - 1:
                x -= nx
            if EY[i] < 0 and yb and ly == 0:
                r += nyf
            if EY[i] > 0 and yt and ly == ty - 1:
                r -= nyf
            assert 0 <= x < nx and 0 <= r < nyf
    # hand-over: neighbour tiles are the tiles of the neighbour nodes
    for d in (-1, 1):
        t = neighbour_tile(x0, d, tx, nx, True)
        assert t == wrap(x0 - 1 if d < 0 else x0 + tx, nx) // tx
        assert 0 <= g.ring_index(R_L, t, 0, nyf - 1, 0) < g.ring_elems(R_L)
        t = neighbour_tile(y0, d, ty, nyf, True)
        assert t == wrap(y0 - 1 if d < 0 else y0 + ty, nyf) // ty
        assert 0 <= g.ring_index(R_T, 0, t, 0, nx - 1) < g.ring_elems(R_T)


def _lattices():
    fixed = [(96, 96, False), (128, 48, False), (96, 50, True), (224, 165, False),
             (160, 100, False), (100, 100, False), (99, 54, True), (134, 77, True),
             (196, 52, False), (192, 98, True), (1000, 1000, False), (500, 200, True),
             (70, 21, False), (5, 5, False), (131, 37, True), (4096, 4096, False)]
    rng = random.Random(1611)
    extra = [(rng.choice([32, 64, 96, 128, 160, 192, 224, 256]) + rng.choice([0, 0, 1, 3, 4, 5, 20]),
              rng.randint(7, 300), rng.random() < 0.5) for _ in range(60)]
    return fixed + extra


@pytest.mark.parametrize("seams", [True, False])
def test_library_classes_follow_the_stated_rules(seams):
    for nx, ny, walls in _lattices():
        g = Geometry(nx, ny, walls)
        for tx, ty in SHAPES:
            got = tile_kinds(nx, ny, walls, (tx, ty), seams)
            want = np.array([[rule_kind(g, tx, ty, bx, by, seams)
                              for bx in range(got.shape[1])] for by in range(got.shape[0])])
            assert got.shape == (-(-g.nyf // ty), -(-nx // tx))
            assert np.array_equal(got, want), (nx, ny, walls, tx, ty)


def test_index_arithmetic_of_tma_tiles():
    checked = 0
    for nx, ny, walls in _lattices():
        if nx * ny > 300 * 300:
            continue
        g = Geometry(nx, ny, walls)
        for tx, ty in SHAPES:
            kinds = tile_kinds(nx, ny, walls, (tx, ty), True)
            for by, bx in zip(*np.nonzero(kinds)):
                check_tile(g, tx, ty, int(bx), int(by), kinds[by, bx] == 1)
                checked += 1
    assert checked > 2000


def test_small_shared_memory_launch_has_no_general_tile():
    # launch_shape asks only for the TMA path's shared memory when both
    # periodic directions are seams over full tiles
    for nx, ny, walls in _lattices():
        for tx, ty in SHAPES:
            g = Geometry(nx, ny, walls)
            if not walls and nx % tx == 0 and g.nyf % ty == 0 and \
                    nx // tx >= 3 and g.nyf // ty >= 3:
                assert tile_kinds(nx, ny, walls, (tx, ty), True).min() >= 1


def test_tile_kinds_rejects_bad_arguments():
    with pytest.raises(LbmError):
        tile_kinds(64, 64, False, (48, 16))
    with pytest.raises(LbmError):
        tile_kinds(4, 64, False, (32, 32))
    lib = _lib.load()
    short = np.zeros(3, dtype=np.int32)
    assert lib.lbm_tile_kinds(128, 128, 0, 32, 32, 1, short.ctypes.data, short.size) != 0
