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
* every halo node the step reads gets exactly the partial sums (class and
  owning tile) that load_rho_stored adds for that node, no more and no fewer,
  from the staged entries that combine_ring adds at that position;
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
    nty = -(-g.nyf // ty)
    sx = seams and nfx >= 3 and (rx == 0 or rx >= 4)
    sy = seams and not g.walls and nfy >= 3 and (ry == 0 or ry >= 4)
    # wall tiles: two tile rows at least, the one above the bottom tile
    # full or at least 4 rows high
    sw = seams and g.walls and (nfy >= 2 or (nfy == 1 and ry >= 4))
    xhi = nfx - 1 if rx >= 4 else nfx - 2
    yhi = nfy - 1 if ry >= 4 else nfy - 2
    ix, iy = 1 <= bx <= xhi, 1 <= by <= yhi
    if ix and iy:
        return 2
    # a one-row top wall tile stays general (its only row is also a tile
    # bottom edge, read by the Eq. 28 average beyond the combined halo)
    wall = sw and (by == 0 or (by == nty - 1 and g.nyf - by * ty >= 2))
    # the ragged last tile of a periodic direction: TMA on 32-wide tiles
    ragged = seams and tx == 32
    if (ix or (sx and (bx < nfx or ragged))) and (iy or (sy and (by < nfy or ragged)) or wall):
        return 1
    return 0


def edge_tile(ci):
    return -1 if ci == 0 else (1 if ci == 3 else 0)


def neighbour_tile(c0, d, t, n, seam):
    c = c0 - 1 if d < 0 else (c0 + t if d > 0 else c0)
    return (wrap(c, n) if seam else c) // t


def pin_col(px, i):   # odd steps
    return px - 1 if EX[i] == 1 else (1 if EX[i] == -1 else 0)


def aa_read_source(g, i, r, x):
    """(plane, row, column) an odd step reads f_i of fluid node (x, r) from
    (aa_read_index): slot opp(i) of x - e_i, or with a solid source row the
    node's own slot i (halfway bounce-back); x and, without walls, y wrap."""
    rs = r - EY[i]
    if g.walls and not 0 <= rs < g.nyf:
        return i, r, x
    return OPP[i], wrap(rs, g.nyf), wrap(x - EX[i], g.nx)


def edge_pos(ci, w):
    """Halo column (row) of edge index ci of a tile w wide (high)."""
    return (1, 2, w + 1, w + 2)[ci]


def combine_model(tx, ty, hx, hy):
    """Staged (row, column) -> the staged entries combine_ring adds there:
    ('col', ci, j), ('row', ri, j), ('corner', ci, ri)."""
    add = {}
    for ci in range(4):
        lx = edge_pos(ci, hx)
        for ly in range(ty + 4):
            e = [("col", ci, ly + 2)]
            if ly in (1, 2, hy + 1, hy + 2):
                ri = (1, 2, hy + 1, hy + 2).index(ly)
                e += [("row", ri, lx + 2), ("corner", ci, ri)]
            add.setdefault((ly, lx + 2), []).extend(e)
    for ri in range(4):
        ly = edge_pos(ri, hy)
        for k in range(hx):
            lx = 0 if k == 0 else (hx + 3 if k == hx - 1 else k + 2)
            add.setdefault((ly, lx + 2), []).append(("row", ri, lx + 2))
    return add


def check_combine(g, tx, ty, bx, by, hx, hy, seam):
    """Every halo node the tile reads gets, from the staged entries
    combine_ring adds at its position, exactly the partial sums
    load_rho_stored adds for it (class and owning tile; entries staged as
    zeros, with no writer, count as absent)."""
    x0, y0 = bx * tx, by * ty
    nx, nyf = g.nx, g.nyf
    wb = g.walls and y0 == 0
    wt = g.walls and y0 + ty >= nyf
    vlo, vhi = (2 if wb else 0), (hy + 2 if wt else ty + 4)

    def resolve(entry):
        kind, a, b = entry
        if kind == "col":
            r = y0 - 4 + b
            if g.walls and not 0 <= r < nyf:
                return None
            t = neighbour_tile(x0, edge_tile(a), tx, nx, True)
            return (R_L if a & 1 else R_R, t, wrap(r, nyf))
        ri = a if kind == "row" else b
        if (wb and ri <= 1) or (wt and ri >= 2):
            return None
        ty_ = neighbour_tile(y0, edge_tile(ri), ty, nyf, not g.walls)
        if kind == "row":
            return (R_B if ri & 1 else R_T, ty_, wrap(x0 - 4 + b, nx))
        ci = a
        tx_ = neighbour_tile(x0, edge_tile(ci), tx, nx, True)
        left, below = ci & 1, ri & 1   # col_is_left, row_is_below
        c = (R_BL if left else R_BR) if below else (R_TL if left else R_TR)
        return (c, tx_, ty_)

    model = combine_model(tx, ty, hx, hy)
    for ly in range(vlo, min(vhi, hy + 4)):
        for c in range(2, hx + 6):
            xs, r = wrap(x0 - 4 + c, nx), y0 - 2 + ly
            rs = r if g.walls else wrap(r, nyf)
            tbx, tby = xs // tx, rs // ty
            wx, wy = min(tx, nx - tbx * tx), min(ty, nyf - tby * ty)
            lxn, lyn = xs - tbx * tx, rs - tby * ty
            left, right = lxn == 0, lxn == wx - 1
            below = lyn == 0 and not (g.walls and rs == 0)
            above = lyn == wy - 1 and not (g.walls and rs == nyf - 1)
            want = []
            if left:
                want.append((R_L, tbx, rs))
            if right:
                want.append((R_R, tbx, rs))
            if below:
                want.append((R_B, tby, xs))
                if left:
                    want.append((R_BL, tbx, tby))
                if right:
                    want.append((R_BR, tbx, tby))
            if above:
                want.append((R_T, tby, xs))
                if left:
                    want.append((R_TL, tbx, tby))
                if right:
                    want.append((R_TR, tbx, tby))
            got = [e for e in map(resolve, model.get((ly, c), [])) if e is not None]
            assert sorted(got) == sorted(want), (g.nx, g.ny, g.walls, tx, ty, bx, by,
                                                 ly, c, got, want)


def check_tile(g, tx, ty, bx, by, seam):
    x0, y0 = bx * tx, by * ty
    nx, nyf = g.nx, g.nyf
    wb = g.walls and y0 == 0
    wt = g.walls and y0 + ty >= nyf
    hx, hy = min(tx, nx - x0), min(ty, nyf - y0)   # columns and fluid rows of the tile
    if tx != 32:
        assert hx == tx, "two-nodes-per-lane TMA tiles are full in x"
        assert hy == ty or wt, "only a top wall tile may be ragged"
    assert hx >= 4 and (hy >= 4 or wt), "a ragged last tile is at least 4 wide"
    assert hy >= 1 and not (wb and wt)
    # the neighbour tiles across the halo are full or at least 4 nodes wide
    for c in (x0 - 1, x0 + tx):
        if seam or 0 <= c < nx:
            t = wrap(c, nx) // tx
            assert min(tx, nx - t * tx) >= 4
    for c in (y0 - 1, y0 + ty):
        if g.walls and not 0 <= c < nyf:
            continue                      # beyond a wall: no tile
        if seam or 0 <= c < nyf:
            t = wrap(c, nyf) // ty
            assert min(ty, nyf - t * ty) >= 4
    check_combine(g, tx, ty, bx, by, hx, hy, seam)
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
    # edge tiles: partial sums staged element by element, wrapped across
    # periodic edges; with walls only fluid rows and existing tile rows
    for ci in range(4):
        c = R_L if ci & 1 else R_R
        t = neighbour_tile(x0, edge_tile(ci), tx, nx, True)
        for j in range(cl):
            r = y0 - 4 + j
            if g.walls and not 0 <= r < nyf:
                continue
            assert 0 <= g.ring_index(c, t, 0, wrap(r, nyf), 0) < g.ring_elems(c)
    for ri in range(4):
        if (wb and ri <= 1) or (wt and ri >= 2):
            continue
        c = R_B if ri & 1 else R_T
        t = neighbour_tile(y0, edge_tile(ri), ty, nyf, not g.walls)
        if g.walls:   # the tile row of the halo node, no wrap
            assert t == by + (-1 if ri == 0 else 1 if ri == 3 else 0)
        for j in range(rl):
            assert 0 <= g.ring_index(c, 0, t, 0, wrap(x0 - 4 + j, nx)) < g.ring_elems(c)
    xl, xr = x0 == 0, x0 + tx >= nx
    yb, yt = not g.walls and y0 == 0, not g.walls and y0 + ty >= nyf
    vlo, vhi = (2 if wb else 0), (hy + 2 if wt else ty + 4)
    # density fix-ups (seam_rho_slot) cover every zero-filled entry read:
    # the fluid rows of the halo and the sources of the Eq. 28 rows
    fixed = set()
    for t in range(2 * (ty + 4) + 2 * (tx + 4) + 4):
        if t < 2 * (ty + 4):
            if not (xl or xr):
                continue
            ly, c = t >> 1, (2 if xl else hx + 4) + (t & 1)
            if not vlo <= ly < vhi:
                continue
        elif t < 2 * (ty + 4) + 2 * (tx + 4):
            if not (yb or yt):
                continue
            q = t - 2 * (ty + 4)
            sel = q // (tx + 4)
            ly, c = (0 if yb else hy + 2) + sel, 2 + q - sel * (tx + 4)
        else:
            k = t - 2 * (ty + 4) - 2 * (tx + 4)
            top, right = k >> 1, k & 1
            if not ((wt if top else wb) and (xr if right else xl)):
                continue
            ly, c = (hy + 1 if top else 2), (hx + 6 if right else 1)
        x, r = wrap(x0 - 4 + c, nx), y0 - 2 + ly
        assert 0 <= x < nx
        assert 0 <= r < nyf if g.walls else True
        fixed.add((ly, c))
    # the halo of the tile's own nodes: columns 2 .. hx + 5, rows up to hy + 3
    read = {(ly, c) for ly in range(vlo, min(vhi, hy + 4)) for c in range(2, hx + 6)}
    if wb:
        read |= {(2, c) for c in range(1, hx + 7)}
    if wt:
        read |= {(hy + 1, c) for c in range(1, hx + 7)}
    for ly, c in read:
        x, r = x0 - 4 + c, y0 - 2 + ly
        assert not (g.walls and not 0 <= r < nyf), "a solid row is read as stored"
        if not (0 <= x < nx and 0 <= r < nyf):
            assert (ly, c) in fixed, (ly, c)
        # entries outside the halo (columns 1 and tx + 6, read only by the
        # Eq. 28 average) get no partial sums: the node there must hold its
        # whole density, i.e. sit on no edge of its own tile that receives
        # partial sums (load_rho_stored)
        if c in (1, hx + 6):
            xs, rr = wrap(x, nx), r
            tx0 = xs // tx * tx
            wxx = min(tx, nx - tx0)
            ty0 = rr // ty * ty
            wyy = min(ty, nyf - ty0)
            lxx, lyy = xs - tx0, rr - ty0
            edge = lxx in (0, wxx - 1) or \
                (lyy == 0 and not (g.walls and rr == 0)) or \
                (lyy == wyy - 1 and not (g.walls and rr == nyf - 1))
            assert not edge, ("Eq. 28 source needs partial sums", ly, c)
    # odd-step population fix-ups (seam_pop_slot) cover every source the
    # TMA box cannot deliver: across a periodic edge, or in a solid row
    fixed = {}
    for t in range(3 * ty + 3 * tx):
        if t < 3 * ty:
            if not (xl or xr):
                continue
            d, ly = t // ty, t % ty
            if ly >= hy:
                continue
            lx = 0 if xl else hx - 1
            i = ([1, 5, 8] if xl else [3, 6, 7])[d]
        else:
            bottom = yb or wb
            if not (bottom or yt or wt):
                continue
            q = t - 3 * ty
            d, lx = q // tx, q % tx
            if lx >= hx:
                continue
            ly = 0 if bottom else hy - 1
            i = ([2, 5, 6] if bottom else [4, 7, 8])[d]
        src = aa_read_source(g, i, y0 + ly, x0 + lx)
        assert 0 <= src[1] < nyf and 0 <= src[2] < nx
        # two slots that name one node and direction fetch the same source
        assert fixed.setdefault((i, ly, lx), src) == src
    for ly in range(hy):
        for lx in range(hx):
            for i in range(1, 9):
                x, r = x0 + lx, y0 + ly
                plane, rs, xs = aa_read_source(g, i, r, x)
                # the TMA box of direction i delivers slot opp(i) at row r -
                # e_y, column x - e_x, inside the lattice only
                boxed = plane == OPP[i] and rs == r - EY[i] and xs == x - EX[i]
                if not boxed:
                    assert (i, ly, lx) in fixed, (i, ly, lx)
                # the staged column matches the box's start
                px = 4
                start = x0 - px if EX[i] == 1 else x0
                assert start + lx + pin_col(px, i) == x0 + lx - EX[i]
                # odd-step writes: into a solid row -> own slot opp(i);
                # across a periodic edge -> corrected back into the lattice
                xt, rt = x + EX[i], r + EY[i]
                if g.walls and not 0 <= rt < nyf:
                    assert (wb and ly == 0 and EY[i] < 0) or (wt and ly == hy - 1 and EY[i] > 0)
                    continue
                if EX[i] < 0 and xl and lx == 0:
                    xt += nx
                if EX[i] > 0 and xr and lx == hx - 1:
                    xt -= nx
                if EY[i] < 0 and yb and ly == 0:
                    rt += nyf
                if EY[i] > 0 and yt and ly == hy - 1:
                    rt -= nyf
                assert 0 <= xt < nx and 0 <= rt < nyf
    # hand-over: neighbour tiles are the tiles of the neighbour nodes
    for d in (-1, 1):
        t = neighbour_tile(x0, d, tx, nx, True)
        assert t == wrap(x0 - 1 if d < 0 else x0 + tx, nx) // tx
        assert 0 <= g.ring_index(R_L, t, 0, nyf - 1, 0) < g.ring_elems(R_L)
        if (d < 0 and wb) or (d > 0 and wt):
            continue                      # no ring row across a wall
        t = neighbour_tile(y0, d, ty, nyf, True)
        assert t == wrap(y0 - 1 if d < 0 else y0 + ty, nyf) // ty
        assert 0 <= g.ring_index(R_T, 0, t, 0, nx - 1) < g.ring_elems(R_T)


def _lattices():
    fixed = [(96, 96, False), (128, 48, False), (96, 50, True), (224, 165, False),
             (160, 100, False), (100, 100, False), (99, 54, True), (134, 77, True),
             (196, 52, False), (192, 98, True), (1000, 1000, False), (500, 200, True),
             (70, 21, False), (5, 5, False), (131, 37, True), (4096, 4096, False),
             # walls: top wall tiles 1 (general), 2, 3, 4 and 16 rows high;
             # two tile rows
             (128, 51, True), (128, 52, True), (128, 53, True), (128, 38, True),
             (192, 66, True), (96, 22, True), (96, 38, True), (512, 256, True)]
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
    checked = wall_tiles = ragged_tops = ragged_x = ragged_y = 0
    for nx, ny, walls in _lattices():
        if nx * ny > 520 * 260:
            continue
        g = Geometry(nx, ny, walls)
        for tx, ty in SHAPES:
            kinds = tile_kinds(nx, ny, walls, (tx, ty), True)
            nty = kinds.shape[0]
            for by, bx in zip(*np.nonzero(kinds)):
                check_tile(g, tx, ty, int(bx), int(by), kinds[by, bx] == 1)
                checked += 1
                if walls and by in (0, nty - 1):
                    wall_tiles += 1
                    ragged_tops += by == nty - 1 and g.nyf % ty != 0
                ragged_x += (bx + 1) * tx > nx
                ragged_y += not walls and (by + 1) * ty > g.nyf
    assert checked > 2000 and wall_tiles > 300 and ragged_tops > 100
    assert ragged_x > 100 and ragged_y > 100, (ragged_x, ragged_y)


def test_small_shared_memory_launch_has_no_general_tile():
    # launch_shape asks only for the TMA path's shared memory when x is
    # periodic seams over full tiles and y either the same or walls with a
    # top tile full or at least 4 rows high
    seen = 0
    for nx, ny, walls in _lattices():
        for tx, ty in SHAPES:
            g = Geometry(nx, ny, walls)
            nfy, ry = g.nyf // ty, g.nyf % ty
            x_ok = nx % tx == 0 and nx // tx >= 3
            if walls:
                y_ok = (nfy >= 2 or (nfy == 1 and ry >= 4)) and (ry == 0 or ry >= 4)
            else:
                y_ok = ry == 0 and nfy >= 3
            if x_ok and y_ok:
                assert tile_kinds(nx, ny, walls, (tx, ty), True).min() >= 1
                seen += walls
    assert seen > 0


def test_tile_kinds_rejects_bad_arguments():
    with pytest.raises(LbmError):
        tile_kinds(64, 64, False, (48, 16))
    with pytest.raises(LbmError):
        tile_kinds(4, 64, False, (32, 32))
    lib = _lib.load()
    short = np.zeros(3, dtype=np.int32)
    assert lib.lbm_tile_kinds(128, 128, 0, 32, 32, 1, short.ctypes.data, short.size) != 0
