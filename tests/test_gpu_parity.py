"""Parity of the CUDA step with the FP64 CPU oracle, through the C ABI.

FP64: one step to 1e-13 and 1000 steps to 1e-10 relative per field (rho, v,
mu and all nine populations), on sizes that span several 64 x 16 tiles with
ragged last tiles, one-node-wide last tiles, the minimum sizes, periodic and
walled geometries and every EOS.  Full size (4096 x 4096, the throughput
workload): one step of sampled nodes against the oracle run on a periodic
patch around each sample (a node's next state depends on its 7 x 7
neighbourhood only), and exact mass conservation.
"""
import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_1611_00907_gb300 import LbmError, Simulation, inputs, tile_kinds

pytestmark = pytest.mark.gpu

# (kind, a, b, Tr, kappa, tau): the paper's parameter sets (Sec. III, V);
# kappa scaled to the EOS's density range so runs stay stable.
EOS_CASES = {
    "cs": ("cs", 1.0, 4.0, 0.85, 0.5, 1.0),
    "vdw": ("vdw", 9 / 49, 2 / 21, 0.85, 0.01, 1.0),
    "pr": ("pr", 2 / 49, 2 / 21, 0.85, 0.01, 1.3),
    "rks": ("rks", 2 / 49, 2 / 21, 0.8, 0.01, 1.3),
}


def _setup(case, nx, ny, walls, mu_shift=0.01, precision="f64", rho_ref=0.0,
           geometry="drop", top_mode=0, mu_top=0.0):
    kind, a, b, Tr, kappa, tau = EOS_CASES[case]
    e = thermo.make_eos(kind, a, b, 1.0, Tr, 0.344)
    rv, rl, mc, _ = thermo.maxwell(e)
    width = 4.0 if kind == "cs" else 2.0
    r = max(2.0, min(nx, ny) / 4)
    if walls:
        rho = inputs.wall_drop(nx, ny, r, rl, rv, width)
    elif geometry == "slab":
        rho = inputs.slab(nx, ny, rl, rv, width)
    else:
        rho = inputs.drop(nx, ny, r, rl, rv, width)
    sim = Simulation(nx, ny, kind, a, b, 1.0, Tr, omega=0.344, tau=tau,
                     kappa=kappa, walls=walls, precision=precision,
                     rho_ref=rho_ref, mu_bottom=mc + mu_shift,
                     top_mode=top_mode, mu_top=mu_top)
    ref = oracle.Lattice(nx, ny, e, tau, kappa, walls=walls,
                         mu_bottom=mc + mu_shift, top_mode=top_mode,
                         mu_top=mu_top)
    return sim, ref, rho


def _rel(got, want):
    scale = np.abs(want).max()
    return np.abs(got - want).max() / (scale if scale > 0 else 1.0)


def _compare(sim, ref, tol):
    g, w = sim.moments(), ref.moments()
    for k in ("rho", "mu", "vx", "vy"):
        assert _rel(g[k], w[k]) < tol, (k, _rel(g[k], w[k]))
    fg, fw = sim.populations(), ref.f
    for i in range(9):
        assert _rel(fg[i], fw[i]) < tol, ("f", i, _rel(fg[i], fw[i]))


SIZES = [(9, 7), (70, 21), (131, 37), (65, 17), (5, 5), (64, 16), (200, 9)]


@pytest.mark.parametrize("case", list(EOS_CASES))
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("size", SIZES)
def test_one_step_fp64(case, walls, size):
    nx, ny = size
    if walls and ny < 7:
        ny = 7
    sim, ref, rho = _setup(case, nx, ny, walls)
    with sim:
        sim.init(rho)
        ref.init_equilibrium(rho)
        _compare(sim, ref, 1e-13)
        sim.step(1)
        ref.step(1)
        _compare(sim, ref, 1e-13)
        sim.step(1)      # odd parity of the in-place pattern
        ref.step(1)
        _compare(sim, ref, 1e-13)


@pytest.mark.parametrize("case,walls,size", [
    ("cs", False, (64, 64)),      # the 64 x 64 slab/drop configuration
    ("cs", True, (131, 37)),
    ("rks", True, (97, 40)),
    ("pr", False, (70, 33)),
    ("vdw", True, (65, 18)),
])
def test_1000_steps_fp64(case, walls, size, oracle_threads):
    nx, ny = size
    sim, ref, rho = _setup(case, nx, ny, walls)
    with sim:
        sim.init(rho).step(1000)
        ref.init_equilibrium(rho).step(1000)
        _compare(sim, ref, 1e-10)


@pytest.mark.parametrize("tile", [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)])
# FP32: mu = psi'(rho) - kappa lap(rho) cancels terms ~100x its size, so
# eps_32 ~ 6e-8 becomes ~1e-5 relative per evaluation and grows over steps.
@pytest.mark.parametrize("precision,tol,steps", [("f64", 1e-12, 60),
                                                 ("f32", 1e-4, 60),
                                                 ("f32_offset", 1e-4, 60)])
def test_every_tile_shape(tile, precision, tol, steps):
    # 230 x 140 with walls: interior tiles (TMA paths), ragged edge tiles,
    # both parities
    ref_rho = 0.5 * sum(_coexistence("cs")) if precision == "f32_offset" else 0.0
    sim, ref, rho = _setup("cs", 230, 140, True, precision=precision,
                           rho_ref=ref_rho)
    with sim:
        sim.set_tile(*tile)
        assert sim.tile == tile
        sim.init(rho).step(steps)
        ref.init_equilibrium(rho).step(steps)
        g, w = sim.moments(), ref.moments()
        for k in ("rho", "mu", "vx", "vy"):
            assert _rel(g[k], w[k]) < tol, (k, _rel(g[k], w[k]))


@pytest.mark.parametrize("tile", [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)])
@pytest.mark.parametrize("walls,size", [(True, (260, 200)), (False, (224, 165))])
def test_interior_tiles_many_steps_fp64(tile, walls, size, oracle_threads):
    # lattices with several rows and columns of interior tiles, 400 steps
    nx, ny = size
    sim, ref, rho = _setup("cs", nx, ny, walls)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho).step(400)
        ref.init_equilibrium(rho).step(400)
        _compare(sim, ref, 1e-11)


def _coexistence(case):
    kind, a, b, Tr, _, _ = EOS_CASES[case]
    rv, rl, _, _ = thermo.maxwell(thermo.make_eos(kind, a, b, 1.0, Tr, 0.344))
    return rv, rl


# FP32 interior tiles take the TMA path (32-wide tiles) or the path with two
# nodes per lane on packed FP32 pairs (64-wide tiles), edge tiles the general
# path.  Two steps (both parities of the in-place pattern) against the
# oracle: the density and populations carry FP32 rounding of a few ulp per
# step, mu (~100x cancellation) and the velocity (small against the
# populations it is summed from) proportionally more.
# Seam tiles: full tiles whose halo wraps around a periodic edge (at least
# three tiles across that edge) take the 32-wide TMA path, with the wrapped
# parts of the halo, the partial sums and the odd-step populations loaded
# element by element and the writes across the edge wrapped.
SEAM_CASES = [
    ((32, 32), False, (96, 96)),    # 3 x 3 tiles: all but the centre wrap
    ((32, 16), False, (128, 48)),   # corners, left/right and bottom/top seams
    ((32, 24), False, (96, 72)),
    ((32, 16), True, (96, 50)),     # walls: left and right seams only
    ((32, 32), False, (160, 100)),  # ragged rows: left and right seams only
]


@pytest.mark.parametrize("tile,walls,size", SEAM_CASES)
def test_seam_tiles_fp64(tile, walls, size, oracle_threads):
    nx, ny = size
    sim, ref, rho = _setup("cs", nx, ny, walls)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho)
        ref.init_equilibrium(rho)
        # both parities of the in-place pattern; the TMA path adds the
        # density hand-over in another order than the oracle, and near
        # coexistence mu (~2e-3 here) is the difference of terms ~50x its
        # size, so one last-bit density difference shows as ~1e-13 in mu
        for _ in range(2):
            sim.step(1)
            ref.step(1)
            _compare(sim, ref, 1e-12)
        sim.step(198)
        ref.step(198)
        _compare(sim, ref, 1e-11)


# A full tile whose right or top neighbour is the ragged last tile of its
# row or column takes the interior paths when that tile is at least 4 nodes
# wide (remainder 4 here; remainder 3 keeps the general path for both).
RAGGED_NEIGHBOUR_CASES = [
    ((32, 32), False, (100, 100)),   # remainders 4 and 4
    ((32, 16), True, (99, 54)),      # x remainder 3, 52 fluid rows: remainder 4
    ((32, 24), True, (134, 77)),     # remainders 6 and 3
]


@pytest.mark.parametrize("tile,walls,size", RAGGED_NEIGHBOUR_CASES)
def test_ragged_neighbour_tiles_fp64(tile, walls, size, oracle_threads):
    nx, ny = size
    sim, ref, rho = _setup("cs", nx, ny, walls)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho)
        ref.init_equilibrium(rho)
        for _ in range(2):      # both parities; tolerance as test_seam_tiles_fp64
            sim.step(1)
            ref.step(1)
            _compare(sim, ref, 1e-12)
        sim.step(198)
        ref.step(198)
        _compare(sim, ref, 1e-11)


# The ragged last tile of a periodic direction (at least 4 nodes) takes the
# 32-wide TMA path itself: its right and top edges, the wrap across them and
# the partial sums there sit at its own width and height, and the lanes and
# rows beyond them store nothing.
RAGGED_TMA_CASES = [
    ((32, 32), False, (100, 100)),   # remainders 4 and 4: the narrowest
    ((32, 16), False, (230, 140)),   # remainders 6 and 12
    ((32, 24), False, (133, 120)),   # x remainder 5, y full
    ((32, 32), False, (128, 115)),   # x full, y remainder 19
    ((32, 24), True, (134, 77)),     # walls: x remainder 6, top wall tile ragged
    ((32, 16), True, (230, 140)),
]


@pytest.mark.parametrize("tile,walls,size", RAGGED_TMA_CASES)
def test_ragged_last_tiles_take_tma_fp64(tile, walls, size, oracle_threads):
    nx, ny = size
    # the ragged last tile of every tile row (column) with TMA tiles is one
    # (a row under a top wall tile of fewer than 4 rows is general whole)
    kinds = np.asarray(tile_kinds(nx, ny, walls, tile))
    tx, ty = tile
    nyf = ny - 2 if walls else ny
    if nx % tx:
        rows = (kinds[:, :-1] != 0).any(axis=1)
        assert rows.sum() >= 2 and (kinds[rows, -1] == 1).all()
    if not walls and nyf % ty:
        cols = (kinds[:-1, :] != 0).any(axis=0)
        assert cols.sum() >= 2 and (kinds[-1, cols] == 1).all()
    sim, ref, rho = _setup("cs", nx, ny, walls)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho)
        ref.init_equilibrium(rho)
        for _ in range(2):      # both parities; tolerance as test_seam_tiles_fp64
            sim.step(1)
            ref.step(1)
            _compare(sim, ref, 1e-12)
        sim.step(198)
        ref.step(198)
        _compare(sim, ref, 1e-11)


# Lattices with ragged last tiles in FP32 arithmetic: on the 32-wide path
# they take the TMA path (odd widths included); on the two-nodes-per-lane
# path they stay general beside TMA neighbours.  Against the oracle
# (tolerance as test_every_tile_shape) and against the same lattice on the
# general path.
RAGGED_FP32_CASES = [
    ((32, 24), False, (133, 120)),   # x remainder 5
    ((32, 16), False, (229, 141)),   # remainders 5 and 13
    ((32, 16), True, (197, 66)),     # walls: x remainder 5
    ((64, 16), False, (229, 141)),   # remainders 37 and 13: general ragged tiles
    ((64, 32), True, (197, 66)),     # walls, x remainder 5
]


@pytest.mark.parametrize("tile,walls,size", RAGGED_FP32_CASES)
@pytest.mark.parametrize("precision", ["f32", "f32_offset"])
def test_ragged_lattices_fp32(tile, walls, size, precision, monkeypatch):
    nx, ny = size
    kinds = np.asarray(tile_kinds(nx, ny, walls, tile))
    if tile[0] == 32:
        assert (kinds[1:-1, -1] == 1).all() and kinds.min() >= 1
    ref_rho = 0.5 * sum(_coexistence("cs")) if precision == "f32_offset" else 0.0
    runs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("CPLBM_NO_TMA", "1")
        sim, ref, rho = _setup("cs", nx, ny, walls, precision=precision,
                               rho_ref=ref_rho)
        with sim:
            sim.set_tile(*tile)
            sim.init(rho).step(61)
            runs.append(sim.moments())
    ref.init_equilibrium(rho).step(61)
    want = ref.moments()
    for k in ("rho", "mu", "vx", "vy"):
        assert _rel(runs[0][k], want[k]) < 1e-4, (k, _rel(runs[0][k], want[k]))
        assert _rel(runs[0][k], runs[1][k]) < 1e-4, (k, _rel(runs[0][k], runs[1][k]))


@pytest.mark.parametrize("tile,walls,size", SEAM_CASES[:2] + SEAM_CASES[3:4] + [
    ((64, 16), False, (192, 48)),   # two nodes per lane: 3 x 3 tiles
    ((64, 32), True, (192, 98)),
    ((64, 16), False, (196, 52)),   # ragged right and top neighbours (remainders 4)
    ((32, 32), True, (100, 102)),
])
@pytest.mark.parametrize("precision", ["f32", "f32_offset"])
def test_seam_tiles_fp32(tile, walls, size, precision, monkeypatch):
    # seam and ragged-neighbour tiles, against the oracle (tolerance as
    # test_every_tile_shape) and against the same lattice with every tile on
    # the general path
    nx, ny = size
    ref_rho = 0.5 * sum(_coexistence("cs")) if precision == "f32_offset" else 0.0
    runs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("CPLBM_NO_TMA", "1")
        sim, ref, rho = _setup("cs", nx, ny, walls, precision=precision,
                               rho_ref=ref_rho)
        with sim:
            sim.set_tile(*tile)
            sim.init(rho).step(60)
            runs.append(sim.moments())
    ref.init_equilibrium(rho).step(60)
    want = ref.moments()
    for k in ("rho", "mu", "vx", "vy"):
        assert _rel(runs[0][k], want[k]) < 1e-4, (k, _rel(runs[0][k], want[k]))
        assert _rel(runs[0][k], runs[1][k]) < 1e-4, (k, _rel(runs[0][k], runs[1][k]))


# Wall tiles: with walls the bottom and top tile rows take the TMA paths as
# edge tiles (the top one may be ragged, down to one fluid row): the Eq. 28
# density row after the partial sums, the surface chemical potential rows,
# odd-step reads and writes through the node's own slots at the wall, the
# bounce-back in the register hand-over, and no partial sums across a wall.
WALL_CASES = [
    ((32, 32), (128, 66)),    # 64 fluid rows: full top tile
    ((32, 16), (128, 51)),    # one-row top wall tile: general path beside TMA tiles
    ((32, 16), (128, 52)),    # two rows
    ((32, 24), (96, 53)),     # three rows (the tile below it general)
    ((32, 32), (160, 38)),    # two tile rows, top 4 rows high
    ((32, 16), (100, 60)),    # ragged last column (general) beside wall tiles
]


@pytest.mark.parametrize("tile,size", WALL_CASES)
@pytest.mark.parametrize("case,top_mode", [("cs", 0), ("cs", 1), ("rks", 0)])
def test_wall_tiles_fp64(tile, size, case, top_mode, oracle_threads):
    nx, ny = size
    kinds = np.asarray(tile_kinds(nx, ny, True, tile))
    assert (kinds[[0, -1]] > 0).sum() >= 4     # wall rows on the TMA paths
    sim, ref, rho = _setup(case, nx, ny, True, top_mode=top_mode,
                           mu_top=0.004 if case == "cs" else -0.05)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho)
        ref.init_equilibrium(rho)
        for _ in range(2):      # both parities; tolerance as test_seam_tiles_fp64
            sim.step(1)
            ref.step(1)
            _compare(sim, ref, 1e-12)
        sim.step(198)
        ref.step(198)
        _compare(sim, ref, 1e-11)


@pytest.mark.parametrize("tile,size", WALL_CASES[:3] + [
    ((64, 16), (192, 66)),    # two nodes per lane: full top tile
    ((64, 16), (192, 53)),    # three-row top tile
    ((64, 32), (192, 100)),   # two-row top tile
    ((64, 16), (256, 39)),    # two tile rows, every tile on the TMA path
])
@pytest.mark.parametrize("precision", ["f32", "f32_offset", "f16_offset"])
def test_wall_tiles_reduced_precision(tile, size, precision, monkeypatch):
    # against the oracle and against the same lattice with every tile on the
    # general path (FP16 storage: its rounding of ~5e-4 per population
    # shows in the density at ~1e-3 after 60 steps; rho only)
    nx, ny = size
    ref_rho = 0.5 * sum(_coexistence("cs")) if precision != "f32" else 0.0
    runs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("CPLBM_NO_TMA", "1")
        sim, ref, rho = _setup("cs", nx, ny, True, precision=precision,
                               rho_ref=ref_rho)
        with sim:
            sim.set_tile(*tile)
            sim.init(rho).step(60)
            runs.append(sim.moments())
    ref.init_equilibrium(rho).step(60)
    want = ref.moments()
    keys, tol = (("rho",), 2e-3) if precision == "f16_offset" else (
        ("rho", "mu", "vx", "vy"), 1e-4)
    for k in keys:
        assert _rel(runs[0][k], want[k]) < tol, (k, _rel(runs[0][k], want[k]))
        assert _rel(runs[0][k], runs[1][k]) < tol, (k, _rel(runs[0][k], runs[1][k]))


@pytest.mark.parametrize("case", list(EOS_CASES))
@pytest.mark.parametrize("precision", ["f32", "f32_offset"])
@pytest.mark.parametrize("tile,walls", [((64, 16), False), ((64, 32), True),
                                        ((32, 32), False)])
def test_fp32_paths_two_steps(case, precision, tile, walls):
    ref_rho = 0.5 * sum(_coexistence(case)) if precision == "f32_offset" else 0.0
    # 330 x 200: three columns of interior 64-wide tiles, ragged last tiles
    sim, ref, rho = _setup(case, 330, 200, walls, precision=precision,
                           rho_ref=ref_rho)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho).step(2)
        ref.init_equilibrium(rho).step(2)
        g, w = sim.moments(), ref.moments()
        assert _rel(g["rho"], w["rho"]) < 2e-6
        assert _rel(g["mu"], w["mu"]) < 1e-4
        for k in ("vx", "vy"):
            assert _rel(g[k], w[k]) < 1e-3, (k, _rel(g[k], w[k]))
        fg = sim.populations()
        for i in range(9):
            assert _rel(fg[i], ref.f[i]) < 5e-6, (i, _rel(fg[i], ref.f[i]))


@pytest.mark.parametrize("tile", [(64, 16), (32, 32)])
def test_fp32_step_is_deterministic(tile):
    # no atomics on the data path: two runs agree bit for bit
    out = []
    for _ in range(2):
        sim, _, rho = _setup("cs", 330, 200, False, precision="f32")
        with sim:
            sim.set_tile(*tile)
            sim.init(rho).step(31)
            out.append(sim.populations())
    assert np.array_equal(out[0], out[1])


def test_tile_switch_mid_run():
    sim, ref, rho = _setup("cs", 200, 90, False)
    with sim:
        sim.set_tile(64, 16)
        sim.init(rho).step(31)
        sim.set_tile(32, 24)        # re-splits the current density
        sim.step(30)
        ref.init_equilibrium(rho).step(61)
        _compare(sim, ref, 1e-12)
        with pytest.raises(LbmError):
            sim.set_tile(48, 16)


def test_autotune_keeps_the_state():
    sim, ref, rho = _setup("cs", 200, 90, True)
    with sim:
        sim.init(rho).step(7)
        before = sim.populations()
        shape = sim.autotune(4)
        assert shape == sim.tile
        assert sim.step_count == 7
        assert np.array_equal(sim.populations(), before)
        sim.step(13)
        ref.init_equilibrium(rho).step(20)
        _compare(sim, ref, 1e-12)


def test_top_wall_with_given_value():
    sim, ref, rho = _setup("cs", 70, 21, True, top_mode=1, mu_top=0.004)
    with sim:
        sim.init(rho).step(25)
        ref.init_equilibrium(rho).step(25)
        _compare(sim, ref, 1e-12)


def test_initial_velocity_field():
    nx, ny = 70, 21
    sim, ref, rho = _setup("cs", nx, ny, False)
    rng = np.random.default_rng(5)
    ux = 0.02 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.02 * rng.uniform(-1, 1, (ny, nx))
    with sim:
        sim.init(rho, ux, uy).step(30)
        ref.init_equilibrium(rho, ux, uy).step(30)
        _compare(sim, ref, 1e-12)


def test_device_tensors_in_and_out():
    torch = pytest.importorskip("torch")
    nx, ny = 70, 21
    sim, ref, rho = _setup("cs", nx, ny, False)
    with sim:
        sim.init(torch.tensor(rho, device="cuda")).step(5)
        ref.init_equilibrium(rho).step(5)
        got = sim.moments(device=True)
        assert got["rho"].is_cuda
        assert _rel(got["rho"].cpu().numpy(), ref.moments()["rho"]) < 1e-13


def test_mass_conservation_and_reduce():
    sim, ref, rho = _setup("cs", 131, 37, True)
    with sim:
        sim.init(rho)
        m0, px, py, d0 = sim.reduce()
        assert m0 == pytest.approx(ref.init_equilibrium(rho).density()[1:-1]
                                   .sum(), rel=1e-14)
        assert d0 == 0.0
        sim.step(500)
        m1, _, _, d1 = sim.reduce()
        assert abs(m1 - m0) / m0 < 1e-13
        assert d1 > 0.0
        _, _, _, d2 = sim.reduce()
        assert d2 == 0.0           # no step since the last call


def _oracle_reduction(ref, rho_prev):
    """(mass, rho v_x, rho v_y, max |rho - rho_prev|) over the fluid nodes of
    the oracle's state, with v = u + F/(2 rho) as the oracle reports it, and
    the sums of magnitudes that bound each sum's rounding."""
    m = ref.moments()
    fl = ref.fluid_rows()
    r, px, py = m["rho"][fl], (m["rho"] * m["vx"])[fl], (m["rho"] * m["vy"])[fl]
    want = (r.sum(), px.sum(), py.sum(), np.abs(r - rho_prev[fl]).max())
    scale = (np.abs(r).sum(), np.abs(px).sum(), np.abs(py).sum())
    return want, scale, m["rho"]


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_reduction_matches_oracle(walls, precision, tol):
    """The FP64 reductions of lbm_reduce (mass, momentum sum rho v with the
    reported velocity of Sec. II, and the convergence measure max |rho_t -
    rho_t'| since the previous call) against the same quantities of the
    oracle's state, from a moving drop so that momentum is not round-off."""
    sim, ref, rho = _setup("cs", 131, 37, walls, precision=precision)
    ny, nx = rho.shape
    ux, uy = np.full((ny, nx), 0.02), np.full((ny, nx), -0.01)
    if walls:
        uy[:] = 0.0
    with sim:
        sim.init(rho, ux, uy)
        ref.init_equilibrium(rho, ux, uy)
        prev = ref.moments()["rho"]
        got = sim.reduce()
        want, scale, _ = _oracle_reduction(ref, prev)
        t0 = 1e-13 if precision == "f64" else tol   # FP32 stores a rounded state
        for k in range(3):
            assert abs(got[k] - want[k]) <= t0 * scale[k], (k, got, want)
        assert got[3] == 0.0
        for n in (1, 40, 161):
            sim.step(n)
            ref.step(n)
            got = sim.reduce()
            want, scale, prev = _oracle_reduction(ref, prev)
            for k in range(3):
                assert abs(got[k] - want[k]) <= tol * scale[k], (n, k, got, want)
            assert want[3] > 1e-6
            # FP32 densities carry their own storage rounding: absolute bound
            dtol = 1e-12 * want[3] if precision == "f64" else 3e-5 * rho.max()
            assert abs(got[3] - want[3]) <= dtol, (n, got[3], want[3])


def test_diverging_lattice_reports_numeric_error():
    """A lattice the scheme cannot hold (van der Waals with kappa = 0.5: its
    density range makes the square-gradient term linearly unstable; the
    oracle goes non-finite within three steps) makes lbm_reduce return
    LBM_ERR_NUMERIC with the count of bad nodes, instead of a value.  The
    failure is the run's own arithmetic; no index depends on a density, so
    nothing is read or written out of place."""
    import ctypes as C
    from paper_1611_00907_gb300 import _lib
    kind, a, b, Tr = "vdw", 9 / 49, 2 / 21, 0.85
    e = thermo.make_eos(kind, a, b, 1.0, Tr)
    rv, rl, _, _ = thermo.maxwell(e)
    nx, ny = 70, 21
    rho = inputs.drop(nx, ny, 6, rl, rv, 2.0)
    ref = oracle.Lattice(nx, ny, e, 1.0, 0.5).init_equilibrium(rho).step(20)
    assert not np.isfinite(ref.density()).all()
    with Simulation(nx, ny, kind, a, b, 1.0, Tr, tau=1.0, kappa=0.5) as sim:
        sim.init(rho)
        sim.reduce()                       # finite initial state: OK
        sim.step(20)
        out = (C.c_double * 4)()
        st = sim._lib.lbm_reduce(sim._ctx, out)
        assert st == _lib.LBM_ERR_NUMERIC
        assert b"non-finite" in sim._lib.lbm_last_error(sim._ctx)
        with pytest.raises(LbmError) as ei:
            sim.reduce()
        assert ei.value.status == _lib.LBM_ERR_NUMERIC
        # the context stays usable: a uniform state runs and reduces again
        flat = np.full((ny, nx), rv)
        sim.init(flat).step(2)
        assert sim.reduce()[0] == pytest.approx(flat.sum(), rel=1e-13)


def test_checkpoint_resume_is_bitwise():
    sim, _, rho = _setup("cs", 131, 37, True)
    with sim:
        sim.init(rho).step(37)     # odd step count
        state = sim.get_state()
        sim.step(13)
        a = sim.populations()
    sim2, _, _ = _setup("cs", 131, 37, True)
    with sim2:
        sim2.set_state(state)
        assert sim2.step_count == 37
        sim2.step(13)
        b = sim2.populations()
    assert np.array_equal(a, b)


def test_zero_steps_and_uniform_fixed_point():
    nx, ny = 70, 21
    sim, _, _ = _setup("cs", nx, ny, False)
    with sim:
        rho = np.full((ny, nx), 0.2)
        sim.init(rho, np.full((ny, nx), 0.03), np.full((ny, nx), -0.01))
        f0 = sim.populations()
        sim.step(0)
        assert np.array_equal(sim.populations(), f0)
        sim.step(20)
        assert np.abs(sim.populations() - f0).max() < 1e-15


def test_invalid_init_is_rejected_without_fault():
    sim, _, rho = _setup("cs", 70, 21, False)
    with sim:
        bad = rho.copy()
        bad[3, 4] = 1.5            # beyond the CS pole 4/b = 1
        with pytest.raises(LbmError) as ei:
            sim.init(bad)
        assert "density" in str(ei.value)
        with pytest.raises(LbmError):
            sim.step(1)            # not initialised
        sim.init(rho).step(2)      # the context stays usable


def _patch_step(e, tau, kappa, fpatch):
    """One oracle step on a periodic patch; returns the centre node."""
    n = fpatch.shape[1]
    L = oracle.Lattice(n, n, e, tau, kappa)
    L.f = np.ascontiguousarray(fpatch)
    L.step(1)
    return L.f[:, n // 2, n // 2]


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_full_size_sampled_one_step(precision, tol):
    # The throughput workload: 4096 x 4096 Carnahan-Starling spinodal
    # decomposition at T_r = 0.85 from rho_c (1 + 0.01 xi).
    n = 4096
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85)
    _, rc = thermo.critical_point("cs", 1.0, 4.0)
    rho = inputs.spinodal_noise(n, n, rc, 0.01, seed=1)
    sim = Simulation(n, n, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0, kappa=0.5,
                     precision=precision)
    with sim:
        sim.init(rho).step(3)
        f0 = sim.populations()
        m0 = sim.reduce()[0]
        sim.step(1)
        f1 = sim.populations()
        rng = np.random.default_rng(7)
        pts = [(0, 0), (n - 1, n - 1), (63, 15), (64, 16), (4095, 16),
               (2047, 2048)] + [tuple(p) for p in rng.integers(0, n, (20, 2))]
        h = 6
        for (y, x) in pts:
            ys = np.arange(y - h, y + h + 1) % n
            xs = np.arange(x - h, x + h + 1) % n
            patch = f0[:, ys][:, :, xs]
            want = _patch_step(e, 1.0, 0.5, patch)
            got = f1[:, y, x]
            assert np.abs(got - want).max() / np.abs(want).max() < tol, (y, x)
        sim.step(96)
        m1 = sim.reduce()[0]
        assert abs(m1 - m0) / m0 < (1e-13 if precision == "f64" else 1e-5)


@pytest.mark.parametrize("tile", [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)])
@pytest.mark.parametrize("size", [(330, 200), (192, 96)])  # 192 x 96: seam tiles
def test_fp16_storage_tma_path(tile, size, monkeypatch):
    # FP16 storage: interior tiles stage the half populations by TMA; the
    # same lattice with every tile on the general path (no tensor maps)
    # does the same FP32 arithmetic on the same half inputs.  The two paths
    # sum the density hand-over in different orders, and an FP32 last-bit
    # difference flips the half rounding of a stored g_i = f_i - w_i rho_ref
    # now and then: one such flip moves rho by ~3e-5 of its largest value.
    rv, rl = _coexistence("cs")
    runs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("CPLBM_NO_TMA", "1")
        sim, ref, rho = _setup("cs", *size, False, precision="f16_offset",
                               rho_ref=0.5 * (rv + rl))
        with sim:
            sim.set_tile(*tile)
            sim.init(rho).step(21)
            runs.append(sim.moments())
    ref.init_equilibrium(rho).step(21)
    want = ref.moments()
    # mu = psi'(rho) - kappa lap(rho) cancels terms ~100x its size, so the
    # same density differences show ~100x larger in mu
    for k, tol in (("rho", 5e-4), ("mu", 3e-2)):
        assert _rel(runs[0][k], runs[1][k]) < tol, (k, _rel(runs[0][k], runs[1][k]))
    # half populations (eps 4.9e-4 on g_i) against the FP64 oracle
    for run in runs:
        assert _rel(run["rho"], want["rho"]) < 2e-3


@pytest.mark.parametrize("tile", [(32, 16), (32, 32), (64, 16), (64, 32)])
# 192 x 96: seam tiles; 330 x 200 and 229 x 141: ragged last tiles (even and
# odd widths; TMA on 32-wide tiles, general on 64-wide ones)
@pytest.mark.parametrize("size", [(330, 200), (192, 96), (229, 141)])
@pytest.mark.parametrize("steps", [20, 21])                 # both in-place parities
def test_fp16_storage_against_the_oracle(tile, size, steps):
    """Density, chemical potential and reported velocity of the FP16-offset
    storage against the FP64 oracle, within the bounds that follow from the
    half-precision unit roundoff (derived in tests/fp16_bounds.py)."""
    from fp16_bounds import check, run_with_bounds
    kind, a, b, Tr, kappa, tau = EOS_CASES["cs"]
    e = thermo.make_eos(kind, a, b, 1.0, Tr, 0.344)
    rv, rl = _coexistence("cs")
    rho_ref = 0.5 * (rv + rl)
    sim, ref, rho = _setup("cs", *size, False, precision="f16_offset",
                           rho_ref=rho_ref)
    with sim:
        sim.set_tile(*tile)
        sim.init(rho).step(steps)
        got = sim.moments()
    want, bounds = run_with_bounds(ref, rho, steps, rho_ref, e, kappa)
    check(got, want, bounds, (tile, size, steps))


def test_moments_subset_into_caller_buffers():
    sim, ref, rho = _setup("cs", 70, 21, True)
    with sim:
        sim.init(rho).step(3)
        full = sim.moments()
        buf = np.zeros((21, 70))
        part = sim.moments(fields=("rho", "mu"), out={"rho": buf})
        assert set(part) == {"rho", "mu"} and part["rho"] is buf
        assert np.array_equal(buf, full["rho"]) and np.array_equal(part["mu"], full["mu"])
        with pytest.raises(ValueError):
            sim.moments(fields=("rho",), out={"rho": np.zeros((21, 70), np.float32)})


@pytest.mark.parametrize("own_stream", [False, True])
def test_step_graphs_follow_every_change(own_stream):
    """lbm_step replays blocks of 16 steps from a captured CUDA graph whose
    kernels hold the lattice's parameters: a change of tile shape, wall
    chemical potential or wait limit between calls must reach the replayed
    steps (the graph is captured again), on the legacy stream and on a
    stream of the caller's, and odd step counts fall back to single
    launches in between."""
    import torch
    nx, ny = 192, 66
    kind, a, b, Tr, kappa, tau = EOS_CASES["cs"]
    e = thermo.make_eos(kind, a, b, 1.0, Tr, 0.344)
    rv, rl, mc, _ = thermo.maxwell(e)
    rho = inputs.wall_drop(nx, ny, 24, rl, rv, 4.0)
    stream = torch.cuda.Stream() if own_stream else None
    sim = Simulation(nx, ny, kind, a, b, 1.0, Tr, omega=0.344, tau=tau, kappa=kappa,
                     walls=True, precision="f64", mu_bottom=mc + 0.01,
                     stream=stream.cuda_stream if stream else None)
    ref = oracle.Lattice(nx, ny, e, tau, kappa, walls=True, mu_bottom=mc + 0.01)
    lib = _lib_module().load()
    with sim:
        sim.init(rho)
        ref.init_equilibrium(rho)
        sim.step(37)                      # graphs, then single launches
        ref.step(37)
        sim.set_tile(64, 32)
        sim.step(33)                      # one single launch, then graphs
        ref.step(33)
        sim.set_wall_mu(mc - 0.02)
        ref.mu_bottom = mc - 0.02
        sim.step(32)
        ref.step(32)
        assert lib.lbm_test_set_wait_cycles(sim._ctx, 1 << 40) == 0
        sim.step(16)
        ref.step(16)
        _compare(sim, ref, 1e-11)


def test_steps_inside_a_callers_graph_capture():
    """A caller capturing lbm_step into its own CUDA graph gets every step
    in it (the library does not capture a graph of its own meanwhile)."""
    import torch
    sim, ref, rho = _setup("cs", 128, 64, False)
    stream = torch.cuda.Stream()
    sim.close()
    kind, a, b, Tr, kappa, tau = EOS_CASES["cs"]
    sim = Simulation(128, 64, kind, a, b, 1.0, Tr, omega=0.344, tau=tau, kappa=kappa,
                     precision="f64", stream=stream.cuda_stream)
    with sim:
        sim.init(rho).step(2)             # kernel attributes set outside the capture
        sim.init(rho)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sim.step(32)                  # captured into g: 32 kernel launches
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        ref.init_equilibrium(rho).step(3 * 32)
        # the capture itself advanced the lattice's step count by 32 without
        # running anything: the replays did the stepping
        _compare(sim, ref, 1e-11)


def _lib_module():
    from paper_1611_00907_gb300 import _lib
    return _lib
