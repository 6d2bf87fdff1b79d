"""Memory safety of the step and field kernels, by the bounds-checked debug
build (libcplbm_checked.so, CPLBM_CHECK_BOUNDS; the stand-in for a memory
checker): every global load, store and copy source of those kernels is
checked against the buffer it belongs to, and one outside it is skipped and
reported as LBM_ERR_CUDA by the next synchronising call.  Every precision,
tile shape, geometry (odd sizes, ragged tiles, periodic seams, walls) and
launch (single lattice, pressure-tensor force, both batch schedules) runs a
few steps of both in-place parities and reads everything back without a
report; FP64 cases match the oracle as the product build does.  A negative
control makes the checks treat a buffer as shorter than it is, so that
legitimate accesses are flagged: no access ever leaves its buffer.

The checked library is built on demand (a few minutes of nvcc) and loaded in
a child process (CPLBM_LIBRARY_VARIANT=checked)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TILES = [(32, 16), (32, 24), (32, 32), (64, 16), (64, 32)]
# (nx, ny, walls): odd and ragged sizes, seam tiles (three or more full
# tiles across), one-node-wide last tiles, walls with ragged top tiles,
# ragged last tiles of periodic directions on the 32-wide TMA path (230 x
# 140; 100 x 100: 4 nodes, the narrowest it takes; 229 x 141 and 197 x 66:
# odd widths)
SIZES = [(9, 7, False), (70, 21, False), (131, 37, False), (65, 17, False),
         (192, 96, False), (256, 128, False), (230, 140, False), (100, 100, False),
         (229, 141, False), (9, 9, True), (131, 37, True), (96, 50, True), (192, 66, True),
         (230, 140, True), (197, 66, True)]


def _child():
    import numpy as np

    import oracle
    from oracle import thermo
    from paper_1611_00907_gb300 import Batch, LbmError, Simulation, _lib, inputs
    assert os.path.basename(_lib.LIB_PATH) == "libcplbm_checked.so"
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.85, 0.344)
    rv, rl, mc, _ = thermo.maxwell(e)
    ref = 0.5 * (rv + rl)

    def field(nx, ny, walls):
        r = max(2.0, min(nx, ny) / 4)
        return (inputs.wall_drop(nx, ny, r, rl, rv, 4.0) if walls
                else inputs.drop(nx, ny, r, rl, rv, 4.0))

    def sim(nx, ny, walls, prec):
        return Simulation(nx, ny, "cs", 1.0, 4.0, 1.0, 0.85, tau=1.0, kappa=0.5,
                          walls=walls, precision=prec, rho_ref=ref,
                          mu_bottom=mc + 0.01)

    runs = 0
    for prec in ("f64", "f32", "f32_offset", "f16_offset"):
        for tile in TILES:
            for nx, ny, walls in SIZES:
                rho = field(nx, ny, walls)
                with sim(nx, ny, walls, prec) as s:
                    s.set_tile(*tile)
                    s.init(rho).step(3)
                    got = s.moments()          # raises on a bounds report
                    s.reduce()
                    s.populations()
                    s.set_state(s.get_state())
                    s.step(2)
                    s.moments()
                    if prec == "f64" and tile == (32, 32) and nx >= 131:
                        o = oracle.Lattice(nx, ny, e, 1.0, 0.5, walls=walls,
                                           mu_bottom=mc + 0.01)
                        o.init_equilibrium(rho).step(3)
                        want = o.moments()
                        for k in ("rho", "mu", "vx", "vy"):
                            err = np.abs(got[k] - want[k]).max() / np.abs(want[k]).max()
                            assert err < 1e-12, (nx, ny, walls, k, err)
                runs += 1
    # the pressure-tensor force (periodic lattices)
    for prec in ("f64", "f32"):
        for nx, ny in ((131, 37), (192, 96)):
            with sim(nx, ny, False, prec) as s:
                s.set_force_model("pressure_tensor")
                s.init(field(nx, ny, False)).step(3)
                s.moments()
                runs += 1
    # batches: a work list with general tiles, and one geometry (grid per lattice)
    mixed = [dict(nx=nx, ny=ny, walls=w, eos="cs", a=1.0, b=4.0, Tr=0.85, tau=1.0,
                  kappa=0.5, mu_bottom=mc + 0.01, rho_ref=ref) for nx, ny, w in SIZES]
    same = [dict(mixed[9], tau=t) for t in (0.9, 1.0, 1.2)]
    for specs in (mixed, same):
        for prec in ("f32", "f16_offset", "f64"):
            for tile in TILES:
                for sched in (0, 1, 3):
                    with Batch(specs, precision=prec) as b:
                        b.set_tile(*tile)
                        b.items_per_cta = sched
                        for k, sp in enumerate(specs):
                            b.init(k, field(sp["nx"], sp["ny"], sp["walls"]))
                        b.step(19)                 # a graph block and direct launches
                        for k in range(len(specs)):
                            b.moments(k)
                    runs += 1
    # negative control: the checks see a density buffer shorter than it is
    lib = _lib.load()
    with sim(131, 37, False, "f32") as s:
        s.init(field(131, 37, False))
        assert lib.lbm_test_shrink_bounds(s._ctx, 1000) == _lib.LBM_OK
        s.step(1)
        try:
            s.moments()
            caught = False
        except LbmError as err:
            caught = "outside its buffer" in str(err)
    print(json.dumps({"runs": runs, "negative_control_caught": caught}))


@pytest.mark.gpu
def test_no_access_leaves_its_buffer():
    subprocess.run([sys.executable, "-m", "paper_1611_00907_gb300._build", "--checked"],
                   cwd=ROOT, check=True, timeout=1800)
    env = dict(os.environ, CPLBM_LIBRARY_VARIANT="checked",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "child"], cwd=ROOT,
                         env=env, capture_output=True, text=True, timeout=1800)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["runs"] == 4 * len(TILES) * len(SIZES) + 4 + 2 * 3 * len(TILES) * 3
    assert out["negative_control_caught"]


if __name__ == "__main__" and sys.argv[1:] == ["child"]:
    _child()
