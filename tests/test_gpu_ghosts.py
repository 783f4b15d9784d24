"""Wall ghosts of the fused D2Q9 kernels on tiles one or two cells wide or
tall.  The ghost cells beyond a wall are extrapolated (quadratically along
the wall normal, Sec. 2.3 with the stencil of eq. flux_DS) from cells staged
in the same tile; for a tile one or two cells across those cells lie in the
tile's halo.  Forced tile heights put one- and two-row tiles against the
north wall, and widths 33, 34, 35 and 65 put one- to three-column tiles
against the east wall (width 3: one tile holding both x walls).

FP64 and double-word kernels against the oracle at the FP64 parity bar
(relative L-infinity 1e-12); the FP32 / BF16 deviation forms against the
oracle within bounds of their storage rounding (measured errors are ~1e-7
and ~1e-4 of max f; a wrong ghost gives errors of order 1e-2)."""
import functools

import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu

STEPS = 4
# (nx, ny, tile height): last tile row 1 or 2 cells tall, last tile column
# 1 to 3 cells wide
CASES = [(33, 13, 12), (34, 14, 12), (33, 17, 8), (65, 6, 5), (3, 5, 4), (35, 9, 4)]
BC = {
    "cavity": [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)],
    "xper_ydiffuse": [(P.PERIODIC, 0, 0), (P.PERIODIC, 0, 0), (P.DIFFUSE, 0, 0),
                      (P.DIFFUSE, 0.04, 0)],
    "xdiffuse_yper": [(P.DIFFUSE, 0, 0.03), (P.DIFFUSE, 0, 0), (P.PERIODIC, 0, 0),
                      (P.PERIODIC, 0, 0)],
}
TOL = {P.FP64: 1e-12, P.F64_DW: 1e-12, P.G_FP32: 2e-6, P.G_BF16: 2e-3}
FORMS = [P.FP64, P.F64_DW, P.G_FP32, P.G_BF16]


@functools.lru_cache(maxsize=None)
def oracle_case(nx, ny, bcname):
    xi, W, RT = OV.d2q9(1 / 3)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.002, 0.004, BC[bcname])
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=7 * nx + ny)
    return f0, O.t3s3_run(f0, o, STEPS)


@pytest.mark.parametrize("storage", FORMS, ids=["fp64", "dw", "fp32", "bf16"])
@pytest.mark.parametrize("bcname", list(BC))
@pytest.mark.parametrize("nx,ny,ty", CASES)
def test_narrow_wall_tiles(cuda, nx, ny, ty, bcname, storage):
    if (bcname == "xdiffuse_yper" and nx < 3) or (bcname == "xper_ydiffuse" and ny < 3):
        pytest.skip("walls need three cells across")
    f0, fo = oracle_case(nx, ny, bcname)
    xi, W, RT = PV.d2q9(1 / 3)
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.002, 0.004, BC[bcname], storage=storage)
    P.dugks_set_tile_height(g.ctx, ty)
    g.set_state(f0)
    g.step(STEPS)
    assert P.dugks_tile_height(g.ctx) == ty
    fg = g.state()
    assert g.check() == P.DUGKS_OK
    g.close()
    err = float(np.abs(fg - fo).max() / np.abs(fo).max())
    assert err <= TOL[storage], err
