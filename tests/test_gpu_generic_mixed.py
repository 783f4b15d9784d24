"""Deviation-storage forms (DUGKS_G_FP32, DUGKS_G_BF16) on the generic
kernels -- Newton-Cotes velocity grids, and D2Q9 on the generic path
(DUGKS_PATH_GENERIC) -- against the FP64 oracle.

These forms store d = f - W_k rho0 in FP32 or BF16 and compute stencils,
face values and the equilibrium assembly in FP32.  The moment sums over the
velocities add blocks of 16 terms in FP32 and fold each block into a
Kahan-compensated FP32 sum, which is rounded to FP64; the splits of a sum
and the face moments built from the cell sums are added in FP64 and FP32
respectively.  They are not bit-for-bit; the bounds are on the relative
L-infinity state error max|f - f_oracle| / max|f_oracle|, the L2 velocity
error E(u) (Sec. 3.1 definition) and the relative mass drift, after the
stated number of steps, each a few times the value measured on GB300
(quoted in each test).  FP32 storage rounds d with relative error 2^-24,
BF16 with 2^-9; the face values are FP32 in both forms."""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu

FORMS = [P.G_FP32, P.G_BF16]
IDS = ["fp32", "bf16"]


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def E_u(u, v, uo, vo):
    return float(np.sqrt(((u - uo) ** 2 + (v - vo) ** 2).sum() / (uo ** 2 + vo ** 2).sum()))


def nc_case(walls, nv1, nx, ny, steps, storage, seed=3):
    """Newton-Cotes nv1 x nv1 grid, RT = 0.5, Kn = 1 (tau = Kn / sqrt(pi RT/2)),
    CFL 0.25, walls as in the rarefied workloads; from a near-equilibrium
    random state.  Returns (state error, E(u), mass drift)."""
    RT = 0.5
    uw = 0.16 * np.sqrt(5 / 3 * RT)
    bc = {"diffuse": [(P.DIFFUSE, 0, 0)] * 3 + [(P.DIFFUSE, uw, 0)],
          "couette": [(P.PERIODIC, 0, 0)] * 2 + [(P.DIFFUSE, -uw, 0), (P.DIFFUSE, uw, 0)],
          "mixed": [(P.BOUNCEBACK, 0, 0), (P.DIFFUSE, 0, 0), (P.DIFFUSE, 0, 0),
                    (P.BOUNCEBACK, uw, 0)],
          "periodic": [(P.PERIODIC, 0, 0)] * 4}[walls]
    tau = 1.0 / np.sqrt(np.pi * RT / 2)
    dt = 0.25 * (1 / nx) / (4 * np.sqrt(RT))
    pg, po = PV.newton_cotes(nv1, RT), OV.newton_cotes_2d(nv1, RT)
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, pg[0], pg[1], pg[2], tau, dt, bc, storage=storage)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], tau, dt, bc)
    f0 = WL.near_equilibrium_state(po[1], ny, nx, amp=0.1, seed=seed)
    g.set_state(f0)
    g.step(steps)
    fg = g.state()
    _, u, v = g.moments()
    g.close()
    fo = O.t3s3_run(f0, o, steps)
    _, uo, vo = O.velocity(fo, o)
    out = rel_linf(fg, fo), E_u(u, v, uo, vo), abs(fg.sum() - fo.sum()) / fo.sum()
    print(f"Newton-Cotes {nv1}x{nv1}, {walls}, {nx}x{ny}, {steps} steps, storage {storage}: "
          f"state {out[0]:.2e}, E(u) {out[1]:.2e}, mass {out[2]:.2e}")
    return out


# 37 x 21 cells: two 32-lane column blocks and three 8-row blocks, each ragged
@pytest.mark.parametrize("storage", FORMS, ids=IDS)
@pytest.mark.parametrize("walls", ["diffuse", "couette", "mixed"])
def test_newton_cotes_deviation_forms(cuda, walls, storage):
    """8 x 8 Newton-Cotes grid (64 velocities), 20 steps.  Measured on GB300
    (state, E(u), mass), over the three wall kinds: FP32 (4.0-5.1e-8,
    1.3-1.9e-7, 1.1-4.6e-11), BF16 (5.1-5.4e-3, 1.0-1.7e-2, 1.4-2.1e-5)."""
    err, e, dm = nc_case(walls, 8, 37, 21, 20, storage)
    b = {P.G_FP32: (5e-7, 2e-6, 1e-8), P.G_BF16: (2e-2, 5e-2, 1e-4)}[storage]
    assert err <= b[0] and e <= b[1] and dm <= b[2], (err, e, dm)


# (nx, ny): three-cell walls (a wall ghost's sources span the mesh), a
# two-column last tile, ragged tiles in both directions
TINY = [(3, 3), (3, 5), (34, 4), (33, 17)]
TINY_BC = {
    "mixed": [(P.BOUNCEBACK, 0, 0), (P.DIFFUSE, 0, 0), (P.DIFFUSE, 0, 0), (P.BOUNCEBACK, 0.05, 0)],
    "xper": [(P.PERIODIC, 0, 0)] * 2 + [(P.DIFFUSE, 0, 0), (P.DIFFUSE, 0.05, 0)],
}


@pytest.mark.parametrize("storage", FORMS, ids=IDS)
@pytest.mark.parametrize("nv1", [5, 6])
@pytest.mark.parametrize("bcname", list(TINY_BC))
@pytest.mark.parametrize("nx,ny", TINY)
def test_class_moment_path_tiny_meshes(cuda, nx, ny, bcname, nv1, storage):
    """The class-moment kernels on meshes of a few cells: wall ghosts whose
    corners take all nine nearest mesh cells, tiles narrower than 32 x 16,
    an odd (25, with tie velocities) and an even (36) velocity count (the
    FP32 update takes the velocities in pairs), mixed wall kinds; 6 steps
    against the oracle.  Bounds as for the 37 x 21 cases above."""
    RT = 0.5
    bc = TINY_BC[bcname]
    tau, dt = 0.2, 0.25 * (1 / max(nx, ny)) / (4 * np.sqrt(RT))
    pg, po = PV.newton_cotes(nv1, RT), OV.newton_cotes_2d(nv1, RT)
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, pg[0], pg[1], pg[2], tau, dt, bc, storage=storage)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], tau, dt, bc)
    f0 = WL.near_equilibrium_state(po[1], ny, nx, amp=0.1, seed=11 * nx + ny)
    g.set_state(f0)
    g.step(6)
    fg = g.state()
    assert g.check() == P.DUGKS_OK
    g.close()
    fo = O.t3s3_run(f0, o, 6)
    err = rel_linf(fg, fo)
    assert err <= {P.G_FP32: 5e-7, P.G_BF16: 2e-2}[storage], err
    assert abs(fg.sum() - fo.sum()) <= {P.G_FP32: 1e-8, P.G_BF16: 1e-3}[storage] * fo.sum()


@pytest.mark.parametrize("storage", FORMS, ids=IDS)
def test_small_velocity_set_deviation_forms(cuda, storage):
    """5 x 5 Newton-Cotes grid (25 velocities; an odd grid, with tie
    velocities xi_x = 0 or xi_y = 0).  Measured: FP32 (4.3e-8, 2.0e-7,
    2.0e-10), BF16 (2.1e-3, 9.4e-3, 1.6e-4): the coarse grid's larger weights
    give larger BF16 deviations."""
    err, e, dm = nc_case("mixed", 5, 37, 21, 20, storage, seed=5)
    b = {P.G_FP32: (5e-7, 2e-6, 2e-8), P.G_BF16: (2e-2, 5e-2, 1e-3)}[storage]
    assert err <= b[0] and e <= b[1] and dm <= b[2], (err, e, dm)


def test_periodic_mass_conservation_fp32(cuda):
    """Periodic box, 16 x 16 grid, 50 steps: the FP32 form keeps mass to the
    rounding of its stored deviations (measured: state 5.5e-8, mass 2.4e-11)."""
    err, e, dm = nc_case("periodic", 16, 40, 33, 50, P.G_FP32, seed=8)
    assert err <= 5e-7 and dm <= 5e-9, (err, e, dm)


def test_rarefied128_fp32_corner_window(cuda):
    """rarefied128 workload at full size (128^2 cells, 64 x 64 Newton-Cotes,
    Kn = 1, diffuse walls) in the FP32 form, one step, against the oracle on
    the 20 x 20 south-west corner (an output cell depends on cells at most 4
    away; the inner 16 x 16 are compared)."""
    c = WL.config("rarefied128_kn1_nv64")
    n = c["nx"]
    pg = PV.newton_cotes(64, c["RT"])
    po = OV.newton_cotes_2d(64, c["RT"])
    g = P.Solver(n, n, 1 / n, 1 / n, pg[0], pg[1], pg[2], c["tau"], c["dt"], c["bc"],
                 storage=P.G_FP32)
    f0 = WL.near_equilibrium_state(po[1], n, n, amp=0.1, seed=9)
    g.set_state(f0)
    g.step(1)
    fg = g.state()
    g.close()
    m = 20
    o = O.Setup(m, m, 1 / n, 1 / n, po[0], po[1], po[2], c["tau"], c["dt"], c["bc"])
    fo = O.t3s3_step(np.ascontiguousarray(f0[:, :m, :m]), o)
    k = m - 4
    assert rel_linf(fg[:, :k, :k], fo[:, :k, :k]) <= 1e-6
    assert abs(fg.sum() - f0.sum()) <= 1e-7 * f0.sum()


@pytest.mark.parametrize("storage", FORMS, ids=IDS)
def test_d2q9_on_generic_deviation_kernels(cuda, storage):
    """D2Q9 on the generic kernels (dugks_init_ex with DUGKS_PATH_GENERIC):
    the Taylor-Green vortex on 32^2, 200 steps, within the bounds of the
    fused deviation kernels."""
    c = WL.config("tgv32")
    xi, W, RT = PV.d2q9(c["RT"])
    fields = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    g = P.Solver(32, 32, 1 / 32, 1 / 32, xi, W, RT, c["tau"], c["dt"], c["bc"], storage=storage,
                 path=P.PATH_GENERIC)
    g.set_equilibrium(*fields)
    m0 = g.moments()[0].sum()
    g.step(200)
    f = g.state()
    r, u, v = g.moments()
    g.close()
    po = OV.d2q9(c["RT"])
    o = O.Setup(32, 32, 1 / 32, 1 / 32, po[0], po[1], po[2], c["tau"], c["dt"], c["bc"])
    fo = O.t3s3_run(O.equilibrium_state(*fields, o), o, 200)
    _, uo, vo = O.velocity(fo, o)
    e, fe, dm = E_u(u, v, uo, vo), rel_linf(f, fo), abs(r.sum() - m0) / m0
    b = {P.G_FP32: (5e-5, 5e-7, 1e-8), P.G_BF16: (1e-2, 2e-4, 1e-5)}[storage]
    assert e <= b[0] and fe <= b[1] and dm <= b[2], (e, fe, dm)


@pytest.mark.parametrize("storage", FORMS, ids=IDS)
def test_non_finite_state_is_reported(cuda, storage):
    """A non-finite entry in the state reaches the FP64 moments as a
    non-finite value and dugks_check reports DUGKS_EUNSTABLE."""
    pg = PV.newton_cotes(8, 0.5)
    n = 24
    g = P.Solver(n, n, 1 / n, 1 / n, pg[0], pg[1], pg[2], 0.1, 0.001,
                 [(P.DIFFUSE, 0, 0)] * 4, storage=storage)
    f0 = WL.near_equilibrium_state(OV.newton_cotes_2d(8, 0.5)[1], n, n, amp=0.05, seed=2)
    f0[10, 12, 12] = np.inf
    g.set_state(f0)
    g.step(1)
    assert g.check() == P.DUGKS_EUNSTABLE
    g.close()
