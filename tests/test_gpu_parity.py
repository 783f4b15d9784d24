"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (floating point, FP64 arithmetic on both sides): relative L-infinity
error  max|f_gpu - f_oracle| / max|f_oracle| <= 1e-12  on the same seeded
inputs.  Each side builds its own velocity set and its own equilibrium; the
state arrays come from ``workloads``.
"""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def pair(nx, ny, vel, RT, tau, dt, bc, Lx=1.0, Ly=1.0, path=P.PATH_AUTO, **vkw):
    """(GPU solver, oracle setup) for the same problem; ``path`` the kernel
    path of dugks_init_ex."""
    if vel == "d2q9":
        pg, po = PV.d2q9(RT), OV.d2q9(RT)
    else:
        pg, po = PV.newton_cotes(vel, RT, **vkw), OV.newton_cotes_2d(vel, RT, **vkw)
    dx, dy = Lx / nx, Ly / ny
    g = P.Solver(nx, ny, dx, dy, pg[0], pg[1], pg[2], tau, dt, bc, path=path)
    o = O.Setup(nx, ny, dx, dy, po[0], po[1], po[2], tau, dt, bc)
    return g, o


def compare_from_state(g, o, f0, steps):
    g.set_state(f0)
    g.step(steps)
    fg = g.state()
    fo = O.t3s3_run(f0, o, steps)
    return rel_linf(fg, fo), fg, fo


PER = [(P.PERIODIC, 0, 0)] * 4


@pytest.mark.parametrize("steps", [1, 10])
def test_tgv_equilibrium_init(cuda, steps):
    """Taylor-Green 32^2 D2Q9 (tgv32 workload), equilibrium initialisation
    done by each side (dugks_set_equilibrium vs the oracle)."""
    c = WL.config("tgv32")
    g, o = pair(32, 32, "d2q9", c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    g.set_equilibrium(rho, u, v)
    f0 = O.equilibrium_state(rho, u, v, o)
    assert rel_linf(g.state(), f0) <= TOL
    g.step(steps)
    assert rel_linf(g.state(), O.t3s3_run(f0, o, steps)) <= TOL


def test_tgv32_full_200_steps(cuda):
    """The tgv32 workload as configured: 200 steps from equilibrium."""
    c = WL.config("tgv32")
    g, o = pair(32, 32, "d2q9", c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    g.set_equilibrium(rho, u, v)
    g.step(c["steps"])
    fo = O.t3s3_run(O.equilibrium_state(rho, u, v, o), o, c["steps"])
    assert rel_linf(g.state(), fo) <= TOL
    # moments through the ABI against the oracle's
    r, ux, uy = g.moments()
    ro, uxo, uyo = O.velocity(fo, o)
    assert np.abs(r - ro).max() <= TOL * np.abs(ro).max()
    assert np.abs(ux - uxo).max() <= 1e-10 * np.abs(uxo).max()


@pytest.mark.parametrize("nx,ny", [(37, 29), (1, 5), (2, 3), (300, 7)])
def test_periodic_random_state_ragged(cuda, nx, ny):
    """Non-equilibrium random state on ragged periodic grids (several
    256-cell tiles plus a tail; degenerate 1- and 2-cell widths)."""
    g, o = pair(nx, ny, "d2q9", 1 / 3, 0.01, 0.03, PER, Lx=nx / 32, Ly=ny / 32)
    _, W, _ = OV.d2q9(1 / 3)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.2, seed=11)
    err, _, _ = compare_from_state(g, o, f0, 5)
    assert err <= TOL


@pytest.mark.parametrize("nx,ny", [(45, 33), (3, 3), (3, 17)])
def test_bounceback_cavity_ragged(cuda, nx, ny):
    """Lid-driven cavity walls (bounce-back, moving north wall)."""
    U = 0.05
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, U, 0)]
    g, o = pair(nx, ny, "d2q9", 1 / 3, 0.002, 0.004, bc)
    _, W, _ = OV.d2q9(1 / 3)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=5)
    err, fg, _ = compare_from_state(g, o, f0, 8)
    assert err <= TOL
    assert abs(fg.sum() - f0.sum()) <= 1e-12 * f0.sum()


def test_cavity256_workload_full_compare(cuda):
    """cavity256 at full size (256^2 D2Q9, Re 1000, lid Ma 0.1) from rest,
    10 steps compared element by element."""
    c = WL.config("cavity256")
    g, o = pair(256, 256, "d2q9", c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.rest_fields(256, 256)
    g.set_equilibrium(rho, u, v)
    g.step(10)
    fo = O.t3s3_run(O.equilibrium_state(rho, u, v, o), o, 10)
    assert rel_linf(g.state(), fo) <= TOL


@pytest.mark.parametrize("kernels", ["optimised", "first"])
@pytest.mark.parametrize("walls", ["diffuse", "couette", "mixed"])
def test_newton_cotes_walls(cuda, walls, kernels):
    """Newton-Cotes velocity grid with diffuse-scattering walls (more than 32
    velocities), on the optimised generic kernels and on the reference
    kernels (DUGKS_PATH_REFERENCE; they also serve the T2 schemes, the
    adjoint's forward recomputation and the allocation-free entry)."""
    path = P.PATH_REFERENCE if kernels == "first" else P.PATH_AUTO
    uw = 0.16 * np.sqrt(5 / 3 * 0.5)
    bc = {"diffuse": [(P.DIFFUSE, 0, 0)] * 3 + [(P.DIFFUSE, uw, 0)],
          "couette": [(P.PERIODIC, 0, 0)] * 2 + [(P.DIFFUSE, -uw, 0), (P.DIFFUSE, uw, 0)],
          "mixed": [(P.BOUNCEBACK, 0, 0), (P.DIFFUSE, 0, 0), (P.DIFFUSE, 0, 0),
                    (P.BOUNCEBACK, uw, 0)]}[walls]
    nx, ny = 21, 18
    tau = 1.0 / np.sqrt(np.pi * 0.5 / 2)
    dt = 0.25 * (1 / 21) / (4 * np.sqrt(0.5))
    g, o = pair(nx, ny, 16, 0.5, tau, dt, bc, path=path)
    f0 = WL.near_equilibrium_state(o.W, ny, nx, amp=0.1, seed=3)
    err, fg, _ = compare_from_state(g, o, f0, 4)
    assert err <= TOL
    assert abs(fg.sum() - f0.sum()) <= 1e-12 * f0.sum()


def test_rarefied128_full_size_corner_window(cuda):
    """rarefied128 workload at full size (128^2 cells, 64x64 Newton-Cotes,
    Kn = 1, diffuse walls), one step.  An output cell depends on cells at
    most 4 away (two stages of the 2-cell stencil), so the oracle runs on the
    20x20 south-west corner with the true west/south walls and its 16x16
    corner cells are compared exactly."""
    c = WL.config("rarefied128_kn1_nv64")
    n = c["nx"]
    pg = PV.newton_cotes(64, c["RT"])
    po = OV.newton_cotes_2d(64, c["RT"])
    g = P.Solver(n, n, 1 / n, 1 / n, pg[0], pg[1], pg[2], c["tau"], c["dt"], c["bc"])
    f0 = WL.near_equilibrium_state(po[1], n, n, amp=0.1, seed=9)
    g.set_state(f0)
    g.step(1)
    fg = g.state()
    m = 20
    o = O.Setup(m, m, 1 / n, 1 / n, po[0], po[1], po[2], c["tau"], c["dt"], c["bc"])
    fo = O.t3s3_step(np.ascontiguousarray(f0[:, :m, :m]), o)
    k = m - 4
    assert rel_linf(fg[:, :k, :k], fo[:, :k, :k]) <= TOL
    assert abs(fg.sum() - f0.sum()) <= 1e-12 * f0.sum()


def test_device_pointer_path(cuda):
    """on_device = 1: state and moments through torch device tensors on the
    solver's own stream."""
    torch = cuda
    s = torch.cuda.Stream()
    xi, W, RT = PV.d2q9(1 / 3)
    nx, ny = 40, 24
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.02, PER, stream=s)
    po = OV.d2q9(1 / 3)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], 0.01, 0.02, PER)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.2, seed=4)
    with torch.cuda.stream(s):
        t0 = torch.from_numpy(f0).cuda()
        g.set_state(t0)
        g.step(3)
        out = torch.empty_like(t0)
        P.dugks_get_state(g.ctx, out)
        rho = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        P.dugks_moments(g.ctx, rho, None, None)
    s.synchronize()
    fo = O.t3s3_run(f0, o, 3)
    assert rel_linf(out.cpu().numpy(), fo) <= TOL
    assert np.abs(rho.cpu().numpy() - fo.sum(axis=0)).max() <= 1e-12


def test_moments_into_one_buffer(cuda):
    """rho, ux, uy as the three planes of one [3][ny][nx] buffer (read back in
    one copy) equal the three separate arrays, on the host and on the device,
    and the oracle's moments (Sec. 2.2)."""
    torch = cuda
    xi, W, RT = PV.d2q9(1 / 3)
    nx, ny = 37, 21
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.02, bc)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.2, seed=6)
    g.set_state(f0)
    g.step(2)
    r, u, v = g.moments()
    packed = np.empty((3, ny, nx))
    P.dugks_moments(g.ctx, packed[0], packed[1], packed[2])
    for a, b in zip(packed, (r, u, v)):
        np.testing.assert_array_equal(a, b)
    dev = torch.empty((3, ny, nx), dtype=torch.float64, device="cuda")
    P.dugks_moments(g.ctx, dev[0], dev[1], dev[2])
    g.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), packed)
    po = OV.d2q9(1 / 3)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], 0.01, 0.02, bc)
    fo = O.t3s3_run(f0, o, 2)
    ro, uo, vo = O.velocity(fo, o)
    assert np.abs(r - fo.sum(axis=0)).max() <= 1e-12
    assert max(np.abs(u - uo).max(), np.abs(v - vo).max()) <= 1e-11
    g.close()


def test_zero_steps_and_state_roundtrip(cuda):
    xi, W, RT = PV.d2q9(1 / 3)
    g = P.Solver(5, 4, .2, .25, xi, W, RT, 0.1, 0.1, PER)
    f0 = WL.near_equilibrium_state(W, 4, 5)
    g.set_state(f0)
    g.step(0)
    np.testing.assert_array_equal(g.state(), f0)


def test_unstable_run_is_detected_on_the_host(cuda):
    """dt/tau ~ 90 (the literal CFL 0.5 reading of the tgv32 workload) is
    beyond the stability bound 12 of Sec. 2.1.1: the run blows up and
    dugks_check reports DUGKS_EUNSTABLE instead of faulting."""
    xi, W, RT = PV.d2q9(1 / 3)
    U = 0.01 * np.sqrt(RT)
    nu = U / 100
    tau = nu / RT
    dt = 0.5 * (1 / 32) / 1.0
    g = P.Solver(32, 32, 1 / 32, 1 / 32, xi, W, RT, tau, dt, PER)
    assert "stability" in g.warning
    rho, u, v = WL.tgv_fields(32, 32, U * 2 * np.pi, RT)
    g.set_equilibrium(rho, u, v)
    assert g.check() == P.DUGKS_OK
    bad = False
    for _ in range(40):
        g.step(50)
        if g.check() == P.DUGKS_EUNSTABLE:
            bad = True
            break
    assert bad


@pytest.mark.parametrize("bcname", ["periodic", "cavity", "diffuse"])
def test_fused_d2q9_matches_generic_path(cuda, bcname):
    """The fused D2Q9 kernels (default for D2Q9) and the generic kernels
    (DUGKS_PATH_GENERIC) agree with each other and with the oracle, on a grid
    that spans several 32 x ty tiles with ragged edges."""
    bc = {"periodic": PER,
          "cavity": [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)],
          "diffuse": [(P.DIFFUSE, 0.0, 0.02), (P.DIFFUSE, 0, 0), (P.DIFFUSE, -0.03, 0),
                      (P.DIFFUSE, 0.05, 0)]}[bcname]
    nx, ny = 70, 45
    _, W, _ = OV.d2q9(1 / 3)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.15, seed=17)
    out = {}
    for mode, path in (("0", P.PATH_AUTO), ("1", P.PATH_GENERIC)):
        g, o = pair(nx, ny, "d2q9", 1 / 3, 0.003, 0.006, bc, path=path)
        g.set_state(f0)
        g.step(6)
        out[mode] = g.state()
        g.close()
    fo = O.t3s3_run(f0, o, 6)
    assert rel_linf(out["0"], fo) <= TOL
    assert rel_linf(out["1"], fo) <= TOL


@pytest.mark.parametrize("form", ["fp64_fused", "fp64_nc", "fp32_fused", "t2s3"])
def test_get_state_of_f(cuda, form):
    """dugks_get_state(which = DUGKS_STATE_F) returns the distribution f
    itself: f = (4 tau f^ + dt feq)/(4 tau + dt) under T3S3 and
    (2 tau f~ + dt feq)/(2 tau + dt) under a T2 scheme (feq of the state's
    moments), against the oracle's conversion of its own state."""
    nx, ny = 37, 23
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    if form == "fp64_nc":
        g, o = pair(nx, ny, 8, 0.5, 0.05, 0.004,
                    [(P.DIFFUSE, 0, 0)] * 3 + [(P.DIFFUSE, 0.1, 0)])
    else:
        g, o = pair(nx, ny, "d2q9", 1 / 3, 0.003, 0.006, bc)
        if form == "fp32_fused":
            g.close()
            pg = PV.d2q9(1 / 3)
            g = P.Solver(nx, ny, 1 / nx, 1 / ny, *pg, 0.003, 0.006, bc, storage=P.G_FP32)
        elif form == "t2s3":
            P.dugks_set_scheme(g.ctx, P.T2S3)
    f0 = WL.near_equilibrium_state(o.W, ny, nx, amp=0.1, seed=8)
    g.set_state(f0)
    g.step(2)
    x = g.state()
    f = g.state(which=P.STATE_F)
    feq, _ = O.equilibrium_of(x, o)
    cdt = (0.5 if form == "t2s3" else 0.25) * o.dt
    fo = (o.tau * x + cdt * feq) / (o.tau + cdt)
    assert rel_linf(f, fo) <= TOL
    if form == "fp64_fused":
        fs = O.t3s3_run(f0, o, 2)
        assert rel_linf(f, O.f_from_fhat(fs, o)) <= TOL
    g.close()
