"""GPU parity of DUGKS_F64_DW -- FP64 arrays, the fused D2Q9 kernels in
double-word (FP32 pair) arithmetic -- against the FP64 oracle.

Bar: the FP64 one, relative L-infinity error
max|f_gpu - f_oracle| / max|f_oracle| <= 1e-12, on the cases of the FP64
parity file that the fused D2Q9 kernels take.  A double-word operation has a
unit roundoff of 2^-48 (about 3.6e-15, against 1.1e-16 for FP64) with
normwise bounds on sums, so a step adds errors of order 1e-14 relative to
max|f|; the measured errors are quoted per test."""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-12
PER = [(P.PERIODIC, 0, 0)] * 4


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def pair(nx, ny, RT, tau, dt, bc, Lx=1.0, Ly=1.0, storage=P.F64_DW):
    pg, po = PV.d2q9(RT), OV.d2q9(RT)
    dx, dy = Lx / nx, Ly / ny
    g = P.Solver(nx, ny, dx, dy, pg[0], pg[1], pg[2], tau, dt, bc, storage=storage)
    o = O.Setup(nx, ny, dx, dy, po[0], po[1], po[2], tau, dt, bc)
    return g, o


@pytest.mark.parametrize("steps", [1, 10])
def test_tgv_equilibrium_init(cuda, steps):
    c = WL.config("tgv32")
    g, o = pair(32, 32, c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    g.set_equilibrium(rho, u, v)
    f0 = O.equilibrium_state(rho, u, v, o)
    g.step(steps)
    assert rel_linf(g.state(), O.t3s3_run(f0, o, steps)) <= TOL
    g.close()


def test_tgv32_full_200_steps(cuda):
    """The tgv32 workload: 200 steps from equilibrium, state and moments."""
    c = WL.config("tgv32")
    g, o = pair(32, 32, c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    g.set_equilibrium(rho, u, v)
    g.step(c["steps"])
    fo = O.t3s3_run(O.equilibrium_state(rho, u, v, o), o, c["steps"])
    assert rel_linf(g.state(), fo) <= TOL
    r, ux, uy = g.moments()
    ro, uxo, uyo = O.velocity(fo, o)
    assert np.abs(r - ro).max() <= TOL * np.abs(ro).max()
    assert np.abs(ux - uxo).max() <= 1e-10 * np.abs(uxo).max()
    g.close()


@pytest.mark.parametrize("nx,ny", [(37, 29), (1, 5), (2, 3), (300, 7)])
def test_periodic_random_state_ragged(cuda, nx, ny):
    g, o = pair(nx, ny, 1 / 3, 0.01, 0.03, PER, Lx=nx / 32, Ly=ny / 32)
    _, W, _ = OV.d2q9(1 / 3)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.2, seed=11)
    g.set_state(f0)
    g.step(5)
    assert rel_linf(g.state(), O.t3s3_run(f0, o, 5)) <= TOL
    g.close()


@pytest.mark.parametrize("bcname", ["cavity", "diffuse"])
@pytest.mark.parametrize("nx,ny", [(45, 33), (3, 3), (70, 45)])
def test_walls_ragged(cuda, bcname, nx, ny):
    """Bounce-back cavity with a moving lid, and diffuse walls moving in
    both directions; mass conserved to 1e-12."""
    bc = {"cavity": [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)],
          "diffuse": [(P.DIFFUSE, 0.0, 0.02), (P.DIFFUSE, 0, 0), (P.DIFFUSE, -0.03, 0),
                      (P.DIFFUSE, 0.05, 0)]}[bcname]
    g, o = pair(nx, ny, 1 / 3, 0.002, 0.004, bc)
    _, W, _ = OV.d2q9(1 / 3)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=5)
    g.set_state(f0)
    g.step(8)
    fg = g.state()
    g.close()
    assert rel_linf(fg, O.t3s3_run(f0, o, 8)) <= TOL
    if bcname == "cavity":
        assert abs(fg.sum() - f0.sum()) <= 1e-12 * f0.sum()


def test_cavity256_workload_full_compare(cuda):
    """cavity256 at full size from rest, 10 steps, element by element."""
    c = WL.config("cavity256")
    g, o = pair(256, 256, c["RT"], c["tau"], c["dt"], c["bc"])
    rho, u, v = WL.rest_fields(256, 256)
    g.set_equilibrium(rho, u, v)
    g.step(10)
    fo = O.t3s3_run(O.equilibrium_state(rho, u, v, o), o, 10)
    assert rel_linf(g.state(), fo) <= TOL
    g.close()


def test_long_run_against_fp64_kernels(cuda):
    """cavity256, 2000 steps from rest: the double-word and FP64 fused
    kernels stay within 1e-12 of each other (the oracle would take
    minutes at this length)."""
    c = WL.config("cavity256")
    out = []
    for st in (P.FP64, P.F64_DW):
        g, _ = pair(256, 256, c["RT"], c["tau"], c["dt"], c["bc"], storage=st)
        g.set_equilibrium(*WL.rest_fields(256, 256))
        g.step(2000)
        out.append(g.state())
        assert g.check() == P.DUGKS_OK
        g.close()
    assert rel_linf(out[1], out[0]) <= TOL


def test_refusals(cuda):
    """The T2 schemes and the adjoint need FP64 arithmetic."""
    c = WL.config("tgv32")
    g, _ = pair(32, 32, c["RT"], c["tau"], c["dt"], c["bc"])
    with pytest.raises(P.DugksError) as e:
        P.dugks_set_scheme(g.ctx, P.T2S2)
    assert e.value.code == P.DUGKS_ENOTIMPL
    lam = np.zeros((9, 32, 32))
    with pytest.raises(P.DugksError) as e:
        P.dugks_adjoint_step(g.ctx, lam, np.empty_like(lam))
    assert e.value.code == P.DUGKS_ENOTIMPL
    g.close()


def test_batch_runs_double_word_instances_on_their_own_launches(cuda):
    """A batch holding a double-word context steps it with its own kernels:
    the result equals the unbatched run bit for bit."""
    import torch
    stream = torch.cuda.Stream()
    c = WL.config("tgv32")
    pg = PV.d2q9(c["RT"])
    fields = WL.tgv_fields(32, 32, c["u0"], c["RT"])
    ref = P.Solver(32, 32, 1 / 32, 1 / 32, *pg, c["tau"], c["dt"], c["bc"], storage=P.F64_DW)
    ref.set_equilibrium(*fields)
    ref.step(7)
    want = ref.state()
    ref.close()
    a = P.Solver(32, 32, 1 / 32, 1 / 32, *pg, c["tau"], c["dt"], c["bc"], stream=stream,
                 storage=P.F64_DW)
    b = P.Solver(32, 32, 1 / 32, 1 / 32, *pg, c["tau"], c["dt"], c["bc"], stream=stream)
    a.set_equilibrium(*fields)
    b.set_equilibrium(*fields)
    bt = P.Batch([a, b])
    bt.step(7)
    stream.synchronize()
    np.testing.assert_array_equal(a.state(), want)
    bt.close()
    a.close()
    b.close()


@pytest.mark.parametrize("storage", [P.FP64, P.F64_DW], ids=["fp64", "dw"])
def test_unequal_weights_take_the_general_kernels(cuda, storage):
    """D2Q9 velocities with weights that differ inside a class (W of +x and
    -x moved by +-0.01, still summing to one): the fused kernels' general
    instantiations (one weight per velocity) against the oracle with the
    same weights, bounce-back cavity, 8 steps."""
    pg, po = PV.d2q9(1 / 3), OV.d2q9(1 / 3)
    W, Wo = np.array(pg[1], dtype=float), np.array(po[1], dtype=float)
    for w in (W, Wo):     # each side perturbs its own set
        w[7] += 0.01      # (+1, 0)
        w[1] -= 0.01      # (-1, 0)
    nx, ny = 45, 33
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, pg[0], W, pg[2], 0.002, 0.004, bc, storage=storage)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], Wo, po[2], 0.002, 0.004, bc)
    f0 = WL.near_equilibrium_state(Wo, ny, nx, amp=0.1, seed=23)
    g.set_state(f0)
    g.step(8)
    fg = g.state()
    g.close()
    assert rel_linf(fg, O.t3s3_run(f0, o, 8)) <= TOL


def test_autotune_keeps_results_identical(cuda):
    """dugks_autotune on a double-word context picks a height in 4..12 and
    later steps equal those of an untuned context bit for bit (the tile
    height changes no arithmetic)."""
    c = WL.config("cavity128")
    runs = []
    for tune in (False, True):
        g, _ = pair(128, 128, c["RT"], c["tau"], 0.5 * c["dt"], c["bc"])
        g.set_equilibrium(*WL.rest_fields(128, 128))
        g.step(3)
        if tune:
            ty = P.dugks_autotune(g.ctx, trials=1)
            assert 4 <= ty <= 12
        g.step(5)
        runs.append(g.state())
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])
