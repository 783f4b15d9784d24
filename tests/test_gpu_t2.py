"""T2S3 and T2S2 (the second-order comparison schemes of Sec. 3, Remark I)
through the C ABI against the oracle's t2 steps: FP64 on both sides, the
same seeded states; bar 1e-12 relative L-infinity (as the T3S3 parity)."""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-12
SCHEMES = [(P.T2S3, "printed"), (P.T2S2, "central")]
IDS = ["t2s3", "t2s2"]


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def pair(nx, ny, vel, RT, tau, dt, bc, scheme):
    if vel == "d2q9":
        pg, po = PV.d2q9(RT), OV.d2q9(RT)
    else:
        pg, po = PV.newton_cotes(vel, RT), OV.newton_cotes_2d(vel, RT)
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, pg[0], pg[1], pg[2], tau, dt, bc, scheme=scheme)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], tau, dt, bc)
    return g, o


@pytest.mark.parametrize("scheme,recon", SCHEMES, ids=IDS)
@pytest.mark.parametrize("case", ["periodic", "cavity", "nc_diffuse"])
def test_t2_parity(cuda, scheme, recon, case):
    if case == "periodic":
        nx, ny, vel, RT, tau, dt, steps = 45, 37, "d2q9", 1 / 3, 0.004, 0.008, 6
        bc = [(P.PERIODIC, 0, 0)] * 4
    elif case == "cavity":
        nx, ny, vel, RT, tau, dt, steps = 33, 29, "d2q9", 1 / 3, 0.003, 0.006, 6
        bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    else:
        nx, ny, vel, RT, steps = 21, 18, 8, 0.5, 3
        tau, dt = 1.0 / np.sqrt(np.pi * 0.5 / 2), 0.25 * (1 / 21) / (4 * np.sqrt(0.5))
        uw = 0.16 * np.sqrt(5 / 3 * 0.5)
        bc = [(P.DIFFUSE, 0, 0), (P.BOUNCEBACK, 0, 0), (P.DIFFUSE, 0, 0), (P.DIFFUSE, uw, 0)]
    g, o = pair(nx, ny, vel, RT, tau, dt, bc, scheme)
    f0 = WL.near_equilibrium_state(o.W, ny, nx, amp=0.1, seed=4)
    g.set_state(f0)
    g.step(steps)
    fg = g.state()
    g.close()
    fo = O.t2_run(f0, o, steps, recon)
    assert rel_linf(fg, fo) <= TOL


def test_scheme_switch_and_back(cuda):
    """T2S2 steps, then back to T3S3 (the fused D2Q9 kernels): each segment
    matches the oracle from the state the previous one left."""
    nx, ny = 40, 34
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    g, o = pair(nx, ny, "d2q9", 1 / 3, 0.003, 0.006, bc, P.T3S3)
    f0 = WL.near_equilibrium_state(o.W, ny, nx, amp=0.1, seed=6)
    g.set_state(f0)
    g.step(3)
    f1 = g.state()
    assert rel_linf(f1, O.t3s3_run(f0, o, 3)) <= TOL
    P.dugks_set_scheme(g.ctx, P.T2S2)
    g.step(4)
    f2 = g.state()
    assert rel_linf(f2, O.t2_run(f1, o, 4, "central")) <= TOL
    P.dugks_set_scheme(g.ctx, P.T3S3)
    g.step(2)
    assert rel_linf(g.state(), O.t3s3_run(f2, o, 2)) <= TOL
    g.close()


def test_t2_refusals(cuda):
    xi, W, RT = PV.d2q9(1 / 3)
    bc = [(P.PERIODIC, 0, 0)] * 4
    g = P.Solver(16, 16, 1 / 16, 1 / 16, xi, W, RT, 0.01, 0.01, bc, storage=P.G_FP32)
    with pytest.raises(P.DugksError) as e:
        P.dugks_set_scheme(g.ctx, P.T2S2)
    assert e.value.code == P.DUGKS_ENOTIMPL
    g.close()
    g = P.Solver(16, 16, 1 / 16, 1 / 16, xi, W, RT, 0.01, 0.01, bc, scheme=P.T2S3)
    lam = np.ones((9, 16, 16))
    with pytest.raises(P.DugksError) as e:
        P.dugks_adjoint_step(g.ctx, lam, np.empty_like(lam))
    assert e.value.code == P.DUGKS_ENOTIMPL
    with pytest.raises(P.DugksError) as e:
        P.dugks_set_scheme(g.ctx, 7)
    assert e.value.code == P.DUGKS_EINVAL
    g.close()
