"""dugks_step_static: the T3S3 step for callers that may not allocate device
memory (e.g. a plugin inside an application that owns all device memory
through its own pool).  Its intermediates live in a fixed 32 MiB array inside
the library.  This file is collected last on purpose.

Checks, through the C ABI, that two calls in a row give the same states as
the allocating path (dugks_init / dugks_set_state / dugks_step /
dugks_get_state) within the parity tolerance, for two problems of different
shape that reuse the same array, and that an oversized problem is refused
with a clear message."""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
import workloads as WL

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _allocating(nx, ny, xi, W, RT, tau, dt, bc, f0, n1, n2):
    g = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, tau, dt, bc)
    g.set_state(f0)
    g.step(n1)
    a = g.state()
    g.step(n2)
    b = g.state()
    g.close()
    return a, b


@pytest.mark.parametrize("case", ["cavity_d2q9", "diffuse_nc"])
def test_static_matches_allocating_path_two_calls(cuda, case):
    torch = cuda
    if case == "cavity_d2q9":
        nx, ny = 48, 40
        xi, W, RT = PV.d2q9(1 / 3)
        bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
        tau, dt = 0.002, 0.004
    else:
        nx, ny = 20, 17
        xi, W, RT = PV.newton_cotes(16, 0.5)
        uw = 0.1
        bc = [(P.DIFFUSE, 0, 0)] * 3 + [(P.DIFFUSE, uw, 0)]
        tau, dt = 0.5, 0.002
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=21)
    ref1, ref2 = _allocating(nx, ny, xi, W, RT, tau, dt, bc, f0, 3, 2)

    s = torch.cuda.Stream()
    fin = torch.from_numpy(f0).cuda()
    out1 = torch.empty_like(fin)
    P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, tau, dt, bc, fin, out1, 3, stream=s)
    s.synchronize()
    out2 = out1.clone()
    P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, tau, dt, bc, out2, out2, 2, stream=s)
    s.synchronize()
    assert rel(out1.cpu().numpy(), ref1) <= TOL
    assert rel(out2.cpu().numpy(), ref2) <= TOL
    np.testing.assert_array_equal(fin.cpu().numpy(), f0)


def test_static_rejects_oversized_problem(cuda):
    torch = cuda
    xi, W, RT = PV.d2q9(1 / 3)
    n = 512                      # 5 * 9 * 512^2 doubles > 32 MiB
    f = torch.empty((9, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(P.DugksError) as e:
        P.dugks_step_static(n, n, 1 / n, 1 / n, xi, W, RT, 0.01, 0.01,
                            [(P.PERIODIC, 0, 0)] * 4, f, f, 1)
    assert e.value.code == P.DUGKS_EINVAL
    assert "bytes of scratch" in str(e.value)
