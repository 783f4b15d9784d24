"""dugks_step_static: the T3S3 step for callers that may not allocate device
memory (e.g. a plugin inside an application that owns all device memory
through its own pool).  Its intermediates live in a fixed 32 MiB array inside
the library.  This file is collected last on purpose.

Checks, through the C ABI, that two calls in a row give the same states as
the allocating path (dugks_init / dugks_set_state / dugks_step /
dugks_get_state) within the parity tolerance, for two problems of different
shape that reuse the same array; that calls after the first allocate no
device memory; and that an oversized problem, partially overlapping buffers,
wrong tensors and a capturing stream are refused with a clear message."""
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


def test_static_call_allocates_no_device_memory(cuda):
    """The property the entry point exists for: after a warm-up call (which
    loads the kernels and looks up the array's address), further calls leave
    the device's free memory and torch's allocator unchanged."""
    torch = cuda
    nx, ny = 40, 36
    xi, W, RT = PV.d2q9(1 / 3)
    bc = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    f = torch.from_numpy(WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=5)).cuda()
    s = torch.cuda.Stream()
    P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.002, 0.004, bc, f, f, 2, stream=s)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.002, 0.004, bc, f, f, 4, stream=s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert bool(torch.isfinite(f).all())


def test_static_rejects_oversized_problem(cuda):
    torch = cuda
    xi, W, RT = PV.d2q9(1 / 3)
    n = 512                      # 5 * 9 * 512^2 doubles > 32 MiB
    f = torch.zeros((9, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(P.DugksError) as e:
        P.dugks_step_static(n, n, 1 / n, 1 / n, xi, W, RT, 0.01, 0.01,
                            [(P.PERIODIC, 0, 0)] * 4, f, f, 1)
    assert e.value.code == P.DUGKS_EINVAL
    assert "bytes of scratch" in str(e.value)


def test_static_rejects_partial_overlap_and_bad_tensors(cuda):
    torch = cuda
    nx, ny = 8, 6
    xi, W, RT = PV.d2q9(1 / 3)
    bc = [(P.PERIODIC, 0, 0)] * 4
    n = 9 * nx * ny
    buf = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    a, b = buf[:n], buf[n // 2:n // 2 + n]          # overlapping, not equal
    with pytest.raises(P.DugksError) as e:
        P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.01, bc, a, b, 1)
    assert e.value.code == P.DUGKS_EINVAL and "overlap" in str(e.value)
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(n, dtype=torch.float64),                   # host tensor
                torch.zeros(n, dtype=torch.float32, device="cuda"),   # wrong dtype
                torch.zeros(n - 1, dtype=torch.float64, device="cuda")):  # wrong size
        with pytest.raises(ValueError):
            P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.01, bc, good, bad, 1)


def test_static_refuses_a_capturing_stream(cuda):
    """Each call uploads its velocity tables from call-local host memory, so
    it refuses to be recorded into a CUDA graph (the copy would point at
    freed memory on replay)."""
    torch = cuda
    nx, ny = 8, 6
    xi, W, RT = PV.d2q9(1 / 3)
    bc = [(P.PERIODIC, 0, 0)] * 4
    f = torch.zeros((9, ny, nx), dtype=torch.float64, device="cuda")
    import gc
    s = torch.cuda.Stream()
    P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.01, bc, f, f, 0, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    # no garbage collection during the capture: a collected object of an
    # earlier test (a solver freeing its buffers) would invalidate it
    gc.collect()
    gc.disable()
    try:
        with pytest.raises(P.DugksError) as e:
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                P.dugks_step_static(nx, ny, 1 / nx, 1 / ny, xi, W, RT, 0.01, 0.01, bc, f, f, 1,
                                    stream=s)
    finally:
        gc.enable()
    assert e.value.code == P.DUGKS_EINVAL and "capturing" in str(e.value)
    torch.cuda.synchronize()
