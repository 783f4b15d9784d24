"""Batched stepping (one persistent launch per stage for the FP64 D2Q9
instances, CUDA graph per step count) and tile autotuning.  The batched
results must be bit-for-bit those of stepping each problem alone (the same
per-face and per-cell arithmetic), and the autotuner must leave the state
and the later results unchanged."""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
from oracle import dugks_oracle as O
from oracle import velocity_sets as OV
import workloads as WL

pytestmark = pytest.mark.gpu


def specs():
    """(nx, ny, velocity set, tau, dt, bc, storage) of uneven instances."""
    d2 = PV.d2q9(1 / 3)
    nc = PV.newton_cotes(16, 0.5)
    per = [(P.PERIODIC, 0, 0)] * 4
    cav = [(P.BOUNCEBACK, 0, 0)] * 3 + [(P.BOUNCEBACK, 0.05, 0)]
    ds = [(P.DIFFUSE, 0, 0)] * 3 + [(P.DIFFUSE, 0.1, 0)]
    return [
        (32, 32, d2, 0.004, 0.01, per, P.FP64),
        (70, 45, d2, 0.003, 0.006, cav, P.FP64),
        (129, 64, d2, 0.002, 0.004, per, P.FP64),
        (40, 33, d2, 0.005, 0.01, cav, P.G_FP32),
        (20, 17, nc, 0.5, 0.002, ds, P.FP64),
        (256, 7, d2, 0.01, 0.02, per, P.FP64),
        (33, 19, nc, 0.5, 0.002, ds, P.G_FP32),
        (21, 40, nc, 0.5, 0.002, per, P.G_FP32),
        (18, 18, nc, 0.5, 0.002, ds, P.G_BF16),
        (26, 14, PV.newton_cotes(5, 0.5), 0.5, 0.002, ds, P.G_FP32),
    ]


def make(spec, stream):
    nx, ny, (xi, W, RT), tau, dt, bc, st = spec
    s = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, tau, dt, bc, stream=stream, storage=st)
    f0 = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=nx * 1000 + ny)
    s.set_state(f0)
    return s, f0


def test_batch_equals_individual_runs(cuda):
    torch = cuda
    stream = torch.cuda.Stream()
    sols, f0s = zip(*[make(sp, stream) for sp in specs()])
    b = P.Batch(sols)
    b.step(3)
    b.step(3)            # graph for nsteps = 3 is replayed
    b.step(2)
    out = [s.state() for s in sols]
    for sp, f0, fb in zip(specs(), f0s, out):
        ref, _ = make(sp, stream)
        ref.set_state(f0)
        ref.step(8)
        np.testing.assert_array_equal(fb, ref.state())
    b.close()
    # one batched instance against the oracle
    nx, ny, _, tau, dt, bc, _ = specs()[1]
    po = OV.d2q9(1 / 3)
    o = O.Setup(nx, ny, 1 / nx, 1 / ny, po[0], po[1], po[2], tau, dt, bc)
    fo = O.t3s3_run(f0s[1], o, 8)
    assert np.abs(out[1] - fo).max() <= 1e-12 * np.abs(fo).max()


def test_autotune_keeps_state_and_results(cuda):
    torch = cuda
    stream = torch.cuda.Stream()
    sp = specs()[2]
    a, f0 = make(sp, stream)
    ty = P.dugks_autotune(a.ctx, trials=2)
    assert 4 <= ty <= 16
    np.testing.assert_array_equal(a.state(), f0)
    a.step(4)
    ref, _ = make(sp, stream)
    ref.step(4)
    np.testing.assert_array_equal(a.state(), ref.state())


@pytest.mark.parametrize("storage", [P.FP64, P.F64_DW], ids=["fp64", "dw"])
def test_fixed_tile_heights_give_identical_results(cuda, storage):
    """Every height dugks_set_tile_height accepts gives the same state bit for
    bit (a ragged bounce-back cavity, 70 x 45, 6 steps); out-of-range
    heights are refused and leave the height unchanged."""
    sp = specs()[1][:6] + (storage,)
    runs = {}
    top = 16 if storage == P.FP64 else 12
    for ty in (4, 5, 7, 11, top):
        a, _ = make(sp, None)
        P.dugks_set_tile_height(a.ctx, ty)
        assert P.dugks_tile_height(a.ctx) == ty
        a.step(6)
        runs[ty] = a.state()
        for bad in (3, top + 1):
            with pytest.raises(P.DugksError) as e:
                P.dugks_set_tile_height(a.ctx, bad)
            assert e.value.code == P.DUGKS_EINVAL
        assert P.dugks_tile_height(a.ctx) == ty
        a.close()
    for ty, f in runs.items():
        np.testing.assert_array_equal(f, runs[4])


def test_batch_needs_a_stream(cuda):
    xi, W, RT = PV.d2q9(1 / 3)
    s = P.Solver(8, 8, 1 / 8, 1 / 8, xi, W, RT, 0.01, 0.01, [(P.PERIODIC, 0, 0)] * 4)
    with pytest.raises(P.DugksError) as e:
        P.Batch([s])
    assert e.value.code == P.DUGKS_EINVAL


def recipe_problem(it):
    """Boundaries and initial fields of one instance of the seeded
    64-instance recipe (workloads.batched_instances), as the benchmark builds
    it: TGV (periodic) or lid cavity (bounce-back for D2Q9, diffuse for
    Newton-Cotes), from equilibrium."""
    N = it["N"]
    if it["kind"] == "tgv":
        return [(P.PERIODIC, 0, 0)] * 4, WL.tgv_fields(N, N, it["U"] * 2 * np.pi, it["RT"])
    kw = P.BOUNCEBACK if it["vel"] == "d2q9" else P.DIFFUSE
    return [(kw, 0, 0)] * 3 + [(kw, it["U"], 0)], WL.rest_fields(N, N)


def recipe_solver(it, stream, storage=P.FP64):
    N = it["N"]
    if it["vel"] == "d2q9":
        xi, W, RT = PV.d2q9(it["RT"])
    else:
        xi, W, RT = PV.newton_cotes(it["nv1"], it["RT"])
    bc, fields = recipe_problem(it)
    s = P.Solver(N, N, 1.0 / N, 1.0 / N, xi, W, RT, it["tau"], it["dt"], bc, stream=stream,
                 storage=storage)
    s.set_equilibrium(*fields)
    return s


@pytest.mark.parametrize("storage", [P.FP64, P.G_FP32], ids=["fp64", "fp32"])
def test_batched64_recipe_matches_individual_runs_and_oracle(cuda, storage):
    """The full 64-instance recipe (seeded grids 32^2-512^2, D2Q9 and
    Newton-Cotes 16^2-32^2 sets) in one batch with its tile height
    autotuned: two batched steps equal, bit for bit, each instance stepped
    alone (FP32: the Newton-Cotes instances through the batched class-moment
    launches, each alone through its own), and the smallest D2Q9 and the
    smallest Newton-Cotes instance match the FP64 oracle (FP64: 1e-12; FP32:
    the state within 1e-6 relative)."""
    torch = cuda
    stream = torch.cuda.Stream()
    insts = WL.config("batched64")["instances"]
    sols = [recipe_solver(it, stream, storage) for it in insts]
    b = P.Batch(sols)
    ty = b.autotune(1)
    assert ty == 0 or 4 <= ty <= 16
    b.step(2)
    torch.cuda.synchronize()
    for it, s in zip(insts, sols):
        got = torch.empty((s.nv, s.ny, s.nx), dtype=torch.float64, device="cuda")
        s.state(got)
        ref = recipe_solver(it, stream, storage)
        ref.step(2)
        want = torch.empty_like(got)
        ref.state(want)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (it["vel"], it["N"])
        ref.close()
        del got, want
    for vel in ("d2q9", "nc"):
        i = min((k for k, it in enumerate(insts) if it["vel"] == vel), key=lambda k: insts[k]["N"])
        it = insts[i]
        bc, fields = recipe_problem(it)
        if vel == "d2q9":
            po = OV.d2q9(it["RT"])
        else:
            po = OV.newton_cotes_2d(it["nv1"], it["RT"])
        N = it["N"]
        o = O.Setup(N, N, 1.0 / N, 1.0 / N, po[0], po[1], po[2], it["tau"], it["dt"], bc)
        fo = O.t3s3_run(O.equilibrium_state(*fields, o), o, 2)
        fg = sols[i].state()
        tol = 1e-12 if storage == P.FP64 else 1e-6
        assert np.abs(fg - fo).max() <= tol * np.abs(fo).max(), (vel, N)
    b.close()
    for s in sols:
        s.close()
