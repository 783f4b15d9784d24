"""Adjoint of the T3S3 step against central finite differences (FP64).

* transpose tests: <lam, J dphi> from central differences of the forward
  step equals <J^T lam, dphi> from dugks_adjoint_step, per wall type and
  velocity set (bar 1e-7 relative);
* parameter adjoints of one step (tau, wall velocity) against central
  differences with relative step 1e-5 (the sweet spot measured on GB300: at
  1e-7 rounding noise of <lam, df> reaches 3e-6, at 1e-5 it is ~1e-8; the
  random-sign lam makes these sums cancel), bar 5e-6;
* the lid-driven cavity on 128^2 D2Q9 over 2000 steps with checkpoints every
  100 (torch.autograd through T3S3Run and Equilibrium): gradients of the
  final kinetic energy and of a lid shear functional with respect to the lid
  velocity, tau and the initial velocity field (a seeded direction) within
  1e-5 relative of central differences (relative step 1e-6).
"""
import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV
import workloads as WL

pytestmark = pytest.mark.gpu


def solver_for(case, tau=None, uw=None):
    if case == "periodic":
        xi, W, RT = PV.d2q9(1 / 3)
        kinds, nx, ny, tau0, dt = [0, 0, 0, 0], 12, 10, 0.004, 0.01
    elif case == "cavity":
        xi, W, RT = PV.d2q9(1 / 3)
        kinds, nx, ny, tau0, dt = [1, 1, 1, 1], 11, 9, 0.004, 0.01
    elif case == "diffuse_d2q9":
        xi, W, RT = PV.d2q9(1 / 3)
        kinds, nx, ny, tau0, dt = [2, 2, 2, 2], 9, 8, 0.004, 0.01
    else:  # diffuse Newton-Cotes with a bounce-back pair
        xi, W, RT = PV.newton_cotes(6, 0.5)
        kinds, nx, ny, tau0, dt = [1, 1, 2, 2], 7, 6, 0.05, 0.01
    uw0 = np.array([[0.0, 0.02], [0.0, -0.01], [-0.03, 0.0], [0.05, 0.0]])
    uw = uw0 if uw is None else uw
    bc = [(kinds[s], uw[s, 0], uw[s, 1]) for s in range(4)]
    t = tau0 if tau is None else tau
    s = P.Solver(nx, ny, 1 / nx, 1 / ny, xi, W, RT, t, dt, bc)
    return s, (xi, W, nx, ny, tau0, uw0)


def step_once(case, f, tau=None, uw=None):
    s, _ = solver_for(case, tau, uw)
    s.set_state(f)
    s.step(1)
    out = s.state()
    s.close()
    return out


@pytest.mark.parametrize("case", ["periodic", "cavity", "diffuse_d2q9", "diffuse_nc"])
def test_adjoint_step_is_the_transpose(cuda, case):
    s, (xi, W, nx, ny, tau0, uw0) = solver_for(case)
    f = WL.near_equilibrium_state(W, ny, nx, amp=0.1, seed=31)
    r = WL.rng(77)
    dphi = r.standard_normal(f.shape) * np.asarray(W)[:, None, None]
    lam = r.standard_normal(f.shape)
    eps = 1e-6
    jd = (step_once(case, f + eps * dphi) - step_once(case, f - eps * dphi)) / (2 * eps)
    s.set_state(f)
    out = np.empty_like(f)
    dtau, duw = P.dugks_adjoint_step(s.ctx, lam, out)
    lhs, rhs = float(np.sum(lam * jd)), float(np.sum(out * dphi))
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs), (lhs, rhs)
    # parameter adjoints of the same step
    ht = 1e-5 * tau0
    jt = np.sum(lam * (step_once(case, f, tau=tau0 + ht) - step_once(case, f, tau=tau0 - ht))) / (2 * ht)
    assert abs(dtau - jt) <= 5e-6 * abs(jt), (dtau, jt)
    for side in range(4):
        if case == "periodic":
            break
        for comp in range(2):
            hu = 1e-5
            up, um = uw0.copy(), uw0.copy()
            up[side, comp] += hu
            um[side, comp] -= hu
            ju = np.sum(lam * (step_once(case, f, uw=up) - step_once(case, f, uw=um))) / (2 * hu)
            assert abs(duw[side, comp] - ju) <= 5e-6 * (abs(ju) + 1e-3 * np.abs(duw).max()), \
                (side, comp, duw[side, comp], ju)


def test_cavity128_gradients_against_finite_differences(cuda):
    """Cavity 128^2 D2Q9 FP64, Re 1000, lid Ma 0.1, CFL 0.25 (dt/tau = 6.5;
    the CFL 0.5 of the 256^2 workload would give dt/tau = 13 > 12 here),
    2000 steps, checkpoints every 100."""
    torch = cuda
    from paper_1709_05458_gb300.autograd import Equilibrium, Problem, T3S3Run
    n = 128
    c = WL.config("cavity128")
    xi, W, RT = PV.d2q9(c["RT"])
    dt = 0.5 * c["dt"]
    prob = Problem(n, n, 1 / n, 1 / n, xi, W, RT, dt, (1, 1, 1, 1))
    dev = "cuda"
    U = c["U"]
    tau0 = c["tau"]
    rho0, ux0, uy0 = (torch.from_numpy(a).to(dev) for a in WL.rest_fields(n, n))
    # a smooth seeded initial velocity perturbation so d/du0 is not trivial
    r = WL.smooth_random_field(2, n, n, seed=5, noise=0.0)
    ux0 = ux0 + 0.01 * U * torch.from_numpy(r[0]).to(dev)
    uy0 = uy0 + 0.01 * U * torch.from_numpy(r[1]).to(dev)
    steps, every = 2000, 100
    dx = 1.0 / n
    cx = torch.tensor(xi[:, 0], device=dev)[:, None, None]
    cy = torch.tensor(xi[:, 1], device=dev)[:, None, None]
    nu = tau0 * RT

    def objectives(f, lid):
        rho = f.sum(0)
        ux, uy = (cx * f).sum(0) / rho, (cy * f).sum(0) / rho
        ke = 0.5 * (rho * (ux * ux + uy * uy)).sum() * dx * dx
        shear = (nu * (lid - ux[-1, :]) / (0.5 * dx)).sum() * dx
        return ke, shear

    def run(tau, lid, ux, uy, grad=False):
        t = torch.tensor(tau, dtype=torch.float64, device=dev, requires_grad=grad)
        uw = torch.zeros((4, 2), dtype=torch.float64, device=dev)
        uw[3, 0] = lid
        uw.requires_grad_(grad)
        u = ux.clone().requires_grad_(grad)
        f0 = Equilibrium.apply(rho0, u, uy, prob)
        fN = T3S3Run.apply(f0, t, uw, prob, steps, every)
        return objectives(fN, uw[3, 0]), t, uw, u

    (ke, sh), t, uw, u = run(tau0, U, ux0, uy0, grad=True)
    dirn = torch.from_numpy(WL.smooth_random_field(1, n, n, seed=8, noise=0.0)[0]).to(dev)
    for J in (ke, sh):
        g_t, g_uw, g_u = torch.autograd.grad(J, (t, uw, u), retain_graph=True)
        ht, hu, he = 1e-6 * tau0, 1e-6 * U, 1e-6 * U
        fd_t = (run(tau0 + ht, U, ux0, uy0)[0][J is sh] - run(tau0 - ht, U, ux0, uy0)[0][J is sh]) / (2 * ht)
        fd_u = (run(tau0, U + hu, ux0, uy0)[0][J is sh] - run(tau0, U - hu, ux0, uy0)[0][J is sh]) / (2 * hu)
        fd_d = (run(tau0, U, ux0 + he * dirn, uy0)[0][J is sh]
                - run(tau0, U, ux0 - he * dirn, uy0)[0][J is sh]) / (2 * he)
        ad_d = float((g_u * dirn).sum())
        for ad, fd in ((float(g_t), float(fd_t)), (float(g_uw[3, 0]), float(fd_u)), (ad_d, float(fd_d))):
            assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)
