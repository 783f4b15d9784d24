"""Plain FP64 CPU oracle of the third-order DUGKS (T3S3) time step.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import anything under
``oracle/``.  The product (the CUDA library and its Python binding) never
imports, links or calls this module, and this module shares no code with it.

What it computes: one two-stage, third-order DUGKS step of the isothermal
BGK-Boltzmann equation (Wu, Shu, Shi, Chen, arXiv:1709.05458), restated
step by step in the paper's order and notation, every named quantity its own
numpy array, no blocking, fusion or reordering:

  Step (1)  f^  -> f-bar^{+,dt/6}          (eq. f_bar_1_6)
            -> f-bar(x_b, t*)              (eqs. interfaceEvof, flux_DS)
            -> f(x_b, t*)                  (eq. recover2f)
            -> L*                          (eq. microflux, midpoint rule)
  Step (2)  f~+(t_n) = 5/4 f-bar^{+,dt/6} - 1/4 f^   (eq. f_tilde_1_3)
            f~(t')   = f~+(t_n) + dt/3 L*           (eq. feqIntD2nd_Explicit, step dt/3)
            dt*Omega(f')                            (eq. collisionterm)
  Step (3)  f~(t') -> f-bar^{+,5dt/12}(t')          (eq. fbp_5_12, see reading Q6)
            -> faces at t** -> L**
  Step (4)  f^+(t_n) = 1/4 f^ + 3/4 f-bar^{+,dt/6}  (eq. fhp)
            f^^{n+1} = f^+ + 3/4 dt Omega' + dt/7 (3 L* + 4 L**)  (eq. feqIntD3rdHat2_DS)

State layout: ``f[k, j, i]`` with velocity k, cell row j (y) and column i (x),
cell centres at ((i+1/2) dx, (j+1/2) dy).

Readings of the paper where it is silent, garbled or inconsistent (each
marked ``Qn`` where it is used):

* Q1  micro-flux sign: L = -(1/|V|) oint (xi.n) f dS, consistent with L = -xi.grad f.
* Q2p eq. flux_DS is taken as printed: f + d.grad f + d^2 : grad^2 f, the
      second-order term the full double contraction (mixed derivative
      included) without a factor 1/2.  Run on the Taylor vortex of Table 1
      this reproduces the printed T3S3 and T2S3 errors on the finer meshes
      (within 25 % for N >= 96 and 13 % for N >= 64); the corrected Taylor
      series with the 1/2 (``recon="quadratic"``, reading Q2) is 40-90x above
      every printed entry.
* Q3  derivatives by second-order central differences on the 3x3
      neighbourhood of the upwind cell.
* Q4  xi.n == 0 at an interior face: average of the two one-sided expansions.
* Q5  eq. f_tilde_1_3 evaluates to f~+(t_n) (not f~); it is used as f~+ and
      eq. ftp is not applied a second time.
* Q6  eq. fbp_5_12 as printed is inconsistent with the definitions
      f~ = f - dt/6 Omega and f-bar^{+,h} = f + h/2 Omega; the consistent map is
      ((24 tau - 5 dt) f~ + 9 dt feq) / (24 tau + 4 dt).  ``fbp='printed'``
      selects the printed coefficients for comparison studies.
* Q7  the T2 explicit step uses the full step times L at the midpoint
      (B~_2 = 1), i.e. f~(t') = f~+(t_n) + (dt/3) L*.
* Q9  face equilibria use the moments of f-bar at the face.
* Q12 walls lie on cell faces; n is the unit normal pointing out of the
      fluid; velocities with xi.n < 0 leave the wall.
* Q13 bounce-back and diffuse scattering are imposed on f-bar at the wall
      face; the face moments and f-bar -> f then follow as at interior faces.
* Q14 rho_w of bounce-back is the density of the wall-adjacent cell at the
      stage's base time (t_n for stage 1, t' for stage 2).
* Q15 diffuse scattering: rho_w = sum_{xi.n>0} (xi.n) f-bar /
      [ - sum_{xi.n<0} (xi.n) feq(xi; 1, u_w) ].
* Q16 stencil ghosts beyond a wall: quadratic extrapolation along the wall
      normal, g_{-1} = 3 g_0 - 3 g_1 + g_2 (corners: both directions).
* Q26 T2S2 (Sec. 3, the second-order comparison method that Remark I
      identifies as the original DUGKS; its reconstruction is not printed):
      the original DUGKS interpolation f-bar^+(x_b - xi h) = f-bar^+(x_b) -
      xi h . grad f-bar^+(x_b), face value and gradient interpolated linearly
      between the two cells of the face (``recon="central"``); beyond a wall
      the cell is the Q16 ghost.  It reproduces Table 1's T2S2 row to 0.02 %.
      T2S3 is the same T2 step with the reconstruction of eq. flux_DS (Q2p).
"""
from __future__ import annotations

import numpy as np

from .velocity_sets import opposite_index

PERIODIC, BOUNCEBACK, DIFFUSE = 0, 1, 2
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3

# Free parameters of the scheme (Sec. 2.1.1): a = 1/3, A = a/2 = 1/6 and
# A = (3K-2)/(6K-3)  =>  K = 3/4.  They give the coefficients used below:
SCHEME = {
    "a": 1.0 / 3.0, "A": 1.0 / 6.0, "K": 3.0 / 4.0,
    "B1": 3.0 / 7.0, "B2": 4.0 / 7.0,          # L(f*) and L(f**) weights
    "Pn": 0.0, "Pp": 3.0 / 4.0, "Pn1": 1.0 / 4.0,  # Omega(t_n), Omega(t'), Omega(t_{n+1})
}


class Setup:
    """Problem definition: uniform mesh, velocity set, tau, dt, 4 walls.

    ``bc`` is a sequence of four ``(kind, uw_x, uw_y)`` in the order
    west, east, south, north.  Periodic sides must come in pairs.
    """

    def __init__(self, nx, ny, dx, dy, xi, W, RT, tau, dt, bc, fbp="derived",
                 recon="printed"):
        self.nx, self.ny = int(nx), int(ny)
        self.dx, self.dy = float(dx), float(dy)
        self.xi = np.asarray(xi, dtype=np.float64)
        self.W = np.asarray(W, dtype=np.float64)
        self.RT = float(RT)
        self.tau, self.dt = float(tau), float(dt)
        self.bc = [(int(b[0]), float(b[1]), float(b[2])) for b in bc]
        self.fbp = fbp
        self.recon = recon            # face reconstruction of the T3S3 step
        if (self.bc[WEST][0] == PERIODIC) != (self.bc[EAST][0] == PERIODIC):
            raise ValueError("periodic x needs both west and east periodic")
        if (self.bc[SOUTH][0] == PERIODIC) != (self.bc[NORTH][0] == PERIODIC):
            raise ValueError("periodic y needs both south and north periodic")
        self.periodic_x = self.bc[WEST][0] == PERIODIC
        self.periodic_y = self.bc[SOUTH][0] == PERIODIC
        self.opp = opposite_index(self.xi)
        # per-velocity columns broadcastable against (nv, ny, nx)
        self.cx = self.xi[:, 0][:, None, None]
        self.cy = self.xi[:, 1][:, None, None]
        self.Wc = self.W[:, None, None]


# ---------------------------------------------------------------- kinetics
def moments(f, s: Setup):
    """rho = sum_k f_k, rho u = sum_k xi_k f_k (Sec. 2.2, discrete moments)."""
    rho = f.sum(axis=0)
    jx = (s.cx * f).sum(axis=0)
    jy = (s.cy * f).sum(axis=0)
    return rho, jx, jy


def equilibrium(rho, ux, uy, s: Setup):
    """Second-order Hermite/Taylor equilibrium (Sec. 2.1.1):

    feq_k = W_k rho [1 + xi.u/RT + (xi.u)^2/(2 RT^2) - |u|^2/(2 RT)].
    """
    eu = s.cx * ux + s.cy * uy
    uu = ux * ux + uy * uy
    return s.Wc * rho * (1.0 + eu / s.RT + eu * eu / (2.0 * s.RT * s.RT)
                         - uu / (2.0 * s.RT))


def equilibrium_of(f, s: Setup):
    rho, jx, jy = moments(f, s)
    return equilibrium(rho, jx / rho, jy / rho, s), rho


# ----------------------------------------------------- interface evolution
def _with_ghosts(g, s: Setup):
    """g with one ghost layer on every side (periodic wrap or Q16)."""
    if s.periodic_x:
        lo, hi = g[:, :, -1:], g[:, :, :1]
    else:
        lo = (3.0 * g[:, :, 0] - 3.0 * g[:, :, 1] + g[:, :, 2])[:, :, None]
        hi = (3.0 * g[:, :, -1] - 3.0 * g[:, :, -2] + g[:, :, -3])[:, :, None]
    gx = np.concatenate([lo, g, hi], axis=2)
    if s.periodic_y:
        lo, hi = gx[:, -1:, :], gx[:, :1, :]
    else:
        lo = (3.0 * gx[:, 0, :] - 3.0 * gx[:, 1, :] + gx[:, 2, :])[:, None, :]
        hi = (3.0 * gx[:, -1, :] - 3.0 * gx[:, -2, :] + gx[:, -3, :])[:, None, :]
    return np.concatenate([lo, gx, hi], axis=1)


def cell_derivatives(g, s: Setup):
    """Value, gradient and Hessian of g at every cell centre (Q3):
    second-order central differences on the 3x3 neighbourhood."""
    ge = _with_ghosts(g, s)
    C = ge[:, 1:-1, 1:-1]
    E, Wd = ge[:, 1:-1, 2:], ge[:, 1:-1, :-2]
    N, S = ge[:, 2:, 1:-1], ge[:, :-2, 1:-1]
    NE, NW = ge[:, 2:, 2:], ge[:, 2:, :-2]
    SE, SW = ge[:, :-2, 2:], ge[:, :-2, :-2]
    dx, dy = s.dx, s.dy
    gx = (E - Wd) / (2.0 * dx)
    gy = (N - S) / (2.0 * dy)
    gxx = (E - 2.0 * C + Wd) / (dx * dx)
    gyy = (N - 2.0 * C + S) / (dy * dy)
    gxy = (NE - NW - SE + SW) / (4.0 * dx * dy)
    return C, gx, gy, gxx, gxy, gyy


def taylor(d, dX, dY):
    """Quadratic Taylor series about a cell centre (reading Q2: eq. flux_DS
    with the factor 1/2), kept for comparison with Q2p."""
    C, gx, gy, gxx, gxy, gyy = d
    return C + dX * gx + dY * gy + 0.5 * (dX * dX * gxx + 2.0 * dX * dY * gxy
                                          + dY * dY * gyy)


def taylor_printed(d, dX, dY):
    """eq. flux_DS as printed (Q2p): the second-order term is the full double
    contraction (x_b - xi h - x_j)^2 : grad^2 f, without a factor 1/2."""
    C, gx, gy, gxx, gxy, gyy = d
    return C + dX * gx + dY * gy + (dX * dX * gxx + 2.0 * dX * dY * gxy + dY * dY * gyy)


def _feq_unit(s: Setup, uwx, uwy):
    """feq(xi_k; rho=1, u_w) as a (nv,) vector."""
    eu = s.xi[:, 0] * uwx + s.xi[:, 1] * uwy
    uu = uwx * uwx + uwy * uwy
    return s.W * (1.0 + eu / s.RT + eu * eu / (2.0 * s.RT * s.RT) - uu / (2.0 * s.RT))


def _wall(fluid, rho_adj, xn, s: Setup, bc):
    """f-bar at a wall face (Q12, Q13).

    ``fluid``: (nv, m) reconstruction from the fluid cell for every velocity;
    ``rho_adj``: (m,) density of the wall-adjacent cells (Q14);
    ``xn``: (nv,) xi_k . n with n the outward normal of the fluid.
    """
    kind, uwx, uwy = bc
    out = xn < 0.0                       # leaving the wall
    inc = xn > 0.0                       # hitting the wall
    fb = fluid.copy()
    if kind == BOUNCEBACK:               # eq. BB applied to f-bar
        eu = s.xi[:, 0] * uwx + s.xi[:, 1] * uwy
        for k in np.nonzero(out)[0]:
            fb[k] = fluid[s.opp[k]] + 2.0 * rho_adj * s.W[k] * eu[k] / s.RT
    elif kind == DIFFUSE:                # diffuse scattering with Q15
        fu = _feq_unit(s, uwx, uwy)
        num = (xn[inc][:, None] * fluid[inc]).sum(axis=0)
        den = -(xn[out] * fu[out]).sum()
        rho_w = num / den
        fb[out] = fu[out][:, None] * rho_w[None, :]
    else:
        raise ValueError("not a wall")
    return fb


RECONS = ("printed", "quadratic", "central")


def _central_faces(g, h, s: Setup):
    """Original DUGKS reconstruction (Remark I's second-order method, T2S2):
    f-bar^+(x_b - xi h) = f-bar^+(x_b) - xi h . grad f-bar^+(x_b) with the
    face value and gradient by linear interpolation between the two cells of
    the face -- value (g_L + g_R)/2, normal derivative (g_R - g_L)/dx,
    tangential derivative the mean of the two cells' central differences.
    Beyond a wall the cell is the Q16 ghost.  Returns (fbx, fby) without the
    wall rule applied."""
    ge = _with_ghosts(g, s)                       # (nv, ny+2, nx+2)
    # x-faces i = 0..nx between ghosted columns i and i+1, rows 1..ny
    L, R = ge[:, 1:-1, :-1], ge[:, 1:-1, 1:]
    gy_all = (ge[:, 2:, :] - ge[:, :-2, :]) / (2.0 * s.dy)   # (nv, ny, nx+2)
    gt = 0.5 * (gy_all[:, :, :-1] + gy_all[:, :, 1:])
    fbx = 0.5 * (L + R) - s.cx * h * (R - L) / s.dx - s.cy * h * gt
    # y-faces j = 0..ny between ghosted rows j and j+1, columns 1..nx
    B, T = ge[:, :-1, 1:-1], ge[:, 1:, 1:-1]
    gx_all = (ge[:, :, 2:] - ge[:, :, :-2]) / (2.0 * s.dx)   # (nv, ny+2, nx)
    gt = 0.5 * (gx_all[:, :-1, :] + gx_all[:, 1:, :])
    fby = 0.5 * (B + T) - s.cy * h * (T - B) / s.dy - s.cx * h * gt
    return fbx, fby


def interface_fbar(g, h, rho_base, s: Setup, recon="printed"):
    """f-bar(x_b, t+h) = f-bar^{+,h}(x_b - xi h, t) on every face
    (eqs. interfaceEvof and flux_DS), given g = f-bar^{+,h}(t) at the cells.

    Returns (fbx, fby): x-faces (nv, ny, nx+1) at x = i dx and y-faces
    (nv, ny+1, nx) at y = j dy.  ``recon`` selects the reconstruction:

    * ``"printed"`` (T3S3, T2S3): eq. flux_DS exactly as printed (Q2p),
      expanded about the upwind cell chosen by the sign of xi.n; Q4 for
      xi.n == 0.
    * ``"quadratic"``: the same with the factor 1/2 on the second-order term
      (reading Q2, for comparison).
    * ``"central"``: the original DUGKS reconstruction (T2S2, Q26).
    """
    nx, ny = s.nx, s.ny
    if recon not in RECONS:
        raise ValueError(recon)
    if recon == "central":
        fbx, fby = _central_faces(g, h, s)
        fromL = fromR = fbx
        fromB = fromT = fby
    else:
        taylor_ = {"quadratic": taylor, "printed": taylor_printed}[recon]
        d = cell_derivatives(g, s)

        # x-faces: face i lies between cell i-1 (left) and cell i (right)
        li = (np.arange(nx + 1) - 1) % nx
        ri = np.arange(nx + 1) % nx
        dL = tuple(a[:, :, li] for a in d)
        dR = tuple(a[:, :, ri] for a in d)
        fromL = taylor_(dL, 0.5 * s.dx - s.cx * h, -s.cy * h)
        fromR = taylor_(dR, -0.5 * s.dx - s.cx * h, -s.cy * h)
        fbx = np.where(s.cx > 0, fromL, np.where(s.cx < 0, fromR, 0.5 * (fromL + fromR)))

        # y-faces: face j lies between cell j-1 (below) and cell j (above)
        lj = (np.arange(ny + 1) - 1) % ny
        rj = np.arange(ny + 1) % ny
        dB = tuple(a[:, lj, :] for a in d)
        dT = tuple(a[:, rj, :] for a in d)
        fromB = taylor_(dB, -s.cx * h, 0.5 * s.dy - s.cy * h)
        fromT = taylor_(dT, -s.cx * h, -0.5 * s.dy - s.cy * h)
        fby = np.where(s.cy > 0, fromB, np.where(s.cy < 0, fromT, 0.5 * (fromB + fromT)))
    if not s.periodic_x:
        fbx[:, :, 0] = _wall(fromR[:, :, 0], rho_base[:, 0], -s.xi[:, 0], s, s.bc[WEST])
        fbx[:, :, nx] = _wall(fromL[:, :, nx], rho_base[:, nx - 1], s.xi[:, 0], s, s.bc[EAST])
    if not s.periodic_y:
        fby[:, 0, :] = _wall(fromT[:, 0, :], rho_base[0, :], -s.xi[:, 1], s, s.bc[SOUTH])
        fby[:, ny, :] = _wall(fromB[:, ny, :], rho_base[ny - 1, :], s.xi[:, 1], s, s.bc[NORTH])
    return fbx, fby


def recover_f(fbar, h, s: Setup):
    """f = 2 tau/(2 tau + h) f-bar + h/(2 tau + h) feq (eq. recover2f),
    feq from the moments of f-bar at the face (Q9)."""
    feq, _ = equilibrium_of(fbar, s)
    return (2.0 * s.tau * fbar + h * feq) / (2.0 * s.tau + h)


def microflux(fx, fy, s: Setup):
    """L_j = -(1/|V_j|) oint (xi.n) f dS, midpoint rule on the four faces (Q1)."""
    return -(s.cx * (fx[:, :, 1:] - fx[:, :, :-1]) / s.dx
             + s.cy * (fy[:, 1:, :] - fy[:, :-1, :]) / s.dy)


def flux_from_g(g, h, rho_base, s: Setup, recon="printed"):
    """The DUGKS reconstruction chain: g -> f-bar(x_b) -> f(x_b) -> L."""
    fbx, fby = interface_fbar(g, h, rho_base, s, recon)
    return microflux(recover_f(fbx, h, s), recover_f(fby, h, s), s)


# ------------------------------------------------------------ T3S3 step
def t3s3_step(fhat, s: Setup, trace=None):
    """One T3S3 step f^(t_n) -> f^(t_{n+1}) (Sec. 2.1.3, Steps (1)-(4))."""
    tau, dt = s.tau, s.dt

    # Step (1): L* at t* = t_n + dt/6
    feq_n, rho_n = equilibrium_of(fhat, s)
    g1 = ((12.0 * tau - dt) * fhat + 4.0 * dt * feq_n) / (12.0 * tau + 3.0 * dt)
    L1 = flux_from_g(g1, dt / 6.0, rho_n, s, s.recon)

    # Step (2): T2 step of size dt/3 to t' = t_n + dt/3, then dt*Omega(f')
    ft_plus = 1.25 * g1 - 0.25 * fhat                       # Q5
    ft_prime = ft_plus + (dt / 3.0) * L1                     # Q7
    feq_p, rho_p = equilibrium_of(ft_prime, s)
    dtOmega_p = -6.0 * dt / (6.0 * tau + dt) * (ft_prime - feq_p)

    # Step (3): L** at t** = t_n + 3 dt/4 from f~(t'), h = 5 dt/12
    if s.fbp == "derived":                                   # Q6
        g2 = ((24.0 * tau - 5.0 * dt) * ft_prime + 9.0 * dt * feq_p) / (24.0 * tau + 4.0 * dt)
    else:
        g2 = ((24.0 * tau - 5.0 * dt) * ft_prime + 15.0 * dt * feq_p) / (24.0 * tau + 10.0 * dt)
    L2 = flux_from_g(g2, 5.0 * dt / 12.0, rho_p, s, s.recon)

    # Step (4)
    fhat_plus = 0.25 * fhat + 0.75 * g1
    out = fhat_plus + 0.75 * dtOmega_p + (dt / 7.0) * (3.0 * L1 + 4.0 * L2)
    if trace is not None:
        trace.update(g1=g1, L1=L1, ft_plus=ft_plus, ft_prime=ft_prime,
                     dtOmega_p=dtOmega_p, g2=g2, L2=L2, fhat_plus=fhat_plus,
                     feq_n=feq_n, feq_p=feq_p)
    return out


def t3s3_run(fhat, s: Setup, nsteps: int):
    f = np.array(fhat, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        f = t3s3_step(f, s)
    return f


# ------------------------------------------------ T2 step (Remark I)
def t2_step(ftilde, s: Setup, delta: float, recon="printed"):
    """Original DUGKS time step of size ``delta`` (Remark I, eq.
    feqIntD2nd_Explicit with Q7) at h = delta/2:
    f~^{n+1} = f~^{+,n} + delta * L(t_n + delta/2); the reconstruction of
    eq. flux_DS (Q2p) gives T2S3, ``recon="central"`` (Q26) gives T2S2.

    Works on f~ = f - delta/2 Omega.
    """
    tau = s.tau
    feq, rho = equilibrium_of(ftilde, s)
    h = 0.5 * delta
    # f-bar^{+,h} from f~ (x = f - (h) Omega here since delta/2 = h):
    # f~ - feq = (f - feq)(1 + h/tau);  f-bar^{+,h} - feq = (f - feq)(1 - h/(2 tau))
    gbar = ((2.0 * tau - h) * ftilde + 3.0 * h * feq) / (2.0 * tau + 2.0 * h)
    L = flux_from_g(gbar, h, rho, s, recon)
    ft_plus = ((2.0 * tau - delta) * ftilde + 2.0 * delta * feq) / (2.0 * tau + delta)
    return ft_plus + delta * L


def t2_run(ftilde, s: Setup, nsteps: int, recon="printed"):
    """nsteps T2 steps of size s.dt (T2S3, or T2S2 with recon="central")."""
    f = np.array(ftilde, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        f = t2_step(f, s, s.dt, recon)
    return f


def ftilde_from_f(f, s: Setup):
    """f~ = f - dt/2 Omega(f) = f + dt/(2 tau) (f - feq(f)), the T2 state."""
    feq, _ = equilibrium_of(f, s)
    return f + s.dt / (2.0 * s.tau) * (f - feq)


# ---------------------------------------------------------- conversions
def fhat_from_f(f, s: Setup):
    """f^ = f - dt/4 Omega(f) = f + dt/(4 tau) (f - feq(f))."""
    feq, _ = equilibrium_of(f, s)
    return f + s.dt / (4.0 * s.tau) * (f - feq)


def f_from_fhat(fhat, s: Setup):
    """f = 4 tau/(4 tau + dt) f^ + dt/(4 tau + dt) feq (the useful equation
    for f^+ after eq. feqIntD3rdHat2, since f^+ = f)."""
    feq, _ = equilibrium_of(fhat, s)
    return (4.0 * s.tau * fhat + s.dt * feq) / (4.0 * s.tau + s.dt)


def equilibrium_state(rho, ux, uy, s: Setup):
    """f^ for an initial state at equilibrium (Sec. 3: f = feq, so f^ = feq)."""
    return equilibrium(np.asarray(rho, float), np.asarray(ux, float),
                       np.asarray(uy, float), s)


def velocity(fhat, s: Setup):
    rho, jx, jy = moments(fhat, s)
    return rho, jx / rho, jy / rho


def stability_factor(D):
    """P^_n of Sec. 2.1.1 at a = 1/3 (von Neumann amplification of the
    non-equilibrium part with L neglected), D = dt/tau."""
    a = 1.0 / 3.0
    return abs((-3 * a * a * D * D + 13 * a * D * D + 10 * a * D - 22 * D + 32)
               / (4 * (a * D + 2) * (D + 4)))
