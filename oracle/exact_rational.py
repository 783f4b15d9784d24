"""Exact-rational brute-force T3S3 step for tiny grids (test infrastructure).

TEST INFRASTRUCTURE: only ``tests/`` may use this file.  It is a second,
independent restatement of one T3S3 step (arXiv:1709.05458, Sec. 2.1.3,
Steps (1)-(4)) written as scalar loops over cells, faces and velocities in
exact ``fractions.Fraction`` arithmetic.  It is used to pin the vectorised
FP64 oracle (``dugks_oracle.py``) on 4x4 grids: any index, sign or
coefficient slip in either restatement makes them disagree.

It follows the same readings of the paper (Q1-Q16 and Q2p in
``dugks_oracle.py``).
Velocity sets must have rational velocities and weights (D2Q9 with RT = 1/3
gives xi in {-1, 0, 1}).
"""
from __future__ import annotations

from fractions import Fraction as Fr

PERIODIC, BOUNCEBACK, DIFFUSE = 0, 1, 2


class ExactSetup:
    def __init__(self, nx, ny, dx, dy, xi, W, RT, tau, dt, bc):
        self.nx, self.ny = nx, ny
        self.dx, self.dy = Fr(dx), Fr(dy)
        self.xi = [(Fr(a), Fr(b)) for a, b in xi]
        self.W = [Fr(w) for w in W]
        self.RT = Fr(RT)
        self.tau, self.dt = Fr(tau), Fr(dt)
        self.bc = [(k, Fr(ux), Fr(uy)) for k, ux, uy in bc]   # W, E, S, N
        self.nv = len(self.xi)
        self.opp = []
        for k in range(self.nv):
            m = [q for q in range(self.nv) if self.xi[q] == (-self.xi[k][0], -self.xi[k][1])]
            self.opp.append(m[0] if m else -1)


def _zeros(s, ny, nx):
    return [[[Fr(0)] * nx for _ in range(ny)] for _ in range(s.nv)]


def feq_point(s, k, rho, ux, uy):
    cx, cy = s.xi[k]
    eu = cx * ux + cy * uy
    return s.W[k] * rho * (1 + eu / s.RT + eu * eu / (2 * s.RT * s.RT)
                           - (ux * ux + uy * uy) / (2 * s.RT))


def cell_moments(s, f):
    out = {}
    for j in range(s.ny):
        for i in range(s.nx):
            rho = sum(f[k][j][i] for k in range(s.nv))
            jx = sum(s.xi[k][0] * f[k][j][i] for k in range(s.nv))
            jy = sum(s.xi[k][1] * f[k][j][i] for k in range(s.nv))
            out[(j, i)] = (rho, jx / rho, jy / rho)
    return out


def _gval(s, g, k, j, i):
    """g at cell (j, i) with one ghost layer: wrap or quadratic extrapolation."""
    px = s.bc[0][0] == PERIODIC
    py = s.bc[2][0] == PERIODIC
    if i < 0 or i >= s.nx:
        if px:
            i %= s.nx
        else:
            a, b, c = (0, 1, 2) if i < 0 else (s.nx - 1, s.nx - 2, s.nx - 3)
            return 3 * _gval(s, g, k, j, a) - 3 * _gval(s, g, k, j, b) + _gval(s, g, k, j, c)
    if j < 0 or j >= s.ny:
        if py:
            j %= s.ny
        else:
            a, b, c = (0, 1, 2) if j < 0 else (s.ny - 1, s.ny - 2, s.ny - 3)
            return 3 * g[k][a][i] - 3 * g[k][b][i] + g[k][c][i]
    return g[k][j][i]


def _expand(s, g, k, j, i, ddx, ddy):
    """eq. flux_DS as printed (reading Q2p) at centre(j, i) + (ddx, ddy):
    value + d.grad + d^2 : grad^2, no factor 1/2 on the second-order term."""
    G = lambda a, b: _gval(s, g, k, j + b, i + a)   # noqa: E731  (a: x offset)
    c = G(0, 0)
    gx = (G(1, 0) - G(-1, 0)) / (2 * s.dx)
    gy = (G(0, 1) - G(0, -1)) / (2 * s.dy)
    gxx = (G(1, 0) - 2 * c + G(-1, 0)) / (s.dx * s.dx)
    gyy = (G(0, 1) - 2 * c + G(0, -1)) / (s.dy * s.dy)
    gxy = (G(1, 1) - G(-1, 1) - G(1, -1) + G(-1, -1)) / (4 * s.dx * s.dy)
    return (c + ddx * gx + ddy * gy
            + (ddx * ddx * gxx + 2 * ddx * ddy * gxy + ddy * ddy * gyy))


def _face_value(s, g, k, cell_a, cell_b, normal_axis, h):
    """f-bar at the face between cell_a (lower index side) and cell_b."""
    cx, cy = s.xi[k]
    ja, ia = cell_a
    jb, ib = cell_b
    if normal_axis == 0:
        va = _expand(s, g, k, ja, ia, s.dx / 2 - cx * h, -cy * h)
        vb = _expand(s, g, k, jb, ib, -s.dx / 2 - cx * h, -cy * h)
        cn = cx
    else:
        va = _expand(s, g, k, ja, ia, -cx * h, s.dy / 2 - cy * h)
        vb = _expand(s, g, k, jb, ib, -cx * h, -s.dy / 2 - cy * h)
        cn = cy
    if cn > 0:
        return va
    if cn < 0:
        return vb
    return (va + vb) / 2


def _wall_face(s, g, k_all_fluid, rho_adj, normal, bc):
    kind, uwx, uwy = bc
    nx_, ny_ = normal
    fb = list(k_all_fluid)
    xn = [s.xi[k][0] * nx_ + s.xi[k][1] * ny_ for k in range(s.nv)]
    if kind == BOUNCEBACK:
        for k in range(s.nv):
            if xn[k] < 0:
                eu = s.xi[k][0] * uwx + s.xi[k][1] * uwy
                fb[k] = k_all_fluid[s.opp[k]] + 2 * rho_adj * s.W[k] * eu / s.RT
    elif kind == DIFFUSE:
        num = sum(xn[k] * k_all_fluid[k] for k in range(s.nv) if xn[k] > 0)
        den = -sum(xn[k] * feq_point(s, k, 1, uwx, uwy) for k in range(s.nv) if xn[k] < 0)
        rw = num / den
        for k in range(s.nv):
            if xn[k] < 0:
                fb[k] = rw * feq_point(s, k, 1, uwx, uwy)
    return fb


def _recover(s, fbar_list, h):
    rho = sum(fbar_list)
    ux = sum(s.xi[k][0] * fbar_list[k] for k in range(s.nv)) / rho
    uy = sum(s.xi[k][1] * fbar_list[k] for k in range(s.nv)) / rho
    return [(2 * s.tau * fbar_list[k] + h * feq_point(s, k, rho, ux, uy)) / (2 * s.tau + h)
            for k in range(s.nv)]


def flux(s, g, h, mom):
    """L for every (k, cell) from g = f-bar^{+,h} at the cells."""
    nx, ny = s.nx, s.ny
    px = s.bc[0][0] == PERIODIC
    py = s.bc[2][0] == PERIODIC
    # x-faces i = 0..nx, between cell i-1 and i
    FX = {}
    for j in range(ny):
        for i in range(nx + 1):
            if not px and i == 0:
                fl = [_expand(s, g, k, j, 0, -s.dx / 2 - s.xi[k][0] * h, -s.xi[k][1] * h)
                      for k in range(s.nv)]
                fbar = _wall_face(s, g, fl, mom[(j, 0)][0], (-1, 0), s.bc[0])
            elif not px and i == nx:
                fl = [_expand(s, g, k, j, nx - 1, s.dx / 2 - s.xi[k][0] * h, -s.xi[k][1] * h)
                      for k in range(s.nv)]
                fbar = _wall_face(s, g, fl, mom[(j, nx - 1)][0], (1, 0), s.bc[1])
            else:
                fbar = [_face_value(s, g, k, (j, (i - 1) % nx), (j, i % nx), 0, h)
                        for k in range(s.nv)]
            FX[(j, i)] = _recover(s, fbar, h)
    FY = {}
    for j in range(ny + 1):
        for i in range(nx):
            if not py and j == 0:
                fl = [_expand(s, g, k, 0, i, -s.xi[k][0] * h, -s.dy / 2 - s.xi[k][1] * h)
                      for k in range(s.nv)]
                fbar = _wall_face(s, g, fl, mom[(0, i)][0], (0, -1), s.bc[2])
            elif not py and j == ny:
                fl = [_expand(s, g, k, ny - 1, i, -s.xi[k][0] * h, s.dy / 2 - s.xi[k][1] * h)
                      for k in range(s.nv)]
                fbar = _wall_face(s, g, fl, mom[(ny - 1, i)][0], (0, 1), s.bc[3])
            else:
                fbar = [_face_value(s, g, k, ((j - 1) % ny, i), (j % ny, i), 1, h)
                        for k in range(s.nv)]
            FY[(j, i)] = _recover(s, fbar, h)
    L = _zeros(s, ny, nx)
    for k in range(s.nv):
        cx, cy = s.xi[k]
        for j in range(ny):
            for i in range(nx):
                L[k][j][i] = -(cx * (FX[(j, i + 1)][k] - FX[(j, i)][k]) / s.dx
                               + cy * (FY[(j + 1, i)][k] - FY[(j, i)][k]) / s.dy)
    return L


def t3s3_step(s, fhat):
    tau, dt = s.tau, s.dt
    nv, nx, ny = s.nv, s.nx, s.ny
    mom = cell_moments(s, fhat)
    g1 = _zeros(s, ny, nx)
    for k in range(nv):
        for j in range(ny):
            for i in range(nx):
                rho, ux, uy = mom[(j, i)]
                fe = feq_point(s, k, rho, ux, uy)
                g1[k][j][i] = ((12 * tau - dt) * fhat[k][j][i] + 4 * dt * fe) / (12 * tau + 3 * dt)
    L1 = flux(s, g1, dt / 6, mom)
    ftp = _zeros(s, ny, nx)
    for k in range(nv):
        for j in range(ny):
            for i in range(nx):
                ftp[k][j][i] = (Fr(5, 4) * g1[k][j][i] - Fr(1, 4) * fhat[k][j][i]
                                + dt / 3 * L1[k][j][i])
    mom2 = cell_moments(s, ftp)
    g2 = _zeros(s, ny, nx)
    om = _zeros(s, ny, nx)
    for k in range(nv):
        for j in range(ny):
            for i in range(nx):
                rho, ux, uy = mom2[(j, i)]
                fe = feq_point(s, k, rho, ux, uy)
                om[k][j][i] = -6 * dt / (6 * tau + dt) * (ftp[k][j][i] - fe)
                g2[k][j][i] = ((24 * tau - 5 * dt) * ftp[k][j][i] + 9 * dt * fe) / (24 * tau + 4 * dt)
    L2 = flux(s, g2, 5 * dt / 12, mom2)
    out = _zeros(s, ny, nx)
    for k in range(nv):
        for j in range(ny):
            for i in range(nx):
                fp = Fr(1, 4) * fhat[k][j][i] + Fr(3, 4) * g1[k][j][i]
                out[k][j][i] = (fp + Fr(3, 4) * om[k][j][i]
                                + dt / 7 * (3 * L1[k][j][i] + 4 * L2[k][j][i]))
    return out
