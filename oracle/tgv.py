"""Taylor-Green vortex helpers for oracle pins (test infrastructure only).

TEST INFRASTRUCTURE: only ``tests/`` and ``bench.py``'s reference arm may
import this file.

Sec. 3.1 of the paper: on [0,1]^2 with A = B = 2 pi,
  u = -(u0/A) cos(Ax) sin(By) e^{-nu alpha t},
  v =  (u0/B) sin(Ax) cos(By) e^{-nu alpha t},
  p = -(u0^2/4) [cos(2Ax)/A^2 + cos(2By)/B^2] e^{-2 nu alpha t},
alpha = A^2 + B^2, initialised by the Chapman-Enskog expansion
f = feq - tau (d_t feq + xi . grad feq), and scored by the relative global
L2 velocity error E(u).  Readings: rho = rho0 + p/RT (Q19) and nu = tau RT
(Q17).
"""
from __future__ import annotations

import numpy as np

from . import dugks_oracle as O


def fields(X, Y, t, u0, nu, RT, A=2 * np.pi, B=2 * np.pi, rho0=1.0):
    """rho, u, v and their x, y, t derivatives (analytic)."""
    al = A * A + B * B
    e1 = np.exp(-nu * al * t)
    e2 = np.exp(-2 * nu * al * t)
    u = -(u0 / A) * np.cos(A * X) * np.sin(B * Y) * e1
    v = (u0 / B) * np.sin(A * X) * np.cos(B * Y) * e1
    p = -(u0 * u0 / 4) * (np.cos(2 * A * X) / A ** 2 + np.cos(2 * B * Y) / B ** 2) * e2
    rho = rho0 + p / RT
    d = {
        "u_x": u0 * np.sin(A * X) * np.sin(B * Y) * e1,
        "u_y": -(u0 / A) * B * np.cos(A * X) * np.cos(B * Y) * e1,
        "v_x": (u0 / B) * A * np.cos(A * X) * np.cos(B * Y) * e1,
        "v_y": -u0 * np.sin(A * X) * np.sin(B * Y) * e1,
        "u_t": -nu * al * u,
        "v_t": -nu * al * v,
        "rho_x": (u0 * u0 / 4) * (2 / A) * np.sin(2 * A * X) * e2 / RT,
        "rho_y": (u0 * u0 / 4) * (2 / B) * np.sin(2 * B * Y) * e2 / RT,
        "rho_t": -2 * nu * al * p / RT,
    }
    return rho, u, v, d


def cell_centres(s: O.Setup):
    x = (np.arange(s.nx) + 0.5) * s.dx
    y = (np.arange(s.ny) + 0.5) * s.dy
    X, Y = np.meshgrid(x, y, indexing="xy")     # shape (ny, nx)
    return X, Y


def chapman_enskog_fhat(s: O.Setup, u0, nu):
    """Initial f^ = f - dt/4 Omega(f) of the Chapman-Enskog state below."""
    return O.fhat_from_f(chapman_enskog_f(s, u0, nu), s)


def chapman_enskog_f(s: O.Setup, u0, nu):
    """Initial f = feq - tau (d_t feq + xi . grad feq) (Sec. 3.1).

    The derivatives of feq follow from the chain rule through (rho, u) of
    the analytic solution.
    """
    X, Y = cell_centres(s)
    rho, u, v, d = fields(X, Y, 0.0, u0, nu, s.RT)
    RT = s.RT
    cx, cy, Wc = s.cx, s.cy, s.Wc
    eu = cx * u + cy * v
    P = 1 + eu / RT + eu * eu / (2 * RT * RT) - (u * u + v * v) / (2 * RT)

    def dfeq(dr, du, dv):
        deu = cx * du + cy * dv
        dP = deu / RT + eu * deu / (RT * RT) - (u * du + v * dv) / RT
        return Wc * (dr * P + rho * dP)

    feq = Wc * rho * P
    ft = dfeq(d["rho_t"], d["u_t"], d["v_t"])
    fx = dfeq(d["rho_x"], d["u_x"], d["v_x"])
    fy = dfeq(d["rho_y"], d["u_y"], d["v_y"])
    return feq - s.tau * (ft + cx * fx + cy * fy)


def error_L2(fhat, s: O.Setup, t, u0, nu):
    """E(u) of Sec. 3.1 against the analytic solution at time t."""
    X, Y = cell_centres(s)
    _, ua, va, _ = fields(X, Y, t, u0, nu, s.RT)
    _, u, v = O.velocity(fhat, s)
    num = np.sqrt(np.sum((u - ua) ** 2 + (v - va) ** 2))
    den = np.sqrt(np.sum(ua ** 2 + va ** 2))
    return num / den
