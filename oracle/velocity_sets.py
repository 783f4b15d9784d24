"""Discrete velocity sets for the oracle (test infrastructure only).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import anything under
``oracle/``.  The product path never does.

A velocity set is the triple ``(xi, W, RT)``:

* ``xi`` -- array (N_xi, 2) of discrete particle velocities,
* ``W``  -- array (N_xi,) of the weights that multiply the equilibrium
  polynomial, i.e. the quadrature weight times the Maxwellian factor
  ``exp(-|xi|^2 / 2RT) / (2 pi RT)`` ("absorbed" weights),
* ``RT`` -- the gas constant times temperature used in the equilibrium.

Sec. 2.2 of the paper (discrete particle velocities):

* continuum flows use the tensor product of the three-point Gauss-Hermite
  rule, ``xi = sqrt(3RT) * {-1, 0, 1}``, giving the D2Q9 set with 2-D
  weights ``{1/36, 1/9, 4/9}``.  The 1-D weights are printed as
  ``{1/3, 2/3, 1/3}``, which neither sum to one nor give the printed 2-D
  weights; the reading here (Q23) takes the printed 2-D table, i.e. the
  standard 1-D Gauss-Hermite weights ``{1/6, 2/3, 1/6}``;
* rarefied flows use a uniform tensor grid with Newton-Cotes weights.

The paper does not say which composite Newton-Cotes rule it uses nor how the
quadrature is folded into the equilibrium weights.  The reading used here:
composite Boole if (n-1) % 4 == 0, else composite Simpson-3/8 if
(n-1) % 3 == 0, else composite Simpson-1/3 if (n-1) is even, else Simpson-1/3
on the first n-4 intervals plus one 3/8 panel on the last 3, averaged with its
mirror image so that the rule stays symmetric (odd moments vanish).  With
``normalize=True`` the weights are scaled so that ``sum W = 1`` and ``RT`` is
replaced by the discrete second moment ``sum W xi_x^2`` so that the BGK
collision conserves mass and momentum exactly on the truncated grid.
"""
from __future__ import annotations

import numpy as np


def d2q9(RT: float):
    """D2Q9 Gauss-Hermite set of Sec. 2.2 in the paper's ordering.

    The paper lists the velocities column by column as
    ``xi_x = c*(-1,-1,-1, 0,0,0, 1,1,1)``, ``xi_y = c*(-1,0,1, -1,0,1, -1,0,1)``
    with ``c = sqrt(3RT)`` and weights ``(1/36,1/9,1/36, 1/9,4/9,1/9,
    1/36,1/9,1/36)``.
    """
    c = np.sqrt(3.0 * RT)
    ex = np.array([-1, -1, -1, 0, 0, 0, 1, 1, 1], dtype=np.float64)
    ey = np.array([-1, 0, 1, -1, 0, 1, -1, 0, 1], dtype=np.float64)
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}   # Q23
    W = np.array([w1[int(a)] * w1[int(b)] for a, b in zip(ex, ey)])
    xi = np.stack([c * ex, c * ey], axis=1)
    return xi, W, float(RT)


def newton_cotes_1d(n: int, a: float, b: float):
    """Nodes and weights of a composite closed Newton-Cotes rule on [a, b].

    ``n`` uniformly spaced nodes including both ends.  The rule choice is the
    reading stated in the module docstring.
    """
    if n < 3:
        raise ValueError("need at least 3 nodes")
    m = n - 1                      # number of intervals
    h = (b - a) / m
    x = a + h * np.arange(n, dtype=np.float64)
    w = np.zeros(n)

    def panel(start, coeffs, scale):
        for k, c in enumerate(coeffs):
            w[start + k] += scale * c * h

    if m % 4 == 0:                                  # composite Boole
        for p in range(0, m, 4):
            panel(p, (7, 32, 12, 32, 7), 2.0 / 45.0)
    elif m % 3 == 0:                                # composite Simpson 3/8
        for p in range(0, m, 3):
            panel(p, (1, 3, 3, 1), 3.0 / 8.0)
    elif m % 2 == 0:                                # composite Simpson 1/3
        for p in range(0, m, 2):
            panel(p, (1, 4, 1), 1.0 / 3.0)
    else:                                           # Simpson 1/3 + one 3/8 panel
        for p in range(0, m - 3, 2):
            panel(p, (1, 4, 1), 1.0 / 3.0)
        panel(m - 3, (1, 3, 3, 1), 3.0 / 8.0)
        w = 0.5 * (w + w[::-1])
    return x, w


def newton_cotes_2d(n: int, RT: float, vmax_over_sqrtRT: float = 4.0,
                    normalize: bool = True):
    """Tensor Newton-Cotes velocity grid on [-v, v]^2, v = vmax*sqrt(RT).

    Velocity index k = ix * n + iy (x-major, same ordering convention as the
    D2Q9 listing).  Returns ``(xi, W, RT_eff)``.
    """
    v = vmax_over_sqrtRT * np.sqrt(RT)
    x1, w1 = newton_cotes_1d(n, -v, v)
    gx, gy = np.meshgrid(x1, x1, indexing="ij")
    wx, wy = np.meshgrid(w1, w1, indexing="ij")
    xi = np.stack([gx.ravel(), gy.ravel()], axis=1)
    maxw = np.exp(-(xi[:, 0] ** 2 + xi[:, 1] ** 2) / (2.0 * RT)) / (2.0 * np.pi * RT)
    W = (wx * wy).ravel() * maxw
    RT_eff = float(RT)
    if normalize:
        W = W / W.sum()
        RT_eff = float(np.sum(W * xi[:, 0] ** 2))
    return xi, W, RT_eff


def opposite_index(xi: np.ndarray) -> np.ndarray:
    """Index of -xi_k for every k (-1 if the set has no such velocity)."""
    opp = -np.ones(len(xi), dtype=np.int64)
    for k in range(len(xi)):
        d = np.abs(xi + xi[k]).sum(axis=1)
        j = int(np.argmin(d))
        if d[j] <= 1e-12 * (1.0 + np.abs(xi[k]).sum()):
            opp[k] = j
    return opp
