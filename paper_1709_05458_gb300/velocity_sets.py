"""Discrete velocity sets for ``dugks_init`` (Sec. 2.2 of arXiv:1709.05458).

Each builder returns ``(xi, W, RT)``: velocities (nv, 2), equilibrium weights
W_k (the Gauss-Hermite weight, or the Newton-Cotes quadrature weight times
the Maxwellian factor), and the RT to pass to the library.

* :func:`d2q9` -- tensor product of the 3-point Gauss-Hermite rule,
  xi = sqrt(3RT) {-1,0,1}^2, 2-D weights 1/36 (corners), 1/9 (axes),
  4/9 (rest), ordered x-major as the paper lists them.
* :func:`newton_cotes` -- uniform n x n grid on [-v, v]^2, v = vmax sqrt(RT),
  with a composite closed Newton-Cotes rule per axis (Boole when n-1 is a
  multiple of 4, else Simpson-3/8 when a multiple of 3, else Simpson-1/3 when
  even, else Simpson-1/3 plus one 3/8 panel, symmetrised by averaging with its
  mirror image).  ``normalize`` rescales W to sum to one and returns the
  discrete second moment as RT, which makes the discrete collision exactly
  conservative on the truncated grid.
"""
from __future__ import annotations

import math

import numpy as np

_D2Q9_UNIT = [(-1, -1, 1 / 36), (-1, 0, 1 / 9), (-1, 1, 1 / 36),
              (0, -1, 1 / 9), (0, 0, 4 / 9), (0, 1, 1 / 9),
              (1, -1, 1 / 36), (1, 0, 1 / 9), (1, 1, 1 / 36)]


def d2q9(RT: float):
    c = math.sqrt(3.0 * RT)
    xi = np.array([[c * a, c * b] for a, b, _ in _D2Q9_UNIT], dtype=np.float64)
    W = np.array([w for _, _, w in _D2Q9_UNIT], dtype=np.float64)
    return xi, W, float(RT)


_PANELS = {
    4: (2.0 / 45.0, (7.0, 32.0, 12.0, 32.0, 7.0)),   # Boole
    3: (3.0 / 8.0, (1.0, 3.0, 3.0, 1.0)),            # Simpson 3/8
    2: (1.0 / 3.0, (1.0, 4.0, 1.0)),                 # Simpson 1/3
}


def _nc_weights(n: int, h: float) -> np.ndarray:
    m = n - 1
    w = np.zeros(n)

    def add(start, width):
        scale, coef = _PANELS[width]
        w[start:start + width + 1] += h * scale * np.asarray(coef)

    for width in (4, 3, 2):
        if m % width == 0:
            for s in range(0, m, width):
                add(s, width)
            return w
    for s in range(0, m - 3, 2):
        add(s, 2)
    add(m - 3, 3)
    return 0.5 * (w + w[::-1])


def newton_cotes(n: int, RT: float, vmax: float = 4.0, normalize: bool = True):
    if n < 3:
        raise ValueError("need at least 3 nodes per axis")
    v = vmax * math.sqrt(RT)
    h = 2.0 * v / (n - 1)
    x = -v + h * np.arange(n, dtype=np.float64)
    w1 = _nc_weights(n, h)
    X = np.repeat(x, n)
    Y = np.tile(x, n)
    Wq = np.repeat(w1, n) * np.tile(w1, n)
    W = Wq * np.exp(-(X * X + Y * Y) / (2.0 * RT)) / (2.0 * math.pi * RT)
    RT_out = float(RT)
    if normalize:
        W = W / W.sum()
        RT_out = float(np.sum(W * X * X))
    return np.stack([X, Y], axis=1), W, RT_out
