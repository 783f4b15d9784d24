"""Run the oracle on the Taylor vortex of Table 1 and print E(u).

TEST INFRASTRUCTURE: calls only ``oracle/`` (and numpy).  It writes the
oracle's Table 1 figures recorded in ``table1_oracle.txt`` beside it.

The setting is the paper's (Sec. 3.1, Table 1): [0, 1]^2 periodic, D2Q9,
A = B = 2 pi, u0 = 1, nu = 0.01, dt = 1e-5, dt/tau = 4 (so RT = nu/tau =
4000 with nu = tau RT), Chapman-Enskog initial state, E(u) at t = 1 s
(1e5 steps).  One line per run:

    scheme recon N E(u) steps seconds

  python tests/golden/table1_oracle.py t3s3 printed 32
  python tests/golden/table1_oracle.py t2 central 64 --steps 20000
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import dugks_oracle as O  # noqa: E402
from oracle import tgv  # noqa: E402
from oracle import velocity_sets as OV  # noqa: E402

NU, DT, U0 = 0.01, 1e-5, 1.0


def run(scheme: str, recon: str, N: int, steps: int = 100_000):
    tau = DT / 4.0
    RT = NU / tau
    xi, W, _ = OV.d2q9(RT)
    s = O.Setup(N, N, 1.0 / N, 1.0 / N, xi, W, RT, tau, DT, [(O.PERIODIC, 0, 0)] * 4,
                recon=recon)
    f = tgv.chapman_enskog_f(s, U0, NU)
    if scheme == "t3s3":
        out = O.t3s3_run(O.fhat_from_f(f, s), s, steps)
    elif scheme == "t2":
        out = O.t2_run(O.ftilde_from_f(f, s), s, steps, recon)
    else:
        raise ValueError(scheme)
    return tgv.error_L2(out, s, steps * DT, U0, NU)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("scheme", choices=["t3s3", "t2"])
    ap.add_argument("recon", choices=list(O.RECONS))
    ap.add_argument("N", type=int)
    ap.add_argument("--steps", type=int, default=100_000)
    a = ap.parse_args()
    t0 = time.time()
    e = run(a.scheme, a.recon, a.N, a.steps)
    print(f"{a.scheme} {a.recon} {a.N} {e:.4e} {a.steps} {time.time() - t0:.0f}", flush=True)


if __name__ == "__main__":
    main()
