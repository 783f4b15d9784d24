"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the method itself (no moments, no
equilibrium, no reconstruction): it only draws seeded random numbers and
evaluates the closed-form test fields of the paper's workloads (Taylor-Green
vortex velocity and pressure, a cavity at rest).  Both the CUDA path and the
CPU oracle take their inputs from here.

Workload recipes (synthetic stand-ins for the paper's test cases, Sec. 3):

* ``tgv``     -- 2-D periodic Taylor-Green vortex (Sec. 3.1), D2Q9;
* ``cavity``  -- lid-driven cavity with bounce-back walls (Sec. 3.3), D2Q9;
* ``rarefied``-- micro-cavity / Couette with diffuse walls on a Newton-Cotes
  velocity grid (Sec. 3.4);
* ``near_equilibrium_state`` -- a positive, smooth-plus-noise distribution
  used by the parity tests so that the non-equilibrium part is non-zero.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1709


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def smooth_random_field(nv: int, ny: int, nx: int, seed: int = SEED,
                        modes: int = 3, noise: float = 0.1) -> np.ndarray:
    """(nv, ny, nx) array, O(1) amplitude: a few random periodic Fourier
    modes per velocity plus white noise of relative size ``noise``."""
    r = rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    out = np.zeros((nv, ny, nx))
    for k in range(nv):
        for _ in range(modes):
            kx, ky = r.integers(0, 3, size=2)
            ph = r.uniform(0, 2 * math.pi)
            a = r.uniform(-1, 1)
            out[k] += a * np.cos(2 * math.pi * (kx * X + ky * Y) + ph)
    out /= modes
    out += noise * r.standard_normal((nv, ny, nx))
    return out


def near_equilibrium_state(W, ny: int, nx: int, amp: float = 0.05,
                           seed: int = SEED) -> np.ndarray:
    """f_k(x) = W_k (1 + amp * r_k(x)) with r from ``smooth_random_field``.

    ``W`` is the weight vector of the velocity set.  The result is positive
    for amp < ~0.5 and has non-zero moments and non-equilibrium parts.
    """
    W = np.asarray(W, dtype=np.float64)
    r = smooth_random_field(len(W), ny, nx, seed=seed)
    return W[:, None, None] * (1.0 + amp * r)


def cell_centres(nx: int, ny: int, Lx: float = 1.0, Ly: float = 1.0):
    x = (np.arange(nx) + 0.5) * (Lx / nx)
    y = (np.arange(ny) + 0.5) * (Ly / ny)
    return np.meshgrid(x, y, indexing="xy")


def tgv_fields(nx: int, ny: int, u0: float, RT: float, rho0: float = 1.0):
    """Taylor-Green vortex at t = 0 on [0,1]^2, A = B = 2 pi (Sec. 3.1):
    u = -(u0/A) cos(Ax) sin(By), v = (u0/B) sin(Ax) cos(By),
    p = -(u0^2/4) [cos(2Ax)/A^2 + cos(2By)/B^2], rho = rho0 + p/RT."""
    A = B = 2 * math.pi
    X, Y = cell_centres(nx, ny)
    u = -(u0 / A) * np.cos(A * X) * np.sin(B * Y)
    v = (u0 / B) * np.sin(A * X) * np.cos(B * Y)
    p = -(u0 * u0 / 4) * (np.cos(2 * A * X) / A ** 2 + np.cos(2 * B * Y) / B ** 2)
    return rho0 + p / RT, u, v


def rest_fields(nx: int, ny: int, rho0: float = 1.0):
    return (np.full((ny, nx), rho0), np.zeros((ny, nx)), np.zeros((ny, nx)))


# Boundary kinds and side order used by both implementations' interfaces.
PERIODIC, BOUNCEBACK, DIFFUSE = 0, 1, 2


def config(name: str) -> dict:
    """Parameters of the benchmark/parity workloads (dimensionless units,
    domain [0,1]^2).  Derived values follow the paper's definitions:
    dt = CFL dx / C (C = largest velocity component), Ma = U/C, Re = U L/nu,
    nu = tau RT, Kn = tau sqrt(pi RT/2) / L."""
    if name == "tgv32":
        # TGV 32^2, u amplitude 0.01 c_s, Re = 100, dt/tau = 4 (the literal
        # CFL 0.5 would give dt/tau ~ 90, beyond the stability bound 12)
        RT = 1.0 / 3.0
        U = 0.01 * math.sqrt(RT)
        nu = U / 100.0
        tau = nu / RT
        return dict(name=name, nx=32, ny=32, RT=RT, vel="d2q9", u0=U * 2 * math.pi,
                    nu=nu, tau=tau, dt=4 * tau, steps=200,
                    bc=[(PERIODIC, 0, 0)] * 4)
    if name.startswith("cavity"):
        n = int(name[len("cavity"):] or 256)
        RT = 1.0 / 3.0
        C = math.sqrt(3 * RT)
        U = 0.1 * C
        nu = U / 1000.0
        tau = nu / RT
        dt = 0.5 * (1.0 / n) / C
        return dict(name=name, nx=n, ny=n, RT=RT, vel="d2q9", U=U, nu=nu,
                    tau=tau, dt=dt, steps=20000,
                    bc=[(BOUNCEBACK, 0, 0), (BOUNCEBACK, 0, 0),
                        (BOUNCEBACK, 0, 0), (BOUNCEBACK, U, 0)])
    if name.startswith("rarefied"):
        # rarefied128_kn1_nv64 style names
        parts = name[len("rarefied"):].split("_")
        n = int(parts[0] or 128)
        kn = float(parts[1][2:]) if len(parts) > 1 else 1.0
        nv1 = int(parts[2][2:]) if len(parts) > 2 else 64
        RT = 0.5
        tau = kn / math.sqrt(math.pi * RT / 2)
        C = 4 * math.sqrt(RT)
        dt = 0.25 * (1.0 / n) / C
        uw = 0.16 * math.sqrt(5.0 / 3.0 * RT)
        return dict(name=name, nx=n, ny=n, RT=RT, vel="nc", nv1=nv1, Kn=kn,
                    tau=tau, dt=dt, steps=5000, U=uw,
                    bc=[(DIFFUSE, 0, 0), (DIFFUSE, 0, 0),
                        (DIFFUSE, 0, 0), (DIFFUSE, uw, 0)])
    if name == "batched64":
        return dict(name=name, instances=batched_instances(64))
    raise KeyError(name)


def batched_instances(n: int, seed: int = SEED):
    """Seeded mix of uneven instances: kind TGV or cavity (p = 1/2), N in
    {32, 64, ..., 512}; D2Q9 (p = 1/2) with Re log-uniform in [100, 1000] and
    dt/tau = 4, else a Newton-Cotes grid n in {16, 22, 28, 32} with Kn
    log-uniform in [0.1, 10] (CFL 0.25)."""
    r = rng(seed)
    out = []
    for _ in range(n):
        kind = "tgv" if r.uniform() < 0.5 else "cavity"
        N = int(32 * r.integers(1, 17))
        if r.uniform() < 0.5:
            RT = 1.0 / 3.0
            C = math.sqrt(3 * RT)
            U = 0.05 * C
            Re = float(np.exp(r.uniform(np.log(100.0), np.log(1000.0))))
            nu = U / Re
            tau = nu / RT
            out.append(dict(kind=kind, N=N, vel="d2q9", RT=RT, U=U, tau=tau, dt=4 * tau))
        else:
            nv1 = int(r.choice([16, 22, 28, 32]))
            RT = 0.5
            Kn = float(np.exp(r.uniform(np.log(0.1), np.log(10.0))))
            tau = Kn / math.sqrt(math.pi * RT / 2)
            dt = 0.25 * (1.0 / N) / (4 * math.sqrt(RT))
            out.append(dict(kind=kind, N=N, vel="nc", nv1=nv1, RT=RT, U=0.1 * math.sqrt(RT),
                            tau=tau, dt=dt, Kn=Kn))
    return out
