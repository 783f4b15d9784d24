"""Python binding of the GB300 third-order DUGKS library (``libdugks.so``).

Argument marshalling only: every step of the DUGKS path runs in the
library's CUDA kernels (see ``include/dugks.h``).  The functions keep the
C-ABI names (``dugks_init``, ``dugks_step``, ...); :class:`Solver` is a small
convenience wrapper that owns one context.  PyTorch is used only for device
buffers and streams.

The library must have been built (``paper_1709_05458_gb300.build``); there is
no fallback: loading fails loudly if ``libdugks.so`` is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import velocity_sets  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdugks.so")

DUGKS_OK, DUGKS_EINVAL, DUGKS_ECUDA, DUGKS_ENOMEM, DUGKS_EUNSTABLE, DUGKS_ENOTIMPL = 0, -1, -2, -3, -4, -5
PERIODIC, BOUNCEBACK, DIFFUSE = 0, 1, 2
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
FP64, G_FP32, G_BF16, F64_DW = 0, 1, 2, 3
T3S3, T2S3, T2S2 = 0, 1, 2
PATH_AUTO, PATH_GENERIC, PATH_REFERENCE = 0, 1, 2

# every symbol include/dugks.h declares
EXPORTS = ("dugks_init", "dugks_init_ex", "dugks_set_equilibrium", "dugks_set_state", "dugks_get_state",
           "dugks_step", "dugks_moments", "dugks_check", "dugks_synchronize",
           "dugks_profile", "dugks_profile_read", "dugks_kernel_name", "dugks_destroy",
           "dugks_last_error", "dugks_step_static", "dugks_adjoint_step", "dugks_adjoint_run",
           "dugks_adjoint_equilibrium", "dugks_autotune", "dugks_set_tile_height",
           "dugks_tile_height", "dugks_batch_create",
           "dugks_batch_step", "dugks_batch_autotune", "dugks_batch_destroy", "dugks_set_scheme",
           "dugks_alu_peak")


class DugksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dugks error {code}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double)]


class VelSet(C.Structure):
    _fields_ = [("nv", C.c_int), ("xi_x", C.POINTER(C.c_double)), ("xi_y", C.POINTER(C.c_double)),
                ("w", C.POINTER(C.c_double)), ("RT", C.c_double)]


class BC(C.Structure):
    _fields_ = [("kind", C.c_int), ("uw_x", C.c_double), ("uw_y", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libdugks.so`` (raises if it is absent: no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run python -m paper_1709_05458_gb300.build")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    sig = {
        "dugks_init": (I, [C.POINTER(Mesh), C.POINTER(VelSet), D, D, C.POINTER(BC), I, P, C.POINTER(P)]),
        "dugks_init_ex": (I, [C.POINTER(Mesh), C.POINTER(VelSet), D, D, C.POINTER(BC), I, I, P,
                              C.POINTER(P)]),
        "dugks_set_equilibrium": (I, [P, P, P, P, I]),
        "dugks_set_state": (I, [P, P, I]),
        "dugks_get_state": (I, [P, P, I, I]),
        "dugks_step": (I, [P, I]),
        "dugks_moments": (I, [P, P, P, P, I]),
        "dugks_check": (I, [P]),
        "dugks_synchronize": (I, [P]),
        "dugks_profile": (I, [P, I]),
        "dugks_profile_read": (I, [P, C.POINTER(C.c_longlong), C.POINTER(C.c_double), I]),
        "dugks_kernel_name": (C.c_char_p, [I]),
        "dugks_destroy": (I, [P]),
        "dugks_last_error": (C.c_char_p, []),
        "dugks_step_static": (I, [C.POINTER(Mesh), C.POINTER(VelSet), D, D, C.POINTER(BC), P, P, I, P]),
        "dugks_adjoint_step": (I, [P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double), I]),
        "dugks_adjoint_run": (I, [P, P, I, I, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double), I]),
        "dugks_adjoint_equilibrium": (I, [P, P, P, P, P, P, P, P, I]),
        "dugks_autotune": (I, [P, I, C.POINTER(C.c_int)]),
        "dugks_set_tile_height": (I, [P, I]),
        "dugks_tile_height": (I, [P, C.POINTER(C.c_int)]),
        "dugks_batch_create": (I, [C.POINTER(P), I, C.POINTER(P)]),
        "dugks_batch_step": (I, [P, I]),
        "dugks_batch_autotune": (I, [P, I, C.POINTER(I)]),
        "dugks_batch_destroy": (I, [P]),
        "dugks_set_scheme": (I, [P, I]),
        "dugks_alu_peak": (I, [I, I, I, P, C.c_longlong, C.POINTER(C.c_double),
                               C.POINTER(C.c_float), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != DUGKS_OK:
        raise DugksError(rc, load().dugks_last_error().decode())
    return rc


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(C.c_void_p)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def _on_device(a):
    return 0 if (a is None or isinstance(a, np.ndarray)) else int(a.is_cuda)


# ------------------------------------------------- C-ABI mirrors
def dugks_init(nx, ny, dx, dy, xi, W, RT, tau, dt, bc, storage=FP64, stream=None,
               path=PATH_AUTO):
    """Returns an opaque context handle (int).  ``bc``: four (kind, uw_x, uw_y)
    in the order west, east, south, north; ``stream``: a torch.cuda.Stream,
    a raw cudaStream_t int, or None; ``path``: the kernel path of
    ``dugks_init_ex`` (PATH_AUTO, PATH_GENERIC, PATH_REFERENCE)."""
    lib = load()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    xx = np.ascontiguousarray(xi[:, 0])
    xy = np.ascontiguousarray(xi[:, 1])
    w = np.ascontiguousarray(W, dtype=np.float64)
    vs = VelSet(len(w), xx.ctypes.data_as(C.POINTER(C.c_double)),
                xy.ctypes.data_as(C.POINTER(C.c_double)),
                w.ctypes.data_as(C.POINTER(C.c_double)), float(RT))
    bcs = (BC * 4)(*[BC(int(b[0]), float(b[1]), float(b[2])) for b in bc])
    mesh = Mesh(int(nx), int(ny), float(dx), float(dy))
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    out = C.c_void_p()
    if path == PATH_AUTO:
        _check(lib.dugks_init(C.byref(mesh), C.byref(vs), float(tau), float(dt), bcs, int(storage),
                              C.c_void_p(s), C.byref(out)))
    else:
        _check(lib.dugks_init_ex(C.byref(mesh), C.byref(vs), float(tau), float(dt), bcs,
                                 int(storage), int(path), C.c_void_p(s), C.byref(out)))
    return out.value


def dugks_set_equilibrium(ctx, rho, ux, uy):
    return _check(load().dugks_set_equilibrium(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _on_device(rho)))


def dugks_set_state(ctx, fhat):
    return _check(load().dugks_set_state(ctx, _ptr(fhat), _on_device(fhat)))


STATE_SCHEME, STATE_F = 0, 1


def dugks_get_state(ctx, out, which=STATE_SCHEME):
    """Copy the state into ``out``: the scheme's variable (f^ under T3S3,
    f~ under T2; ``which=STATE_SCHEME``) or the distribution f itself
    (``which=STATE_F``)."""
    return _check(load().dugks_get_state(ctx, _ptr(out), int(which), _on_device(out)))


def dugks_step(ctx, n=1):
    return _check(load().dugks_step(ctx, int(n)))


def dugks_moments(ctx, rho=None, ux=None, uy=None):
    ref = next((a for a in (rho, ux, uy) if a is not None), None)
    return _check(load().dugks_moments(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _on_device(ref)))


def dugks_check(ctx):
    return load().dugks_check(ctx)


def dugks_synchronize(ctx):
    return _check(load().dugks_synchronize(ctx))


def dugks_profile(ctx, enable=True):
    return _check(load().dugks_profile(ctx, int(bool(enable))))


def dugks_profile_read(ctx):
    """{kernel name: (launches, total ms)} since profiling was enabled."""
    lib = load()
    n = 128
    la = (C.c_longlong * n)()
    ms = (C.c_double * n)()
    k = lib.dugks_profile_read(ctx, la, ms, n)
    if k < 0:
        _check(k)
    return {lib.dugks_kernel_name(i).decode(): (int(la[i]), float(ms[i])) for i in range(min(k, n))}


def dugks_destroy(ctx):
    return _check(load().dugks_destroy(ctx))


def dugks_set_scheme(ctx, scheme):
    """T3S3 (default), T2S3 or T2S2; under a T2 scheme the state is f~."""
    return _check(load().dugks_set_scheme(ctx, int(scheme)))


def dugks_last_error():
    return load().dugks_last_error().decode()


def dugks_adjoint_step(ctx, lam_in, lam_out):
    """lam_out = (d step / d f^)^T lam_in at the current state; returns
    (dJ/dtau, dJ/duw[4][2]) contributions of this step."""
    t = (C.c_double * 1)(0.0)
    u = (C.c_double * 8)(*([0.0] * 8))
    _check(load().dugks_adjoint_step(ctx, _ptr(lam_in), _ptr(lam_out), t, u, _on_device(lam_in)))
    return t[0], np.array(list(u)).reshape(4, 2)


def dugks_adjoint_run(ctx, fhat0, nsteps, every, lam_final, lam0):
    """Checkpointed forward + reverse sweep; returns (dJ/dtau, dJ/duw[4][2])."""
    t = (C.c_double * 1)(0.0)
    u = (C.c_double * 8)(*([0.0] * 8))
    _check(load().dugks_adjoint_run(ctx, _ptr(fhat0), int(nsteps), int(every), _ptr(lam_final),
                                    _ptr(lam0), t, u, _on_device(fhat0)))
    return t[0], np.array(list(u)).reshape(4, 2)


def dugks_adjoint_equilibrium(ctx, rho, ux, uy, lam, drho=None, dux=None, duy=None):
    return _check(load().dugks_adjoint_equilibrium(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(lam),
                                                   _ptr(drho), _ptr(dux), _ptr(duy),
                                                   _on_device(lam)))


def dugks_autotune(ctx, trials=3):
    """Time tile heights 4..16 (4..12 for the double-word form) for this
    context's fused D2Q9 kernels and keep the fastest (state unchanged);
    returns the chosen height."""
    ty = C.c_int(0)
    _check(load().dugks_autotune(ctx, int(trials), C.byref(ty)))
    return ty.value


def dugks_set_tile_height(ctx, ty):
    """Fix the fused D2Q9 kernels' tile height (4..16; 4..12 double-word)."""
    return _check(load().dugks_set_tile_height(ctx, int(ty)))


def dugks_tile_height(ctx):
    ty = C.c_int(0)
    _check(load().dugks_tile_height(ctx, C.byref(ty)))
    return ty.value


def dugks_batch_create(ctxs):
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    out = C.c_void_p()
    _check(load().dugks_batch_create(arr, len(ctxs), C.byref(out)))
    return out.value


def dugks_batch_step(batch, nsteps=1):
    return _check(load().dugks_batch_step(batch, int(nsteps)))


def dugks_batch_autotune(batch, trials=3):
    """Tile height of the batch's persistent launch: the fastest over
    ``trials`` timed steps (0 without fused instances)."""
    ty = C.c_int(0)
    _check(load().dugks_batch_autotune(batch, int(trials), C.byref(ty)))
    return ty.value


def dugks_batch_destroy(batch):
    return _check(load().dugks_batch_destroy(batch))


ALU_FP64, ALU_FP32, ALU_FP32X2 = 0, 1, 2


def dugks_alu_peak(kind, iters, blocks_per_sm, out, stream=None):
    """One launch of the FMA-throughput microbenchmark; ``out`` is a CUDA
    float64 tensor of at least SMs x blocks_per_sm x 256 elements.  Returns
    (flops, ms)."""
    import torch
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64:
        raise ValueError("out must be a CUDA float64 tensor")
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    fl, ms = C.c_double(0.0), C.c_float(0.0)
    _check(load().dugks_alu_peak(int(kind), int(iters), int(blocks_per_sm), _ptr(out),
                                 out.numel(), C.byref(fl), C.byref(ms), C.c_void_p(s)))
    return fl.value, float(ms.value)


class Batch:
    """Many Solvers advanced together (one persistent launch per stage for
    the FP64 D2Q9 ones, everything inside one CUDA graph per step count).
    The solvers must share one non-default stream."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = dugks_batch_create([s.ctx for s in self.solvers])

    def step(self, n=1):
        dugks_batch_step(self.handle, n)

    def autotune(self, trials=3):
        """Tile height of the persistent launch (see dugks_batch_autotune)."""
        return dugks_batch_autotune(self.handle, trials)

    def close(self):
        if self.handle:
            dugks_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_static_tensor(name, t, numel):
    """dugks_step_static takes raw device pointers: refuse anything but a
    contiguous float64 CUDA tensor of the right size on the current device."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, the problem needs {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, not the current device "
                         f"cuda:{torch.cuda.current_device()}")


def dugks_step_static(nx, ny, dx, dy, xi, W, RT, tau, dt, bc, fhat_in, fhat_out, nsteps,
                      stream=None):
    """T3S3 steps with no device allocation (library-internal fixed 32 MiB
    scratch); ``fhat_in``/``fhat_out`` are CUDA tensors [nv][ny][nx]
    (may be the same tensor).  For callers that may not allocate device
    memory; calls must not overlap on the GPU."""
    lib = load()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    xx, xy = np.ascontiguousarray(xi[:, 0]), np.ascontiguousarray(xi[:, 1])
    w = np.ascontiguousarray(W, dtype=np.float64)
    _check_static_tensor("fhat_in", fhat_in, len(w) * int(ny) * int(nx))
    _check_static_tensor("fhat_out", fhat_out, len(w) * int(ny) * int(nx))
    vs = VelSet(len(w), xx.ctypes.data_as(C.POINTER(C.c_double)),
                xy.ctypes.data_as(C.POINTER(C.c_double)),
                w.ctypes.data_as(C.POINTER(C.c_double)), float(RT))
    bcs = (BC * 4)(*[BC(int(b[0]), float(b[1]), float(b[2])) for b in bc])
    mesh = Mesh(int(nx), int(ny), float(dx), float(dy))
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    return _check(lib.dugks_step_static(C.byref(mesh), C.byref(vs), float(tau), float(dt), bcs,
                                        _ptr(fhat_in), _ptr(fhat_out), int(nsteps), C.c_void_p(s)))


class Solver:
    """One DUGKS context: ``Solver(nx, ny, dx, dy, xi, W, RT, tau, dt, bc)``."""

    def __init__(self, nx, ny, dx, dy, xi, W, RT, tau, dt, bc, stream=None, storage=FP64,
                 scheme=T3S3, path=PATH_AUTO):
        self.nx, self.ny, self.nv = int(nx), int(ny), len(W)
        self.ctx = None
        self.ctx = dugks_init(nx, ny, dx, dy, xi, W, RT, tau, dt, bc, storage, stream, path)
        self.warning = dugks_last_error()
        if scheme != T3S3:
            dugks_set_scheme(self.ctx, scheme)

    def set_equilibrium(self, rho, ux, uy):
        a = [np.ascontiguousarray(x, dtype=np.float64) if isinstance(x, np.ndarray) else x
             for x in (rho, ux, uy)]
        dugks_set_equilibrium(self.ctx, *a)

    def set_state(self, fhat):
        if isinstance(fhat, np.ndarray):
            fhat = np.ascontiguousarray(fhat, dtype=np.float64)
        dugks_set_state(self.ctx, fhat)

    def state(self, out=None, which=STATE_SCHEME):
        if out is None:
            out = np.empty((self.nv, self.ny, self.nx))
        dugks_get_state(self.ctx, out, which)
        return out

    def step(self, n=1):
        dugks_step(self.ctx, n)

    def moments(self):
        r, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        dugks_moments(self.ctx, r, u, v)
        return r, u, v

    def check(self):
        return dugks_check(self.ctx)

    def synchronize(self):
        dugks_synchronize(self.ctx)

    def close(self):
        if self.ctx:
            dugks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
