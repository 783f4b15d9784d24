"""The C-ABI library loads, exports every declared entry point, and rejects
bad problems on the host before touching the GPU (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import paper_1709_05458_gb300 as P
from paper_1709_05458_gb300 import velocity_sets as PV

HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")


def declared():
    names = set()
    for f in os.listdir(HDR):
        if f.endswith(".h"):
            txt = open(os.path.join(HDR, f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(dugks_\w+)\s*\(", txt, re.M))
    return names


def test_header_declares_the_binding_names():
    assert declared() == set(P.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def _init(**kw):
    xi, W, RT = PV.d2q9(1 / 3)
    a = dict(nx=8, ny=8, dx=1 / 8, dy=1 / 8, xi=xi, W=W, RT=RT, tau=0.01, dt=0.01,
             bc=[(P.PERIODIC, 0, 0)] * 4)
    a.update(kw)
    return P.dugks_init(**a)


@pytest.mark.parametrize("kw,frag", [
    (dict(tau=0.0), "tau"),
    (dict(dt=-1.0), "tau"),
    (dict(nx=0), "nx"),
    (dict(dx=0.0), "dx"),
    (dict(RT=0.0), "RT"),
    (dict(bc=[(P.PERIODIC, 0, 0), (P.BOUNCEBACK, 0, 0), (P.PERIODIC, 0, 0), (P.PERIODIC, 0, 0)]), "west"),
    (dict(bc=[(P.PERIODIC, 0, 0)] * 2 + [(P.DIFFUSE, 0, 0), (P.PERIODIC, 0, 0)]), "south"),
    (dict(bc=[(7, 0, 0)] * 4), "kind"),
    (dict(nx=2, bc=[(P.BOUNCEBACK, 0, 0)] * 4), "nx >= 3"),
    (dict(tau=float("nan")), "tau"),
], ids=["tau0", "dtneg", "nx0", "dx0", "RT0", "halfperiodic_x", "halfperiodic_y", "kind", "narrow", "nan"])
def test_init_rejects_bad_problems(lib, kw, frag):
    with pytest.raises(P.DugksError) as e:
        _init(**kw)
    assert e.value.code == P.DUGKS_EINVAL
    assert frag in str(e.value)


def test_bounceback_needs_opposite_velocities(lib):
    xi = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    W = np.array([0.25, 0.25, 0.5])
    with pytest.raises(P.DugksError) as e:
        P.dugks_init(8, 8, .1, .1, xi, W, 1.0, .1, .1, [(P.BOUNCEBACK, 0, 0)] * 4)
    assert "bounce-back" in str(e.value)


def test_unknown_storage_form_not_provided(lib):
    with pytest.raises(P.DugksError) as e:
        _init(storage=4)
    assert e.value.code == P.DUGKS_ENOTIMPL


def test_double_word_form_needs_the_d2q9_set(lib):
    """DUGKS_F64_DW runs on the fused D2Q9 kernels only; a Newton-Cotes set
    is refused before any device work."""
    xi, W, RT = PV.newton_cotes(4, 0.5)
    with pytest.raises(P.DugksError) as e:
        _init(xi=xi, W=W, RT=RT, storage=P.F64_DW)
    assert e.value.code == P.DUGKS_ENOTIMPL
    assert "D2Q9" in str(e.value)


def test_kernel_path_is_checked_on_the_host(lib):
    """dugks_init_ex refuses an unknown kernel path (EINVAL) and the
    reference kernels with a deviation storage form (ENOTIMPL) before any
    device work; the double-word form needs the automatic path."""
    xi, W, RT = PV.d2q9(1 / 3)
    for path, storage, code in ((7, P.FP64, P.DUGKS_EINVAL), (-1, P.FP64, P.DUGKS_EINVAL),
                                (P.PATH_REFERENCE, P.G_FP32, P.DUGKS_ENOTIMPL),
                                (P.PATH_GENERIC, P.F64_DW, P.DUGKS_ENOTIMPL)):
        with pytest.raises(P.DugksError) as e:
            P.dugks_init(8, 8, .1, .1, xi, W, RT, .1, .1, [(P.PERIODIC, 0, 0)] * 4,
                         storage=storage, path=path)
        assert e.value.code == code


def test_product_velocity_sets_match_oracle():
    """The product and oracle velocity sets are built independently."""
    from oracle import velocity_sets as V
    for n in (12, 16, 22, 28, 32, 64):
        a, b = PV.newton_cotes(n, 0.5), V.newton_cotes_2d(n, 0.5)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_allclose(a[1], b[1], rtol=1e-14, atol=0)
        assert a[2] == pytest.approx(b[2], rel=1e-14)
    a, b = PV.d2q9(0.4), V.d2q9(0.4)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_set_scheme_needs_a_context(lib):
    with pytest.raises(P.DugksError) as e:
        P.dugks_set_scheme(None, P.T2S2)
    assert e.value.code == P.DUGKS_EINVAL


def test_alu_peak_rejects_bad_arguments_on_the_host(lib):
    """Argument checks run before any CUDA call (no GPU needed)."""
    import ctypes as C
    fl, ms = C.c_double(0.0), C.c_float(0.0)
    for kind, iters, bps in ((3, 10, 4), (0, 0, 4), (0, 10, 0), (0, 10, 33)):
        rc = lib.dugks_alu_peak(kind, iters, bps, C.c_void_p(1), 1 << 20, C.byref(fl),
                                C.byref(ms), None)
        assert rc == P.DUGKS_EINVAL
