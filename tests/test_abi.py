"""Host-side checks of the C ABI: the library loads, exports every function the
header declares, and rejects bad arguments before touching the GPU."""

import ctypes
import os
import re

import pytest

from paper_2101_11680_gb300 import build as B
from paper_2101_11680_gb300 import ctof

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ctof_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctof.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert lib.ctof_status_string(s)
    assert lib.ctof_status_string(-99) == b"unknown status"


def _build(lib, optics, grid, flags=0):
    h = ctypes.c_void_p()
    st = lib.ctof_build_kernel(ctypes.byref(optics) if optics else None, ctypes.byref(grid) if grid else None,
                               flags, None, ctypes.byref(h))
    return st, h


def test_build_rejects_bad_arguments(lib):
    good_o = ctof.make_optics()
    good_g = ctof.make_grid(32, 16, 64, 1.0, 1.0, 1.0, 50.0)
    assert _build(lib, None, good_g)[0] == ctof.EINVAL
    assert _build(lib, good_o, None)[0] == ctof.EINVAL
    for bad in (dict(mua=-1.0), dict(musp=0.0), dict(n=0.5), dict(mua=float("nan"))):
        assert _build(lib, ctof.make_optics(**bad), good_g)[0] == ctof.EINVAL, bad
    for bad in (dict(n=0), dict(nz=0), dict(nt=-1), dict(dx=0.0), dict(dz=-1.0), dict(z_first=0.0), dict(dt=0.0)):
        kw = dict(n=32, nz=16, nt=64, dx=1.0, dz=1.0, z_first=1.0, dt=50.0)
        kw.update(bad)
        assert _build(lib, good_o, ctof.make_grid(**kw))[0] == ctof.EINVAL, bad
    g = ctof.make_grid(32, 16, 64, 1.0, 1.0, 1.0, 50.0)
    g.ny = 16
    assert _build(lib, good_o, g)[0] == ctof.EUNSUPPORTED
    assert _build(lib, good_o, ctof.make_grid(300, 16, 64, 1.0, 1.0, 1.0, 50.0))[0] == ctof.EUNSUPPORTED
    assert _build(lib, good_o, ctof.make_grid(32, 65, 64, 1.0, 1.0, 1.0, 50.0))[0] == ctof.EUNSUPPORTED
    assert _build(lib, good_o, ctof.make_grid(48, 16, 64, 1.0, 1.0, 1.0, 50.0, mode="circular"))[0] \
        == ctof.EUNSUPPORTED
    assert _build(lib, good_o, good_g, flags=8)[0] == ctof.EINVAL


def test_calls_reject_null_handles(lib):
    assert lib.ctof_forward(None, None, None, None) == ctof.EINVAL
    assert lib.ctof_adjoint(None, None, None, None) == ctof.EINVAL
    p = ctof.admm_params()
    assert lib.ctof_reconstruct(None, None, ctypes.byref(p), None, None, None) == ctof.EINVAL
    assert lib.ctof_reconstruct_host(None, None, ctypes.byref(p), None, None, None) == ctof.EINVAL
    assert lib.ctof_kernel_get_info(None, None) == ctof.EINVAL
    lib.ctof_kernel_destroy(None)  # no-op


def test_learned_parameter_count_matches_oracle(lib):
    from oracle import learned as ln
    for s in (1, 3, 10):
        assert lib.ctof_learned_param_count(s) == ln.param_count(s)
    out = ctypes.c_void_p(1)
    import numpy as np
    p = np.zeros(ln.param_count(3), dtype=np.float32)
    assert lib.ctof_learned_create(0, p.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(out)) != 0
    assert lib.ctof_learned_loss_grad(None, None, 1, None, None, None, None, None) != 0
    bad = ctof.LearnedOptions(0.0, 2, 0.0)  # data-consistency steps need a positive lambda
    assert lib.ctof_learned_create(3, p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(bad), ctypes.byref(out)) != 0


def test_learned_checked_reconstruct_rejects_bad_arguments(lib):
    """ctof_learned_reconstruct_checked validates its pointers and batch size before any device call."""
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert lib.ctof_learned_reconstruct_checked(None, fake, 1, fake, fake, fake, None) == ctof.EINVAL
    assert lib.ctof_learned_reconstruct_checked(fake, None, 1, fake, fake, fake, None) == ctof.EINVAL
    assert lib.ctof_learned_reconstruct_checked(fake, fake, 0, fake, fake, fake, None) == ctof.EINVAL
    assert lib.ctof_learned_reconstruct_checked(fake, fake, 1, None, fake, fake, None) == ctof.EINVAL
    assert lib.ctof_learned_reconstruct_checked(fake, fake, 1, fake, None, fake, None) == ctof.EINVAL
    assert lib.ctof_learned_reconstruct_checked(fake, fake, 1, fake, fake, None, None) == ctof.EINVAL


def test_fluorescence_build_rejects_bad_emission(lib):
    """Argument checks of ctof_build_kernel_fluorescence run before any device call."""
    o = ctof.make_optics()
    g = ctof.make_grid(32, 16, 64, 1.0, 1.0, 1.0, 50.0)
    h = ctypes.c_void_p(1)
    assert lib.ctof_build_kernel_fluorescence(ctypes.byref(o), None, ctypes.byref(g), 0, None,
                                              ctypes.byref(h)) == ctof.EINVAL
    assert h.value is None
    for bad in (dict(mua=-0.1), dict(musp=0.0), dict(tau=-1.0), dict(tau=float("inf")), dict(mua=float("nan"))):
        h = ctypes.c_void_p()
        st = lib.ctof_build_kernel_fluorescence(ctypes.byref(o), ctypes.byref(ctof.make_emission(**bad)),
                                                ctypes.byref(g), 0, None, ctypes.byref(h))
        assert st == ctof.EINVAL, bad


def test_build_ex_rejects_bad_average(lib):
    """Voxel-averaging options are checked before any device call."""
    o = ctof.make_optics()
    g = ctof.make_grid(32, 16, 64, 1.0, 1.0, 1.0, 50.0)
    shallow = ctof.make_grid(32, 16, 64, 1.0, 1.0, 0.4, 50.0)  # top layer reaches above the surface
    for grid, layers, nodes in ((g, -1, 4), (g, 17, 4), (g, 2, 0), (g, 2, 9), (shallow, 1, 4)):
        h = ctypes.c_void_p()
        av = ctof.VoxelAverage(layers, nodes)
        st = lib.ctof_build_kernel_ex(ctypes.byref(o), None, ctypes.byref(av), ctypes.byref(grid), 0, None,
                                      ctypes.byref(h))
        assert st == ctof.EINVAL, (layers, nodes)
