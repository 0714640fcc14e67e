"""Voxel-averaged kernel near the surface on the device against the FP64 oracle.

Both sides apply a tensor Gauss-Legendre rule over the voxel to the same
point response (own node generators: Newton iteration in CUDA,
numpy's leggauss here), so the tables agree to FP64 rounding: bound 1e-12 of
the maximum for the absorption kernel (as the plain kernel table), the
fluorescence bound (1e-10 of the maximum) for the fluorescence kernel.
"""

import functools

import numpy as np
import pytest

from gpu_common import CASES, CFG1_OPTICS, medium, oracle_grid, rel_l2
from oracle import operators as op
from oracle import physics as ph
from paper_2101_11680_gb300 import ctof

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# name -> (case, layers, nodes, fluorescence lifetime or None)
AVG = {
    "sub_abs": ("sub", 2, 4, None),
    "ragged_abs": ("ragged", 5, 2, None),
    "sub_fl": ("sub", 1, 3, 400.0),
}
EMISSION = dict(mua=0.005, musp=0.8)


@functools.lru_cache(maxsize=None)
def oracle_avg(name):
    case, layers, nodes, tau = AVG[name]
    kw = CASES[case]
    g = oracle_grid(kw)
    mx = medium(grid_kw=kw)
    em = None
    if tau is not None:
        em = (ph.Medium(EMISSION["mua"], EMISSION["musp"], CFG1_OPTICS["n"], r_min=mx.r_min), tau)
    w = op.kernel_offsets_averaged(g, mx, layers, nodes, emission=em)
    return g, w, op.kernel_spectrum(w, g)


def device_avg(name):
    from paper_2101_11680_gb300 import build as B
    B.build()
    case, layers, nodes, tau = AVG[name]
    kw = CASES[case]
    grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"],
                          dy=kw.get("dy"), mode=kw.get("mode", "linear"))
    em = None if tau is None else ctof.make_emission(EMISSION["mua"], EMISSION["musp"], tau)
    return ctof.Kernel(ctof.make_optics(**CFG1_OPTICS), grid, keep_w=True, emission=em, average=(layers, nodes))


@pytest.mark.parametrize("name", list(AVG))
def test_averaged_kernel_table(name):
    g, w, _ = oracle_avg(name)
    k = device_avg(name)
    n = g.n
    want = w[:, :, n - 1:, n - 1:]
    got = k.get_w()
    assert got.shape == want.shape
    bound = 1e-12 if AVG[name][3] is None else 1e-10
    assert np.abs(got - want).max() <= bound * np.abs(want).max()


@pytest.mark.parametrize("name", ["sub_abs", "sub_fl"])
def test_averaged_kernel_operators(name):
    g, _, wh = oracle_avg(name)
    k = device_avg(name)
    rng = np.random.default_rng(31)
    mu = rng.uniform(0.0, 0.02, (g.nz, g.n, g.n))
    want = op.forward_fft(wh, mu, g)
    got = k.forward(torch.tensor(mu, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got, want) <= 1e-5
    m = rng.standard_normal((g.nt, g.n, g.n))
    got_a = k.adjoint(torch.tensor(m, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got_a, op.adjoint_fft(wh, m, g)) <= 1e-5


def test_one_node_equals_plain_build():
    """average=(nz, 1) is the centre-value kernel: the same table as the plain build."""
    from paper_2101_11680_gb300 import build as B
    B.build()
    kw = CASES["sub"]
    grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"])
    opt = ctof.make_optics(**CFG1_OPTICS)
    a = ctof.Kernel(opt, grid, keep_w=True).get_w()
    b = ctof.Kernel(opt, grid, keep_w=True, average=(kw["nz"], 1)).get_w()
    assert np.array_equal(a, b)
