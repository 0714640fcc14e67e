"""Fluorescence-mode kernel (Section 5, simulator paragraph) on the device against the FP64 oracle.

Both sides evaluate Phi0_ex (*) L_tau (*) R_em through the product of Laplace
transforms and a 24-term fixed-Talbot inversion at the bin edges, in
independent code (NumPy here, CUDA FP64 there).  The Talbot sum cancels
terms up to e^(2M/5) ~ 1.5e4 times larger than its result, so ulp-level
differences of exp/sin/sqrt between the two give ~1e-12 of the cumulative
response: the table bound is 1e-10 of its maximum (1e-8 relative on entries
above 1 % of it).  Everything downstream is the absorption-mode code, held
to the same FP32 bounds as in the other parity tests.
"""

import functools

import numpy as np
import pytest

from gpu_common import CASES, CFG1_OPTICS, oracle_grid, rel_l2
from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so
from paper_2101_11680_gb300 import ctof, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EMISSION = dict(mua=0.005, musp=0.8)
FL_CASES = {"sub": 300.0, "ragged": 0.0, "circ": 1000.0, "cfg1": 500.0}


def _media(kw, em=EMISSION):
    dy = kw.get("dy", kw["dx"])
    rmin = 0.5 * min(kw["dx"], dy, kw["dz"])
    mx = ph.Medium(CFG1_OPTICS["mua"], CFG1_OPTICS["musp"], CFG1_OPTICS["n"], r_min=rmin)
    mm = ph.Medium(em["mua"], em["musp"], CFG1_OPTICS["n"], r_min=rmin)
    return mx, mm


@functools.lru_cache(maxsize=None)
def oracle_fl(name):
    kw = CASES[name]
    g = oracle_grid(kw)
    mx, mm = _media(kw)
    w = op.kernel_offsets_fluorescence(g, mx, mm, FL_CASES[name])
    return g, w, op.kernel_spectrum(w, g)


_dev = {}


def device_fl(name):
    from paper_2101_11680_gb300 import build as B
    if name not in _dev:
        B.build()
        kw = CASES[name]
        grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"],
                              dy=kw.get("dy"), mode=kw.get("mode", "linear"))
        em = ctof.make_emission(EMISSION["mua"], EMISSION["musp"], FL_CASES[name])
        _dev[name] = ctof.Kernel(ctof.make_optics(**CFG1_OPTICS), grid, keep_w=True, emission=em)
    return _dev[name]


@pytest.mark.parametrize("name", ["sub", "ragged", "circ", "cfg1"])
def test_fluorescence_kernel_table(name):
    g, w, _ = oracle_fl(name)
    k = device_fl(name)
    wd = k.get_w()
    n = g.n
    if g.mode == "linear":
        want = w[:, :, n - 1:, n - 1:]
    else:
        q = g.p // 2 + 1
        want = w[:, :, n - 1:n - 1 + q, n - 1:n - 1 + q]
    assert wd.shape == want.shape
    mx = np.abs(want).max()
    assert np.abs(wd - want).max() <= 1e-10 * mx
    big = np.abs(want) > 1e-2 * mx
    assert np.all(np.abs(wd[big] - want[big]) <= 1e-8 * np.abs(want[big]))


@pytest.mark.parametrize("name", ["sub", "ragged", "circ"])
def test_fluorescence_operators(name):
    g, _, wh = oracle_fl(name)
    k = device_fl(name)
    rng = np.random.default_rng(21)
    mu = rng.uniform(0.0, 0.02, (g.nz, g.n, g.n)) * (rng.uniform(size=(g.nz, g.n, g.n)) < 0.3)
    want = op.forward_fft(wh, mu, g)
    got = k.forward(torch.tensor(mu, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got, want) <= 1e-5
    m = rng.standard_normal((g.nt, g.n, g.n)) * np.abs(want).max()
    got_a = k.adjoint(torch.tensor(m, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got_a, op.adjoint_fft(wh, m, g)) <= 1e-5


def test_fluorescence_tikhonov_cfg1():
    g, _, wh = oracle_fl("cfg1")
    mu = synth.phantom_spheres(g.n, g.nz, g.dx, g.dz, g.z_first, seed=4)
    m = synth.poisson_noise(np.clip(op.forward_fft(wh, mu, g), 0, None), 1e4, 104)
    want, lam, _ = so.tikhonov(wh, m, g)
    k = device_fl("cfg1")
    got, rep = k.reconstruct(torch.tensor(m, dtype=torch.float32, device="cuda"), ctof.tikhonov_params(),
                             report=True)
    assert rep.lambda_ == pytest.approx(lam, rel=1e-10)
    assert rel_l2(got.cpu().numpy(), want) <= 1e-5


def test_lifetime_delays_the_response():
    """Same optics as the absorption kernel and tau > 0: every column keeps its total over a
    long window and its mean arrival time grows by tau.  Means are taken at the bin centres,
    which misplaces a response that sits inside one bin by up to half a bin (the tau = 0
    response of the shallow voxels is a few ps wide), hence the bound dt/2."""
    kw = dict(n=8, nz=3, nt=300, dx=1.0, dz=1.0, z_first=1.0, dt=50.0)
    grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"])
    opt = ctof.make_optics(**CFG1_OPTICS)
    same = dict(mua=CFG1_OPTICS["mua"], musp=CFG1_OPTICS["musp"])
    k0 = ctof.Kernel(opt, grid, keep_w=True, emission=ctof.make_emission(tau=0.0, **same))
    k1 = ctof.Kernel(opt, grid, keep_w=True, emission=ctof.make_emission(tau=800.0, **same))
    w0, w1 = k0.get_w(), k1.get_w()
    t = (np.arange(kw["nt"]) + 0.5) * kw["dt"]
    s0, s1 = w0.sum(axis=0), w1.sum(axis=0)
    assert np.allclose(s1, s0, rtol=1e-6)
    m0 = np.tensordot(t, w0, axes=1) / s0
    m1 = np.tensordot(t, w1, axes=1) / s1
    assert np.abs(m1 - m0 - 800.0).max() <= 0.5 * kw["dt"]
    assert np.all(m1 > m0 + 700.0)
