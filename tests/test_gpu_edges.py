"""Edge cases of the CUDA path against the FP64 oracle: degenerate sizes (one depth,
one time bin, the smallest lateral grid), the largest per-class block the
contraction kernels accept (nt = 512 at nz = 64: one CTA per SM, single
buffer), and an all-zero measurement (every solver must return exactly zero,
with no division by the zero data scale).  Tolerances as in test_gpu_parity.py,
scaled by sqrt(nt / 64) above 64 bins: the FP32 sums of W^T m run over nt
terms, so their rounding grows as sqrt(nt) (the 1e-5 of the parity tests is
set at config 1's 64 bins; at nt = 512 Tikhonov measured 1.01e-5).
"""

import numpy as np
import pytest

from gpu_common import CFG1_OPTICS, medium, oracle_grid, rel_l2
from oracle import operators as op
from oracle import solvers as so
from paper_2101_11680_gb300 import ctof

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGE = {
    "one_bin_one_depth": dict(n=4, nz=1, nt=1, dx=1.0, dz=1.0, z_first=1.0, dt=50.0),
    "one_depth": dict(n=5, nz=1, nt=7, dx=0.8, dz=1.0, z_first=1.0, dt=40.0),
    "one_bin": dict(n=6, nz=3, nt=1, dx=1.0, dz=0.7, z_first=0.7, dt=300.0),
    "circ_one_bin_one_depth": dict(n=32, nz=1, nt=1, dx=1.0, dz=1.0, z_first=1.0, dt=60.0, mode="circular"),
    "largest_block": dict(n=8, nz=64, nt=512, dx=1.0, dz=0.5, z_first=0.5, dt=20.0),
}

_cache = {}


def pair(name):
    if name not in _cache:
        from paper_2101_11680_gb300 import build as B
        B.build()
        kw = EDGE[name]
        g = oracle_grid(kw)
        w = op.kernel_offsets(g, medium(grid_kw=kw))
        grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"],
                              mode=kw.get("mode", "linear"))
        k = ctof.Kernel(ctof.make_optics(**CFG1_OPTICS), grid, keep_w=True)
        _cache[name] = (g, w, op.kernel_spectrum(w, g), k)
    return _cache[name]


def _phantom(g, seed):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.0, 0.02, (g.nz, g.n, g.n))
    return mu * (rng.uniform(size=mu.shape) < 0.4)


@pytest.mark.parametrize("name", list(EDGE))
def test_edge_kernel_and_operators(name):
    g, w, wh, k = pair(name)
    n = g.n
    want_w = w[:, :, n - 1:, n - 1:] if g.mode == "linear" else \
        w[:, :, n - 1:n - 1 + g.p // 2 + 1, n - 1:n - 1 + g.p // 2 + 1]
    assert np.abs(k.get_w() - want_w).max() <= 1e-12 * np.abs(want_w).max()
    mu = _phantom(g, 5)
    want = op.forward_fft(wh, mu, g)
    got = k.forward(torch.tensor(mu, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got, want) <= 1e-5
    m = np.random.default_rng(6).standard_normal((g.nt, g.n, g.n))
    got_a = k.adjoint(torch.tensor(m, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(got_a, op.adjoint_fft(wh, m, g)) <= 1e-5


def _bound(g):
    return 1e-5 * max(1.0, np.sqrt(g.nt / 64.0))


@pytest.mark.parametrize("name", list(EDGE))
def test_edge_solvers(name):
    g, _, wh, k = pair(name)
    tol = _bound(g)
    m = op.forward_fft(wh, _phantom(g, 7), g)
    m = m + 1e-3 * np.abs(m).max() * np.random.default_rng(8).standard_normal(m.shape)
    dm = torch.tensor(m, dtype=torch.float32, device="cuda")
    want, lam, _ = so.tikhonov(wh, m, g)
    got, rep = k.reconstruct(dm, ctof.tikhonov_params(), report=True)
    assert rep.lambda_ == pytest.approx(lam, rel=1e-10)
    assert rel_l2(got.cpu().numpy(), want) <= tol
    iters = 20
    want, info = so.admm(wh, m, g, iters)
    got, rep = k.reconstruct(dm, ctof.admm_params(iters=iters), report=True)
    assert rep.beta == pytest.approx(info["beta"], rel=1e-5)
    assert rel_l2(got.cpu().numpy(), want) <= tol
    want, info = so.fista_l1(wh, m, g, iters, lam_rel=1e-2)
    got = k.reconstruct(dm, ctof.fista_params(iters=iters, lam_rel=1e-2))
    assert rel_l2(got.cpu().numpy(), want) <= max(tol, 5e-7 * iters)


@pytest.mark.parametrize("name", ["one_bin_one_depth", "largest_block"])
def test_zero_measurement_gives_zero(name):
    g, _, _, k = pair(name)
    zero = torch.zeros((g.nt, g.n, g.n), device="cuda")
    for p in (ctof.tikhonov_params(), ctof.admm_params(iters=5), ctof.fista_params(iters=5)):
        out = k.reconstruct(zero, p)
        assert torch.count_nonzero(out).item() == 0
    assert torch.count_nonzero(k.forward(torch.zeros((g.nz, g.n, g.n), device="cuda"))).item() == 0
