"""Parity at the benchmark workload (128 x 128 scan at 0.5 mm, 48 depths, 256
bins of 25 ps) on outputs the oracle can compute one by one, and properties
that hold at any size for the rest.

* W_hat: for sampled (bin, depth) planes the oracle evaluates the kernel at
  all 128 x 128 non-negative offsets from the closed form, places it on the
  256 x 256 periodic grid and takes numpy's FFT; every frequency class on the
  device must match.
* forward: a sparse volume (40 absorbers) makes each measurement sample a
  40-term sum of closed-form kernel values the oracle computes directly.
* adjoint: a sparse measurement (40 nonzero samples) makes each output voxel
  a 40-term sum of closed-form kernel values, likewise.
* adjoint identity at full size; ADMM (the bench launch configuration,
  100 iterations) is finite, non-negative, reproducible and reduces the data
  residual.
"""

import numpy as np
import pytest

from oracle import physics as ph
from paper_2101_11680_gb300 import ctof, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NZ, NT, DX, DZ, ZF, DT = 128, 48, 256, 0.5, 0.5, 0.5, 25.0


@pytest.fixture(scope="module")
def kern():
    from paper_2101_11680_gb300 import build as B
    B.build()
    k = ctof.Kernel(ctof.make_optics(), ctof.make_grid(N, NZ, NT, DX, DZ, ZF, DT))
    yield k
    k.close()


def _medium():
    return ph.Medium(0.01, 1.0, 1.4, r_min=0.25)


def _bin_value(med, rho, z, k):
    """Oracle kernel value for bin k at lateral offset rho (array) and depth z."""
    ts, ws = ph.bin_nodes(k, DT)
    acc = np.zeros_like(np.asarray(rho, dtype=np.float64))
    for t, w in zip(ts, ws):
        acc = acc + w * ph.conv_closed(rho, z, t, med)
    return acc * DX * DX * DZ


@pytest.mark.parametrize("k,j", [(3, 0), (40, 7), (120, 25), (255, 47)])
def test_what_planes_full_size(kern, k, j):
    med = _medium()
    q = np.arange(N)
    rho = np.sqrt((q[None, :] * DX) ** 2 + (q[:, None] * DX) ** 2)
    wq = _bin_value(med, rho, ZF + j * DZ, k)  # [|oy|][|ox|]
    p = kern.info.p
    per = np.zeros((p, p))
    o = np.arange(-(N - 1), N)
    per[np.mod(o, p)[:, None], np.mod(o, p)[None, :]] = wq[np.abs(o)[:, None], np.abs(o)[None, :]]
    wh = np.fft.fft2(per)
    assert np.abs(wh.imag).max() <= 1e-14 * np.abs(wh).max()
    mem = kern.get_classes()
    what = kern.get_what()
    h = p // 2 + 1
    got = np.repeat(what[:, k, j][:, None], 4, axis=1)
    valid = mem >= 0
    ky, kx = np.divmod(mem[valid], h)
    assert np.abs(got[valid] - wh.real[ky, kx]).max() <= 1e-6 * np.abs(wh).max()


def test_forward_sampled_full_size(kern):
    rng = np.random.default_rng(11)
    nvox = 40
    vz = rng.integers(0, NZ, nvox)
    vy = rng.integers(0, N, nvox)
    vx = rng.integers(0, N, nvox)
    val = rng.uniform(0.005, 0.02, nvox)
    mu = np.zeros((NZ, N, N))
    mu[vz, vy, vx] = val
    m = kern.forward(torch.tensor(mu, dtype=torch.float32, device="cuda")).cpu().numpy()
    med = _medium()
    sk = rng.integers(0, NT, 150)
    sy = rng.integers(0, N, 150)
    sx = rng.integers(0, N, 150)
    scale = np.abs(m).max()
    for k, y, x in zip(sk, sy, sx):
        rho = np.sqrt(((x - vx) * DX) ** 2 + ((y - vy) * DX) ** 2)
        want = 0.0
        for zz in np.unique(vz):
            sel = vz == zz
            want += float(np.sum(_bin_value(med, rho[sel], ZF + zz * DZ, int(k)) * val[sel]))
        assert abs(m[k, y, x] - want) <= 2e-6 * scale + 1e-5 * abs(want)


def test_adjoint_sampled_full_size(kern):
    """A^T m at 150 sampled voxels: vol[z][y][x] = sum_k sum_(y',x') W(x'-x, y'-y, z_j, k) m[k][y'][x']
    (the transpose of Eq. 11), a 40-term sum for a measurement with 40 nonzero samples."""
    rng = np.random.default_rng(12)
    nmeas = 40
    mk = rng.integers(0, NT, nmeas)
    my = rng.integers(0, N, nmeas)
    mx = rng.integers(0, N, nmeas)
    val = rng.uniform(0.5, 2.0, nmeas)
    m = np.zeros((NT, N, N))
    m[mk, my, mx] = val
    vol = kern.adjoint(torch.tensor(m, dtype=torch.float32, device="cuda")).cpu().numpy()
    med = _medium()
    sz = rng.integers(0, NZ, 150)
    sy = rng.integers(0, N, 150)
    sx = rng.integers(0, N, 150)
    scale = np.abs(vol).max()
    for z, y, x in zip(sz, sy, sx):
        rho = np.sqrt(((mx - x) * DX) ** 2 + ((my - y) * DX) ** 2)
        want = 0.0
        for kk in np.unique(mk):
            sel = mk == kk
            want += float(np.sum(_bin_value(med, rho[sel], ZF + z * DZ, int(kk)) * val[sel]))
        assert abs(vol[z, y, x] - want) <= 2e-6 * scale + 1e-5 * abs(want)


def test_adjoint_identity_full_size(kern):
    gen = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand((NZ, N, N), device="cuda", generator=gen)
    y = torch.randn((NT, N, N), device="cuda", generator=gen)
    ax = kern.forward(x)
    aty = kern.adjoint(y)
    lhs = float((ax.double() * y.double()).sum())
    rhs = float((x.double() * aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(ax.double().norm()) * float(y.double().norm())


def test_admm_full_size_properties(kern):
    mu = synth.phantom_shapes(N, NZ, DX, DZ, ZF, seed=1001)
    mu_d = torch.tensor(mu, dtype=torch.float32, device="cuda")
    clean = kern.forward(mu_d).double().clamp_(min=0).cpu().numpy()
    m = torch.tensor(synth.poisson_noise(clean, 1e5, seed=11001), dtype=torch.float32, device="cuda")
    p = ctof.admm_params(iters=100)
    rec, rep = kern.reconstruct(m, p, report=True)
    rec2 = kern.reconstruct(m, p)
    assert torch.isfinite(rec).all()
    assert float(rec.min()) >= 0.0
    assert torch.equal(rec, rec2)
    assert rep.iters_done == 100 and rep.beta > 0
    r0 = float(m.double().norm())
    r1 = float((kern.forward(rec) - m).double().norm())
    assert r1 < r0


def test_fista_full_size_properties(kern):
    """The paper's FISTA (Eq. 10) at the benchmark size: finite, with exact zeros,
    reproducible, and it lowers the data residual."""
    mu = synth.phantom_shapes(N, NZ, DX, DZ, ZF, seed=1002)
    mu_d = torch.tensor(mu, dtype=torch.float32, device="cuda")
    clean = kern.forward(mu_d).double().clamp_(min=0).cpu().numpy()
    m = torch.tensor(synth.poisson_noise(clean, 1e5, seed=11002), dtype=torch.float32, device="cuda")
    p = ctof.fista_params(iters=100)
    rec, rep = kern.reconstruct(m, p, report=True)
    assert torch.isfinite(rec).all()
    assert rep.iters_done == 100 and rep.beta > 0
    assert bool((rec == 0).any())  # the L1 weight zeroes voxels exactly
    assert torch.equal(rec, kern.reconstruct(m, p))
    r0 = float(m.double().norm())
    r1 = float((kern.forward(rec) - m).double().norm())
    assert r1 < r0
