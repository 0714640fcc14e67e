"""Batched per-frequency contractions (ctof_contract_forward_batch / _adjoint_batch)
against the FP64 oracle spectrum.

From 4 volumes on the library runs them as 128-wide tcgen05 GEMMs (16 volumes x
one frequency class, 3xTF32); below that on the FP32 CUDA-core path.  Both are
held to rel-L2 1e-5 (3xTF32 measured ~5e-7 in isolation).  Padding entries of
the input rows (z >= nz, t >= nt) are NaN and must be ignored; padding entries
of the output rows must stay untouched.  Cases cover ragged Z / T (padding to
the MMA's K = 8 and N = 16), the anisotropic pitch (4-fold classes), the
circular grid, the largest per-class block (nt 512, nz 64: four 128-row tiles,
K = 64) and a volume count that is not a multiple of the 16-volume chunk.
"""

import functools

import numpy as np
import pytest

from gpu_common import CASES, CFG1_OPTICS, device_kernel, medium, oracle_grid, oracle_kernel
from oracle import operators as op
from paper_2101_11680_gb300 import ctof

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LARGEST = dict(n=8, nz=64, nt=512, dx=1.0, dz=0.5, z_first=0.5, dt=20.0)


@functools.lru_cache(maxsize=None)
def case(name):
    """(half-plane W_hat [F][T][Z] real, device kernel) for a case."""
    if name == "largest":
        g = oracle_grid(LARGEST)
        wh = op.kernel_spectrum(op.kernel_offsets(g, medium(grid_kw=LARGEST)), g)
        grid = ctof.make_grid(LARGEST["n"], LARGEST["nz"], LARGEST["nt"], LARGEST["dx"], LARGEST["dz"],
                              LARGEST["z_first"], LARGEST["dt"])
        from paper_2101_11680_gb300 import build as B
        B.build()
        k = ctof.Kernel(ctof.make_optics(**CFG1_OPTICS), grid)
    else:
        g, _, wh = oracle_kernel(name)
        k = device_kernel(name)
    p, h = g.p, g.p // 2 + 1
    wf = wh[:, :, :, :h].real.reshape(g.nt, g.nz, p * h)  # [T][Z][f], f = ky * h + kx
    return np.ascontiguousarray(np.transpose(wf, (2, 0, 1))), k, g


def _spectra(rng, nvol, nf, ld, valid):
    x = rng.standard_normal((nvol, nf, ld, 2)).astype(np.float32)
    x[:, :, valid:, :] = np.nan
    return x


@pytest.mark.parametrize("name", ["cfg1", "ragged", "aniso", "circ", "largest"])
@pytest.mark.parametrize("nvol", [1, 4, 16, 21])
def test_batched_contractions(name, nvol):
    wf, k, g = case(name)
    nf, nt, nz = wf.shape
    rng = np.random.default_rng(100 + nvol)
    xz = _spectra(rng, nvol, nf, k.ldz, nz)
    got = k.contract_forward_batch(torch.tensor(xz, device="cuda")).cpu().numpy()
    xc = xz[..., :nz, 0].astype(np.float64) + 1j * xz[..., :nz, 1]
    want = np.einsum("ftz,vfz->vft", wf, xc)
    gc = got[..., :nt, 0] + 1j * got[..., :nt, 1]
    assert np.linalg.norm(gc - want) <= 1e-5 * np.linalg.norm(want)
    assert not np.any(got[..., nt:, :])  # padding of the output rows untouched
    xt = _spectra(rng, nvol, nf, k.ldt, nt)
    got = k.contract_adjoint_batch(torch.tensor(xt, device="cuda")).cpu().numpy()
    xc = xt[..., :nt, 0].astype(np.float64) + 1j * xt[..., :nt, 1]
    want = np.einsum("ftz,vft->vfz", wf, xc)
    gc = got[..., :nz, 0] + 1j * got[..., :nz, 1]
    assert np.linalg.norm(gc - want) <= 1e-5 * np.linalg.norm(want)
    assert not np.any(got[..., nz:, :])


def test_batched_equals_single_volume_calls():
    """Volume v of a 16-volume call equals the FP32 path on that volume alone (to 3xTF32 rounding)."""
    wf, k, g = case("cfg1")
    nf, nt, nz = wf.shape
    rng = np.random.default_rng(5)
    xz = torch.tensor(_spectra(rng, 16, nf, k.ldz, nz), device="cuda")
    batch = k.contract_forward_batch(xz)
    for v in (0, 7, 15):
        one = k.contract_forward_batch(xz[v:v + 1].contiguous())
        d = (batch[v, :, :nt] - one[0, :, :nt]).norm() / one[0, :, :nt].norm()
        assert float(d) <= 2e-6


def test_bounded_wait_gives_up_and_reports_timeout():
    """A completion wait that runs out stops the tensor-core kernel and is reported.

    With the poll limit at 0 every MMA-completion wait of the tcgen05 kernels
    gives up at once: the kernel sets the handle's sticky flag, waits (with the
    fixed drain limit) for the MMAs in flight, frees its TMEM and returns.  The
    next synchronising call reports CTOF_ETIMEOUT and clears the flag; with the
    default limit the same calls are correct again.
    """
    wf, k, g = case("cfg1")
    nf, nt, nz = wf.shape
    rng = np.random.default_rng(9)
    xz = torch.tensor(_spectra(rng, 4, nf, k.ldz, nz), device="cuda")
    xt = torch.tensor(_spectra(rng, 4, nf, k.ldt, nt), device="cuda")
    k.sync_status()  # nothing pending
    k.set_wait_limit(0)
    try:
        for call in (k.contract_forward_batch, k.contract_adjoint_batch):
            call(xz if call == k.contract_forward_batch else xt)
            with pytest.raises(ctof.CtofError) as e:
                k.sync_status()
            assert e.value.status == ctof.ETIMEOUT
            k.sync_status()  # the flag was cleared by the read
    finally:
        k.set_wait_limit(1 << 24)
    got = k.contract_forward_batch(xz).cpu().numpy()
    k.sync_status()
    xc = xz.cpu().numpy()[..., :nz, 0].astype(np.float64) + 1j * xz.cpu().numpy()[..., :nz, 1]
    want = np.einsum("ftz,vfz->vft", wf, xc)
    gc = got[..., :nt, 0] + 1j * got[..., :nt, 1]
    assert np.linalg.norm(gc - want) <= 1e-5 * np.linalg.norm(want)
