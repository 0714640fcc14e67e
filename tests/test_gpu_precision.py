"""Precision form: batched Tikhonov with the contraction on the tcgen05 tensor
cores in BF16 or FP8 (e4m3) and iterative refinement of the Z x Z solve.

Every volume of a batch must match the FP64 oracle's Tikhonov solution to
rel-L2 <= 1e-3 after two refinement steps (the bound stated for the BF16 and
FP8 paths); refinement must improve on the unrefined solve; the FP32 branch
of the same entry point must meet the FP32 bound (1e-5).  Batches of more
than 16 volumes span several 128-wide right-hand-side chunks.
"""

import numpy as np
import pytest

from gpu_common import device_kernel, oracle_kernel, rel_l2
from oracle import operators as op
from oracle import solvers as so
from paper_2101_11680_gb300 import ctof, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(name, count, seed0):
    g, _, wh = oracle_kernel(name)
    ms, wants = [], []
    for i in range(count):
        mu = synth.phantom_shapes(g.n, g.nz, g.dx, g.dz, g.z_first, seed=seed0 + i)
        m = synth.poisson_noise(np.clip(op.forward_fft(wh, mu, g), 0, None), 1e4, seed0 + 50 + i)
        ms.append(m)
        wants.append(so.tikhonov(wh, m, g)[0])
    return g, np.stack(ms), wants


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("name,count", [("cfg1", 3), ("ragged", 3), ("admm16", 4), ("admm16", 21)])
def test_batch_refined_matches_oracle(name, count, prec):
    g, ms, wants = _batch(name, count, seed0=300)
    k = device_kernel(name)
    m_d = torch.tensor(ms, dtype=torch.float32, device="cuda")
    p = ctof.BF16 if prec == "bf16" else ctof.FP8E4M3
    out2, lam = k.reconstruct_batch_tikhonov(m_d, precision=p, refine=2)
    out0, _ = k.reconstruct_batch_tikhonov(m_d, precision=p, refine=0)
    torch.cuda.synchronize()
    e2 = [rel_l2(out2[i].cpu().numpy(), wants[i]) for i in range(count)]
    e0 = [rel_l2(out0[i].cpu().numpy(), wants[i]) for i in range(count)]
    assert max(e2) <= 1e-3, e2
    assert max(e2) < max(e0), (e2, e0)


def test_batch_fp32_branch_matches_oracle():
    g, ms, wants = _batch("cfg1", 2, seed0=400)
    k = device_kernel("cfg1")
    out, _ = k.reconstruct_batch_tikhonov(torch.tensor(ms, dtype=torch.float32, device="cuda"),
                                          precision=ctof.FP32)
    torch.cuda.synchronize()
    for i in range(2):
        assert rel_l2(out[i].cpu().numpy(), wants[i]) <= 1e-5


def test_class_shape_64_depths_512_bins():
    """The 64-depth x 512-bin class block of the 256 x 256 x 64 x 512 workload.

    FP64 oracle solutions of two measurement volumes on a 32 x 32 scan (all
    2112 lateral frequencies solved exactly) are stored in tests/golden by
    make_oracle_fixtures.py.  The batch holds 18 volumes (two right-hand-side
    chunks, the second partial): volume i is a_i times stored volume i mod 2,
    with distinct a_i of both signs; Tikhonov is linear, so the oracle's
    answer for it is a_i times the stored solution.  BF16 and FP8 after two
    refinement steps: rel-L2 <= 1e-3 for every volume.
    """
    import os
    from paper_2101_11680_gb300 import build as B
    fx = np.load(os.path.join(os.path.dirname(__file__), "golden", "tikhonov_n32_z64_t512.npz"))
    n, nz, nt = (int(v) for v in fx["grid"])
    dx, dz, zf, dt = (float(v) for v in fx["pitch"])
    base = [fx["counts"][i].astype(np.float64) * float(fx["unit"][i]) for i in range(2)]
    alpha = [(1.0 + 0.25 * i) * (-1.0 if i % 3 == 2 else 1.0) for i in range(18)]
    ms = np.stack([alpha[i] * base[i % 2] for i in range(18)])
    B.build()
    k = ctof.Kernel(ctof.make_optics(), ctof.make_grid(n, nz, nt, dx, dz, zf, dt))
    try:
        m_d = torch.tensor(ms, dtype=torch.float32, device="cuda")
        for p in (ctof.BF16, ctof.FP8E4M3):
            out, lam = k.reconstruct_batch_tikhonov(m_d, precision=p, refine=2)
            assert lam == pytest.approx(float(fx["lam"]), rel=1e-10)
            torch.cuda.synchronize()
            errs = [rel_l2(out[i].cpu().numpy(), alpha[i] * fx["want"][i % 2].astype(np.float64))
                    for i in range(18)]
            assert max(errs) <= 1e-3, (p, errs)
    finally:
        k.close()
