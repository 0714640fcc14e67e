"""Precision form: batched BF16 tensor-core Tikhonov with iterative refinement.

Every volume of a batch must match the FP64 oracle's Tikhonov solution to
rel-L2 <= 1e-3 after two refinement steps (the bound stated for the BF16
path); refinement must improve on the unrefined BF16 solve; the FP32 branch
of the same entry point must meet the FP32 bound (1e-5).
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


@pytest.mark.parametrize("name,count", [("cfg1", 3), ("ragged", 3), ("admm16", 4)])
def test_batch_bf16_refined_matches_oracle(name, count):
    g, ms, wants = _batch(name, count, seed0=300)
    k = device_kernel(name)
    m_d = torch.tensor(ms, dtype=torch.float32, device="cuda")
    out2, lam = k.reconstruct_batch_tikhonov(m_d, precision=ctof.BF16, refine=2)
    out0, _ = k.reconstruct_batch_tikhonov(m_d, precision=ctof.BF16, refine=0)
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


def test_batch_fp8_not_built():
    k = device_kernel("sub")
    m = torch.zeros((1, 16, 8, 8), device="cuda")
    with pytest.raises(ctof.CtofError) as e:
        k.reconstruct_batch_tikhonov(m, precision=ctof.FP8E4M3)
    assert e.value.status == ctof.EUNSUPPORTED
