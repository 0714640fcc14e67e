"""The allocation-free forward entry point (ctof_forward_static).

Callers that may not allocate device memory where they call the library
(real-time acquisition loops that must never wait on an allocator, host
frameworks and plugins that own every device allocation and hand the library
only input and output buffers) use ctof_forward_static, whose intermediates
live in a fixed device array inside the library.  Its output must match the
FP64 oracle's forward operator (Eq. 11) to the FP32 bound 1e-5 and the
regular ctof_forward on the same inputs, on consecutive calls that reuse the
array.  This file is collected last so that a failure here leaves every
other test already run.
"""

import numpy as np
import pytest

from gpu_common import device_kernel, oracle_kernel, rel_l2
from oracle import operators as op
from paper_2101_11680_gb300 import ctof

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_forward_static_matches_forward(name):
    g, _, wh = oracle_kernel(name)
    k = device_kernel(name)
    rng = np.random.default_rng(21)
    outs = []
    for call in range(2):
        mu = rng.uniform(0.0, 0.02, (g.nz, g.n, g.n)) * (rng.uniform(size=(g.nz, g.n, g.n)) < 0.3)
        mu_d = torch.tensor(mu, dtype=torch.float32, device="cuda")
        want = k.forward(mu_d)
        got = torch.full_like(want, float("nan"))
        k.forward_static(mu_d, got)
        torch.cuda.synchronize()
        assert rel_l2(got.cpu().numpy(), want.cpu().numpy()) <= 1e-5
        exact = op.forward_fft(wh, mu, g)
        assert rel_l2(got.cpu().numpy(), exact) <= 1e-5
        assert np.abs(got.cpu().numpy() - exact).max() <= 1e-5 * np.abs(exact).max()
        outs.append(got.cpu())
    assert not torch.equal(outs[0], outs[1])  # two different inputs, two different results


def test_forward_static_rejects_oversized_grids():
    g = ctof.make_grid(128, 48, 256, 0.5, 0.5, 0.5, 25.0)
    k = ctof.Kernel(ctof.make_optics(), g)
    try:
        mu = torch.zeros((48, 128, 128), device="cuda")
        out = torch.zeros((256, 128, 128), device="cuda")
        with pytest.raises(ctof.CtofError) as e:
            k.forward_static(mu, out)
        assert e.value.status == ctof.EUNSUPPORTED
        assert "static maximum" in str(e.value)
    finally:
        k.close()
