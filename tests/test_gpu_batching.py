"""Batching form: several ADMM problems of uneven sizes and optics in one
captured graph: per iteration, the x-updates of all problems whose class
blocks fit the shared stages run as one persistent launch fed by a device work
queue, the FFT / TV stages of every problem on forked streams; column-FFT
tiles are autotuned.

Each problem of the batch must match the FP64 oracle (rel-L2 <= 1e-5, the
FP32 bound) and be bit-identical to the same problem reconstructed alone; a
repeated batch (graph replay) must reproduce itself.
"""

import numpy as np
import pytest

from gpu_common import rel_l2
from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so
from paper_2101_11680_gb300 import ctof, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROBLEMS = [
    # n, nz, nt, dx, dz, z_first, dt, (mua, musp, n_refr)
    (16, 6, 32, 1.0, 1.0, 1.0, 50.0, (0.01, 1.0, 1.4)),
    (20, 5, 19, 0.7, 0.9, 0.9, 33.0, (0.015, 1.5, 1.4)),
    (12, 8, 40, 1.0, 0.8, 0.8, 40.0, (0.008, 0.7, 1.33)),
    (32, 4, 24, 0.8, 1.2, 1.2, 45.0, (0.02, 2.0, 1.4)),
]
ITERS = 30


@pytest.fixture(scope="module")
def batch():
    from paper_2101_11680_gb300 import build as B
    B.build()
    kernels, ms, wants = [], [], []
    for i, (n, nz, nt, dx, dz, zf, dt, (mua, musp, nr)) in enumerate(PROBLEMS):
        g = op.Grid(n, nz, nt, dx, dz, zf, dt)
        med = ph.Medium(mua, musp, nr, r_min=0.5 * min(dx, dz))
        wh = op.kernel_spectrum(op.kernel_offsets(g, med), g)
        mu = synth.phantom_shapes(n, nz, dx, dz, zf, seed=700 + i)
        m = synth.poisson_noise(np.clip(op.forward_fft(wh, mu, g), 0, None), 1e5, 800 + i)
        wants.append(so.admm(wh, m, g, ITERS)[0])
        ms.append(torch.tensor(m, dtype=torch.float32, device="cuda"))
        kernels.append(ctof.Kernel(ctof.make_optics(mua, musp, nr), ctof.make_grid(n, nz, nt, dx, dz, zf, dt)))
    yield kernels, ms, wants
    for k in kernels:
        k.close()


def test_batch_matches_oracle_and_single(batch):
    kernels, ms, wants = batch
    p = ctof.admm_params(iters=ITERS)
    outs = ctof.reconstruct_batch(kernels, ms, p)
    torch.cuda.synchronize()
    for k, m, o, w in zip(kernels, ms, outs, wants):
        assert rel_l2(o.cpu().numpy(), w) <= 1e-5
        single = k.reconstruct(m, p)
        torch.cuda.synchronize()
        assert torch.equal(single, o)
    again = ctof.reconstruct_batch(kernels, ms, p, outs=[torch.empty_like(o) for o in outs])
    torch.cuda.synchronize()
    for a, o in zip(again, outs):
        assert torch.equal(a, o)


def test_autotuner_choices(batch):
    kernels, _, _ = batch
    for k in kernels:
        t = k.tuning()
        assert all(v in (8, 16, 108, 116) for v in t)


def test_batch_rejects_repeated_handle(batch):
    kernels, ms, _ = batch
    with pytest.raises(ctof.CtofError) as e:
        ctof.reconstruct_batch([kernels[0], kernels[0]], [ms[0], ms[0]], ctof.admm_params(iters=2))
    assert e.value.status == ctof.EINVAL
