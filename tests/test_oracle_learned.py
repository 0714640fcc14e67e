"""Pins of the learned-solver oracle: the 3-D convolution against
scipy.ndimage.correlate, and the analytic gradients of the unrolled loss
against central finite differences in FP64."""

import numpy as np
import pytest
from scipy import ndimage

from oracle import learned as ln
from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so
from paper_2101_11680_gb300 import synth


def test_conv3d_is_zero_padded_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 7))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    y = ln.conv3d(x, w, b)
    for o in range(3):
        want = np.full(x.shape[1:], b[o])
        for c in range(2):
            want += ndimage.correlate(x[c], w[o, c].reshape(3, 3, 3), mode="constant", cval=0.0)
        assert np.abs(y[o] - want).max() <= 1e-12


def test_param_count():
    assert ln.param_count(10) == 14688 + 49 + 10


def _tiny_problem(stages=3):
    g = op.Grid(6, 3, 10, 1.0, 1.0, 1.0, 50.0)
    med = ph.Medium(0.01, 1.0, 1.4, r_min=0.5)
    wh = op.kernel_spectrum(op.kernel_offsets(g, med), g)
    s = so.spectral_norm(wh)
    fwd = lambda v: op.forward_fft(wh / s, v, g)
    adj = lambda r: op.adjoint_fft(wh / s, r, g)
    rng = np.random.default_rng(1)
    mu = rng.uniform(0, 0.02, (g.nz, g.n, g.n)) * (rng.uniform(size=(g.nz, g.n, g.n)) < 0.4)
    m_n = fwd(mu)
    theta = synth.learned_init(stages, seed=5)
    theta[-stages:] = [0.9, 1.1, 0.8][:stages]
    return theta, stages, fwd, adj, m_n, mu


def test_gradients_match_finite_differences():
    theta, stages, fwd, adj, m_n, mu = _tiny_problem()
    loss, grad = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu)
    rng = np.random.default_rng(2)
    idx = list(rng.choice(len(theta) - stages, 12, replace=False)) + list(range(len(theta) - stages, len(theta)))
    for i in idx:
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = ln.loss_and_grad(tp, stages, fwd, adj, m_n, mu)[0]
        lm = ln.loss_and_grad(tm, stages, fwd, adj, m_n, mu)[0]
        fd = (lp - lm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))


def test_initial_parameters_layout():
    for stages in (1, 3, 10):
        theta = synth.learned_init(stages, seed=stages)
        assert theta.size == ln.param_count(stages)
        layers, eta = ln.unpack(theta, stages)
        assert [w.shape for w, _ in layers] == [(16, 1, 27), (16, 16, 27), (16, 16, 27), (1, 16, 27)]
        assert np.all(eta == 1.0) and all(np.all(b == 0) for _, b in layers)
    # 14,688 weights, 49 biases
    assert ln.param_count(0) == 14688 + 49


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38, -1e-40]])
    want = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ln.bf16(v), want)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert ln.bf16(1.0 + 2.0 ** -8) == 1.0 and ln.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    norm = np.abs(v) > 1e-37
    assert np.max(np.abs(ln.bf16(v[norm]) / v[norm] - 1.0)) <= 2.0 ** -8


def test_rounded_network_is_close_and_identity_rounding_is_exact():
    theta, stages, fwd, adj, m_n, mu = _tiny_problem()
    l0, g0 = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu)
    l1, g1 = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu, rnd=lambda v: v)
    assert l0 == l1 and np.array_equal(g0, g1)
    l2, g2 = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu, rnd=ln.bf16)
    assert abs(l2 / l0 - 1) < 1e-2
    assert np.linalg.norm(g2 - g0) < 5e-2 * np.linalg.norm(g0)


def test_gradients_with_tikhonov_start_match_finite_differences():
    theta, stages, fwd, adj, m_n, mu = _tiny_problem()
    g = op.Grid(6, 3, 10, 1.0, 1.0, 1.0, 50.0)
    wh = op.kernel_spectrum(op.kernel_offsets(g, ph.Medium(0.01, 1.0, 1.4, r_min=0.5)), g)
    x0 = so.tikhonov(wh, m_n, g, 1e-3)[0]
    # the start is the Tikhonov solution, not zero: the first stage sees it
    assert not np.allclose(ln.unrolled(theta, stages, fwd, adj, m_n, x0=x0), ln.unrolled(theta, stages, fwd, adj, m_n))
    loss, grad = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu, x0=x0)
    for i in [3, 500, 5000, 14000, len(theta) - 1]:
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ln.loss_and_grad(tp, stages, fwd, adj, m_n, mu, x0=x0)[0]
              - ln.loss_and_grad(tm, stages, fwd, adj, m_n, mu, x0=x0)[0]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))


def test_data_consistency_step():
    """From x = 0 one step is the Tikhonov solution; on a periodic grid each step
    multiplies the residual spectrum by lambda / (sigma^2 + lambda) <= 1."""
    g = op.Grid(8, 3, 10, 1.0, 1.0, 1.0, 50.0, mode="circular")
    wh = op.kernel_spectrum(op.kernel_offsets(g, ph.Medium(0.01, 1.0, 1.4, r_min=0.5)), g)
    s = so.spectral_norm(wh)
    fwd = lambda v: op.forward_fft(wh / s, v, g)
    adj = lambda r: op.adjoint_fft(wh / s, r, g)
    tik = lambda r: so.tikhonov(wh / s, r, g, 1e-3)[0]
    rng = np.random.default_rng(4)
    mu = rng.uniform(0, 0.02, (g.nz, g.n, g.n))
    m_n = fwd(mu) + 1e-4 * rng.standard_normal((g.nt, g.n, g.n))
    theta = synth.learned_init(2, seed=3)
    theta[:-2] *= 0.0  # f = 0: the stages are plain gradient steps
    x_tik = so.tikhonov(wh, m_n * s, g, 1e-3)[0]
    theta_zero_eta = theta.copy()
    theta_zero_eta[-2:] = 0.0
    # zero stages' effect (eta = 0, f = 0): one step from x_0 = 0 gives T m
    assert np.allclose(ln.unrolled(theta_zero_eta, 2, fwd, adj, m_n, dc_steps=1, dc_solve=tik), x_tik, rtol=1e-9,
                       atol=1e-12 * np.abs(x_tik).max())
    x = rng.uniform(0, 0.02, (g.nz, g.n, g.n))
    r0 = np.linalg.norm(fwd(x) - m_n)
    x1 = x - tik(fwd(x) - m_n)
    r1 = np.linalg.norm(fwd(x1) - m_n)
    assert r1 < 0.5 * r0
